/*
 * mlb_oracle.c -- plain FP64 CPU oracle for one time step of the multispecies
 * Enskog/RPA lattice Boltzmann method of Marini Bettolo Marconi & Melchionna,
 * "Multicomponent Diffusion in Nanosystems" (arXiv:1105.3634).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant with the CUDA path; it builds its own velocity set
 * and stencils by enumeration, and is written to be read against the paper,
 * not to be fast (OpenMP over sites is the only concession).
 *
 * What is computed, step by step (all FP64):
 *   R1  moments            n^a = sum_v f^a,  n^a u^a = sum_v v f^a,
 *                          u = sum_a m^a n^a u^a / sum_a m^a n^a      (Eq. colonna, Eq. massdensity ff.)
 *   R2  contact values     n-bar^c = mean of n^c over the ball |d| <= kappa sigma_c,
 *                          xi_k = (pi/6) sum_c sigma_c^k n-bar^c,
 *                          g_ab = BMCSL contact value at (xi_2, xi_3)  (Sec. II: "smoothing procedure";
 *                          the paper gives no formula -- reading)
 *   R3  contact sphere     integral over the unit sphere  ->  sum over lattice shell
 *                          S_ab = {d : sigma_ab - 1/2 <= |d| < sigma_ab + 1/2},
 *                          s = d/|d|, uniform weight 4 pi / |S_ab|       (reading)
 *   R4  hard-core force    Eq. potmeanforce, first term
 *   R5  velocity exchange  Eq. gammaab + Eq. viscousforce (drag + viscous with the
 *                          partner velocity at the contact point); drag only with
 *                          the flag drag_only (partner velocity at r)
 *   R6  attraction (RPA)   G^ab = sum_d n^b(r+d) (-grad U^ab)(d), U = -eps (sigma/r)^6
 *                          on sigma_ab <= |d| <= lambda_c sigma_ab  (Eq. potmeanforce, G term)
 *   R7  psi_perp           second-order Hermite projection of Eq. prefactor
 *   R8  forcing            second-order Hermite projection of (Phi/kT).(v-u) psi  (Eq. evolution)
 *   R8' time integration   semi-implicit half-force shift: psi_perp and S are taken at
 *                          u^a + a^a/2, S carries (1 - omega/2), and a is the effective
 *                          field after one Jacobi sweep of u* = u + a(u*)/2 followed by
 *                          the velocity-exchange operator applied to u* (predictor_sweeps > 1:
 *                          further Jacobi sweeps with the partners' u*); forward Euler
 *                          (a at u, no shift) with the flag explicit_force
 *   R9  collide + stream   f(r+c_i, t+1) = f - omega (f - psi_perp) + S, periodic,
 *                          halfway bounce-back on moving walls
 *   R10 initial state      f := psi_perp(n, u)
 *
 * Pair contact value between two sites is the symmetric mean
 * (g_ab(r) + g_ab(r+d))/2; sites beyond a wall hold no particles (n = 0).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define ORC_Q 19
#define ORC_MAXS 8

typedef struct {
    int32_t nx, ny, nz, nspecies;
    int32_t wall_axis;          /* -1: periodic in all directions; 0,1,2: walls normal to that axis */
    int32_t drag_only;          /* 1: partner velocity taken at r (Eq. gammaab alone) */
    int32_t explicit_force;     /* 1: forward-Euler forcing (R8); 0: semi-implicit half-force shift (R8') */
    int32_t predictor_sweeps;   /* Jacobi sweeps of u* = u + a(u*)/2 (R8'); 0 or 1: one */
    double wall_u_lo[3], wall_u_hi[3];
    double tau, kT, kappa;
    double sigma[ORC_MAXS], mass[ORC_MAXS];
    double eps[ORC_MAXS * ORC_MAXS], lambda_c[ORC_MAXS * ORC_MAXS];
} orc_params;

static const double ORC_PI = 3.14159265358979323846;
static const double CS2 = 1.0 / 3.0;   /* lattice sound speed squared of D3Q19 */

/* ---------------- velocity set: D3Q19 by enumeration ---------------- */
static int VC[ORC_Q][3];
static double VW[ORC_Q];
static int v_ready = 0;

static void build_velocities(void)
{
    if (v_ready) return;
    int k = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int q = dx * dx + dy * dy + dz * dz;
                if (q > 2) continue;
                VC[k][0] = dx; VC[k][1] = dy; VC[k][2] = dz;
                VW[k] = (q == 0) ? 1.0 / 3.0 : (q == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
                ++k;
            }
    v_ready = 1;
}

int orc_velocities(int32_t *c, double *w)
{
    build_velocities();
    for (int i = 0; i < ORC_Q; ++i) {
        for (int a = 0; a < 3; ++a) c[3 * i + a] = VC[i][a];
        w[i] = VW[i];
    }
    return ORC_Q;
}

static int opposite(int i)
{
    for (int k = 0; k < ORC_Q; ++k)
        if (VC[k][0] == -VC[i][0] && VC[k][1] == -VC[i][1] && VC[k][2] == -VC[i][2]) return k;
    return -1;
}

/* ---------------- geometry ---------------- */
static long nsites(const orc_params *p) { return (long)p->nx * p->ny * p->nz; }

static long site(const orc_params *p, int x, int y, int z) { return x + (long)p->nx * (y + (long)p->ny * z); }

static int wrap(int x, int L) { int m = x % L; return m < 0 ? m + L : m; }

/* Index of r+d, or -1 when r+d lies beyond a wall (no particles there). */
static long neighbour(const orc_params *p, int x, int y, int z, int dx, int dy, int dz)
{
    int c[3] = {x + dx, y + dy, z + dz};
    int L[3] = {p->nx, p->ny, p->nz};
    for (int a = 0; a < 3; ++a) {
        if (a == p->wall_axis) {
            if (c[a] < 0 || c[a] >= L[a]) return -1;
        } else {
            c[a] = wrap(c[a], L[a]);
        }
    }
    return site(p, c[0], c[1], c[2]);
}

static void coords(const orc_params *p, long s, int *x, int *y, int *z)
{
    *x = (int)(s % p->nx);
    *y = (int)((s / p->nx) % p->ny);
    *z = (int)(s / ((long)p->nx * p->ny));
}

/* ---------------- stencils by enumeration ---------------- */
typedef struct { int n; int (*d)[3]; } orc_set;

static void set_free(orc_set *s) { free(s->d); s->d = NULL; s->n = 0; }

/* all integer offsets with lo2 <= |d|^2 (strict: lo2 < |d|^2 if lo_strict) and |d|^2 <= hi2 (or < hi2) */
static orc_set enumerate(double lo2, int lo_strict, double hi2, int hi_strict, int exclude_zero)
{
    orc_set s = {0, NULL};
    int R = (int)ceil(sqrt(hi2)) + 1;
    long cap = (long)(2 * R + 1) * (2 * R + 1) * (2 * R + 1);
    s.d = (int (*)[3])malloc(sizeof(int[3]) * cap);
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                double q = (double)(dx * dx + dy * dy + dz * dz);
                if (exclude_zero && q == 0.0) continue;
                if (lo_strict ? !(q > lo2) : !(q >= lo2)) continue;
                if (hi_strict ? !(q < hi2) : !(q <= hi2)) continue;
                s.d[s.n][0] = dx; s.d[s.n][1] = dy; s.d[s.n][2] = dz;
                ++s.n;
            }
    return s;
}

/* contact shell S_ab (R3) */
static orc_set contact_shell(double sab)
{
    double lo = sab - 0.5, hi = sab + 0.5;
    return enumerate(lo > 0 ? lo * lo : 0.0, 0, hi * hi, 1, 1);
}

/* smoothing ball B_c (R2): |d| <= kappa sigma_c, origin included */
static orc_set smoothing_ball(double radius) { return enumerate(0.0, 0, radius * radius, 0, 0); }

/* attraction region (R6): sigma_ab <= |d| <= lambda_c sigma_ab */
static orc_set attraction_ball(double sab, double lc)
{
    return enumerate(sab * sab, 0, (lc * sab) * (lc * sab), 0, 1);
}

int orc_shell(double sab, int32_t *out, int cap)
{
    orc_set s = contact_shell(sab);
    int n = s.n;
    for (int k = 0; k < n && k < cap; ++k) for (int a = 0; a < 3; ++a) out[3 * k + a] = s.d[k][a];
    set_free(&s);
    return n;
}

int orc_attraction_set(double sab, double lc, int32_t *out, int cap)
{
    orc_set s = attraction_ball(sab, lc);
    int n = s.n;
    for (int k = 0; k < n && k < cap; ++k) for (int a = 0; a < 3; ++a) out[3 * k + a] = s.d[k][a];
    set_free(&s);
    return n;
}

/* ---------------- R2: BMCSL contact value ---------------- */
/* Boublik-Mansoori-Carnahan-Starling-Leland contact value of the a-b pair of a
 * hard-sphere mixture with diameters sa, sb at packing moments xi2, xi3. */
double orc_bmcsl(double sa, double sb, double xi2, double xi3)
{
    double h = sa * sb / (sa + sb);
    double one = 1.0 - xi3;
    return 1.0 / one + 3.0 * h * xi2 / (one * one) + 2.0 * h * h * xi2 * xi2 / (one * one * one);
}

/* ---------------- R1: moments ---------------- */
/* f: [S][19][N];  n: [S][N];  j: [S][3][N] (j = n u) */
int orc_moments(const orc_params *p, const double *f, double *n, double *j)
{
    build_velocities();
    long N = nsites(p);
    int S = p->nspecies;
#pragma omp parallel for schedule(static)
    for (long r = 0; r < N; ++r) {
        for (int a = 0; a < S; ++a) {
            double m0 = 0.0, m1[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < ORC_Q; ++i) {
                double fi = f[((long)a * ORC_Q + i) * N + r];
                m0 += fi;
                for (int k = 0; k < 3; ++k) m1[k] += VC[i][k] * fi;
            }
            n[(long)a * N + r] = m0;
            for (int k = 0; k < 3; ++k) j[((long)a * 3 + k) * N + r] = m1[k];
        }
    }
    return 0;
}

/* barycentric velocity and species velocities at one site */
static void site_velocities(const orc_params *p, const double *n, const double *j, long r, double ua[][3], double u[3])
{
    long N = nsites(p);
    int S = p->nspecies;
    double rho = 0.0, mom[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < S; ++a) {
        rho += p->mass[a] * n[(long)a * N + r];
        for (int k = 0; k < 3; ++k) mom[k] += p->mass[a] * j[((long)a * 3 + k) * N + r];
    }
    for (int k = 0; k < 3; ++k) u[k] = rho > 0.0 ? mom[k] / rho : 0.0;
    for (int a = 0; a < S; ++a) {
        double na = n[(long)a * N + r];
        for (int k = 0; k < 3; ++k) ua[a][k] = (na > 1e-300) ? j[((long)a * 3 + k) * N + r] / na : u[k];
    }
}

/* ---------------- R2: smoothed densities and contact values ---------------- */
/* g: [S][S][N] (full symmetric matrix);  xi: [2][N] = (xi2, xi3), either may be NULL */
int orc_gfield(const orc_params *p, const double *n, double *g, double *xi)
{
    long N = nsites(p);
    int S = p->nspecies;
    orc_set ball[ORC_MAXS];
    for (int c = 0; c < S; ++c) ball[c] = smoothing_ball(p->kappa * p->sigma[c]);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (long r = 0; r < N; ++r) {
        int x, y, z;
        coords(p, r, &x, &y, &z);
        double xi2 = 0.0, xi3 = 0.0;
        for (int c = 0; c < S; ++c) {
            double sum = 0.0;
            for (int k = 0; k < ball[c].n; ++k) {
                long r2 = neighbour(p, x, y, z, ball[c].d[k][0], ball[c].d[k][1], ball[c].d[k][2]);
                if (r2 >= 0) sum += n[(long)c * N + r2];
            }
            double nbar = sum / ball[c].n;
            double sc = p->sigma[c];
            xi2 += ORC_PI / 6.0 * sc * sc * nbar;
            xi3 += ORC_PI / 6.0 * sc * sc * sc * nbar;
        }
        if (!(xi3 < 1.0)) bad = 1;
        if (xi) { xi[r] = xi2; xi[N + r] = xi3; }
        for (int a = 0; a < S; ++a)
            for (int b = 0; b < S; ++b)
                g[((long)a * S + b) * N + r] = orc_bmcsl(p->sigma[a], p->sigma[b], xi2, xi3);
    }
    for (int c = 0; c < S; ++c) set_free(&ball[c]);
    return bad ? 1 : 0;
}

/* ---------------- R4-R6: effective field ---------------- */
typedef struct {
    orc_set shell[ORC_MAXS][ORC_MAXS];
    orc_set attr[ORC_MAXS][ORC_MAXS];
} orc_tables;

static void tables_build(const orc_params *p, orc_tables *t)
{
    int S = p->nspecies;
    for (int a = 0; a < S; ++a)
        for (int b = 0; b < S; ++b) {
            double sab = 0.5 * (p->sigma[a] + p->sigma[b]);
            t->shell[a][b] = contact_shell(sab);
            if (p->eps[a * S + b] != 0.0)
                t->attr[a][b] = attraction_ball(sab, p->lambda_c[a * S + b]);
            else {
                t->attr[a][b].n = 0; t->attr[a][b].d = NULL;
            }
        }
}

static void tables_free(const orc_params *p, orc_tables *t)
{
    for (int a = 0; a < p->nspecies; ++a)
        for (int b = 0; b < p->nspecies; ++b) { set_free(&t->shell[a][b]); set_free(&t->attr[a][b]); }
}

static double reduced_mass(const orc_params *p, int a, int b) { return p->mass[a] * p->mass[b] / (p->mass[a] + p->mass[b]); }

/* Hard-core contact force (R4, Eq. potmeanforce first term) and attractive
 * mean field (R6, the G term) on species a at site r. */
static void rest_force_site(const orc_params *p, const orc_tables *t, const double *n, const double *g,
                            long r, int a, double hc[3], double at[3])
{
    long N = nsites(p);
    int S = p->nspecies;
    int x, y, z;
    coords(p, r, &x, &y, &z);
    for (int q = 0; q < 3; ++q) { hc[q] = 0.0; at[q] = 0.0; }
    for (int b = 0; b < S; ++b) {
        double sab = 0.5 * (p->sigma[a] + p->sigma[b]);
        const orc_set *sh = &t->shell[a][b];
        double wS = 4.0 * ORC_PI / sh->n;
        double gr = g[((long)a * S + b) * N + r];
        double acc[3] = {0, 0, 0};
        for (int k = 0; k < sh->n; ++k) {
            const int *d = sh->d[k];
            long r2 = neighbour(p, x, y, z, d[0], d[1], d[2]);
            if (r2 < 0) continue;
            double len = sqrt((double)(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
            double gbar = 0.5 * (gr + g[((long)a * S + b) * N + r2]);
            double nb = n[(long)b * N + r2];
            for (int q = 0; q < 3; ++q) acc[q] += (d[q] / len) * gbar * nb;
        }
        for (int q = 0; q < 3; ++q) hc[q] += -p->kT * sab * sab * wS * acc[q];
        double e = p->eps[a * S + b];
        if (e != 0.0) {
            double s6 = pow(sab, 6.0);
            const orc_set *ab = &t->attr[a][b];
            for (int k = 0; k < ab->n; ++k) {
                const int *d = ab->d[k];
                long r2 = neighbour(p, x, y, z, d[0], d[1], d[2]);
                if (r2 < 0) continue;
                double q2 = (double)(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                /* -grad U(r - r') at r' = r + d, U = -eps (sigma/|x|)^6:  6 eps sigma^6 d / |d|^8 */
                double coef = 6.0 * e * s6 / (q2 * q2 * q2 * q2);
                double nb = n[(long)b * N + r2];
                for (int q = 0; q < 3; ++q) at[q] += coef * d[q] * nb;
            }
        }
    }
}

/* Velocity exchange (R5, Eqs. gammaab + viscousforce) for species a at site r,
 * written as  F^v = gain - Gamma u^a(r)  with
 *   gain  = sum_b K_ab wS sum_d s (s . v^b(partner)) gbar n^b(r+d)
 *   Gamma = sum_b K_ab wS sum_d s s^T gbar n^b(r+d)
 * where the partner velocity is v^b(r+d) (drag + viscous) or v^b(r) (drag only).
 * vel: [S][3][N] velocity field. */
static void exchange_site(const orc_params *p, const orc_tables *t, const double *n, const double *g,
                          const double *vel, long r, int a, double gain[3], double Gam[3][3])
{
    long N = nsites(p);
    int S = p->nspecies;
    int x, y, z;
    coords(p, r, &x, &y, &z);
    for (int q = 0; q < 3; ++q) { gain[q] = 0.0; for (int s = 0; s < 3; ++s) Gam[q][s] = 0.0; }
    for (int b = 0; b < S; ++b) {
        double sab = 0.5 * (p->sigma[a] + p->sigma[b]);
        const orc_set *sh = &t->shell[a][b];
        double wS = 4.0 * ORC_PI / sh->n;
        double Kab = 2.0 * sab * sab * sqrt(2.0 * reduced_mass(p, a, b) * p->kT / ORC_PI);
        double gr = g[((long)a * S + b) * N + r];
        for (int k = 0; k < sh->n; ++k) {
            const int *d = sh->d[k];
            long r2 = neighbour(p, x, y, z, d[0], d[1], d[2]);
            if (r2 < 0) continue;
            double len = sqrt((double)(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
            double s[3] = {d[0] / len, d[1] / len, d[2] / len};
            double gbar = 0.5 * (gr + g[((long)a * S + b) * N + r2]);
            double wgt = Kab * wS * gbar * n[(long)b * N + r2];
            long rp = p->drag_only ? r : r2;
            double sv = 0.0;
            for (int q = 0; q < 3; ++q) sv += s[q] * vel[((long)b * 3 + q) * N + rp];
            for (int q = 0; q < 3; ++q) {
                gain[q] += wgt * s[q] * sv;
                for (int c = 0; c < 3; ++c) Gam[q][c] += wgt * s[q] * s[c];
            }
        }
    }
}

/* species velocity field u^a = j^a/n^a (R1), [S][3][N] */
static void velocity_field(const orc_params *p, const double *n, const double *j, double *vel)
{
    long N = nsites(p);
    int S = p->nspecies;
#pragma omp parallel for schedule(static)
    for (long r = 0; r < N; ++r) {
        double ua[ORC_MAXS][3], u[3];
        site_velocities(p, n, j, r, ua, u);
        for (int a = 0; a < S; ++a)
            for (int q = 0; q < 3; ++q) vel[((long)a * 3 + q) * N + r] = ua[a][q];
    }
}

/* The effective field Phi = F^hc + G + F^v at the velocities of the state
 * (Eq. splitforce).  phi, hc, vx, at: [S][3][M] (any may be NULL except phi);
 * sites == NULL means every site. */
int orc_forces_sites(const orc_params *p, const double *n, const double *j, const double *g,
                     long nlist, const int64_t *sites,
                     double *phi, double *hc, double *vx, double *at)
{
    long N = nsites(p);
    int S = p->nspecies;
    orc_tables t;
    tables_build(p, &t);
    double *vel = (double *)malloc(sizeof(double) * S * 3 * N);
    velocity_field(p, n, j, vel);
    long M = sites ? nlist : N;
#pragma omp parallel for schedule(dynamic, 64)
    for (long k = 0; k < M; ++k) {
        long r = sites ? (long)sites[k] : k;
        for (int a = 0; a < S; ++a) {
            double h[3], A[3], gain[3], Gam[3][3];
            rest_force_site(p, &t, n, g, r, a, h, A);
            exchange_site(p, &t, n, g, vel, r, a, gain, Gam);
            for (int q = 0; q < 3; ++q) {
                double v = gain[q];
                for (int c = 0; c < 3; ++c) v -= Gam[q][c] * vel[((long)a * 3 + c) * N + r];
                long o = ((long)a * 3 + q) * M + k;
                phi[o] = h[q] + v + A[q];
                if (hc) hc[o] = h[q];
                if (vx) vx[o] = v;
                if (at) at[o] = A[q];
            }
        }
    }
    free(vel);
    tables_free(p, &t);
    return 0;
}

int orc_forces(const orc_params *p, const double *n, const double *j, const double *g,
               double *phi, double *hc, double *vx, double *at)
{
    return orc_forces_sites(p, n, j, g, 0, NULL, phi, hc, vx, at);
}

/* solve (I + G/(2m)) x = b for a symmetric 3x3 G by Gaussian elimination */
static void solve3(double Gam[3][3], double m, const double b[3], double x[3])
{
    double A[3][4];
    for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k) A[i][k] = (i == k ? 1.0 : 0.0) + Gam[i][k] / (2.0 * m);
        A[i][3] = b[i];
    }
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        for (int i = c + 1; i < 3; ++i) if (fabs(A[i][c]) > fabs(A[piv][c])) piv = i;
        if (piv != c) for (int k = 0; k < 4; ++k) { double tmp = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = tmp; }
        for (int i = c + 1; i < 3; ++i) {
            double f = A[i][c] / A[c][c];
            for (int k = c; k < 4; ++k) A[i][k] -= f * A[c][k];
        }
    }
    for (int i = 2; i >= 0; --i) {
        double s = A[i][3];
        for (int k = i + 1; k < 3; ++k) s -= A[i][k] * x[k];
        x[i] = s / A[i][i];
    }
}

/* Acceleration a^a = (Phi^a + F_ext^a)/m^a that one step applies (R8'):
 *
 *  explicit_force = 1:  Phi evaluated at the current velocities.
 *  otherwise (semi-implicit half-force shift):
 *    pass 1  u* solves (I + Gamma/2m) u* = u + (F^hc + G + F_ext + gain(u))/2m
 *            (one Jacobi sweep of u* = u + a(u*)/2, partners held at u)
 *    pass 2  a = (F^hc + G + F_ext + gain(u*) - Gamma u*)/m,
 *            i.e. the velocity-exchange operator evaluated on the field u*.
 *
 * fext: [S][3][N] or NULL.  acc: [S][3][M].  ustar (optional): [S][3][N].
 * sites != NULL: acc only at the listed sites (pass 1 is done where needed). */
int orc_accel_sites(const orc_params *p, const double *n, const double *j, const double *g, const double *fext,
                    long nlist, const int64_t *sites, double *acc, double *ustar_out)
{
    long N = nsites(p);
    int S = p->nspecies;
    orc_tables t;
    tables_build(p, &t);
    double *vel = (double *)malloc(sizeof(double) * S * 3 * N);
    double *ust = (double *)calloc((size_t)S * 3 * N, sizeof(double));
    double *rest = (double *)calloc((size_t)S * 3 * N, sizeof(double));
    unsigned char *need = (unsigned char *)calloc((size_t)N, 1);
    velocity_field(p, n, j, vel);
    long M = sites ? nlist : N;

    /* sites where pass 1 is needed: the listed sites and their contact shells
       (every site when more than one predictor sweep is taken) */
    const int sweeps = p->predictor_sweeps > 1 ? p->predictor_sweeps : 1;
    if (!sites || sweeps > 1) {
        memset(need, 1, (size_t)N);
    } else {
        for (long k = 0; k < M; ++k) {
            long r = (long)sites[k];
            int x, y, z;
            coords(p, r, &x, &y, &z);
            need[r] = 1;
            for (int a = 0; a < S; ++a)
                for (int b = 0; b < S; ++b)
                    for (int m = 0; m < t.shell[a][b].n; ++m) {
                        const int *d = t.shell[a][b].d[m];
                        long r2 = neighbour(p, x, y, z, d[0], d[1], d[2]);
                        if (r2 >= 0) need[r2] = 1;
                    }
        }
    }

#pragma omp parallel for schedule(dynamic, 64)
    for (long r = 0; r < N; ++r) {
        if (!need[r]) continue;
        for (int a = 0; a < S; ++a) {
            double h[3], A[3], gain[3], Gam[3][3], b[3], xs[3];
            rest_force_site(p, &t, n, g, r, a, h, A);
            for (int q = 0; q < 3; ++q)
                rest[((long)a * 3 + q) * N + r] = h[q] + A[q] + (fext ? fext[((long)a * 3 + q) * N + r] : 0.0);
            if (p->explicit_force) continue;
            exchange_site(p, &t, n, g, vel, r, a, gain, Gam);
            for (int q = 0; q < 3; ++q)
                b[q] = vel[((long)a * 3 + q) * N + r] + (rest[((long)a * 3 + q) * N + r] + gain[q]) / (2.0 * p->mass[a]);
            solve3(Gam, p->mass[a], b, xs);
            for (int q = 0; q < 3; ++q) ust[((long)a * 3 + q) * N + r] = xs[q];
        }
    }
    /* further Jacobi sweeps: the partners' velocities from the previous sweep */
    if (!p->explicit_force && sweeps > 1) {
        double *prev = (double *)malloc(sizeof(double) * S * 3 * N);
        for (int k = 1; k < sweeps; ++k) {
            memcpy(prev, ust, sizeof(double) * S * 3 * N);
#pragma omp parallel for schedule(dynamic, 64)
            for (long r = 0; r < N; ++r)
                for (int a = 0; a < S; ++a) {
                    double gain[3], Gam[3][3], b[3], xs[3];
                    exchange_site(p, &t, n, g, prev, r, a, gain, Gam);
                    for (int q = 0; q < 3; ++q)
                        b[q] = vel[((long)a * 3 + q) * N + r] + (rest[((long)a * 3 + q) * N + r] + gain[q]) / (2.0 * p->mass[a]);
                    solve3(Gam, p->mass[a], b, xs);
                    for (int q = 0; q < 3; ++q) ust[((long)a * 3 + q) * N + r] = xs[q];
                }
        }
        free(prev);
    }

    const double *vfield = p->explicit_force ? vel : ust;
#pragma omp parallel for schedule(dynamic, 64)
    for (long k = 0; k < M; ++k) {
        long r = sites ? (long)sites[k] : k;
        for (int a = 0; a < S; ++a) {
            double gain[3], Gam[3][3];
            exchange_site(p, &t, n, g, vfield, r, a, gain, Gam);
            for (int q = 0; q < 3; ++q) {
                double v = gain[q];
                for (int c = 0; c < 3; ++c) v -= Gam[q][c] * vfield[((long)a * 3 + c) * N + r];
                acc[((long)a * 3 + q) * M + k] = (rest[((long)a * 3 + q) * N + r] + v) / p->mass[a];
            }
        }
    }
    if (ustar_out) memcpy(ustar_out, ust, sizeof(double) * S * 3 * N);
    free(vel); free(ust); free(rest); free(need);
    tables_free(p, &t);
    return 0;
}

/* ---------------- R7, R8: equilibrium and forcing at one site ---------------- */
/* Q_i : M with Q_i = c_i c_i - cs2 I */
static double q_contract(int i, double M[3][3])
{
    double s = 0.0;
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y)
            s += (VC[i][x] * VC[i][y] - (x == y ? CS2 : 0.0)) * M[x][y];
    return s;
}

/* psi_perp_i (R7) and forcing S_i (R8) of species a at one site */
static void equilibrium_site(double na, const double ua[3], const double u[3], const double acc[3],
                             double *psi, double *src)
{
    double Mpsi[3][3], Ms[3][3];
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) {
            /* second moment of psi_perp minus its isotropic part, per unit density */
            Mpsi[x][y] = ua[x] * u[y] + u[x] * ua[y] - u[x] * u[y];
            /* second moment of the forcing term, per unit density */
            Ms[x][y] = u[x] * acc[y] + acc[x] * u[y];
        }
    for (int i = 0; i < ORC_Q; ++i) {
        double cu = 0.0, ca = 0.0;
        for (int k = 0; k < 3; ++k) { cu += VC[i][k] * ua[k]; ca += VC[i][k] * acc[k]; }
        psi[i] = VW[i] * na * (1.0 + cu / CS2 + q_contract(i, Mpsi) / (2.0 * CS2 * CS2));
        src[i] = VW[i] * na * (ca / CS2 + q_contract(i, Ms) / (2.0 * CS2 * CS2));
    }
}

/* Post-collision populations of species a at one site (R9 with R8'):
 *   fpost_i = f_i - omega (f_i - psi_perp_i(n, u_eq^a, u_eq)) + k S_i(a, u_eq)
 * semi-implicit shift (default): u_eq^b = u^b + acc^b/2 for every species b,
 *   u_eq their barycentre, k = 1 - omega/2;
 * explicit_force:  u_eq^b = u^b, u_eq = u, k = 1.
 * ua_all/acc_all: [S][3] velocities and accelerations of all species at the site. */
static void collide_site(const orc_params *p, const double *fa, int a, const double *n_all,
                         double ua_all[][3], double acc_all[][3], double *fpost)
{
    int S = p->nspecies;
    double omega = 1.0 / p->tau;
    double half = p->explicit_force ? 0.0 : 0.5;
    double ueq[ORC_MAXS][3], u[3] = {0, 0, 0}, rho = 0.0;
    for (int b = 0; b < S; ++b) {
        rho += p->mass[b] * n_all[b];
        for (int q = 0; q < 3; ++q) {
            ueq[b][q] = ua_all[b][q] + half * acc_all[b][q];
            u[q] += p->mass[b] * n_all[b] * ueq[b][q];
        }
    }
    for (int q = 0; q < 3; ++q) u[q] = rho > 0.0 ? u[q] / rho : 0.0;
    double psi[ORC_Q], src[ORC_Q];
    equilibrium_site(n_all[a], ueq[a], u, acc_all[a], psi, src);
    double k = p->explicit_force ? 1.0 : 1.0 - 0.5 * omega;
    for (int i = 0; i < ORC_Q; ++i) fpost[i] = fa[i] - omega * (fa[i] - psi[i]) + k * src[i];
}

/* Post-collision populations at a list of sites from local data only:
 * f: [nlist][S][19], n: [nlist][S], j: [nlist][S][3],
 * acc: [nlist][S][3] accelerations (Phi + F_ext)/m;  out: [nlist][S][19]. */
int orc_collide_local(const orc_params *p, long nlist, const double *f, const double *n, const double *j,
                      const double *acc, double *out)
{
    build_velocities();
    int S = p->nspecies;
    for (long t = 0; t < nlist; ++t) {
        double rho = 0.0, mom[3] = {0, 0, 0}, u[3], ua[ORC_MAXS][3], ac[ORC_MAXS][3];
        for (int a = 0; a < S; ++a) {
            rho += p->mass[a] * n[t * S + a];
            for (int k = 0; k < 3; ++k) mom[k] += p->mass[a] * j[(t * S + a) * 3 + k];
        }
        for (int k = 0; k < 3; ++k) u[k] = rho > 0 ? mom[k] / rho : 0.0;
        for (int a = 0; a < S; ++a)
            for (int k = 0; k < 3; ++k) {
                ua[a][k] = n[t * S + a] > 1e-300 ? j[(t * S + a) * 3 + k] / n[t * S + a] : u[k];
                ac[a][k] = acc[(t * S + a) * 3 + k];
            }
        for (int a = 0; a < S; ++a)
            collide_site(p, f + (t * S + a) * ORC_Q, a, n + t * S, ua, ac, out + (t * S + a) * ORC_Q);
    }
    return 0;
}

/* ---------------- R9: collide and stream over the whole lattice ---------------- */
/* acc: [S][3][N] accelerations from orc_accel_sites */
static void collide_stream(const orc_params *p, const double *f, const double *n, const double *j,
                           const double *acc, double *fnew)
{
    long N = nsites(p);
    int S = p->nspecies;
#pragma omp parallel for schedule(static)
    for (long r = 0; r < N; ++r) {
        int x, y, z;
        coords(p, r, &x, &y, &z);
        int xr[3] = {x, y, z};
        double ua[ORC_MAXS][3], u[3], ac[ORC_MAXS][3], nn[ORC_MAXS];
        site_velocities(p, n, j, r, ua, u);
        for (int a = 0; a < S; ++a) {
            nn[a] = n[(long)a * N + r];
            for (int k = 0; k < 3; ++k) ac[a][k] = acc[((long)a * 3 + k) * N + r];
        }
        for (int a = 0; a < S; ++a) {
            double fa[ORC_Q], fpost[ORC_Q];
            for (int i = 0; i < ORC_Q; ++i) fa[i] = f[((long)a * ORC_Q + i) * N + r];
            collide_site(p, fa, a, nn, ua, ac, fpost);
            for (int i = 0; i < ORC_Q; ++i) {
                long r2 = neighbour(p, x, y, z, VC[i][0], VC[i][1], VC[i][2]);
                if (r2 >= 0) {
                    fnew[((long)a * ORC_Q + i) * N + r2] = fpost[i];
                } else {
                    /* link crosses a wall: halfway bounce-back with the wall's velocity */
                    int ax = p->wall_axis;
                    const double *uw = (xr[ax] + VC[i][ax] < 0) ? p->wall_u_lo : p->wall_u_hi;
                    double cuw = VC[i][0] * uw[0] + VC[i][1] * uw[1] + VC[i][2] * uw[2];
                    fnew[((long)a * ORC_Q + opposite(i)) * N + r] = fpost[i] - 2.0 * VW[i] * nn[a] * cuw / CS2;
                }
            }
        }
    }
}

/* ---------------- R10: initial populations ---------------- */
/* n: [S][N]; u: [S][3][N] species velocities or NULL (rest) */
int orc_init(const orc_params *p, const double *n, const double *u_species, double *f)
{
    build_velocities();
    long N = nsites(p);
    int S = p->nspecies;
    double *j = (double *)calloc((size_t)S * 3 * N, sizeof(double));
    if (!j) return -1;
    if (u_species)
        for (int a = 0; a < S; ++a)
            for (int k = 0; k < 3; ++k)
                for (long r = 0; r < N; ++r)
                    j[((long)a * 3 + k) * N + r] = n[(long)a * N + r] * u_species[((long)a * 3 + k) * N + r];
    for (long r = 0; r < N; ++r) {
        double ua[ORC_MAXS][3], u[3], zero[3] = {0, 0, 0};
        site_velocities(p, n, j, r, ua, u);
        for (int a = 0; a < S; ++a) {
            double psi[ORC_Q], src[ORC_Q];
            equilibrium_site(n[(long)a * N + r], ua[a], u, zero, psi, src);
            for (int i = 0; i < ORC_Q; ++i) f[((long)a * ORC_Q + i) * N + r] = psi[i];
        }
    }
    free(j);
    return 0;
}

/* ---------------- full step ---------------- */
/* fext: [S][3][N] or NULL.  Returns 0, or 1 if xi3 >= 1 was met (the state is then invalid). */
int orc_step(const orc_params *p, double *f, const double *fext, int nsteps)
{
    build_velocities();
    long N = nsites(p);
    int S = p->nspecies;
    double *n = (double *)malloc(sizeof(double) * S * N);
    double *j = (double *)malloc(sizeof(double) * S * 3 * N);
    double *g = (double *)malloc(sizeof(double) * S * S * N);
    double *acc = (double *)malloc(sizeof(double) * S * 3 * N);
    double *fnew = (double *)malloc(sizeof(double) * S * ORC_Q * N);
    if (!n || !j || !g || !acc || !fnew) { free(n); free(j); free(g); free(acc); free(fnew); return -1; }
    int status = 0;
    for (int t = 0; t < nsteps; ++t) {
        orc_moments(p, f, n, j);                                  /* R1 */
        if (orc_gfield(p, n, g, NULL)) status = 1;                /* R2 */
        orc_accel_sites(p, n, j, g, fext, 0, NULL, acc, NULL);    /* R3-R6, R8' */
        collide_stream(p, f, n, j, acc, fnew);                    /* R7, R9 */
        memcpy(f, fnew, sizeof(double) * S * ORC_Q * N);
    }
    free(n); free(j); free(g); free(acc); free(fnew);
    return status;
}

/* threads the OpenMP loops use from now on (n >= 1); a no-op without OpenMP */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
