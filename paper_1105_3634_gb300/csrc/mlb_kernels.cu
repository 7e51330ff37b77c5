// mlb_kernels.cu -- sm_103a kernels of the multispecies Enskog/RPA lattice
// Boltzmann step (arXiv:1105.3634, Secs. II-III and V).
//
// Storage (structure of arrays, x fastest, site r = x + nx (y + ny z)):
//   f[a][i][r]  FP32 populations minus w_i n_ref^a      (76 B per species-site)
//   mom[a][r]   float4 (n - n_ref, u_x, u_y, u_z)        (16 B per species-site)
//   dg[p][r]    g_ab - g_ab(reference densities)          (per unordered pair)
//   frest[a][r] F^hc + G + F_ext - Gamma du               (pass 1 -> pass 2)
//   pst[a][r]   (n - n_ref, u + du)                       (pass 1 -> pass 2)
//
// One step (all launches on one stream):
//   k_moments        f -> mom                                    (Eq. colonna)
//   k_gfield         mom -> dg: smoothed densities, BMCSL g       (Sec. II smoothing)
//   (k_moments_g     the two above in one pass when g is site-local)
//   k_pass1          mom, dg -> frest, pst: hard core + attraction  (Eqs. potmeanforce, gammaab,
//                    + velocity exchange at u, then the one-sweep    viscousforce)
//                    half-step predictor
//   k_pass2          velocity exchange at u + du -> acc
//   k_collide        collision toward psi_perp at u + a/2 with      (Eqs. evolution, prefactor)
//                    (1 - omega/2) forcing, push streaming /
//                    halfway bounce-back
// Deviations from reference values (n - n_ref, g - g_ref) and velocities
// (rather than momenta) keep the FP32 differences that the contact sums take
// between neighbouring sites small and exact.
#include "mlb_internal.h"

#include <math.h>

namespace {

// D3Q19 velocities: rest, 6 axis links, 12 face diagonals; opposite of i >= 1 is i^1 shifted
__device__ constexpr int CX[MLBI_Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__device__ constexpr int CY[MLBI_Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__device__ constexpr int CZ[MLBI_Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
__device__ constexpr float WQ[MLBI_Q] = {1.f / 3.f,
                                         1.f / 18.f, 1.f / 18.f, 1.f / 18.f, 1.f / 18.f, 1.f / 18.f, 1.f / 18.f,
                                         1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f,
                                         1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};

__device__ __forceinline__ int opposite(int i) { return i == 0 ? 0 : (((i - 1) ^ 1) + 1); }

// the same velocity set for a runtime index, from bit tables (no memory access):
// component = (bit of "plus" mask) - (bit of "minus" mask)
__device__ __forceinline__ int comp_of(int i, unsigned plus, unsigned minus)
{
    return (int)((plus >> i) & 1u) - (int)((minus >> i) & 1u);
}
__device__ __forceinline__ int CXv(int i) { return comp_of(i, 0x2A82u, 0x5504u); }
__device__ __forceinline__ int CYv(int i) { return comp_of(i, 0x28488u, 0x50310u); }
__device__ __forceinline__ int CZv(int i) { return comp_of(i, 0x4C820u, 0x33040u); }
__device__ __forceinline__ float WQv(int i) { return i == 0 ? 1.f / 3.f : (i < 7 ? 1.f / 18.f : 1.f / 36.f); }

constexpr int kBlock = 256;
constexpr float kTinyDensity = 1e-12f;

inline unsigned grid_for(long long N)
{
    long long g = (N + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    if (g > (1ll << 30)) g = 1ll << 30;
    return (unsigned)g;
}

// r + d with periodic wrap (|d| < extent is guaranteed by the host) or -1 beyond a wall
__device__ __forceinline__ long long neighbour(const mlbi_params &p, int x, int y, int z, int dx, int dy, int dz)
{
    int c0 = x + dx, c1 = y + dy, c2 = z + dz;
    if (p.wall_axis == 0) { if (c0 < 0 || c0 >= p.nx) return -1; }
    else { c0 += (c0 < 0) ? p.nx : 0; c0 -= (c0 >= p.nx) ? p.nx : 0; }
    if (p.wall_axis == 1) { if (c1 < 0 || c1 >= p.ny) return -1; }
    else { c1 += (c1 < 0) ? p.ny : 0; c1 -= (c1 >= p.ny) ? p.ny : 0; }
    if (p.wall_axis == 2) { if (c2 < 0 || c2 >= p.nz) return -1; }
    else { c2 += (c2 < 0) ? p.nz : 0; c2 -= (c2 >= p.nz) ? p.nz : 0; }
    return c0 + (long long)p.nx * (c1 + (long long)p.ny * c2);
}

// ------------------------------------------------------------------ moments
// dn = sum_i f_i (f stored minus w_i n_ref), j = sum_i c_i f_i taken as the
// differences of opposite links first, u = j / n (the barycentric velocity
// where n is tiny).  Writes (dn, u) of every species.
template <int S>
__device__ __forceinline__ void site_moments(const mlbi_params &p, const float *__restrict__ f, long long r,
                                             float (&dn)[S], float (&u)[S][3])
{
    const long long N = p.N;
    float jx[S], jy[S], jz[S], rho = 0.f, m[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float *fa = f + (long long)a * MLBI_Q * N + r;
        float v[MLBI_Q];
#pragma unroll
        for (int i = 0; i < MLBI_Q; ++i) v[i] = __ldg(fa + i * N);
        float m0 = v[0], mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
        for (int i = 1; i < MLBI_Q; i += 2) {
            m0 += v[i] + v[i + 1];
            const float d = v[i] - v[i + 1];          // opposite links i, i + 1
            if (CX[i]) mx += CX[i] * d;
            if (CY[i]) my += CY[i] * d;
            if (CZ[i]) mz += CZ[i] * d;
        }
        dn[a] = m0;
        jx[a] = mx; jy[a] = my; jz[a] = mz;
        rho += p.nref[a] + m0;
        m[0] += mx; m[1] += my; m[2] += mz;
    }
    const float irho = rho > 0.f ? 1.f / rho : 0.f;
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float n = p.nref[a] + dn[a];
        const bool ok = n > kTinyDensity;
        const float in = ok ? 1.f / n : 0.f;
        u[a][0] = ok ? jx[a] * in : m[0] * irho;
        u[a][1] = ok ? jy[a] * in : m[1] * irho;
        u[a][2] = ok ? jz[a] * in : m[2] * irho;
    }
}

template <int S>
__global__ void __launch_bounds__(kBlock) k_moments(const mlbi_params p, const float *__restrict__ f,
                                                    float4 *__restrict__ mom)
{
    const long long N = p.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        float dn[S], u[S][3];
        site_moments<S>(p, f, r, dn, u);
#pragma unroll
        for (int a = 0; a < S; ++a) mom[a * N + r] = make_float4(dn[a], u[a][0], u[a][1], u[a][2]);
    }
}

// ------------------------------------------------------------------ site mapping of the stencil kernels
// Blocks of 32 x 4 sites (x fastest): a warp covers 32 consecutive x, so
// every stream of the structure of arrays is read in 128-byte rows.  Sites
// farther than `reach` from every face (the interior) address neighbours by
// the precomputed linear offset of each stencil entry; the others wrap or
// stop at walls through `neighbour`.
constexpr int kBX = 32, kBY = 4;

struct Loc {
    int x, y, z;
    long long r;
    bool interior;
};

__device__ __forceinline__ bool locate(const mlbi_params &p, Loc &L)
{
    L.x = blockIdx.x * kBX + threadIdx.x;
    L.y = blockIdx.y * kBY + threadIdx.y;
    L.z = blockIdx.z;
    if (L.x >= p.nx || L.y >= p.ny) return false;
    L.r = L.x + (long long)p.nx * (L.y + (long long)p.ny * L.z);
    const int R = p.reach;
    L.interior = L.x >= R && L.x < p.nx - R && L.y >= R && L.y < p.ny - R && L.z >= R && L.z < p.nz - R;
    return true;
}

// index of r + sign*d for table entry (e0, e1), or -1 beyond a wall
__device__ __forceinline__ long long nbr(const mlbi_params &p, const Loc &L, const float4 &e0, const float4 &e1,
                                         int sign)
{
    if (L.interior) return L.r + sign * (long long)__float_as_int(e1.x);
    int dx, dy, dz;
    mlbi_unpack(__float_as_int(e0.w), dx, dy, dz);
    return neighbour(p, L.x, L.y, L.z, sign * dx, sign * dy, sign * dz);
}

__host__ __device__ constexpr int pair_of(int a, int b, int S)
{
    return a <= b ? a * S - a * (a - 1) / 2 + (b - a) : b * S - b * (b - 1) / 2 + (a - b);
}

// ------------------------------------------------------------------ contact values
// g_ab(xi) - g_ab(xi_ref) of the BMCSL contact value
//   g = 1/o + 3 h xi2 / o^2 + 2 h^2 xi2^2 / o^3,   o = 1 - xi3,
// expanded exactly in the deviations d2 = xi2 - xi2_ref, d3 = xi3 - xi3_ref
// so that its FP32 value is accurate relative to the deviation itself.
__device__ __forceinline__ float bmcsl_dev(float h, float xi2r, float xi3r, float d2, float d3)
{
    float orf = 1.f - xi3r;
    float o = orf - d3;
    float xi2 = xi2r + d2;
    float o2 = o * o, or2 = orf * orf;
    float dA = d3 / (o * orf);
    float dB = 3.f * h * (d2 / o2 + xi2r * d3 * (orf + o) / (o2 * or2));
    float dC = 2.f * h * h * (d2 * (xi2 + xi2r) / (o2 * o) + xi2r * xi2r * d3 * (or2 + orf * o + o2) / (o2 * o * or2 * orf));
    return dA + dB + dC;
}

__global__ void __launch_bounds__(kBX * kBY) k_gfield(mlbi_params p, const float4 *__restrict__ mom,
                                                      const mlbi_entry *__restrict__ tab, float *__restrict__ dg,
                                                      unsigned int *__restrict__ flags)
{
    Loc L;
    if (!locate(p, L)) return;
    const long long N = p.N, r = L.r;
    float d2 = 0.f, d3 = 0.f;
    for (int c = 0; c < p.S; ++c) {
        float sum = 0.f;
        int outside = 0;
        for (int k = 0; k < p.ball_count[c]; ++k) {
            const int e = p.ball_start[c] + k;
            const long long q = nbr(p, L, __ldg(&tab[2 * e]), __ldg(&tab[2 * e + 1]), 1);
            if (q < 0) ++outside;
            else sum += mom[c * N + q].x;
        }
        // smoothed density minus n_ref; sites beyond a wall hold no particles
        const float dnbar = (sum - (float)outside * p.nref[c]) * p.ball_inv[c];
        d2 += p.xi2_coef[c] * dnbar;
        d3 += p.xi3_coef[c] * dnbar;
    }
    if (!(p.xi3_ref + d3 < 1.f)) atomicOr(flags, MLBI_FLAG_XI3);
    for (int q = 0; q < p.npairs; ++q) dg[q * N + r] = bmcsl_dev(p.pair[q].h, p.xi2_ref, p.xi3_ref, d2, d3);
}

// ------------------------------------------------------------------ centre moments
template <int S>
struct Centre {
    float n[S], dn[S], u[S][3];
};

template <int S>
__device__ __forceinline__ void load_centre(const mlbi_params &p, const float4 *__restrict__ mom, long long r,
                                            Centre<S> &c)
{
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 v = mom[a * p.N + r];
        c.dn[a] = v.x;
        c.n[a] = p.nref[a] + v.x;
        c.u[a][0] = v.y; c.u[a][1] = v.z; c.u[a][2] = v.w;
    }
}

// ------------------------------------------------------------------ moments with local contact values
// When every smoothing ball is the single site (kappa sigma < 1), g_ab at r
// depends on the moments at r only: one pass over f gives both.
template <int S>
__global__ void __launch_bounds__(kBlock) k_moments_g(const mlbi_params p, const float *__restrict__ f,
                                                      float4 *__restrict__ mom, float *__restrict__ dg,
                                                      unsigned int *__restrict__ flags)
{
    constexpr int NP = S * (S + 1) / 2;
    const long long N = p.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        float dn[S], u[S][3];
        site_moments<S>(p, f, r, dn, u);
        float d2 = 0.f, d3 = 0.f;
#pragma unroll
        for (int a = 0; a < S; ++a) {
            mom[a * N + r] = make_float4(dn[a], u[a][0], u[a][1], u[a][2]);
            d2 += p.xi2_coef[a] * dn[a];
            d3 += p.xi3_coef[a] * dn[a];
        }
        if (!(p.xi3_ref + d3 < 1.f)) atomicOr(flags, MLBI_FLAG_XI3);
#pragma unroll
        for (int q = 0; q < NP; ++q) dg[q * N + r] = bmcsl_dev(p.pair[q].h, p.xi2_ref, p.xi3_ref, d2, d3);
    }
}

// ------------------------------------------------------------------ pass 1
// Solve (I + G/2) x = b for symmetric G = (xx, yy, zz, xy, xz, yz).
__device__ __forceinline__ void solve_sym3(const float G[6], const float b[3], float x[3])
{
    float a00 = 1.f + 0.5f * G[0], a11 = 1.f + 0.5f * G[1], a22 = 1.f + 0.5f * G[2];
    float a01 = 0.5f * G[3], a02 = 0.5f * G[4], a12 = 0.5f * G[5];
    float c00 = a11 * a22 - a12 * a12;
    float c01 = a02 * a12 - a01 * a22;
    float c02 = a01 * a12 - a02 * a11;
    float c11 = a00 * a22 - a02 * a02;
    float c12 = a01 * a02 - a00 * a12;
    float c22 = a00 * a11 - a01 * a01;
    float inv = 1.f / (a00 * c00 + a01 * c01 + a02 * c02);
    x[0] = (c00 * b[0] + c01 * b[1] + c02 * b[2]) * inv;
    x[1] = (c01 * b[0] + c11 * b[1] + c12 * b[2]) * inv;
    x[2] = (c02 * b[0] + c12 * b[1] + c22 * b[2]) * inv;
}

// neighbour data of species b at r + sign*d (zero density beyond a wall)
struct Nb {
    float Dn, n, u0, u1, u2;
    long long q;
};

template <bool INTERIOR>
__device__ __forceinline__ Nb fetch_nb(const mlbi_params &p, const Loc &L, const float4 &e0, const float4 &e1,
                                       int sign, const float4 *__restrict__ fld, float nref, float dn0, float n0)
{
    Nb o;
    o.q = INTERIOR ? L.r + sign * (long long)__float_as_int(e1.x) : nbr(p, L, e0, e1, sign);
    if (INTERIOR || o.q >= 0) {
        const float4 v = fld[o.q];
        o.Dn = v.x - dn0; o.n = nref + v.x; o.u0 = v.y; o.u1 = v.z; o.u2 = v.w;
    } else {
        o.Dn = -n0; o.n = 0.f; o.u0 = 0.f; o.u1 = 0.f; o.u2 = 0.f;
    }
    return o;
}

// Shell sums of pass 1 for every species a over neighbour species b:
//   hard core  -hc_ab sum_{+-d} s (g(r)+g(r+d))/2 n^b(r+d)                   (Eq. potmeanforce)
//   exchange   vx_ab sum_{+-d} s s.[(g(r)+g(r+d))/2 n^b(r+d) (u^b(r+d) - u^a)]  (Eqs. gammaab, viscousforce)
//   friction   Gamma^a = vx_ab sum_{+-d} s s^T (g(r)+g(r+d))/2 n^b(r+d)
template <int S, bool INTERIOR>
__device__ __forceinline__ void pass1_shells(const mlbi_params &p, const Loc &L, const Centre<S> &c,
                                             const float *dgc, const float4 *__restrict__ mom,
                                             const float *__restrict__ dg, const mlbi_entry *__restrict__ tab,
                                             float (&hc)[S][3], float (&fv)[S][3], float (&G)[S][6])
{
    const long long N = p.N;
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const float n0 = c.n[b], dn0 = c.dn[b];
        const int k0 = p.ushell_start[b], k1 = k0 + p.ushell_count[b];
        const float4 *fb = mom + b * N;
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const float4 e0 = __ldg(&tab[2 * k]);
            const float4 e1 = __ldg(&tab[2 * k + 1]);
            const int mask = __float_as_int(e1.y);
            const Nb P = fetch_nb<INTERIOR>(p, L, e0, e1, 1, fb, p.nref[b], dn0, n0);
            const Nb M = fetch_nb<INTERIOR>(p, L, e0, e1, -1, fb, p.nref[b], dn0, n0);
            const float sx = e0.x, sy = e0.y, sz = e0.z;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                if (!(mask & (1 << a))) continue;
                const int q = pair_of(a, b, S);
                const mlbi_pair &pr = p.pair[q];
                const float *dgq = dg + q * N;
                const float Dgp = (INTERIOR || P.q >= 0) ? dgq[P.q] - dgc[q] : 0.f;
                const float Dgm = (INTERIOR || M.q >= 0) ? dgq[M.q] - dgc[q] : 0.f;
                const float g0 = pr.g_ref + dgc[q];
                // (g(r)+g(r+d))/2 n(r+d) - (g(r)+g(r-d))/2 n(r-d), expanded about site r
                const float t = -pr.hc_pre * (g0 * (P.Dn - M.Dn) + 0.5f * n0 * (Dgp - Dgm) +
                                              0.5f * (Dgp * P.Dn - Dgm * M.Dn));
                hc[a][0] += sx * t; hc[a][1] += sy * t; hc[a][2] += sz * t;
                const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                const float wn = gp * P.n + gm * M.n;
                float w0, w1, w2;
                if (p.drag_only) {
                    w0 = wn * (c.u[b][0] - c.u[a][0]);
                    w1 = wn * (c.u[b][1] - c.u[a][1]);
                    w2 = wn * (c.u[b][2] - c.u[a][2]);
                } else {
                    const float hp = gp * P.n, hm = gm * M.n;
                    w0 = hp * (P.u0 - c.u[a][0]) + hm * (M.u0 - c.u[a][0]);
                    w1 = hp * (P.u1 - c.u[a][1]) + hm * (M.u1 - c.u[a][1]);
                    w2 = hp * (P.u2 - c.u[a][2]) + hm * (M.u2 - c.u[a][2]);
                }
                const float sd = sx * w0 + sy * w1 + sz * w2;
                fv[a][0] += sx * sd; fv[a][1] += sy * sd; fv[a][2] += sz * sd;
                G[a][0] += wn * sx * sx; G[a][1] += wn * sy * sy; G[a][2] += wn * sz * sz;
                G[a][3] += wn * sx * sy; G[a][4] += wn * sx * sz; G[a][5] += wn * sy * sz;
            }
        }
    }
}

// attraction sum_{+d} K_ab(d) (n^b(r+d) - n^b(r-d))  (G term of Eq. potmeanforce, RPA)
template <int S, bool INTERIOR>
__device__ __forceinline__ void pass1_attraction(const mlbi_params &p, const Loc &L,
                                                 const float4 *__restrict__ mom,
                                                 const mlbi_entry *__restrict__ tab, float (&at)[S][3])
{
    const long long N = p.N;
#pragma unroll
    for (int a = 0; a < S; ++a) {
#pragma unroll
        for (int b = 0; b < S; ++b) {
            const mlbi_pair &pr = p.pair[pair_of(a, b, S)];
            const float *nb = reinterpret_cast<const float *>(mom + b * N);
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll 4
            for (int k = pr.attr_start; k < pr.attr_start + pr.attr_count; ++k) {
                const float4 e0 = __ldg(&tab[2 * k]);
                const float4 e1 = __ldg(&tab[2 * k + 1]);
                float vp, vm;
                if (INTERIOR) {
                    const long long o = __float_as_int(e1.x);
                    vp = nb[4 * (L.r + o)];
                    vm = nb[4 * (L.r - o)];
                } else {
                    const long long ip = nbr(p, L, e0, e1, 1), im = nbr(p, L, e0, e1, -1);
                    // beyond a wall n = 0, i.e. n - n_ref = -n_ref
                    vp = ip >= 0 ? nb[4 * ip] : -p.nref[b];
                    vm = im >= 0 ? nb[4 * im] : -p.nref[b];
                }
                const float d = vp - vm;        // deviations cancel n_ref exactly inside the fluid
                s0 += e0.x * d; s1 += e0.y * d; s2 += e0.z * d;
            }
            at[a][0] += s0; at[a][1] += s1; at[a][2] += s2;
        }
    }
}

// pass 1: the shell and attraction sums at u, then du from
// (I + Gamma/2) du = (rest + exchange)/2 (one Jacobi sweep of u* = u + a(u*)/2
// with partner velocities held at u) and the inputs of pass 2.
template <int S>
__global__ void __launch_bounds__(kBX * kBY) k_pass1(const mlbi_params p, const float4 *__restrict__ mom,
                                                     const float *__restrict__ dg,
                                                     const mlbi_entry *__restrict__ tab,
                                                     const float4 *__restrict__ fext, float4 *__restrict__ frest,
                                                     float4 *__restrict__ pst, float4 *__restrict__ du_out)
{
    constexpr int NP = S * (S + 1) / 2;
    Loc L;
    if (!locate(p, L)) return;
    const long long N = p.N, r = L.r;
    Centre<S> c;
    load_centre<S>(p, mom, r, c);
    float dgc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) dgc[q] = dg[q * N + r];
    float hc[S][3], fv[S][3], G[S][6], at[S][3];
#pragma unroll
    for (int a = 0; a < S; ++a) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { hc[a][k] = 0.f; fv[a][k] = 0.f; at[a][k] = 0.f; }
#pragma unroll
        for (int k = 0; k < 6; ++k) G[a][k] = 0.f;
    }
    if (L.interior) pass1_shells<S, true>(p, L, c, dgc, mom, dg, tab, hc, fv, G);
    else pass1_shells<S, false>(p, L, c, dgc, mom, dg, tab, hc, fv, G);
    if (p.has_attraction) {
        if (L.interior) pass1_attraction<S, true>(p, L, mom, tab, at);
        else pass1_attraction<S, false>(p, L, mom, tab, at);
    }
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 fe = p.has_fext ? fext[a * N + r] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float fr[3] = {hc[a][0] + at[a][0] + fe.x, hc[a][1] + at[a][1] + fe.y, hc[a][2] + at[a][2] + fe.z};
        float d[3] = {0.f, 0.f, 0.f};
        if (p.semi_implicit) {
            const float rhs[3] = {0.5f * (fr[0] + fv[a][0]), 0.5f * (fr[1] + fv[a][1]), 0.5f * (fr[2] + fv[a][2])};
            solve_sym3(G[a], rhs, d);
        }
        // pass 2 evaluates the exchange with the centre velocity u^a; -Gamma du completes it to u*
        const float gd0 = G[a][0] * d[0] + G[a][3] * d[1] + G[a][4] * d[2];
        const float gd1 = G[a][3] * d[0] + G[a][1] * d[1] + G[a][5] * d[2];
        const float gd2 = G[a][4] * d[0] + G[a][5] * d[1] + G[a][2] * d[2];
        if (p.drag_only) {
            frest[a * N + r] = make_float4(fr[0], fr[1], fr[2], 0.f);
            du_out[a * N + r] = make_float4(d[0], d[1], d[2], 0.f);
        } else {
            frest[a * N + r] = make_float4(fr[0] - gd0, fr[1] - gd1, fr[2] - gd2, 0.f);
        }
        pst[a * N + r] = make_float4(c.dn[a], c.u[a][0] + d[0], c.u[a][1] + d[1], c.u[a][2] + d[2]);
    }
}

// ------------------------------------------------------------------ pass 2: acceleration
// a^a = frest^a + vx_ab sum_{+-d} s s.[(g(r)+g(r+d))/2 n^b(r+d) (u*^b(r+d) - u^a)]
// with u* = u + du from pass 1 (drag only: partner velocity u*^b(r)).
template <int S, bool INTERIOR>
__device__ __forceinline__ void pass2_shells(const mlbi_params &p, const Loc &L, const Centre<S> &c,
                                             const float *dgc, const float (&us)[S][3],
                                             const float4 *__restrict__ pst, const float *__restrict__ dg,
                                             const mlbi_entry *__restrict__ tab, float (&acc)[S][3])
{
    const long long N = p.N;
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const int k0 = p.ushell_start[b], k1 = k0 + p.ushell_count[b];
        const float4 *fb = pst + b * N;
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const float4 e0 = __ldg(&tab[2 * k]);
            const float4 e1 = __ldg(&tab[2 * k + 1]);
            const int mask = __float_as_int(e1.y);
            const Nb P = fetch_nb<INTERIOR>(p, L, e0, e1, 1, fb, p.nref[b], 0.f, 0.f);
            const Nb M = fetch_nb<INTERIOR>(p, L, e0, e1, -1, fb, p.nref[b], 0.f, 0.f);
            const float sx = e0.x, sy = e0.y, sz = e0.z;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                if (!(mask & (1 << a))) continue;
                const int q = pair_of(a, b, S);
                const mlbi_pair &pr = p.pair[q];
                const float *dgq = dg + q * N;
                const float Dgp = (INTERIOR || P.q >= 0) ? dgq[P.q] - dgc[q] : 0.f;
                const float Dgm = (INTERIOR || M.q >= 0) ? dgq[M.q] - dgc[q] : 0.f;
                const float g0 = pr.g_ref + dgc[q];
                const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                const float wn = gp * P.n + gm * M.n;
                float w0, w1, w2;
                if (p.drag_only) {
                    w0 = wn * (us[b][0] - us[a][0]);
                    w1 = wn * (us[b][1] - us[a][1]);
                    w2 = wn * (us[b][2] - us[a][2]);
                } else {
                    const float hp = gp * P.n, hm = gm * M.n;
                    w0 = hp * (P.u0 - c.u[a][0]) + hm * (M.u0 - c.u[a][0]);
                    w1 = hp * (P.u1 - c.u[a][1]) + hm * (M.u1 - c.u[a][1]);
                    w2 = hp * (P.u2 - c.u[a][2]) + hm * (M.u2 - c.u[a][2]);
                }
                const float sd = sx * w0 + sy * w1 + sz * w2;
                acc[a][0] += sx * sd; acc[a][1] += sy * sd; acc[a][2] += sz * sd;   // masses are 1
            }
        }
    }
}

template <int S>
__global__ void __launch_bounds__(kBX * kBY) k_pass2(const mlbi_params p, const float4 *__restrict__ mom,
                                                     const float *__restrict__ dg,
                                                     const mlbi_entry *__restrict__ tab,
                                                     const float4 *__restrict__ frest,
                                                     const float4 *__restrict__ pst,
                                                     const float4 *__restrict__ du, float4 *__restrict__ acc_f,
                                                     double *__restrict__ acc_out)
{
    constexpr int NP = S * (S + 1) / 2;
    Loc L;
    if (!locate(p, L)) return;
    const long long N = p.N, r = L.r;
    Centre<S> c;
    load_centre<S>(p, mom, r, c);
    float dgc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) dgc[q] = dg[q * N + r];
    float us[S][3];                 // partner velocities at r (drag only)
#pragma unroll
    for (int a = 0; a < S; ++a) {
        if (p.drag_only) {
            const float4 v = du[a * N + r];
            us[a][0] = c.u[a][0] + v.x; us[a][1] = c.u[a][1] + v.y; us[a][2] = c.u[a][2] + v.z;
        } else {
            us[a][0] = 0.f; us[a][1] = 0.f; us[a][2] = 0.f;
        }
    }
    float acc[S][3];
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 fr = frest[a * N + r];
        acc[a][0] = fr.x; acc[a][1] = fr.y; acc[a][2] = fr.z;
    }
    if (L.interior) pass2_shells<S, true>(p, L, c, dgc, us, pst, dg, tab, acc);
    else pass2_shells<S, false>(p, L, c, dgc, us, pst, dg, tab, acc);
#pragma unroll
    for (int a = 0; a < S; ++a) {
        if (acc_out) {
#pragma unroll
            for (int q = 0; q < 3; ++q) acc_out[(a * 3 + q) * N + r] = (double)acc[a][q];
        } else {
            acc_f[a * N + r] = make_float4(acc[a][0], acc[a][1], acc[a][2], 0.f);
        }
    }
}

// The 13 canonical half offsets of the 3x3x3 cube (first non-zero of (dz, dy, dx)
// positive); with reach 1 every contact shell is a subset of them.
__device__ constexpr int KX[13] = {1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1};
__device__ constexpr int KY[13] = {0, 1, 1, 1, -1, -1, -1, 0, 0, 0, 1, 1, 1};
__device__ constexpr int KZ[13] = {0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1};

__device__ __forceinline__ float cube_inv_len(int k)
{
    const int q = KX[k] * KX[k] + KY[k] * KY[k] + KZ[k] * KZ[k];
    return q == 1 ? 1.0f : (q == 2 ? 0.70710678118654752f : 0.57735026918962576f);
}

// ------------------------------------------------------------------ shared-memory tiles (z marching)
// A block of 32 x 4 threads owns a 32 x 4 column of sites and marches up z
// through `zchunk` planes.  The stencil field of every species (float4: the
// moments in pass 1, (n - n_ref, p*) in pass 2) and the contact-value
// deviations of every pair are staged in shared memory as a ring of planes
// of (32 + 2R) x (4 + 2R) sites: 2R + 1 planes in use and one more being
// filled by cp.async while the current plane is computed.  Every shell
// neighbour is then read from shared memory.
template <int S, int R>
struct Tile {
    static constexpr int TX = kBX, TY = kBY;
    static constexpr int TXH = TX + 2 * R, TYH = TY + 2 * R, PLANE = TXH * TYH;
    static constexpr int NSLOT = 2 * R + 2;
    static constexpr int NP = S * (S + 1) / 2;
    static constexpr size_t bytes = (size_t)NSLOT * PLANE * (S * sizeof(float4) + NP * sizeof(float));
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ int wrap_or_out(int c, int L, bool wall)
{
    if (wall) return (c < 0 || c >= L) ? -1 : c;
    c %= L;
    return c < 0 ? c + L : c;
}

// Stage plane gz of the tile with corner (x0 - R, y0 - R) into ring slot `slot`.
// Sites beyond a wall get n = 0 (n - n_ref = -n_ref), zero momentum and g = g_ref.
template <int S, int R>
__device__ __forceinline__ void stage_plane(const mlbi_params &p, int x0, int y0, int gz, int slot,
                                            const float4 *__restrict__ fld, const float *__restrict__ dg,
                                            float4 *sf, float *sg)
{
    using T = Tile<S, R>;
    const long long N = p.N;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const int z = wrap_or_out(gz, p.nz, p.wall_axis == 2);
    for (int idx = tid; idx < T::PLANE; idx += kBX * kBY) {
        const int hx = idx % T::TXH, hy = idx / T::TXH;
        const int x = wrap_or_out(x0 - R + hx, p.nx, p.wall_axis == 0);
        const int y = wrap_or_out(y0 - R + hy, p.ny, p.wall_axis == 1);
        float4 *df = sf + (size_t)slot * S * T::PLANE + idx;
        float *dgs = sg + (size_t)slot * T::NP * T::PLANE + idx;
        if (x < 0 || y < 0 || z < 0) {
#pragma unroll
            for (int b = 0; b < S; ++b) df[b * T::PLANE] = make_float4(-p.nref[b], 0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < T::NP; ++q) dgs[q * T::PLANE] = 0.f;
        } else {
            const long long g = x + (long long)p.nx * (y + (long long)p.ny * z);
#pragma unroll
            for (int b = 0; b < S; ++b) cp_async16(df + b * T::PLANE, fld + b * N + g);
#pragma unroll
            for (int q = 0; q < T::NP; ++q) cp_async4(dgs + q * T::PLANE, dg + q * N + g);
        }
    }
}

// ring slot of plane z0 - R + k
__device__ __forceinline__ int ring(int k, int nslot) { return k % nslot; }

// Shell sums of pass 1 from the tile (same sums as pass1_shells).
template <int S, int R>
__device__ __forceinline__ void pass1_tile_shells(const mlbi_params &p, const mlbi_entry *__restrict__ tab,
                                                  const float4 *sf, const float *sg, int kz,
                                                  int cidx, const Centre<S> &c, const float *dgc,
                                                  float (&hc)[S][3], float (&fv)[S][3], float (&G)[S][6])
{
    using T = Tile<S, R>;
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const float n0 = c.n[b], dn0 = c.dn[b], nr = p.nref[b];
        const int k0 = p.ushell_start[b], k1 = k0 + p.ushell_count[b];
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const float4 e0 = __ldg(&tab[2 * k]);
            const float4 e1 = __ldg(&tab[2 * k + 1]);
            const int mask = __float_as_int(e1.y), off = __float_as_int(e1.z), dz = __float_as_int(e1.w);
            const int sp = ring(kz + dz, T::NSLOT), sm = ring(kz - dz, T::NSLOT);   // ring slots of the +-d planes
            const float4 vp = sf[sp * S * T::PLANE + b * T::PLANE + cidx + off];
            const float4 vm = sf[sm * S * T::PLANE + b * T::PLANE + cidx - off];
            const float Dnp = vp.x - dn0, np = nr + vp.x, Dnm = vm.x - dn0, nm = nr + vm.x;
            const float sx = e0.x, sy = e0.y, sz = e0.z;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                if (!(mask & (1 << a))) continue;
                const int q = pair_of(a, b, S);
                const mlbi_pair &pr = p.pair[q];
                const float Dgp = sg[sp * T::NP * T::PLANE + q * T::PLANE + cidx + off] - dgc[q];
                const float Dgm = sg[sm * T::NP * T::PLANE + q * T::PLANE + cidx - off] - dgc[q];
                const float g0 = pr.g_ref + dgc[q];
                const float t = -pr.hc_pre * (g0 * (Dnp - Dnm) + 0.5f * n0 * (Dgp - Dgm) +
                                              0.5f * (Dgp * Dnp - Dgm * Dnm));
                hc[a][0] += sx * t; hc[a][1] += sy * t; hc[a][2] += sz * t;
                const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                const float wn = gp * np + gm * nm;
                float w0, w1, w2;
                if (p.drag_only) {
                    w0 = wn * (c.u[b][0] - c.u[a][0]);
                    w1 = wn * (c.u[b][1] - c.u[a][1]);
                    w2 = wn * (c.u[b][2] - c.u[a][2]);
                } else {
                    const float hp = gp * np, hm = gm * nm;
                    w0 = hp * (vp.y - c.u[a][0]) + hm * (vm.y - c.u[a][0]);
                    w1 = hp * (vp.z - c.u[a][1]) + hm * (vm.z - c.u[a][1]);
                    w2 = hp * (vp.w - c.u[a][2]) + hm * (vm.w - c.u[a][2]);
                }
                const float sd = sx * w0 + sy * w1 + sz * w2;
                fv[a][0] += sx * sd; fv[a][1] += sy * sd; fv[a][2] += sz * sd;
                G[a][0] += wn * sx * sx; G[a][1] += wn * sy * sy; G[a][2] += wn * sz * sz;
                G[a][3] += wn * sx * sy; G[a][4] += wn * sx * sz; G[a][5] += wn * sy * sz;
            }
        }
    }
}

// Pass-1 shell sums for reach 1: the 13 half offsets of the 3x3x3 cube are
// compile-time constants, so the unit vectors are immediates and their zero
// components drop out; cube_mask[pair] selects the offsets of each shell.
template <int S>
__device__ __forceinline__ void pass1_cube_shells(const mlbi_params &p, const float4 *sf, const float *sg, int kz,
                                                  int cidx, const Centre<S> &c, const float *dgc,
                                                  float (&hc)[S][3], float (&fv)[S][3], float (&G)[S][6])
{
    using T = Tile<S, 1>;
    // ring slots of the planes z - 1, z, z + 1 as element offsets (32-bit)
    const int s4[3] = {ring(kz - 1, T::NSLOT) * S * T::PLANE + cidx, ring(kz, T::NSLOT) * S * T::PLANE + cidx,
                       ring(kz + 1, T::NSLOT) * S * T::PLANE + cidx};
    const int s1[3] = {ring(kz - 1, T::NSLOT) * T::NP * T::PLANE + cidx, ring(kz, T::NSLOT) * T::NP * T::PLANE + cidx,
                       ring(kz + 1, T::NSLOT) * T::NP * T::PLANE + cidx};
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const float n0 = c.n[b], dn0 = c.dn[b], nr = p.nref[b];
        int any = 0;
#pragma unroll
        for (int a = 0; a < S; ++a) any |= p.cube_mask[pair_of(a, b, S)];
#pragma unroll
        for (int k = 0; k < 13; ++k) {
            if (!((any >> k) & 1)) continue;
            const int off = KX[k] + T::TXH * KY[k];
            const float4 vp = sf[s4[1 + KZ[k]] + b * T::PLANE + off];
            const float4 vm = sf[s4[1 - KZ[k]] + b * T::PLANE - off];
            const float dDn = vp.x - vm.x, np = nr + vp.x, nm = nr + vm.x;
            const float il = cube_inv_len(k);
            const float sx = KX[k] * il, sy = KY[k] * il, sz = KZ[k] * il;
            const bool hx = KX[k] != 0, hy = KY[k] != 0, hz = KZ[k] != 0;
            // s . u at +-d, shared by every species a
            float sjp = 0.f, sjm = 0.f;
            if (hx) { sjp += sx * vp.y; sjm += sx * vm.y; }
            if (hy) { sjp += sy * vp.z; sjm += sy * vm.z; }
            if (hz) { sjp += sz * vp.w; sjm += sz * vm.w; }
#pragma unroll
            for (int a = 0; a < S; ++a) {
                const int q = pair_of(a, b, S);
                if (!((p.cube_mask[q] >> k) & 1)) continue;
                const mlbi_pair &pr = p.pair[q];
                const float Dgp = sg[s1[1 + KZ[k]] + q * T::PLANE + off] - dgc[q];
                const float Dgm = sg[s1[1 - KZ[k]] + q * T::PLANE - off] - dgc[q];
                const float g0 = pr.g_ref + dgc[q];
                // (g(r)+g(r+d))/2 n(r+d) - (g(r)+g(r-d))/2 n(r-d) = g0 (n+ - n-) + (n+ Dg+ - n- Dg-)/2
                const float t = -pr.hc_pre * (g0 * dDn + 0.5f * (np * Dgp - nm * Dgm));
                if (hx) hc[a][0] += sx * t;
                if (hy) hc[a][1] += sy * t;
                if (hz) hc[a][2] += sz * t;
                const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                const float wn = gp * np + gm * nm;
                float su = 0.f;                    // s . u^a (drag only: s . (u^b - u^a))
                if (p.drag_only) {
                    if (hx) su += sx * (c.u[a][0] - c.u[b][0]);
                    if (hy) su += sy * (c.u[a][1] - c.u[b][1]);
                    if (hz) su += sz * (c.u[a][2] - c.u[b][2]);
                } else {
                    if (hx) su += sx * c.u[a][0];
                    if (hy) su += sy * c.u[a][1];
                    if (hz) su += sz * c.u[a][2];
                }
                const float sd = p.drag_only ? -wn * su : gp * np * (sjp - su) + gm * nm * (sjm - su);
                if (hx) fv[a][0] += sx * sd;
                if (hy) fv[a][1] += sy * sd;
                if (hz) fv[a][2] += sz * sd;
                if (hx) G[a][0] += wn * (sx * sx);
                if (hy) G[a][1] += wn * (sy * sy);
                if (hz) G[a][2] += wn * (sz * sz);
                if (hx && hy) G[a][3] += wn * (sx * sy);
                if (hx && hz) G[a][4] += wn * (sx * sz);
                if (hy && hz) G[a][5] += wn * (sy * sz);
            }
        }
    }
}

// Pass-2 exchange sums for reach 1 (the cube specialisation of the table loop).
template <int S>
__device__ __forceinline__ void pass2_cube_shells(const mlbi_params &p, const float4 *sf, const float *sg, int kz,
                                                  int cidx, const Centre<S> &c, const float *dgc,
                                                  const float (&us)[S][3], float (&acc)[S][3])
{
    using T = Tile<S, 1>;
    const int s4[3] = {ring(kz - 1, T::NSLOT) * S * T::PLANE + cidx, ring(kz, T::NSLOT) * S * T::PLANE + cidx,
                       ring(kz + 1, T::NSLOT) * S * T::PLANE + cidx};
    const int s1[3] = {ring(kz - 1, T::NSLOT) * T::NP * T::PLANE + cidx, ring(kz, T::NSLOT) * T::NP * T::PLANE + cidx,
                       ring(kz + 1, T::NSLOT) * T::NP * T::PLANE + cidx};
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const float nr = p.nref[b];
        int any = 0;
#pragma unroll
        for (int a = 0; a < S; ++a) any |= p.cube_mask[pair_of(a, b, S)];
#pragma unroll
        for (int k = 0; k < 13; ++k) {
            if (!((any >> k) & 1)) continue;
            const int off = KX[k] + T::TXH * KY[k];
            const float4 vp = sf[s4[1 + KZ[k]] + b * T::PLANE + off];
            const float4 vm = sf[s4[1 - KZ[k]] + b * T::PLANE - off];
            const float np = nr + vp.x, nm = nr + vm.x;
            const float il = cube_inv_len(k);
            const float sx = KX[k] * il, sy = KY[k] * il, sz = KZ[k] * il;
            const bool hx = KX[k] != 0, hy = KY[k] != 0, hz = KZ[k] != 0;
            float sjp = 0.f, sjm = 0.f;              // s . u* at +-d, shared by every species a
            if (hx) { sjp += sx * vp.y; sjm += sx * vm.y; }
            if (hy) { sjp += sy * vp.z; sjm += sy * vm.z; }
            if (hz) { sjp += sz * vp.w; sjm += sz * vm.w; }
#pragma unroll
            for (int a = 0; a < S; ++a) {
                const int q = pair_of(a, b, S);
                if (!((p.cube_mask[q] >> k) & 1)) continue;
                const mlbi_pair &pr = p.pair[q];
                const float Dgp = sg[s1[1 + KZ[k]] + q * T::PLANE + off] - dgc[q];
                const float Dgm = sg[s1[1 - KZ[k]] + q * T::PLANE - off] - dgc[q];
                const float g0 = pr.g_ref + dgc[q];
                const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                const float wn = gp * np + gm * nm;
                float su = 0.f;                    // s . u^a (drag only: s . (u*^a - u*^b))
                if (p.drag_only) {
                    if (hx) su += sx * (us[a][0] - us[b][0]);
                    if (hy) su += sy * (us[a][1] - us[b][1]);
                    if (hz) su += sz * (us[a][2] - us[b][2]);
                } else {
                    if (hx) su += sx * c.u[a][0];
                    if (hy) su += sy * c.u[a][1];
                    if (hz) su += sz * c.u[a][2];
                }
                const float sd = p.drag_only ? -wn * su : gp * np * (sjp - su) + gm * nm * (sjm - su);
                if (hx) acc[a][0] += sx * sd;     // masses are 1
                if (hy) acc[a][1] += sy * sd;
                if (hz) acc[a][2] += sz * sd;
            }
        }
    }
}

template <int S>
__device__ __forceinline__ void centre_from(const mlbi_params &p, const float4 (&v)[S], Centre<S> &c)
{
#pragma unroll
    for (int a = 0; a < S; ++a) {
        c.dn[a] = v[a].x;
        c.n[a] = p.nref[a] + v[a].x;
        c.u[a][0] = v[a].y; c.u[a][1] = v[a].z; c.u[a][2] = v[a].w;
    }
}

// finish pass 1 at one site: predictor and outputs (shared by both pass-1 kernels)
template <int S>
__device__ __forceinline__ void pass1_finish(const mlbi_params &p, long long r, const Centre<S> &c,
                                             const float (&hc)[S][3], const float (&fv)[S][3],
                                             const float (&G)[S][6], const float (&at)[S][3],
                                             const float4 *__restrict__ fext, float4 *__restrict__ frest,
                                             float4 *__restrict__ pst, float4 *__restrict__ du_out)
{
    const long long N = p.N;
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 fe = p.has_fext ? fext[a * N + r] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float fr[3] = {hc[a][0] + at[a][0] + fe.x, hc[a][1] + at[a][1] + fe.y, hc[a][2] + at[a][2] + fe.z};
        float d[3] = {0.f, 0.f, 0.f};
        if (p.semi_implicit) {
            // one Jacobi sweep of u* = u + a(u*)/2 with partner velocities held at u
            const float rhs[3] = {0.5f * (fr[0] + fv[a][0]), 0.5f * (fr[1] + fv[a][1]), 0.5f * (fr[2] + fv[a][2])};
            solve_sym3(G[a], rhs, d);
        }
        // pass 2 evaluates the exchange with the centre velocity u^a; -Gamma du completes it to u*
        const float gd0 = G[a][0] * d[0] + G[a][3] * d[1] + G[a][4] * d[2];
        const float gd1 = G[a][3] * d[0] + G[a][1] * d[1] + G[a][5] * d[2];
        const float gd2 = G[a][4] * d[0] + G[a][5] * d[1] + G[a][2] * d[2];
        if (p.drag_only) {
            frest[a * N + r] = make_float4(fr[0], fr[1], fr[2], 0.f);
            du_out[a * N + r] = make_float4(d[0], d[1], d[2], 0.f);
        } else {
            frest[a * N + r] = make_float4(fr[0] - gd0, fr[1] - gd1, fr[2] - gd2, 0.f);
        }
        pst[a * N + r] = make_float4(c.dn[a], c.u[a][0] + d[0], c.u[a][1] + d[1], c.u[a][2] + d[2]);
    }
}

template <int S, int R>
__global__ void __launch_bounds__(kBX * kBY, 4) k_pass1_tiled(const mlbi_params p, const float4 *__restrict__ mom,
                                                              const float *__restrict__ dg,
                                                              const mlbi_entry *__restrict__ tab,
                                                              const float4 *__restrict__ fext,
                                                              float4 *__restrict__ frest, float4 *__restrict__ pst,
                                                              float4 *__restrict__ du_out)
{
    using T = Tile<S, R>;
    extern __shared__ float4 smem[];
    float4 *sf = smem;                                                      // [NSLOT][S][PLANE]
    float *sg = reinterpret_cast<float *>(smem + (size_t)T::NSLOT * S * T::PLANE);   // [NSLOT][NP][PLANE]
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY, z0 = blockIdx.z * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = x < p.nx && y < p.ny;
    const int cidx = (threadIdx.y + R) * T::TXH + threadIdx.x + R;
    for (int k = 0; k < 2 * R + 1; ++k) stage_plane<S, R>(p, x0, y0, z0 - R + k, ring(k, T::NSLOT), mom, dg, sf, sg);
    cp_async_commit();
    for (int z = z0; z < z1; ++z) {
        cp_async_wait_all();
        __syncthreads();
        const int kz = z - z0 + R;                      // ring position of plane z
        if (z + 1 < z1) {
            stage_plane<S, R>(p, x0, y0, z + R + 1, ring(kz + R + 1, T::NSLOT), mom, dg, sf, sg);
            cp_async_commit();
        }
        if (!active) continue;
        const int cs = ring(kz, T::NSLOT);
        float4 cv[S];
#pragma unroll
        for (int a = 0; a < S; ++a) cv[a] = sf[cs * S * T::PLANE + a * T::PLANE + cidx];
        Centre<S> c;
        centre_from<S>(p, cv, c);
        float dgc[T::NP];
#pragma unroll
        for (int q = 0; q < T::NP; ++q) dgc[q] = sg[cs * T::NP * T::PLANE + q * T::PLANE + cidx];
        float hc[S][3], fv[S][3], G[S][6], at[S][3];
#pragma unroll
        for (int a = 0; a < S; ++a) {
#pragma unroll
            for (int k = 0; k < 3; ++k) { hc[a][k] = 0.f; fv[a][k] = 0.f; at[a][k] = 0.f; }
#pragma unroll
            for (int k = 0; k < 6; ++k) G[a][k] = 0.f;
        }
        if constexpr (R == 1) pass1_cube_shells<S>(p, sf, sg, kz, cidx, c, dgc, hc, fv, G);
        else pass1_tile_shells<S, R>(p, tab, sf, sg, kz, cidx, c, dgc, hc, fv, G);
        const long long r = x + (long long)p.nx * (y + (long long)p.ny * z);
        if (p.has_attraction) {
            Loc L;
            L.x = x; L.y = y; L.z = z; L.r = r;
            const int Rr = p.reach;
            L.interior = x >= Rr && x < p.nx - Rr && y >= Rr && y < p.ny - Rr && z >= Rr && z < p.nz - Rr;
            if (L.interior) pass1_attraction<S, true>(p, L, mom, tab, at);
            else pass1_attraction<S, false>(p, L, mom, tab, at);
        }
        pass1_finish<S>(p, r, c, hc, fv, G, at, fext, frest, pst, du_out);
    }
}

template <int S, int R>
__global__ void __launch_bounds__(kBX * kBY, 4) k_pass2_tiled(const mlbi_params p, const float4 *__restrict__ mom,
                                                              const float *__restrict__ dg,
                                                              const mlbi_entry *__restrict__ tab,
                                                              const float4 *__restrict__ frest,
                                                              const float4 *__restrict__ pst,
                                                              const float4 *__restrict__ du,
                                                              float4 *__restrict__ acc_f, double *__restrict__ acc_out)
{
    using T = Tile<S, R>;
    extern __shared__ float4 smem[];
    float4 *sf = smem;
    float *sg = reinterpret_cast<float *>(smem + (size_t)T::NSLOT * S * T::PLANE);
    const long long N = p.N;
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY, z0 = blockIdx.z * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = x < p.nx && y < p.ny;
    const int cidx = (threadIdx.y + R) * T::TXH + threadIdx.x + R;
    for (int k = 0; k < 2 * R + 1; ++k) stage_plane<S, R>(p, x0, y0, z0 - R + k, ring(k, T::NSLOT), pst, dg, sf, sg);
    cp_async_commit();
    for (int z = z0; z < z1; ++z) {
        cp_async_wait_all();
        __syncthreads();
        const int kz = z - z0 + R;
        if (z + 1 < z1) {
            stage_plane<S, R>(p, x0, y0, z + R + 1, ring(kz + R + 1, T::NSLOT), pst, dg, sf, sg);
            cp_async_commit();
        }
        if (!active) continue;
        const int cs = ring(kz, T::NSLOT);
        const long long r = x + (long long)p.nx * (y + (long long)p.ny * z);
        Centre<S> c;
        load_centre<S>(p, mom, r, c);
        float dgc[T::NP];
#pragma unroll
        for (int q = 0; q < T::NP; ++q) dgc[q] = sg[cs * T::NP * T::PLANE + q * T::PLANE + cidx];
        float us[S][3];
#pragma unroll
        for (int a = 0; a < S; ++a) {
            if (p.drag_only) {
                const float4 v = du[a * N + r];
                us[a][0] = c.u[a][0] + v.x; us[a][1] = c.u[a][1] + v.y; us[a][2] = c.u[a][2] + v.z;
            } else {
                us[a][0] = 0.f; us[a][1] = 0.f; us[a][2] = 0.f;
            }
        }
        float acc[S][3];
#pragma unroll
        for (int a = 0; a < S; ++a) {
            const float4 fr = frest[a * N + r];
            acc[a][0] = fr.x; acc[a][1] = fr.y; acc[a][2] = fr.z;
        }
        if constexpr (R == 1) {
            pass2_cube_shells<S>(p, sf, sg, kz, cidx, c, dgc, us, acc);
        } else {
#pragma unroll
        for (int b = 0; b < S; ++b) {
            const float nr = p.nref[b];
            const int k0 = p.ushell_start[b], k1 = k0 + p.ushell_count[b];
#pragma unroll 2
            for (int k = k0; k < k1; ++k) {
                const float4 e0 = __ldg(&tab[2 * k]);
                const float4 e1 = __ldg(&tab[2 * k + 1]);
                const int mask = __float_as_int(e1.y), off = __float_as_int(e1.z), dz = __float_as_int(e1.w);
                const int sp = ring(kz + dz, T::NSLOT), sm = ring(kz - dz, T::NSLOT);
                const float4 vp = sf[sp * S * T::PLANE + b * T::PLANE + cidx + off];
                const float4 vm = sf[sm * S * T::PLANE + b * T::PLANE + cidx - off];
                const float np = nr + vp.x, nm = nr + vm.x;
                const float sx = e0.x, sy = e0.y, sz = e0.z;
#pragma unroll
                for (int a = 0; a < S; ++a) {
                    if (!(mask & (1 << a))) continue;
                    const int q = pair_of(a, b, S);
                    const mlbi_pair &pr = p.pair[q];
                    const float Dgp = sg[sp * T::NP * T::PLANE + q * T::PLANE + cidx + off] - dgc[q];
                    const float Dgm = sg[sm * T::NP * T::PLANE + q * T::PLANE + cidx - off] - dgc[q];
                    const float g0 = pr.g_ref + dgc[q];
                    const float gp = pr.vx_pre * (g0 + 0.5f * Dgp), gm = pr.vx_pre * (g0 + 0.5f * Dgm);
                    const float wn = gp * np + gm * nm;
                    float w0, w1, w2;
                    if (p.drag_only) {
                        w0 = wn * (us[b][0] - us[a][0]);
                        w1 = wn * (us[b][1] - us[a][1]);
                        w2 = wn * (us[b][2] - us[a][2]);
                    } else {
                        const float hp = gp * np, hm = gm * nm;
                        w0 = hp * (vp.y - c.u[a][0]) + hm * (vm.y - c.u[a][0]);
                        w1 = hp * (vp.z - c.u[a][1]) + hm * (vm.z - c.u[a][1]);
                        w2 = hp * (vp.w - c.u[a][2]) + hm * (vm.w - c.u[a][2]);
                    }
                    const float sd = sx * w0 + sy * w1 + sz * w2;
                    acc[a][0] += sx * sd; acc[a][1] += sy * sd; acc[a][2] += sz * sd;   // masses are 1
                }
            }
        }
        }
#pragma unroll
        for (int a = 0; a < S; ++a) {
            if (acc_out) {
#pragma unroll
                for (int q = 0; q < 3; ++q) acc_out[(a * 3 + q) * N + r] = (double)acc[a][q];
            } else {
                acc_f[a * N + r] = make_float4(acc[a][0], acc[a][1], acc[a][2], 0.f);
            }
        }
    }
}

// ------------------------------------------------------------------ collide + stream
// Collision toward psi_perp at u + a/2 (Eq. prefactor, Hermite-2) with the
// forcing of Eq. evolution scaled by (1 - omega/2), then push streaming:
// f(r + c_i) with periodic wrap by selects, or halfway bounce-back at walls.
template <int S>
__device__ __forceinline__ void collide_push(const mlbi_params &p, int x, int y, int z, long long r,
                                             const Centre<S> &c, const float (&acc)[S][3],
                                             const float *__restrict__ fin, float *__restrict__ fout)
{
    const long long N = p.N;
    const float half = p.semi_implicit ? 0.5f : 0.f;
    float ueq[S][3];
    float ub[3] = {0.f, 0.f, 0.f}, rho = 0.f;
#pragma unroll
    for (int a = 0; a < S; ++a) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            ueq[a][q] = c.u[a][q] + half * acc[a][q];
            ub[q] += c.n[a] * ueq[a][q];
        }
        rho += c.n[a];
    }
    const float irho = rho > 0.f ? 1.f / rho : 0.f;
    ub[0] *= irho; ub[1] *= irho; ub[2] *= irho;
    const float ubub = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
    const float omega = p.omega;
    const long long sy = p.nx, sz = (long long)p.nx * p.ny;
    // links that wrap around a periodic face move by -+ the extent; sites next
    // to a wall take the compact bounce-back path
    const bool wall_site = (p.wall_axis == 0 && (x == 0 || x == p.nx - 1)) ||
                           (p.wall_axis == 1 && (y == 0 || y == p.ny - 1)) ||
                           (p.wall_axis == 2 && (z == 0 || z == p.nz - 1));
    const long long wxm = x == 0 ? p.nx : 0, wxp = x == p.nx - 1 ? -(long long)p.nx : 0;
    const long long wym = y == 0 ? sz : 0, wyp = y == p.ny - 1 ? -sz : 0;
    const long long wzm = z == 0 ? N : 0, wzp = z == p.nz - 1 ? -N : 0;
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float na = c.n[a], dna = c.dn[a];
        float *oa = fout + (long long)a * MLBI_Q * N;
        const float *fa = fin + (long long)a * MLBI_Q * N + r;
        float fi[MLBI_Q];
#pragma unroll
        for (int i = 0; i < MLBI_Q; ++i) fi[i] = __ldg(fa + i * N);
        const float ua0 = ueq[a][0], ua1 = ueq[a][1], ua2 = ueq[a][2];
        const float a0 = acc[a][0], a1 = acc[a][1], a2 = acc[a][2];
        const float trM = 2.f * (ua0 * ub[0] + ua1 * ub[1] + ua2 * ub[2]) - ubub;   // tr(ua u + u ua - u u)
        const float trS = 2.f * (ub[0] * a0 + ub[1] * a1 + ub[2] * a2);             // tr(u a + a u)
        const float ks = p.src_scale * na;
        if (!wall_site) {
            // psi_perp and the forcing split into parts even and odd in c_i:
            // direction i and its opposite share the even part and flip the odd one.
            const float om1 = 1.f - omega;
            const float K1 = dna - 1.5f * na * trM;          // even part of psi at c = 0
            const float K2 = -1.5f * ks * trS;                // even part of the forcing at c = 0
            float *o = oa + r;
            o[0] = om1 * fi[0] + WQ[0] * (omega * K1 + K2);
#pragma unroll
            for (int i = 1; i < MLBI_Q; i += 2) {
                const float cu = CX[i] * ua0 + CY[i] * ua1 + CZ[i] * ua2;
                const float cb = CX[i] * ub[0] + CY[i] * ub[1] + CZ[i] * ub[2];
                const float ca = CX[i] * a0 + CY[i] * a1 + CZ[i] * a2;
                const float even = omega * (K1 + 4.5f * na * (2.f * cu * cb - cb * cb)) + (K2 + 9.f * ks * cb * ca);
                const float odd = 3.f * (omega * na * cu + ks * ca);
                long long dp = CX[i] + CY[i] * sy + CZ[i] * sz;       // i: +c, i + 1: -c
                long long dm = -dp;
                if (CX[i] > 0) { dp += wxp; dm += wxm; }
                if (CX[i] < 0) { dp += wxm; dm += wxp; }
                if (CY[i] > 0) { dp += wyp; dm += wym; }
                if (CY[i] < 0) { dp += wym; dm += wyp; }
                if (CZ[i] > 0) { dp += wzp; dm += wzm; }
                if (CZ[i] < 0) { dp += wzm; dm += wzp; }
                o[i * N + dp] = om1 * fi[i] + WQ[i] * (even + odd);
                o[(i + 1) * N + dm] = om1 * fi[i + 1] + WQ[i] * (even - odd);
            }
        } else {
#pragma unroll 1
            for (int i = 0; i < MLBI_Q; ++i) {
                const int cx = CXv(i), cy = CYv(i), cz = CZv(i);
                const float w = WQv(i);
                const float cu = cx * ua0 + cy * ua1 + cz * ua2;
                const float cb = cx * ub[0] + cy * ub[1] + cz * ub[2];
                const float ca = cx * a0 + cy * a1 + cz * a2;
                const float psi = w * (dna + na * (3.f * cu + 4.5f * (2.f * cu * cb - cb * cb) - 1.5f * trM));
                const float src = w * ks * (3.f * ca + 9.f * cb * ca - 1.5f * trS);
                const float fv = __ldg(fa + i * N);
                const float post = fv - omega * (fv - psi) + src;
                const long long q = neighbour(p, x, y, z, cx, cy, cz);
                if (q >= 0) {
                    oa[i * N + q] = post;
                } else {
                    const int ax = p.wall_axis;
                    const int cax = ax == 0 ? cx : (ax == 1 ? cy : cz);
                    const int xa = ax == 0 ? x : (ax == 1 ? y : z);
                    const float *uw = (xa + cax < 0) ? p.wall_lo : p.wall_hi;
                    const float cuw = cx * uw[0] + cy * uw[1] + cz * uw[2];
                    oa[opposite(i) * N + r] = post - 6.f * w * na * cuw;
                }
            }
        }
    }
}

template <int S>
__global__ void __launch_bounds__(kBX * kBY, 6) k_collide(const mlbi_params p, const float *__restrict__ fin,
                                                          float *__restrict__ fout, const float4 *__restrict__ mom,
                                                          const float4 *__restrict__ accf)
{
    Loc L;
    if (!locate(p, L)) return;
    const long long N = p.N, r = L.r;
    Centre<S> c;
    load_centre<S>(p, mom, r, c);
    float acc[S][3];
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 v = accf[a * N + r];
        acc[a][0] = v.x; acc[a][1] = v.y; acc[a][2] = v.z;
    }
    collide_push<S>(p, L.x, L.y, L.z, r, c, acc, fin, fout);
}

// ------------------------------------------------------------------ initial populations
__global__ void __launch_bounds__(kBlock) k_init(mlbi_params p, const double *__restrict__ nin,
                                                 const double *__restrict__ uin, float *__restrict__ f)
{
    const long long N = p.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < p.S; ++a) {
            double na = nin[a * N + r];
            rho += na;
            if (uin)
                for (int q = 0; q < 3; ++q) m[q] += na * uin[(a * 3 + q) * N + r];
        }
        float ub[3];
        for (int q = 0; q < 3; ++q) ub[q] = rho > 0.0 ? (float)(m[q] / rho) : 0.f;
        const float ubub = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
        for (int a = 0; a < p.S; ++a) {
            const double nad = nin[a * N + r];
            const float na = (float)nad;
            const float dna = (float)(nad - (double)p.nref[a]);
            float ua[3];
            for (int q = 0; q < 3; ++q) ua[q] = uin ? (float)uin[(a * 3 + q) * N + r] : 0.f;
            if (!(nad > (double)kTinyDensity)) { ua[0] = ub[0]; ua[1] = ub[1]; ua[2] = ub[2]; }
            const float trM = 2.f * (ua[0] * ub[0] + ua[1] * ub[1] + ua[2] * ub[2]) - ubub;
            float *fa = f + (long long)a * MLBI_Q * N + r;
#pragma unroll
            for (int i = 0; i < MLBI_Q; ++i) {
                const float cu = CX[i] * ua[0] + CY[i] * ua[1] + CZ[i] * ua[2];
                const float cb = CX[i] * ub[0] + CY[i] * ub[1] + CZ[i] * ub[2];
                fa[i * N] = WQ[i] * (dna + na * (3.f * cu + 4.5f * (2.f * cu * cb - cb * cb) - 1.5f * trM));
            }
        }
    }
}

// ------------------------------------------------------------------ host transfers
__global__ void __launch_bounds__(kBlock) k_export_moments(mlbi_params p, const float4 *__restrict__ mom,
                                                           double *__restrict__ nout, double *__restrict__ uout,
                                                           unsigned int *__restrict__ flags)
{
    const long long N = p.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < p.S; ++a) {
            const float4 v = mom[a * N + r];
            if (!isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w)) atomicOr(flags, MLBI_FLAG_NAN);
            if (nout) nout[a * N + r] = (double)p.nref[a] + (double)v.x;
            if (uout) {
                uout[(a * 3 + 0) * N + r] = v.y;
                uout[(a * 3 + 1) * N + r] = v.z;
                uout[(a * 3 + 2) * N + r] = v.w;
            }
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_import_fext(mlbi_params p, const double *__restrict__ fe,
                                                        float4 *__restrict__ out)
{
    const long long N = p.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x)
        for (int a = 0; a < p.S; ++a)
            out[a * N + r] = make_float4((float)fe[(a * 3 + 0) * N + r], (float)fe[(a * 3 + 1) * N + r],
                                         (float)fe[(a * 3 + 2) * N + r], 0.f);
}

// ------------------------------------------------------------------ FP64 conservation sums
// Block b sums sites r = b*256 + t, strided by the grid, in a fixed order, then
// a single block adds the block sums in order: the result is deterministic.
__global__ void __launch_bounds__(kBlock) k_conservation(mlbi_params p, const float4 *__restrict__ mom,
                                                         double *__restrict__ partial,
                                                         unsigned int *__restrict__ flags)
{
    const int W = p.S + 3;
    double acc[MLBI_MAXS + 3];
    for (int k = 0; k < W; ++k) acc[k] = 0.0;
    bool bad = false;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < p.N;
         r += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < p.S; ++a) {
            float4 v = mom[a * p.N + r];
            bad |= !isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w);
            const double n = (double)p.nref[a] + (double)v.x;
            acc[a] += (double)v.x;
            acc[p.S + 0] += n * (double)v.y;
            acc[p.S + 1] += n * (double)v.z;
            acc[p.S + 2] += n * (double)v.w;
        }
    }
    if (bad) atomicOr(flags, MLBI_FLAG_NAN);
    __shared__ double sh[kBlock];
    for (int k = 0; k < W; ++k) {
        sh[threadIdx.x] = acc[k];
        __syncthreads();
        for (int s = kBlock / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[blockIdx.x * W + k] = sh[0];
        __syncthreads();
    }
}

__global__ void k_conservation_final(mlbi_params p, const double *__restrict__ partial, int nblocks,
                                     double *__restrict__ sums)
{
    const int W = p.S + 3;
    if (threadIdx.x < W) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[b * W + threadIdx.x];
        if (threadIdx.x < p.S) s += (double)p.nref[threadIdx.x] * (double)p.N;   // mass = N n_ref + sum dn
        sums[threadIdx.x] = s;
    }
}

}  // namespace

cudaError_t mlbi_launch_moments(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s)
{
    switch (p.S) {
    case 1: k_moments<1><<<grid_for(p.N), kBlock, 0, s>>>(p, b.f[cur], b.mom); break;
    case 2: k_moments<2><<<grid_for(p.N), kBlock, 0, s>>>(p, b.f[cur], b.mom); break;
    case 3: k_moments<3><<<grid_for(p.N), kBlock, 0, s>>>(p, b.f[cur], b.mom); break;
    case 4: k_moments<4><<<grid_for(p.N), kBlock, 0, s>>>(p, b.f[cur], b.mom); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

dim3 tiled_grid(const mlbi_params &p)
{
    return dim3((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + kBY - 1) / kBY), (unsigned)p.nz);
}

cudaError_t mlbi_launch_gfield(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    k_gfield<<<tiled_grid(p), dim3(kBX, kBY), 0, s>>>(p, b.mom, b.table, b.dg, b.flags);
    return cudaGetLastError();
}

#define MLBI_DISPATCH_S(...)                                                                       \
    switch (p.S) {                                                                                 \
    case 1: { constexpr int SS = 1; __VA_ARGS__; } break;                                          \
    case 2: { constexpr int SS = 2; __VA_ARGS__; } break;                                          \
    case 3: { constexpr int SS = 3; __VA_ARGS__; } break;                                          \
    case 4: { constexpr int SS = 4; __VA_ARGS__; } break;                                          \
    default: return cudaErrorInvalidValue;                                                         \
    }

cudaError_t mlbi_launch_moments_g(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s)
{
    MLBI_DISPATCH_S((k_moments_g<SS><<<grid_for(p.N), kBlock, 0, s>>>(p, b.f[cur], b.mom, b.dg, b.flags)));
    return cudaGetLastError();
}

template <int S, int R>
cudaError_t launch_pass1_tiled(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    using T = Tile<S, R>;
    auto k = k_pass1_tiled<S, R>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::bytes);
    if (e != cudaSuccess) return e;
    const dim3 g((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + kBY - 1) / kBY),
                 (unsigned)((p.nz + p.zchunk - 1) / p.zchunk));
    k<<<g, dim3(kBX, kBY), T::bytes, s>>>(p, b.mom, b.dg, b.table, b.fext, b.frest, b.pst, b.du);
    return cudaGetLastError();
}

template <int S, int R>
cudaError_t launch_pass2_tiled(const mlbi_params &p, const mlbi_buffers &b, double *acc_out, cudaStream_t s)
{
    using T = Tile<S, R>;
    auto k = k_pass2_tiled<S, R>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::bytes);
    if (e != cudaSuccess) return e;
    const dim3 g((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + kBY - 1) / kBY),
                 (unsigned)((p.nz + p.zchunk - 1) / p.zchunk));
    k<<<g, dim3(kBX, kBY), T::bytes, s>>>(p, b.mom, b.dg, b.table, b.frest, b.pst, b.du, b.acc, acc_out);
    return cudaGetLastError();
}

cudaError_t mlbi_launch_pass1(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    if (p.tile_r == 1) { MLBI_DISPATCH_S(return launch_pass1_tiled<SS, 1>(p, b, s)); }
    if (p.tile_r == 2) { MLBI_DISPATCH_S(return launch_pass1_tiled<SS, 2>(p, b, s)); }
    const dim3 g = tiled_grid(p), t(kBX, kBY);
    MLBI_DISPATCH_S((k_pass1<SS><<<g, t, 0, s>>>(p, b.mom, b.dg, b.table, b.fext, b.frest, b.pst, b.du)));
    return cudaGetLastError();
}

cudaError_t mlbi_launch_pass2(const mlbi_params &p, const mlbi_buffers &b, double *acc_out, cudaStream_t s)
{
    if (p.tile_r == 1) { MLBI_DISPATCH_S(return launch_pass2_tiled<SS, 1>(p, b, acc_out, s)); }
    if (p.tile_r == 2) { MLBI_DISPATCH_S(return launch_pass2_tiled<SS, 2>(p, b, acc_out, s)); }
    const dim3 g = tiled_grid(p), t(kBX, kBY);
    MLBI_DISPATCH_S((k_pass2<SS><<<g, t, 0, s>>>(p, b.mom, b.dg, b.table, b.frest, b.pst, b.du, b.acc, acc_out)));
    return cudaGetLastError();
}

cudaError_t mlbi_launch_collide(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s)
{
    const dim3 g = tiled_grid(p), t(kBX, kBY);
    MLBI_DISPATCH_S((k_collide<SS><<<g, t, 0, s>>>(p, b.f[cur], b.f[cur ^ 1], b.mom, b.acc)));
    return cudaGetLastError();
}

cudaError_t mlbi_launch_init(const mlbi_params &p, const mlbi_buffers &b, int cur, const double *n,
                             const double *u, cudaStream_t s)
{
    k_init<<<grid_for(p.N), kBlock, 0, s>>>(p, n, u, b.f[cur]);
    return cudaGetLastError();
}

cudaError_t mlbi_launch_export_moments(const mlbi_params &p, const mlbi_buffers &b, double *n_out, double *u_out,
                                       cudaStream_t s)
{
    k_export_moments<<<grid_for(p.N), kBlock, 0, s>>>(p, b.mom, n_out, u_out, b.flags);
    return cudaGetLastError();
}

cudaError_t mlbi_launch_import_fext(const mlbi_params &p, const mlbi_buffers &b, const double *fext,
                                    cudaStream_t s)
{
    k_import_fext<<<grid_for(p.N), kBlock, 0, s>>>(p, fext, b.fext);
    return cudaGetLastError();
}

cudaError_t mlbi_launch_conservation(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    k_conservation<<<MLBI_RED_BLOCKS, kBlock, 0, s>>>(p, b.mom, b.partial, b.flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_conservation_final<<<1, 32, 0, s>>>(p, b.partial, MLBI_RED_BLOCKS, b.sums);
    return cudaGetLastError();
}
