// mlb_kernels.cu -- sm_103a kernels of the multispecies Enskog/RPA lattice
// Boltzmann step (arXiv:1105.3634, Secs. II-III and V).
//
// Storage (structure of arrays, x fastest, site r = x + nx (y + ny z)):
//   f[a][i][r]  FP32 populations minus w_i n_ref^a      (76 B per species-site)
//   mom[a][r]   float4 (n - n_ref, j_x, j_y, j_z)        (16 B per species-site)
//   dg[p][r]    g_ab - g_ab(reference densities)          (per unordered pair)
//   frest[a][r] hard core + attraction + external force  (pass 1 -> pass 2)
//   du[a][r]    half-step velocity shift of pass 1       (pass 1 -> pass 2)
//
// One step (all launches on one stream):
//   k_moments        f -> mom                                    (Eq. colonna)
//   k_gfield         mom -> dg: smoothed densities, BMCSL g       (Sec. II smoothing)
//   k_pass1          mom, dg -> frest, du                         (Eqs. potmeanforce, gammaab,
//                    hard core + attraction + velocity exchange    viscousforce)
//                    at u, then the one-sweep half-step predictor
//   k_pass2_collide  velocity exchange at u + du, collision toward (Eqs. evolution, prefactor)
//                    psi_perp at u + a/2 with (1 - omega/2) forcing,
//                    push-streaming / halfway bounce-back
// Deviations from reference values (n - n_ref, g - g_ref) keep the FP32
// differences that the contact sums take small and exact where they cancel.
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

constexpr int kBlock = 256;
constexpr float kTinyDensity = 1e-12f;

__device__ __forceinline__ void site_coords(const mlbi_params &p, long long r, int &x, int &y, int &z)
{
    x = (int)(r % p.nx);
    long long t = r / p.nx;
    y = (int)(t % p.ny);
    z = (int)(t / p.ny);
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

struct SiteState {                 // moments of every species at one site
    float n[MLBI_MAXS];            // full density
    float dn[MLBI_MAXS];           // n - n_ref
    float u[MLBI_MAXS][3];         // species velocity (barycentric where n is tiny)
    float j[MLBI_MAXS][3];
};

__device__ __forceinline__ void load_site(const mlbi_params &p, const float4 *__restrict__ mom, long long r,
                                          SiteState &s)
{
    float rho = 0.f, m[3] = {0.f, 0.f, 0.f};
    for (int a = 0; a < p.S; ++a) {
        float4 v = mom[a * p.N + r];
        s.dn[a] = v.x;
        s.n[a] = p.nref[a] + v.x;
        s.j[a][0] = v.y; s.j[a][1] = v.z; s.j[a][2] = v.w;
        rho += s.n[a];
        m[0] += v.y; m[1] += v.z; m[2] += v.w;
    }
    float inv = rho > 0.f ? 1.f / rho : 0.f;
    for (int a = 0; a < p.S; ++a) {
        bool ok = s.n[a] > kTinyDensity;
        float in = ok ? 1.f / s.n[a] : 0.f;
        for (int k = 0; k < 3; ++k) s.u[a][k] = ok ? s.j[a][k] * in : m[k] * inv;
    }
}

// ------------------------------------------------------------------ moments
__global__ void __launch_bounds__(kBlock) k_moments(mlbi_params p, const float *__restrict__ f,
                                                    float4 *__restrict__ mom)
{
    const long long N = p.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < p.S; ++a) {
            const float *fa = f + (long long)a * MLBI_Q * N + r;
            float m0 = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
            for (int i = 0; i < MLBI_Q; ++i) {
                float v = __ldg(fa + i * N);
                m0 += v;
                if (CX[i]) mx += CX[i] * v;
                if (CY[i]) my += CY[i] * v;
                if (CZ[i]) mz += CZ[i] * v;
            }
            mom[a * N + r] = make_float4(m0, mx, my, mz);
        }
    }
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

__global__ void __launch_bounds__(kBlock) k_gfield(mlbi_params p, const float4 *__restrict__ mom,
                                                   const mlbi_entry *__restrict__ tab, float *__restrict__ dg,
                                                   unsigned int *__restrict__ flags)
{
    const long long N = p.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        site_coords(p, r, x, y, z);
        float d2 = 0.f, d3 = 0.f;
        for (int c = 0; c < p.S; ++c) {
            float sum = 0.f;
            int outside = 0;
            for (int k = 0; k < p.ball_count[c]; ++k) {
                int dx, dy, dz;
                mlbi_unpack(__float_as_int(__ldg(&tab[p.ball_start[c] + k].w)), dx, dy, dz);
                long long q = neighbour(p, x, y, z, dx, dy, dz);
                if (q < 0) ++outside;
                else sum += mom[c * N + q].x;
            }
            // smoothed density minus n_ref; sites beyond a wall hold no particles
            float dnbar = (sum - (float)outside * p.nref[c]) * p.ball_inv[c];
            d2 += p.xi2_coef[c] * dnbar;
            d3 += p.xi3_coef[c] * dnbar;
        }
        if (!(p.xi3_ref + d3 < 1.f)) atomicOr(flags, MLBI_FLAG_XI3);
        for (int q = 0; q < p.npairs; ++q)
            dg[q * N + r] = bmcsl_dev(p.pair[q].h, p.xi2_ref, p.xi3_ref, d2, d3);
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

__global__ void __launch_bounds__(kBlock) k_pass1(mlbi_params p, const float4 *__restrict__ mom,
                                                  const float *__restrict__ dg, const mlbi_entry *__restrict__ tab,
                                                  const float4 *__restrict__ fext, float4 *__restrict__ frest,
                                                  float4 *__restrict__ du)
{
    const long long N = p.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        site_coords(p, r, x, y, z);
        SiteState c;
        load_site(p, mom, r, c);
        for (int a = 0; a < p.S; ++a) {
            float hc[3] = {0.f, 0.f, 0.f}, at[3] = {0.f, 0.f, 0.f}, fv[3] = {0.f, 0.f, 0.f};
            float G[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int b = 0; b < p.S; ++b) {
                const int pi = p.pair_index[a][b];
                const mlbi_pair pr = p.pair[pi];
                const float *dgp = dg + pi * N;
                const float dg0 = dgp[r];
                const float g0 = pr.g_ref + dg0;
                const float n0 = c.n[b], dn0 = c.dn[b];
                float shc[3] = {0.f, 0.f, 0.f}, sv[3] = {0.f, 0.f, 0.f};
                float sG[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                for (int k = 0; k < pr.shell_count; ++k) {
                    const float4 e = __ldg(&tab[pr.shell_start + k]);
                    int dx, dy, dz;
                    mlbi_unpack(__float_as_int(e.w), dx, dy, dz);
                    const long long ip = neighbour(p, x, y, z, dx, dy, dz);
                    const long long im = neighbour(p, x, y, z, -dx, -dy, -dz);
                    float Dnp = -n0, Dgp = 0.f, np = 0.f, jp0 = 0.f, jp1 = 0.f, jp2 = 0.f;
                    float Dnm = -n0, Dgm = 0.f, nm = 0.f, jm0 = 0.f, jm1 = 0.f, jm2 = 0.f;
                    if (ip >= 0) {
                        float4 v = mom[b * N + ip];
                        Dnp = v.x - dn0; np = p.nref[b] + v.x; jp0 = v.y; jp1 = v.z; jp2 = v.w;
                        Dgp = dgp[ip] - dg0;
                    }
                    if (im >= 0) {
                        float4 v = mom[b * N + im];
                        Dnm = v.x - dn0; nm = p.nref[b] + v.x; jm0 = v.y; jm1 = v.z; jm2 = v.w;
                        Dgm = dgp[im] - dg0;
                    }
                    // (g(r)+g(r+d))/2 n(r+d) - (g(r)+g(r-d))/2 n(r-d), expanded about site r
                    const float t = g0 * (Dnp - Dnm) + 0.5f * n0 * (Dgp - Dgm) + 0.5f * (Dgp * Dnp - Dgm * Dnm);
                    shc[0] += e.x * t; shc[1] += e.y * t; shc[2] += e.z * t;
                    const float gp = g0 + 0.5f * Dgp, gm = g0 + 0.5f * Dgm;
                    float vp0, vp1, vp2, vm0, vm1, vm2;
                    if (p.drag_only) {
                        const float w0 = c.u[b][0] - c.u[a][0], w1 = c.u[b][1] - c.u[a][1], w2 = c.u[b][2] - c.u[a][2];
                        vp0 = np * w0; vp1 = np * w1; vp2 = np * w2;
                        vm0 = nm * w0; vm1 = nm * w1; vm2 = nm * w2;
                    } else {
                        vp0 = jp0 - np * c.u[a][0]; vp1 = jp1 - np * c.u[a][1]; vp2 = jp2 - np * c.u[a][2];
                        vm0 = jm0 - nm * c.u[a][0]; vm1 = jm1 - nm * c.u[a][1]; vm2 = jm2 - nm * c.u[a][2];
                    }
                    const float w0 = gp * vp0 + gm * vm0, w1 = gp * vp1 + gm * vm1, w2 = gp * vp2 + gm * vm2;
                    const float sd = e.x * w0 + e.y * w1 + e.z * w2;
                    sv[0] += e.x * sd; sv[1] += e.y * sd; sv[2] += e.z * sd;
                    const float wn = gp * np + gm * nm;
                    sG[0] += wn * e.x * e.x; sG[1] += wn * e.y * e.y; sG[2] += wn * e.z * e.z;
                    sG[3] += wn * e.x * e.y; sG[4] += wn * e.x * e.z; sG[5] += wn * e.y * e.z;
                }
                for (int q = 0; q < 3; ++q) {
                    hc[q] -= pr.hc_pre * shc[q];
                    fv[q] += pr.vx_pre * sv[q];
                }
                for (int q = 0; q < 6; ++q) G[q] += pr.vx_pre * sG[q];
                if (pr.attr_count > 0) {
                    float sa[3] = {0.f, 0.f, 0.f};
                    for (int k = 0; k < pr.attr_count; ++k) {
                        const float4 e = __ldg(&tab[pr.attr_start + k]);
                        int dx, dy, dz;
                        mlbi_unpack(__float_as_int(e.w), dx, dy, dz);
                        const long long ip = neighbour(p, x, y, z, dx, dy, dz);
                        const long long im = neighbour(p, x, y, z, -dx, -dy, -dz);
                        // n(r+d) - n(r-d): deviations cancel n_ref exactly inside the fluid
                        const float np = ip >= 0 ? mom[b * N + ip].x : -p.nref[b];
                        const float nm = im >= 0 ? mom[b * N + im].x : -p.nref[b];
                        const float dn = np - nm;
                        sa[0] += e.x * dn; sa[1] += e.y * dn; sa[2] += e.z * dn;
                    }
                    for (int q = 0; q < 3; ++q) at[q] += sa[q];
                }
            }
            float fr[3];
            float4 fe = p.has_fext ? fext[a * N + r] : make_float4(0.f, 0.f, 0.f, 0.f);
            fr[0] = hc[0] + at[0] + fe.x;
            fr[1] = hc[1] + at[1] + fe.y;
            fr[2] = hc[2] + at[2] + fe.z;
            frest[a * N + r] = make_float4(fr[0], fr[1], fr[2], 0.f);
            float s[3] = {0.f, 0.f, 0.f};
            if (p.semi_implicit) {
                // one Jacobi sweep of u* = u + a(u*)/2 with partner velocities held at u
                const float rhs[3] = {0.5f * (fr[0] + fv[0]), 0.5f * (fr[1] + fv[1]), 0.5f * (fr[2] + fv[2])};
                solve_sym3(G, rhs, s);
            }
            du[a * N + r] = make_float4(s[0], s[1], s[2], 0.f);
        }
    }
}

// ------------------------------------------------------------------ pass 2 + collide + stream
__global__ void __launch_bounds__(kBlock) k_pass2_collide(mlbi_params p, const float *__restrict__ fin,
                                                          float *__restrict__ fout, const float4 *__restrict__ mom,
                                                          const float *__restrict__ dg,
                                                          const mlbi_entry *__restrict__ tab,
                                                          const float4 *__restrict__ frest,
                                                          const float4 *__restrict__ du, double *__restrict__ acc_out)
{
    const long long N = p.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        site_coords(p, r, x, y, z);
        SiteState c;
        load_site(p, mom, r, c);
        float acc[MLBI_MAXS][3];
        float duc[MLBI_MAXS][3];
        for (int a = 0; a < p.S; ++a) {
            float4 v = du[a * N + r];
            duc[a][0] = v.x; duc[a][1] = v.y; duc[a][2] = v.z;
        }
        for (int a = 0; a < p.S; ++a) {
            float4 fr = frest[a * N + r];
            float fv[3] = {0.f, 0.f, 0.f};
            for (int b = 0; b < p.S; ++b) {
                const int pi = p.pair_index[a][b];
                const mlbi_pair pr = p.pair[pi];
                const float *dgp = dg + pi * N;
                const float dg0 = dgp[r];
                const float g0 = pr.g_ref + dg0;
                float sv[3] = {0.f, 0.f, 0.f};
                for (int k = 0; k < pr.shell_count; ++k) {
                    const float4 e = __ldg(&tab[pr.shell_start + k]);
                    int dx, dy, dz;
                    mlbi_unpack(__float_as_int(e.w), dx, dy, dz);
                    const long long ip = neighbour(p, x, y, z, dx, dy, dz);
                    const long long im = neighbour(p, x, y, z, -dx, -dy, -dz);
                    float w0 = 0.f, w1 = 0.f, w2 = 0.f;
                    if (ip >= 0) {
                        const float4 v = mom[b * N + ip];
                        const float np = p.nref[b] + v.x;
                        const float gp = g0 + 0.5f * (dgp[ip] - dg0);
                        float v0, v1, v2;
                        if (p.drag_only) {
                            v0 = np * (c.u[b][0] + duc[b][0] - c.u[a][0] - duc[a][0]);
                            v1 = np * (c.u[b][1] + duc[b][1] - c.u[a][1] - duc[a][1]);
                            v2 = np * (c.u[b][2] + duc[b][2] - c.u[a][2] - duc[a][2]);
                        } else {
                            const float4 d = du[b * N + ip];
                            v0 = (v.y - np * c.u[a][0]) + np * (d.x - duc[a][0]);
                            v1 = (v.z - np * c.u[a][1]) + np * (d.y - duc[a][1]);
                            v2 = (v.w - np * c.u[a][2]) + np * (d.z - duc[a][2]);
                        }
                        w0 += gp * v0; w1 += gp * v1; w2 += gp * v2;
                    }
                    if (im >= 0) {
                        const float4 v = mom[b * N + im];
                        const float nm = p.nref[b] + v.x;
                        const float gm = g0 + 0.5f * (dgp[im] - dg0);
                        float v0, v1, v2;
                        if (p.drag_only) {
                            v0 = nm * (c.u[b][0] + duc[b][0] - c.u[a][0] - duc[a][0]);
                            v1 = nm * (c.u[b][1] + duc[b][1] - c.u[a][1] - duc[a][1]);
                            v2 = nm * (c.u[b][2] + duc[b][2] - c.u[a][2] - duc[a][2]);
                        } else {
                            const float4 d = du[b * N + im];
                            v0 = (v.y - nm * c.u[a][0]) + nm * (d.x - duc[a][0]);
                            v1 = (v.z - nm * c.u[a][1]) + nm * (d.y - duc[a][1]);
                            v2 = (v.w - nm * c.u[a][2]) + nm * (d.z - duc[a][2]);
                        }
                        w0 += gm * v0; w1 += gm * v1; w2 += gm * v2;
                    }
                    const float sd = e.x * w0 + e.y * w1 + e.z * w2;
                    sv[0] += e.x * sd; sv[1] += e.y * sd; sv[2] += e.z * sd;
                }
                for (int q = 0; q < 3; ++q) fv[q] += pr.vx_pre * sv[q];
            }
            acc[a][0] = fr.x + fv[0];     // masses are 1
            acc[a][1] = fr.y + fv[1];
            acc[a][2] = fr.z + fv[2];
        }
        if (acc_out) {
            for (int a = 0; a < p.S; ++a)
                for (int q = 0; q < 3; ++q) acc_out[(a * 3 + q) * N + r] = (double)acc[a][q];
            continue;
        }

        // velocities of the equilibrium: u^a + a^a/2 (semi-implicit) or u^a, and their barycentre
        const float half = p.semi_implicit ? 0.5f : 0.f;
        float ueq[MLBI_MAXS][3];
        float ub[3] = {0.f, 0.f, 0.f}, rho = 0.f;
        for (int a = 0; a < p.S; ++a) {
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

        for (int a = 0; a < p.S; ++a) {
            const float na = c.n[a], dna = c.dn[a];
            const float *fa = fin + (long long)a * MLBI_Q * N + r;
            float *oa = fout + (long long)a * MLBI_Q * N;
            const float ua0 = ueq[a][0], ua1 = ueq[a][1], ua2 = ueq[a][2];
            const float a0 = acc[a][0], a1 = acc[a][1], a2 = acc[a][2];
            const float trM = 2.f * (ua0 * ub[0] + ua1 * ub[1] + ua2 * ub[2]) - ubub;   // tr(ua u + u ua - u u)
            const float trS = 2.f * (ub[0] * a0 + ub[1] * a1 + ub[2] * a2);             // tr(u a + a u)
            const float ks = p.src_scale * na;
#pragma unroll
            for (int i = 0; i < MLBI_Q; ++i) {
                const float cu = CX[i] * ua0 + CY[i] * ua1 + CZ[i] * ua2;
                const float cb = CX[i] * ub[0] + CY[i] * ub[1] + CZ[i] * ub[2];
                const float ca = CX[i] * a0 + CY[i] * a1 + CZ[i] * a2;
                // psi_perp - w n_ref  (1/cs2 = 3, 1/(2 cs4) = 4.5, 1/(2 cs2) = 1.5)
                const float psi = WQ[i] * (dna + na * (3.f * cu + 4.5f * (2.f * cu * cb - cb * cb) - 1.5f * trM));
                const float src = WQ[i] * ks * (3.f * ca + 9.f * cb * ca - 1.5f * trS);
                const float fi = __ldg(fa + i * N);
                const float post = fi - omega * (fi - psi) + src;
                const long long q = neighbour(p, x, y, z, CX[i], CY[i], CZ[i]);
                if (q >= 0) {
                    oa[i * N + q] = post;
                } else {
                    const int ax = p.wall_axis;
                    const int cax = ax == 0 ? CX[i] : (ax == 1 ? CY[i] : CZ[i]);
                    const int xa = ax == 0 ? x : (ax == 1 ? y : z);
                    const float *uw = (xa + cax < 0) ? p.wall_lo : p.wall_hi;
                    const float cuw = CX[i] * uw[0] + CY[i] * uw[1] + CZ[i] * uw[2];
                    oa[opposite(i) * N + r] = post - 6.f * WQ[i] * na * cuw;
                }
            }
        }
    }
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
        double n[MLBI_MAXS], j[MLBI_MAXS][3], rho = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < p.S; ++a) {
            float4 v = mom[a * N + r];
            if (!isfinite(v.x) || !isfinite(v.y) || !isfinite(v.z) || !isfinite(v.w)) atomicOr(flags, MLBI_FLAG_NAN);
            n[a] = (double)p.nref[a] + (double)v.x;
            j[a][0] = v.y; j[a][1] = v.z; j[a][2] = v.w;
            rho += n[a];
            for (int q = 0; q < 3; ++q) m[q] += j[a][q];
        }
        for (int a = 0; a < p.S; ++a) {
            if (nout) nout[a * N + r] = n[a];
            if (uout) {
                const bool ok = n[a] > (double)kTinyDensity;
                for (int q = 0; q < 3; ++q)
                    uout[(a * 3 + q) * N + r] = ok ? j[a][q] / n[a] : (rho > 0.0 ? m[q] / rho : 0.0);
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
            acc[a] += (double)v.x;
            acc[p.S + 0] += (double)v.y;
            acc[p.S + 1] += (double)v.z;
            acc[p.S + 2] += (double)v.w;
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

inline unsigned grid_for(long long N)
{
    long long g = (N + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    if (g > (1ll << 30)) g = 1ll << 30;
    return (unsigned)g;
}

}  // namespace

cudaError_t mlbi_launch_moments(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s)
{
    k_moments<<<grid_for(p.N), kBlock, 0, s>>>(p, b.f[cur], b.mom);
    return cudaGetLastError();
}

cudaError_t mlbi_launch_gfield(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    k_gfield<<<grid_for(p.N), kBlock, 0, s>>>(p, b.mom, b.table, b.dg, b.flags);
    return cudaGetLastError();
}

cudaError_t mlbi_launch_pass1(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    k_pass1<<<grid_for(p.N), kBlock, 0, s>>>(p, b.mom, b.dg, b.table, b.fext, b.frest, b.du);
    return cudaGetLastError();
}

cudaError_t mlbi_launch_pass2_collide(const mlbi_params &p, const mlbi_buffers &b, int cur, double *acc_out,
                                      cudaStream_t s)
{
    k_pass2_collide<<<grid_for(p.N), kBlock, 0, s>>>(p, b.f[cur], b.f[cur ^ 1], b.mom, b.dg, b.table, b.frest,
                                                     b.du, acc_out);
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
