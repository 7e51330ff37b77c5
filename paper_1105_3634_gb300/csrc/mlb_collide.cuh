// mlb_collide.cuh -- the moments, site-local contact values, collision and
// push streaming of one site, shared by the stand-alone kernels
// (mlb_kernels.cu) and the fused pass-2 + collision kernels (mlb_pass2.cu),
// which must agree bit for bit.  Internal header.
#pragma once

#include "mlb_internal.h"
#include "mlb_device.cuh"

namespace {

// ------------------------------------------------------------------ moments
// dn = sum_i f_i (f stored minus w_i n_ref), j = sum_i c_i f_i taken as the
// differences of opposite links first, u = j / n (the barycentric velocity
// where n is tiny), for every species.
// j: the momentum densities themselves, sum_i c_i f_i
template <int S, class Pops>
__device__ __forceinline__ void site_moments(const mlbi_params &p, const Pops &pops, float (&dn)[S], float (&u)[S][3],
                                             float (&j)[S][3])
{
    float jx[S], jy[S], jz[S], rho = 0.f, m[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < S; ++a) {
        float v[MLBI_Q];
#pragma unroll
        for (int i = 0; i < MLBI_Q; ++i) v[i] = pops(a, i);
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
        j[a][0] = jx[a]; j[a][1] = jy[a]; j[a][2] = jz[a];
        const float n = p.nref[a] + dn[a];
        const bool ok = n > kTinyDensity;
        const float in = ok ? 1.f / n : 0.f;
        u[a][0] = ok ? jx[a] * in : m[0] * irho;
        u[a][1] = ok ? jy[a] * in : m[1] * irho;
        u[a][2] = ok ? jz[a] * in : m[2] * irho;
    }
}

template <int S, class Pops>
__device__ __forceinline__ void site_moments(const mlbi_params &p, const Pops &pops, float (&dn)[S], float (&u)[S][3])
{
    float j[S][3];
    site_moments<S>(p, pops, dn, u, j);
}

// ------------------------------------------------------------------ collide + stream
// Collision toward psi_perp at u + a/2 (Eq. prefactor, Hermite-2) with the
// forcing of Eq. evolution scaled by (1 - omega/2), then push streaming:
// f(r + c_i) with periodic wrap by selects, or halfway bounce-back at walls.
// population sources: pops(a, i) = f_i^a at the site
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

// Contact values of a site whose smoothing balls are the site itself:
// dg_q = g_q(xi) - g_q(xi_ref) from the density deviations dn.  Returns
// false where xi3 >= 1.
template <int S>
__device__ __forceinline__ bool site_contact(const mlbi_params &p, const float (&dn)[S],
                                             float (&dg)[S * (S + 1) / 2])
{
    float d2 = 0.f, d3 = 0.f;
#pragma unroll
    for (int a = 0; a < S; ++a) {
        d2 += p.xi2_coef[a] * dn[a];
        d3 += p.xi3_coef[a] * dn[a];
    }
#pragma unroll
    for (int q = 0; q < S * (S + 1) / 2; ++q) dg[q] = bmcsl_dev(p.pair[q].h, p.xi2_ref, p.xi3_ref, d2, d3);
    return p.xi3_ref + d3 < 1.f;
}

struct GlobalPops {
    const float *__restrict__ f;         // f + r
    long long N;
    __device__ __forceinline__ float operator()(int a, int i) const { return __ldg(f + ((long long)a * MLBI_Q + i) * N); }
};
struct SharedPops {
    const float *f;                      // tile slot of the site, stride nt per (a, i)
    int nt;
    __device__ __forceinline__ float operator()(int a, int i) const { return f[(a * MLBI_Q + i) * nt]; }
};

template <int S, class Pops>
__device__ __forceinline__ void collide_push(const mlbi_params &p, int x, int y, int z, long long r,
                                             const Centre<S> &c, const float (&acc)[S][3], const Pops &pops,
                                             float *__restrict__ fout)
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
    // links that wrap around a periodic face move by -+ the extent; sites next
    // to a wall take the compact bounce-back path
    const bool wall_site = (p.wall_axis == 0 && (x == 0 || x == p.nx - 1)) ||
                           (p.wall_axis == 1 && (y == 0 || y == p.ny - 1)) ||
                           (p.wall_axis == 2 && (z == 0 || z == p.nz - 1));
    // target site of every moving link (32-bit: the lattice has fewer than
    // 2^31 sites), the same for every species: tgt[i - 1] for link i
    int tgt[MLBI_Q - 1];
    if (!wall_site) {
        const int sy = p.nx, sz = p.nx * p.ny, r32 = (int)r;
        const int wxm = x == 0 ? p.nx : 0, wxp = x == p.nx - 1 ? -p.nx : 0;
        const int wym = y == 0 ? sz : 0, wyp = y == p.ny - 1 ? -sz : 0;
        const int wzm = z == 0 ? (int)N : 0, wzp = z == p.nz - 1 ? -(int)N : 0;
#pragma unroll
        for (int i = 1; i < MLBI_Q; i += 2) {
            int dp = CX[i] + CY[i] * sy + CZ[i] * sz;                  // i: +c, i + 1: -c
            int dm = -dp;
            if (CX[i] > 0) { dp += wxp; dm += wxm; }
            if (CX[i] < 0) { dp += wxm; dm += wxp; }
            if (CY[i] > 0) { dp += wyp; dm += wym; }
            if (CY[i] < 0) { dp += wym; dm += wyp; }
            if (CZ[i] > 0) { dp += wzp; dm += wzm; }
            if (CZ[i] < 0) { dp += wzm; dm += wzp; }
            tgt[i - 1] = r32 + dp;
            tgt[i] = r32 + dm;
        }
    }
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float na = c.n[a], dna = c.dn[a];
        float *oa = fout + (long long)a * MLBI_Q * N;
        float fi[MLBI_Q];
#pragma unroll
        for (int i = 0; i < MLBI_Q; ++i) fi[i] = pops(a, i);
        const float ua0 = ueq[a][0], ua1 = ueq[a][1], ua2 = ueq[a][2];
        const float a0 = acc[a][0], a1 = acc[a][1], a2 = acc[a][2];
        const float trM = 2.f * (ua0 * ub[0] + ua1 * ub[1] + ua2 * ub[2]) - ubub;   // tr(ua u + u ua - u u)
        const float trS = 2.f * (ub[0] * a0 + ub[1] * a1 + ub[2] * a2);             // tr(u a + a u)
        const float ks = p.src_scale * na;
        if (!wall_site) {
            // psi_perp and the forcing split into parts even and odd in c_i:
            // direction i and its opposite share the even part and flip the odd one.
            // (Collecting the Hermite-2 terms into one quadratic form per species
            // saves arithmetic but doubles the FP32 velocity error at 500 steps
            // against the FP64 oracle: this order is kept.)
            const float om1 = 1.f - omega;
            const float K1 = dna - 1.5f * na * trM;          // even part of psi at c = 0
            const float K2 = -1.5f * ks * trS;                // even part of the forcing at c = 0
            oa[r] = om1 * fi[0] + WQ[0] * (omega * K1 + K2);
#pragma unroll
            for (int i = 1; i < MLBI_Q; i += 2) {
                const float cu = CX[i] * ua0 + CY[i] * ua1 + CZ[i] * ua2;
                const float cb = CX[i] * ub[0] + CY[i] * ub[1] + CZ[i] * ub[2];
                const float ca = CX[i] * a0 + CY[i] * a1 + CZ[i] * a2;
                const float even = omega * (K1 + 4.5f * na * (2.f * cu * cb - cb * cb)) + (K2 + 9.f * ks * cb * ca);
                const float odd = 3.f * (omega * na * cu + ks * ca);
                (oa + i * N)[tgt[i - 1]] = om1 * fi[i] + WQ[i] * (even + odd);
                (oa + (i + 1) * N)[tgt[i]] = om1 * fi[i + 1] + WQ[i] * (even - odd);
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
                const float fv = pops(a, i);
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

}  // namespace
