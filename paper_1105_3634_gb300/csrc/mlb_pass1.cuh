// mlb_pass1.cuh -- device code of pass 1 of a time step on sm_103a: the
// hard-core force (Eq. potmeanforce), the velocity exchange (Eqs. gammaab,
// viscousforce) at u, the friction matrix Gamma^a, the attraction read-in,
// and the half-step predictor du of the semi-implicit forcing.  Three
// variants of the shell sums: global-memory (any reach), shared-memory tile
// with the stencil table (reach 2, 3), and the compile-time 3x3x3 cube
// (reach 1).  The kernels come in three modes:
//   kExact      the method's pass 1 (mlb_pass1.cu)
//   kSurrogate  F^hc taken from attr (the learned surrogate's), no hard-core sums
//   kSweep      a further Jacobi sweep of the half step u* = u + a(u*)/2: the
//               staged field holds the previous sweep's (n - n_ref, u*), the
//               centre keeps its own u (from the moments), the rest force comes
//               from frest; only the exchange and Gamma are summed (mlb_sweep.cu)
// Internal header: each including unit instantiates the kernels it launches.
#pragma once

#include "mlb_passes.cuh"

namespace {

constexpr int kExact = 0, kSurrogate = 1, kSweep = 2;

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

// per species: hf[q] = (F^hc_q, F^v_q), G = friction matrix packed as
// (xx, yy), (zz, xy), (xz, yz) (see add_pass1), at = attraction
template <int S>
struct Acc1 {
    float2 hf[S][3], G[S][3];
    float at[S][3];
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int a = 0; a < S; ++a) {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                hf[a][k] = make_float2(0.f, 0.f);
                G[a][k] = make_float2(0.f, 0.f);
                at[a][k] = 0.f;
            }
        }
    }
};

// Shell sums from global memory, for every species a over neighbour species b:
//   hard core  -hc_ab sum_{+-d} s (g(r)+g(r+d))/2 n^b(r+d)                          (Eq. potmeanforce)
//   exchange   vx_ab sum_{+-d} s s.[(g(r)+g(r+d))/2 n^b(r+d) (u^b(r+d) - u^a(r))]  (Eqs. gammaab, viscousforce)
//   friction   Gamma^a = vx_ab sum_{+-d} s s^T (g(r)+g(r+d))/2 n^b(r+d)
template <int S, bool DRAG, bool INTERIOR, bool HC>
__device__ __forceinline__ void pass1_shells(const mlbi_params &p, const Loc &L, const Centre<S> &c,
                                             const float (&ub)[S][3], const PairW<S> &w,
                                             const float4 *__restrict__ mom, const float *__restrict__ dg,
                                             const mlbi_entry *__restrict__ tab, Acc1<S> &A)
{
    const long long N = p.N;
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const int k0 = p.ushell_start[b], k1 = k0 + p.ushell_count[b];
        const float4 *fb = mom + b * N;
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const float4 e0 = __ldg(&tab[2 * k]);
            const float4 e1 = __ldg(&tab[2 * k + 1]);
            const int mask = __float_as_int(e1.y);
            const Nb P = fetch_nb<INTERIOR>(p, L, e0, e1, 1, fb, p.nref[b]);
            const Nb M = fetch_nb<INTERIOR>(p, L, e0, e1, -1, fb, p.nref[b]);
            const float sx = e0.x, sy = e0.y, sz = e0.z;
            const float jp = DRAG ? 0.f : sx * P.u0 + sy * P.u1 + sz * P.u2;
            const float jm = DRAG ? 0.f : sx * M.u0 + sy * M.u1 + sz * M.u2;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                if (!(mask & (1 << a))) continue;
                const int q = pair_of(a, b, S);
                const float su = DRAG ? 0.f : sx * c.u[a][0] + sy * c.u[a][1] + sz * c.u[a][2];
                const float *dgq = dg + q * N;
                const float dgp = (INTERIOR || P.q >= 0) ? dgq[P.q] : 0.f;
                const float dgm = (INTERIOR || M.q >= 0) ? dgq[M.q] : 0.f;
                const float sdu = DRAG ? sx * (c.u[a][0] - ub[b][0]) + sy * (c.u[a][1] - ub[b][1]) +
                                             sz * (c.u[a][2] - ub[b][2])
                                       : 0.f;
                float t, sd, wn;
                pass1_point<DRAG>(P.n, M.n, P.dn - M.dn, jp - su, jm - su, dgp, dgm, w.kp[q], 0.5f * p.pair[q].vx_pre, w.h[q],
                                  -0.5f * p.pair[q].hc_pre, sdu, t, sd, wn);
                add_pass1(sx, sy, sz, HC ? t : 0.f, sd, wn, A.hf[a], A.G[a]);
            }
        }
    }
}

// attraction sum_{+d} K_ab(d) (n^b(r+d) - n^b(r-d)) from global memory (G term
// of Eq. potmeanforce, RPA), for reaches the column kernel does not serve
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

// Finish pass 1 at one site.  rest = F^hc + G + F_ext and the exchange at u
// (the shell sums of sd) give the predictor du from (I + Gamma/2) du =
// (rest + exchange)/2: one Jacobi sweep of u* = u + a(u*)/2 with partner
// velocities held at u.  Outputs for pass 2: frest = rest, pst = (n - n_ref,
// u* = u + du).
template <int S, bool DRAG>
__device__ __forceinline__ void pass1_finish(const mlbi_params &p, long long r, const Centre<S> &c, const Acc1<S> &A,
                                             const float4 *__restrict__ fext, float4 *__restrict__ frest,
                                             float4 *__restrict__ pst)
{
    const long long N = p.N;
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 fe = p.has_fext ? fext[a * N + r] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float fr[3] = {A.hf[a][0].x + A.at[a][0] + fe.x, A.hf[a][1].x + A.at[a][1] + fe.y,
                             A.hf[a][2].x + A.at[a][2] + fe.z};
        float d[3] = {0.f, 0.f, 0.f};
        if (p.semi_implicit) {
            const float rhs[3] = {0.5f * (fr[0] + A.hf[a][0].y), 0.5f * (fr[1] + A.hf[a][1].y),
                                  0.5f * (fr[2] + A.hf[a][2].y)};
            const float G[6] = {A.G[a][0].x, A.G[a][0].y, A.G[a][1].x, A.G[a][1].y, A.G[a][2].x, A.G[a][2].y};
            solve_sym3(G, rhs, d);
        }
        frest[a * N + r] = make_float4(fr[0], fr[1], fr[2], 0.f);
        pst[a * N + r] = make_float4(c.dn[a], c.u[a][0] + d[0], c.u[a][1] + d[1], c.u[a][2] + d[2]);
    }
}

// Finish a further sweep at one site: rest = frest (pass 1's), the exchange
// with the partners at the previous sweep's u*, the same Gamma; pst_out =
// (n - n_ref, u + du).
template <int S>
__device__ __forceinline__ void sweep_finish(const mlbi_params &p, long long r, const Centre<S> &c, const Acc1<S> &A,
                                             const float4 *__restrict__ frest, float4 *__restrict__ pst_out)
{
    const long long N = p.N;
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 fr = frest[a * N + r];
        const float rhs[3] = {0.5f * (fr.x + A.hf[a][0].y), 0.5f * (fr.y + A.hf[a][1].y),
                              0.5f * (fr.z + A.hf[a][2].y)};
        const float G[6] = {A.G[a][0].x, A.G[a][0].y, A.G[a][1].x, A.G[a][1].y, A.G[a][2].x, A.G[a][2].y};
        float d[3];
        solve_sym3(G, rhs, d);
        pst_out[a * N + r] = make_float4(c.dn[a], c.u[a][0] + d[0], c.u[a][1] + d[1], c.u[a][2] + d[2]);
    }
}

// the centre of a site: densities from the staged field; velocities from it
// too, except in a sweep, where the centre keeps its own u (mom_c) and the
// staged u* of the previous sweep is the partners' (ub, used by drag only)
template <int S, int MODE>
__device__ __forceinline__ void centre_of(const mlbi_params &p, const float4 (&cv)[S], const float4 *__restrict__ mom_c,
                                          long long r, Centre<S> &c, float (&ub)[S][3])
{
#pragma unroll
    for (int a = 0; a < S; ++a) {
        c.dn[a] = cv[a].x;
        c.n[a] = p.nref[a] + cv[a].x;
        ub[a][0] = cv[a].y; ub[a][1] = cv[a].z; ub[a][2] = cv[a].w;
        if constexpr (MODE == kSweep) {
            const float4 m = mom_c[a * p.N + r];
            c.u[a][0] = m.y; c.u[a][1] = m.z; c.u[a][2] = m.w;
        } else {
            c.u[a][0] = cv[a].y; c.u[a][1] = cv[a].z; c.u[a][2] = cv[a].w;
        }
    }
}

template <int S, bool DRAG, int MODE>
__global__ void __launch_bounds__(kBX * kBY) k_pass1(const mlbi_params p, const float4 *__restrict__ mom,
                                                     const float *__restrict__ dg,
                                                     const mlbi_entry *__restrict__ tab,
                                                     const float4 *__restrict__ fext,
                                                     const float4 *__restrict__ attr,
                                                     const float4 *__restrict__ mom_c, float4 *__restrict__ frest,
                                                     float4 *__restrict__ pst)
{
    constexpr int NP = S * (S + 1) / 2;
    Loc L;
    if (!locate(p, L)) return;
    const long long N = p.N, r = L.r;
    Centre<S> c;
    float ub[S][3];
    {
        float4 cv[S];
#pragma unroll
        for (int a = 0; a < S; ++a) cv[a] = mom[a * N + r];
        centre_of<S, MODE>(p, cv, mom_c, r, c, ub);
    }
    float dgc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) dgc[q] = dg[q * N + r];
    PairW<S> w;
    pair_weights<S>(p, dgc, w);
    Acc1<S> A;
    A.zero();
    constexpr bool HC = MODE == kExact;
    if (L.interior) pass1_shells<S, DRAG, true, HC>(p, L, c, ub, w, mom, dg, tab, A);
    else pass1_shells<S, DRAG, false, HC>(p, L, c, ub, w, mom, dg, tab, A);
    if constexpr (MODE == kSweep) {
        sweep_finish<S>(p, r, c, A, frest, pst);
        return;
    }
    if (MODE == kSurrogate || p.attr_r) {
#pragma unroll
        for (int a = 0; a < S; ++a) {
            const float4 v = attr[a * N + r];
            A.at[a][0] = v.x; A.at[a][1] = v.y; A.at[a][2] = v.z;
        }
    } else if (p.has_attraction) {
        if (L.interior) pass1_attraction<S, true>(p, L, mom, tab, A.at);
        else pass1_attraction<S, false>(p, L, mom, tab, A.at);
    }
    pass1_finish<S, DRAG>(p, r, c, A, fext, frest, pst);
}

// ------------------------------------------------------------------ tiled variants
// Shell sums from the tile with the stencil table (same sums as pass1_shells).
template <int S, int R, bool DRAG, int TY, bool HC>
__device__ __forceinline__ void pass1_tile_shells(const mlbi_params &p, const mlbi_entry *tab,
                                                  const float4 *sf, const float *sg, int kz, int cidx,
                                                  const Centre<S> &c, const float (&ub)[S][3], const PairW<S> &w,
                                                  Acc1<S> &A)
{
    using T = Tile<S, R, TY>;
#pragma unroll
    for (int b = 0; b < S; ++b) {
        const float nr = p.nref[b];
        const int k0 = p.ushell_start[b], k1 = k0 + p.ushell_count[b];
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const float4 e0 = tab[2 * k];                   // global or shared (stage_table)
            const float4 e1 = tab[2 * k + 1];
            const int mask = __float_as_int(e1.y), off = __float_as_int(e1.z), dz = __float_as_int(e1.w);
            const int sp = ring(kz + dz, T::NSLOT), sm = ring(kz - dz, T::NSLOT);   // ring slots of the +-d planes
            const float4 vp = sf[sp * S * T::PLANE + b * T::PLANE + cidx + off];
            const float4 vm = sf[sm * S * T::PLANE + b * T::PLANE + cidx - off];
            const float np = nr + vp.x, nm = nr + vm.x, dd = vp.x - vm.x;
            const float sx = e0.x, sy = e0.y, sz = e0.z;
            const float jp = DRAG ? 0.f : sx * vp.y + sy * vp.z + sz * vp.w;
            const float jm = DRAG ? 0.f : sx * vm.y + sy * vm.z + sz * vm.w;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                if (!(mask & (1 << a))) continue;
                const int q = pair_of(a, b, S);
                const float su = DRAG ? 0.f : sx * c.u[a][0] + sy * c.u[a][1] + sz * c.u[a][2];
                const float dgp = sg[sp * T::NP * T::PLANE + q * T::PLANE + cidx + off];
                const float dgm = sg[sm * T::NP * T::PLANE + q * T::PLANE + cidx - off];
                const float sdu = DRAG ? sx * (c.u[a][0] - ub[b][0]) + sy * (c.u[a][1] - ub[b][1]) +
                                             sz * (c.u[a][2] - ub[b][2])
                                       : 0.f;
                float t, sd, wn;
                pass1_point<DRAG>(np, nm, dd, jp - su, jm - su, dgp, dgm, w.kp[q], 0.5f * p.pair[q].vx_pre, w.h[q],
                                  -0.5f * p.pair[q].hc_pre, sdu, t, sd, wn);
                add_pass1(sx, sy, sz, HC ? t : 0.f, sd, wn, A.hf[a], A.G[a]);
            }
        }
    }
}

// Shell sums for reach 1 by offset class (axis, face, corner): the offsets
// and unit vectors are compile-time constants and cube_mask selects the
// classes of each pair's shell.  The +-d data of a class is read once per
// neighbour species and shared by every species a.  f[3], g[3]: element
// offsets of the planes z - 1, z, z + 1 of the float4 and dg tiles.
template <int S, bool DRAG, int CL, bool HC>
__device__ __forceinline__ void pass1_cube_class(const mlbi_params &p, const float4 *sf, const float *sg, int b,
                                                 const int (&f)[3], const int (&g)[3], const Centre<S> &c, const float (&ub)[S][3],
                                                 const PairW<S> &w, Acc1<S> &A)
{
    using T = Tile<S, 1>;
    constexpr float il = cls_il(CL);
    bool has[S];
    bool any = false;
#pragma unroll
    for (int a = 0; a < S; ++a) {
        has[a] = (p.cube_mask[pair_of(a, b, S)] >> cls_bit(CL)) & 1;
        any |= has[a];
    }
    if (!any) return;
    const float nr = p.nref[b];
    static_for<0, cls_n(CL)>([&](auto I) {
        constexpr int k = cls_k(CL, decltype(I)::value);
        constexpr int off = cube_kx(k) + T::TXH * cube_ky(k), dz = cube_kz(k);
        const float4 vp = sf[f[1 + dz] + b * T::PLANE + off];
        const float4 vm = sf[f[1 - dz] + b * T::PLANE - off];
        // the arithmetic of pass1_point with the +d and -d lanes packed
        const float2 npm = add2(f2(nr, nr), f2(vp.x, vm.x));            // (n(r+d), n(r-d))
        const float dd = vp.x - vm.x;
        float2 jpm = f2(0.f, 0.f);                                          // s.u^b(r +- d)
        if constexpr (!DRAG) {
            if constexpr (cube_kx(k) != 0) jpm = fma2(f2(cube_kx(k) * il, cube_kx(k) * il), f2(vp.y, vm.y), jpm);
            if constexpr (cube_ky(k) != 0) jpm = fma2(f2(cube_ky(k) * il, cube_ky(k) * il), f2(vp.z, vm.z), jpm);
            if constexpr (cube_kz(k) != 0) jpm = fma2(f2(cube_kz(k) * il, cube_kz(k) * il), f2(vp.w, vm.w), jpm);
        }
#pragma unroll
        for (int a = 0; a < S; ++a) {
            if (!has[a]) continue;
            const int q = pair_of(a, b, S);
            const float2 dg2 = f2(sg[g[1 + dz] + q * T::PLANE + off], sg[g[1 - dz] + q * T::PLANE - off]);
            const float k1 = 0.5f * p.pair[q].vx_pre;
            const float2 gpm = fma2(f2(k1, k1), dg2, f2(w.kp[q], w.kp[q]));   // exchange weights at r +- d
            const float2 hpm = mul2(gpm, npm);
            const float wn = hpm.x + hpm.y;
            float sd;
            if constexpr (DRAG) {
                const float sdu = cube_dot<k>(il, c.u[a][0] - ub[b][0], c.u[a][1] - ub[b][1], c.u[a][2] - ub[b][2]);
                sd = -wn * sdu;
            } else {
                const float su = cube_dot<k>(il, c.u[a][0], c.u[a][1], c.u[a][2]);
                const float2 j2 = add2(jpm, f2(-su, -su));                   // s.(u^b(r +- d) - u^a(r))
                sd = fmaf(hpm.x, j2.x, hpm.y * j2.y);
            }
            const float t = HC ? fmaf(w.h[q], dd, (-0.5f * p.pair[q].hc_pre) * fmaf(npm.x, dg2.x, -npm.y * dg2.y))
                               : 0.f;
            cube_add2<k>(il, f2(t, sd), A.hf[a]);
            cube_add_ss<k>(il, wn, A.G[a]);
        }
    });
}

template <int S, bool DRAG, bool HC>
__device__ __forceinline__ void pass1_cube(const mlbi_params &p, const float4 *sf, const float *sg, int kz, int cidx,
                                           const Centre<S> &c, const float (&ub)[S][3], const PairW<S> &w,
                                           Acc1<S> &A)
{
    using T = Tile<S, 1>;
    const int f[3] = {ring(kz - 1, T::NSLOT) * S * T::PLANE + cidx, ring(kz, T::NSLOT) * S * T::PLANE + cidx,
                      ring(kz + 1, T::NSLOT) * S * T::PLANE + cidx};
    const int g[3] = {ring(kz - 1, T::NSLOT) * T::NP * T::PLANE + cidx, ring(kz, T::NSLOT) * T::NP * T::PLANE + cidx,
                      ring(kz + 1, T::NSLOT) * T::NP * T::PLANE + cidx};
#pragma unroll
    for (int b = 0; b < S; ++b) {
        pass1_cube_class<S, DRAG, 0, HC>(p, sf, sg, b, f, g, c, ub, w, A);
        pass1_cube_class<S, DRAG, 1, HC>(p, sf, sg, b, f, g, c, ub, w, A);
        pass1_cube_class<S, DRAG, 2, HC>(p, sf, sg, b, f, g, c, ub, w, A);
    }
}

// MODE: kExact; kSurrogate (no hard-core sums, attr holds F^hc); kSweep (mom
// is the previous sweep's (n - n_ref, u*) field, mom_c the moments, frest is
// read, pst receives the sweep's u*)
// the tile (bx, by, bz) of the tiled pass 1
template <int S, int R, bool DRAG, int TY, int MODE>
__device__ __forceinline__ void pass1_tile(const mlbi_params &p, const float4 *__restrict__ mom,
                                           const float *__restrict__ dg, const mlbi_entry *__restrict__ tab,
                                           const float4 *__restrict__ fext, const float4 *__restrict__ attr,
                                           const float4 *__restrict__ mom_c, float4 *__restrict__ frest,
                                           float4 *__restrict__ pst, int bx, int by, int bz)
{
    constexpr bool HC = MODE == kExact;
    using T = Tile<S, R, TY>;
    extern __shared__ float4 smem[];
    float4 *sf = smem;                                                      // [NSLOT][S][PLANE]
    float *sg = reinterpret_cast<float *>(smem + (size_t)T::NSLOT * S * T::PLANE);   // [NSLOT][NP][PLANE]
    const int x0 = bx * kBX, y0 = by * TY, z0 = bz * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = x < p.nx && y < p.ny;
    const int cidx = (threadIdx.y + R) * T::TXH + threadIdx.x + R;
    const mlbi_entry *stab =
        stage_table<T, R>(p, tab, reinterpret_cast<float4 *>(reinterpret_cast<char *>(smem) + T::bytes));
    int xy[T::J];
    stage_sites<S, R, TY>(p, x0, y0, xy);
    for (int k = 0; k < 2 * R + 1; ++k)
        stage_plane<S, R, TY>(p, xy, z0 - R + k, ring(k, T::NSLOT), mom, dg, sf, sg);
    cp_async_commit();
    for (int z = z0; z < z1; ++z) {
        cp_async_wait_all();
        __syncthreads();
        const int kz = z - z0 + R;                      // ring position of plane z
        if (z + 1 < z1) {
            stage_plane<S, R, TY>(p, xy, z + R + 1, ring(kz + R + 1, T::NSLOT), mom, dg, sf, sg);
            cp_async_commit();
        }
        if (!active) continue;
        const int cs = ring(kz, T::NSLOT);
        const long long r = x + (long long)p.nx * (y + (long long)p.ny * z);
        float4 cv[S];
#pragma unroll
        for (int a = 0; a < S; ++a) cv[a] = sf[cs * S * T::PLANE + a * T::PLANE + cidx];
        Centre<S> c;
        float ub[S][3];
        centre_of<S, MODE>(p, cv, mom_c, r, c, ub);
        float dgc[T::NP];
#pragma unroll
        for (int q = 0; q < T::NP; ++q) dgc[q] = sg[cs * T::NP * T::PLANE + q * T::PLANE + cidx];
        PairW<S> w;
        pair_weights<S>(p, dgc, w);
        Acc1<S> A;
        A.zero();
        if constexpr (R == 1 && TY == kBY) pass1_cube<S, DRAG, HC>(p, sf, sg, kz, cidx, c, ub, w, A);
        else pass1_tile_shells<S, R, DRAG, TY, HC>(p, stab, sf, sg, kz, cidx, c, ub, w, A);
        if constexpr (MODE == kSweep) {
            sweep_finish<S>(p, r, c, A, frest, pst);
            continue;
        }
        if (MODE == kSurrogate || p.attr_r) {
#pragma unroll
            for (int a = 0; a < S; ++a) {
                const float4 v = attr[a * p.N + r];
                A.at[a][0] = v.x; A.at[a][1] = v.y; A.at[a][2] = v.z;
            }
        } else if (p.has_attraction) {
            Loc L;
            L.x = x; L.y = y; L.z = z; L.r = r;
            const int Rr = p.reach;
            L.interior = x >= Rr && x < p.nx - Rr && y >= Rr && y < p.ny - Rr && z >= Rr && z < p.nz - Rr;
            if (L.interior) pass1_attraction<S, true>(p, L, mom, tab, A.at);
            else pass1_attraction<S, false>(p, L, mom, tab, A.at);
        }
        pass1_finish<S, DRAG>(p, r, c, A, fext, frest, pst);
    }
}

template <int S, int R, bool DRAG, int TY, int MODE>
__global__ void __launch_bounds__(kBX * TY, tile_blocks(Tile<S, R, TY>::bytes, S <= 2 ? (MODE == kSweep ? 4 : 6) : 2))
    k_pass1_tiled(const mlbi_params p, const float4 *__restrict__ mom, const float *__restrict__ dg,
                  const mlbi_entry *__restrict__ tab, const float4 *__restrict__ fext, const float4 *__restrict__ attr,
                  const float4 *__restrict__ mom_c, float4 *__restrict__ frest, float4 *__restrict__ pst)
{
    pass1_tile<S, R, DRAG, TY, MODE>(p, mom, dg, tab, fext, attr, mom_c, frest, pst, blockIdx.x, blockIdx.y,
                                     blockIdx.z);
}

// every member of a group (block table entries {member, bx, by, bz}), the exact pass
template <int S, int R, bool DRAG, int TY>
__global__ void __launch_bounds__(kBX * TY, tile_blocks(Tile<S, R, TY>::bytes + sizeof(mlbi_params), S <= 2 ? 6 : 2))
    k_pass1_group(const mlbi_member *__restrict__ mem, const int4 *__restrict__ blk)
{
    __shared__ mlbi_params sp;
    const int4 e = blk[blockIdx.x];
    const mlbi_member *m = mem + e.x;
    group_params(m, sp);
    const mlbi_buffers &b = m->b;
    pass1_tile<S, R, DRAG, TY, kExact>(sp, b.mom, b.dg, b.table, b.fext, b.attr, b.mom, b.frest, b.pst, e.y, e.z,
                                       e.w);
}

}  // namespace
