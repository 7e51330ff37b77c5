// mlb_pass2.cu -- pass 2 of a time step on sm_103a: the velocity exchange
// (Eqs. gammaab, viscousforce) at the predicted velocities u* of pass 1,
// completed to the acceleration a^a = frest^a + sum_points s sd (masses 1).
// Same three variants as pass 1: global memory, tile with the stencil table
// (reach 2, 3), compile-time 3x3x3 cube (reach 1).  The tiled variants also come
// fused with the collision (k_pass2_collide): the acceleration is not stored,
// the same thread collides and streams its site right away (the collision
// needs only the site's own acceleration).
#include "mlb_passes.cuh"
#include "mlb_collide.cuh"

namespace {

// centre velocities u*^a(r) from pass 1's (n - n_ref, u*) field
template <int S>
__device__ __forceinline__ void centre_ustar(const mlbi_params &p, const float4 *__restrict__ pst, long long r,
                                             float (&us)[S][3])
{
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 v = pst[a * p.N + r];
        us[a][0] = v.y; us[a][1] = v.z; us[a][2] = v.w;
    }
}

template <int S>
__device__ __forceinline__ void store_acc(const mlbi_params &p, long long r, const float (&acc)[S][3],
                                          float4 *__restrict__ acc_f, double *__restrict__ acc_out)
{
    const long long N = p.N;
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

template <int S>
__device__ __forceinline__ void zero_acc(float (&acc)[S][3])
{
#pragma unroll
    for (int a = 0; a < S; ++a) acc[a][0] = acc[a][1] = acc[a][2] = 0.f;
}

// the rest force F^hc + G + F_ext is added after the shell sums (the same
// order in every variant, so the fused and split launches agree bit for bit)
__device__ __forceinline__ void add_rest(float (&acc)[3], const float4 fr)
{
    acc[0] = fr.x + acc[0];
    acc[1] = fr.y + acc[1];
    acc[2] = fr.z + acc[2];
}

// a^a = frest^a + vx_ab sum_{+-d} s s.[(g(r)+g(r+d))/2 n^b(r+d) (u*^b(r+d) - u*^a(r))]
// (drag only: -wn s.(u*^a - u*^b)(r) per point)
template <int S, bool DRAG, bool INTERIOR>
__device__ __forceinline__ void pass2_shells(const mlbi_params &p, const Loc &L, const PairW<S> &w,
                                             const float (&us)[S][3], const float4 *__restrict__ pst,
                                             const float *__restrict__ dg, const mlbi_entry *__restrict__ tab,
                                             float (&acc)[S][3])
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
            const Nb P = fetch_nb<INTERIOR>(p, L, e0, e1, 1, fb, p.nref[b]);
            const Nb M = fetch_nb<INTERIOR>(p, L, e0, e1, -1, fb, p.nref[b]);
            const float sx = e0.x, sy = e0.y, sz = e0.z;
            const float jp = DRAG ? 0.f : sx * P.u0 + sy * P.u1 + sz * P.u2;
            const float jm = DRAG ? 0.f : sx * M.u0 + sy * M.u1 + sz * M.u2;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                if (!(mask & (1 << a))) continue;
                const int q = pair_of(a, b, S);
                const float su = DRAG ? 0.f : sx * us[a][0] + sy * us[a][1] + sz * us[a][2];
                const float *dgq = dg + q * N;
                const float dgp = (INTERIOR || P.q >= 0) ? dgq[P.q] : 0.f;
                const float dgm = (INTERIOR || M.q >= 0) ? dgq[M.q] : 0.f;
                const float sdu = DRAG ? sx * (us[a][0] - us[b][0]) + sy * (us[a][1] - us[b][1]) +
                                             sz * (us[a][2] - us[b][2])
                                       : 0.f;
                const float sd = pass2_point<DRAG>(P.n, M.n, jp - su, jm - su, dgp, dgm, w.kp[q],
                                                   0.5f * p.pair[q].vx_pre, sdu);
                acc[a][0] = fmaf(sx, sd, acc[a][0]);
                acc[a][1] = fmaf(sy, sd, acc[a][1]);
                acc[a][2] = fmaf(sz, sd, acc[a][2]);
            }
        }
    }
}

template <int S, bool DRAG>
__global__ void __launch_bounds__(kBX * kBY) k_pass2(const mlbi_params p, const float *__restrict__ dg,
                                                     const mlbi_entry *__restrict__ tab,
                                                     const float4 *__restrict__ frest,
                                                     const float4 *__restrict__ pst, float4 *__restrict__ acc_f,
                                                     double *__restrict__ acc_out)
{
    constexpr int NP = S * (S + 1) / 2;
    Loc L;
    if (!locate(p, L)) return;
    const long long N = p.N, r = L.r;
    float dgc[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) dgc[q] = dg[q * N + r];
    PairW<S> w;
    pair_weights<S>(p, dgc, w);
    float us[S][3];
    centre_ustar<S>(p, pst, r, us);
    float acc[S][3];
    zero_acc<S>(acc);
    if (L.interior) pass2_shells<S, DRAG, true>(p, L, w, us, pst, dg, tab, acc);
    else pass2_shells<S, DRAG, false>(p, L, w, us, pst, dg, tab, acc);
#pragma unroll
    for (int a = 0; a < S; ++a) add_rest(acc[a], frest[a * N + r]);
    store_acc<S>(p, r, acc, acc_f, acc_out);
}

// ------------------------------------------------------------------ tiled variants
template <int S, int R, bool DRAG, int TY, int NSL = 2 * R + 2>
__device__ __forceinline__ void pass2_tile_shells(const mlbi_params &p, const mlbi_entry *tab,
                                                  const float4 *sf, const float *sg, int kz, int cidx,
                                                  const PairW<S> &w, const float (&us)[S][3], float (&acc)[S][3])
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
            const int sp = ring(kz + dz, NSL), sm = ring(kz - dz, NSL);
            const float4 vp = sf[sp * S * T::PLANE + b * T::PLANE + cidx + off];
            const float4 vm = sf[sm * S * T::PLANE + b * T::PLANE + cidx - off];
            const float np = nr + vp.x, nm = nr + vm.x;
            const float sx = e0.x, sy = e0.y, sz = e0.z;
            const float jp = DRAG ? 0.f : sx * vp.y + sy * vp.z + sz * vp.w;
            const float jm = DRAG ? 0.f : sx * vm.y + sy * vm.z + sz * vm.w;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                if (!(mask & (1 << a))) continue;
                const int q = pair_of(a, b, S);
                const float su = DRAG ? 0.f : sx * us[a][0] + sy * us[a][1] + sz * us[a][2];
                const float dgp = sg[sp * T::NP * T::PLANE + q * T::PLANE + cidx + off];
                const float dgm = sg[sm * T::NP * T::PLANE + q * T::PLANE + cidx - off];
                const float sdu = DRAG ? sx * (us[a][0] - us[b][0]) + sy * (us[a][1] - us[b][1]) +
                                             sz * (us[a][2] - us[b][2])
                                       : 0.f;
                const float sd = pass2_point<DRAG>(np, nm, jp - su, jm - su, dgp, dgm, w.kp[q],
                                                   0.5f * p.pair[q].vx_pre, sdu);
                acc[a][0] = fmaf(sx, sd, acc[a][0]);
                acc[a][1] = fmaf(sy, sd, acc[a][1]);
                acc[a][2] = fmaf(sz, sd, acc[a][2]);
            }
        }
    }
}

// reach 1 by offset class (see pass1_cube_class)
template <int S, bool DRAG, int CL>
__device__ __forceinline__ void pass2_cube_class(const mlbi_params &p, const float4 *sf, const float *sg, int b,
                                                 const int (&f)[3], const int (&g)[3], const PairW<S> &w,
                                                 const float (&us)[S][3], float (&acc)[S][3])
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
        // the arithmetic of pass2_point with the +d and -d lanes packed
        const float2 npm = add2(f2(nr, nr), f2(vp.x, vm.x));
        float2 jpm = f2(0.f, 0.f);
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
            const float2 hpm = mul2(fma2(f2(k1, k1), dg2, f2(w.kp[q], w.kp[q])), npm);
            float sd;
            if constexpr (DRAG) {
                const float sdu = cube_dot<k>(il, us[a][0] - us[b][0], us[a][1] - us[b][1], us[a][2] - us[b][2]);
                sd = -(hpm.x + hpm.y) * sdu;
            } else {
                const float su = cube_dot<k>(il, us[a][0], us[a][1], us[a][2]);
                const float2 j2 = add2(jpm, f2(-su, -su));
                sd = fmaf(hpm.x, j2.x, hpm.y * j2.y);
            }
            cube_add<k>(il, sd, acc[a]);
        }
    });
}

template <int S, bool DRAG, int NSL = 4>
__device__ __forceinline__ void pass2_cube(const mlbi_params &p, const float4 *sf, const float *sg, int kz, int cidx,
                                           const PairW<S> &w, const float (&us)[S][3], float (&acc)[S][3])
{
    using T = Tile<S, 1>;
    const int f[3] = {ring(kz - 1, NSL) * S * T::PLANE + cidx, ring(kz, NSL) * S * T::PLANE + cidx,
                      ring(kz + 1, NSL) * S * T::PLANE + cidx};
    const int g[3] = {ring(kz - 1, NSL) * T::NP * T::PLANE + cidx, ring(kz, NSL) * T::NP * T::PLANE + cidx,
                      ring(kz + 1, NSL) * T::NP * T::PLANE + cidx};
#pragma unroll
    for (int b = 0; b < S; ++b) {
        pass2_cube_class<S, DRAG, 0>(p, sf, sg, b, f, g, w, us, acc);
        pass2_cube_class<S, DRAG, 1>(p, sf, sg, b, f, g, w, us, acc);
        pass2_cube_class<S, DRAG, 2>(p, sf, sg, b, f, g, w, us, acc);
    }
}

// the shell sums of the acceleration of the site at ring position kz of the
// tile (centre slot cs), added to acc
template <int S, int R, bool DRAG, int TY, int NSL = 2 * R + 2>
__device__ __forceinline__ void pass2_site(const mlbi_params &p, const mlbi_entry *tab, const float4 *sf,
                                           const float *sg, int kz, int cidx, float (&acc)[S][3])
{
    using T = Tile<S, R, TY>;
    const int cs = ring(kz, NSL);
    float dgc[T::NP];
#pragma unroll
    for (int q = 0; q < T::NP; ++q) dgc[q] = sg[cs * T::NP * T::PLANE + q * T::PLANE + cidx];
    PairW<S> w;
    pair_weights<S>(p, dgc, w);
    float us[S][3];
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 v = sf[cs * S * T::PLANE + a * T::PLANE + cidx];
        us[a][0] = v.y; us[a][1] = v.z; us[a][2] = v.w;
    }
    if constexpr (R == 1 && TY == kBY) pass2_cube<S, DRAG, NSL>(p, sf, sg, kz, cidx, w, us, acc);
    else pass2_tile_shells<S, R, DRAG, TY, NSL>(p, tab, sf, sg, kz, cidx, w, us, acc);
}

template <int S, int R, bool DRAG, int TY>
__global__ void __launch_bounds__(kBX * TY, tile_blocks(Tile<S, R, TY>::bytes, S <= 2 ? 4 : 2))
    k_pass2_tiled(const mlbi_params p, const float *__restrict__ dg, const mlbi_entry *__restrict__ tab,
                  const float4 *__restrict__ frest, const float4 *__restrict__ pst, float4 *__restrict__ acc_f,
                  double *__restrict__ acc_out)
{
    using T = Tile<S, R, TY>;
    extern __shared__ float4 smem[];
    float4 *sf = smem;
    float *sg = reinterpret_cast<float *>(smem + (size_t)T::NSLOT * S * T::PLANE);
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * TY, z0 = blockIdx.z * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = x < p.nx && y < p.ny;
    const int cidx = (threadIdx.y + R) * T::TXH + threadIdx.x + R;
    const mlbi_entry *stab =
        stage_table<T, R>(p, tab, reinterpret_cast<float4 *>(reinterpret_cast<char *>(smem) + T::bytes));
    int xy[T::J];
    stage_sites<S, R, TY>(p, x0, y0, xy);
    for (int k = 0; k < 2 * R + 1; ++k)
        stage_plane<S, R, TY>(p, xy, z0 - R + k, ring(k, T::NSLOT), pst, dg, sf, sg);
    cp_async_commit();
    for (int z = z0; z < z1; ++z) {
        cp_async_wait_all();
        __syncthreads();
        const int kz = z - z0 + R;
        if (z + 1 < z1) {
            stage_plane<S, R, TY>(p, xy, z + R + 1, ring(kz + R + 1, T::NSLOT), pst, dg, sf, sg);
            cp_async_commit();
        }
        if (!active) continue;
        const long long r = x + (long long)p.nx * (y + (long long)p.ny * z);
        float acc[S][3];
        zero_acc<S>(acc);
        pass2_site<S, R, DRAG, TY>(p, stab, sf, sg, kz, cidx, acc);
#pragma unroll
        for (int a = 0; a < S; ++a) add_rest(acc[a], frest[a * p.N + r]);
        store_acc<S>(p, r, acc, acc_f, acc_out);
    }
}

// ------------------------------------------------------------------ pass 2 fused with the collision
// Per plane, each thread computes the acceleration of its site and at once
// collides and streams the site.  Its own populations and moments for the
// next plane are prefetched by cp.async into a per-thread slot of shared
// memory while this plane's shell sums run.  Two cp.async groups per plane,
// committed by every thread (empty where there is nothing to copy):
//   A(z) = halo plane z + R of the stencil ring and the site's frest(z),
//   P(z) = the site's populations and moments of plane z.
// They alternate A(z), P(z), A(z+1), P(z+1), ..., so "all but the newest
// group" is A(z) at the top of plane z and P(z) before its collision.
template <int S, int R>
struct FusedTile {
    using T = Tile<S, R>;
    static constexpr size_t pops_off = T::bytes;                                   // float [S*19][NT]
    static constexpr size_t mom_off = pops_off + (size_t)S * MLBI_Q * T::NT * sizeof(float);   // float4 [S][NT]
    static constexpr size_t rest_off = mom_off + (size_t)S * T::NT * sizeof(float4);           // float4 [S][NT]
    static constexpr size_t bytes = rest_off + (size_t)S * T::NT * sizeof(float4);
};

template <int S>
__device__ __forceinline__ void stage_pops(const mlbi_params &p, long long r, int tid, int nt,
                                           const float *__restrict__ fin, const float4 *__restrict__ mom, float *sF,
                                           float4 *sM)
{
#pragma unroll
    for (int a = 0; a < S; ++a) {
        cp_async16(sM + a * nt + tid, mom + a * p.N + r);
#pragma unroll
        for (int i = 0; i < MLBI_Q; ++i)
            cp_async4(sF + (a * MLBI_Q + i) * nt + tid, fin + ((long long)a * MLBI_Q + i) * p.N + r);
    }
}

template <int S>
__device__ __forceinline__ void stage_rest(const mlbi_params &p, long long r, int tid, int nt,
                                           const float4 *__restrict__ frest, float4 *sR)
{
#pragma unroll
    for (int a = 0; a < S; ++a) cp_async16(sR + a * nt + tid, frest + a * p.N + r);
}

__device__ __forceinline__ void cp_async_wait_all_but_newest() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

template <int S, int R, bool DRAG>
__global__ void __launch_bounds__(kBX * kBY, S <= 2 ? 3 : 2) k_pass2_collide(const mlbi_params p,
                                                                            const float *__restrict__ dg,
                                                                            const mlbi_entry *__restrict__ tab,
                                                                            const float4 *__restrict__ frest,
                                                                            const float4 *__restrict__ pst,
                                                                            const float4 *__restrict__ mom,
                                                                            const float *__restrict__ fin,
                                                                            float *__restrict__ fout)
{
    using T = Tile<S, R>;
    using F = FusedTile<S, R>;
    extern __shared__ float4 smem[];
    float4 *sf = smem;
    float *sg = reinterpret_cast<float *>(smem + (size_t)T::NSLOT * S * T::PLANE);
    float *sF = reinterpret_cast<float *>(reinterpret_cast<char *>(smem) + F::pops_off);
    float4 *sM = reinterpret_cast<float4 *>(reinterpret_cast<char *>(smem) + F::mom_off);
    float4 *sR = reinterpret_cast<float4 *>(reinterpret_cast<char *>(smem) + F::rest_off);
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY, z0 = blockIdx.z * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const bool active = x < p.nx && y < p.ny;
    const int cidx = (threadIdx.y + R) * T::TXH + threadIdx.x + R;
    const long long sxy = x + (long long)p.nx * y, nxy = (long long)p.nx * p.ny;
    int xy[T::J];
    stage_sites<S, R>(p, x0, y0, xy);
    for (int k = 0; k < 2 * R + 1; ++k) stage_plane<S, R>(p, xy, z0 - R + k, ring(k, T::NSLOT), pst, dg, sf, sg);
    if (active) stage_rest<S>(p, sxy + nxy * z0, tid, T::NT, frest, sR);
    cp_async_commit();                                                  // A(z0)
    if (active) stage_pops<S>(p, sxy + nxy * z0, tid, T::NT, fin, mom, sF, sM);
    cp_async_commit();                                                  // P(z0)
    float rest[S][3];
    for (int z = z0; z < z1; ++z) {
        cp_async_wait_all_but_newest();                                 // A(z) landed
        __syncthreads();
        const int kz = z - z0 + R;
        const long long r = sxy + nxy * z;
        float acc[S][3];
        zero_acc<S>(acc);
        if (active) {
#pragma unroll
            for (int a = 0; a < S; ++a) {
                const float4 v = sR[a * T::NT + tid];
                rest[a][0] = v.x; rest[a][1] = v.y; rest[a][2] = v.z;
            }
        }
        if (z + 1 < z1) {
            stage_plane<S, R>(p, xy, z + R + 1, ring(kz + R + 1, T::NSLOT), pst, dg, sf, sg);
            if (active) stage_rest<S>(p, r + nxy, tid, T::NT, frest, sR);
        }
        cp_async_commit();                                              // A(z + 1)
        if (active) {
            pass2_site<S, R, DRAG, kBY>(p, tab, sf, sg, kz, cidx, acc);
#pragma unroll
            for (int a = 0; a < S; ++a) add_rest(acc[a], make_float4(rest[a][0], rest[a][1], rest[a][2], 0.f));
        }
        cp_async_wait_all_but_newest();                                 // P(z) landed (own slots only)
        if (active) {
            Centre<S> c;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                const float4 v = sM[a * T::NT + tid];
                c.dn[a] = v.x;
                c.n[a] = p.nref[a] + v.x;
                c.u[a][0] = v.y; c.u[a][1] = v.z; c.u[a][2] = v.w;
            }
            collide_push<S>(p, x, y, z, r, c, acc, SharedPops{sF + tid, T::NT}, fout);
            if (z + 1 < z1) stage_pops<S>(p, r + nxy, tid, T::NT, fin, mom, sF, sM);
        }
        cp_async_commit();                                              // P(z + 1)
    }
    cp_async_wait_all();
}

// ------------------------------------------------------------------ fused, with bulk tensor copies
// The same per-site arithmetic as k_pass2_collide.  The site's own data of a
// plane -- its 19 S populations, moments and rest force -- arrive as three
// bulk tensor (TMA) copies of the block's 32 x 4 sites, issued by one thread
// at the top of the plane and waited on (mbarrier, bounded) only before the
// collision, so they land while the plane's shell sums run.  Shared layouts
// are those of the cp.async variant: population (a, i) of thread t at
// sF[(a * 19 + i) * 128 + t], moments and rest force at sM / sR[a * 128 + t].
// The stencil ring holds 2R + 1 planes only: the next plane is staged into
// the slot of plane z - R once every thread has finished plane z's shell
// sums (a second barrier per plane), and lands during the collisions.  The
// 9 KB this saves (R = 1, S = 2) and a 128-register bound give 4 resident
// blocks per SM instead of 3.
template <int S, int R>
struct TmaTile {
    using T = Tile<S, R>;
    static constexpr int NSL = 2 * R + 1;
    static constexpr size_t pad(size_t b) { return (b + 127) / 128 * 128; }
    static constexpr size_t ring_bytes = (size_t)NSL * T::PLANE * (S * sizeof(float4) + T::NP * sizeof(float));
    static constexpr uint32_t pops_bytes = (uint32_t)S * MLBI_Q * T::NT * 4;
    static constexpr uint32_t v4_bytes = (uint32_t)S * T::NT * 16;
    static constexpr size_t pops_off = pad(ring_bytes);
    static constexpr size_t mom_off = pops_off + pops_bytes;
    static constexpr size_t rest_off = mom_off + v4_bytes;
    static constexpr size_t bytes = rest_off + v4_bytes + 128;       // + alignment slack of the base
    static constexpr uint32_t tx_bytes = pops_bytes + 2 * v4_bytes;
};

// the tile (bx, by, bz) of the fused pass; the maps are kernel parameters or
// (grouped launches) global-memory copies the issuing thread has acquired
template <int S, int R, bool DRAG>
__device__ __forceinline__ void pass2_collide_tma_tile(const mlbi_params &p, const float *__restrict__ dg,
                                                       const mlbi_entry *__restrict__ tab,
                                                       const float4 *__restrict__ pst, float *__restrict__ fout,
                                                       unsigned int *__restrict__ flags, const CUtensorMap *map_f,
                                                       const CUtensorMap *map_mom, const CUtensorMap *map_rest,
                                                       int bx, int by, int bz)
{
    using T = Tile<S, R>;
    using F = TmaTile<S, R>;
    extern __shared__ float4 smem_raw[];
    __shared__ __align__(8) uint64_t bar_mem;
    // the bulk copies want 128-byte aligned destinations
    char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    constexpr int NSL = F::NSL;
    float4 *sf = reinterpret_cast<float4 *>(base);
    float *sg = reinterpret_cast<float *>(sf + (size_t)NSL * S * T::PLANE);
    float *sF = reinterpret_cast<float *>(base + F::pops_off);
    float4 *sM = reinterpret_cast<float4 *>(base + F::mom_off);
    float4 *sR = reinterpret_cast<float4 *>(base + F::rest_off);
    __shared__ int s_fail;                                       // a wait gave up (read after a barrier)
    const uint32_t bar = smem_u32(&bar_mem);
    const int x0 = bx * kBX, y0 = by * kBY, z0 = bz * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const bool active = x < p.nx && y < p.ny;
    const int cidx = (threadIdx.y + R) * T::TXH + threadIdx.x + R;
    const int sxy = x + p.nx * y, nxy = p.nx * p.ny;
    auto issue = [&](int z) {
        mbar_expect_tx(bar, F::tx_bytes);
        tma_load_4d(smem_u32(sF), map_f, bar, x0, y0, z, 0);
        tma_load_5d(smem_u32(sM), map_mom, bar, 0, x0, y0, z, 0);
        tma_load_5d(smem_u32(sR), map_rest, bar, 0, x0, y0, z, 0);
    };
    if (tid == 0) {
        mbar_init(bar, 1);
        s_fail = 0;
    }
    int xy[T::J];
    stage_sites<S, R>(p, x0, y0, xy);
    for (int k = 0; k < 2 * R + 1; ++k) stage_plane<S, R>(p, xy, z0 - R + k, ring(k, NSL), pst, dg, sf, sg);
    cp_async_commit();
    __syncthreads();                                            // the barrier is initialised
    if (tid == 0) issue(z0);
    uint32_t phase = 0;
    for (int z = z0; z < z1; ++z) {
        cp_async_wait_all();
        __syncthreads();              // ring planes up to z + R in; every thread is done with plane z - 1
        if (s_fail) break;            // uniform: read after the barrier
        if (tid == 0 && z > z0) issue(z);
        const int kz = z - z0 + R;
        float acc[S][3];
        zero_acc<S>(acc);
        if (active) pass2_site<S, R, DRAG, kBY, NSL>(p, tab, sf, sg, kz, cidx, acc);
        __syncthreads();              // every thread is done with plane z - R: its slot takes plane z + R + 1
        if (z + 1 < z1) stage_plane<S, R>(p, xy, z + R + 1, ring(kz + R + 1, NSL), pst, dg, sf, sg);
        cp_async_commit();
        // each thread waits for the copies itself, so warps move on to their
        // collisions independently; a wait that gives up marks the block failed,
        // and every thread leaves at the next barrier
        const bool ok = mbar_wait(bar, phase);
        phase ^= 1u;
        if (!ok) {
            s_fail = 1;
            if (tid == 0) atomicOr(flags, MLBI_FLAG_TIMEOUT);
            continue;
        }
        if (active) {
            Centre<S> c;
#pragma unroll
            for (int a = 0; a < S; ++a) {
                const float4 v = sM[a * T::NT + tid];
                c.dn[a] = v.x;
                c.n[a] = p.nref[a] + v.x;
                c.u[a][0] = v.y; c.u[a][1] = v.z; c.u[a][2] = v.w;
                add_rest(acc[a], sR[a * T::NT + tid]);
            }
            collide_push<S>(p, x, y, z, sxy + nxy * z, c, acc, SharedPops{sF + tid, T::NT}, fout);
        }
    }
    cp_async_wait_all();
    if (s_fail && tid == 0) mbar_wait(bar, phase ^ 1u);       // one more bounded wait for the copy in flight
}

template <int S, int R, bool DRAG>
__global__ void __launch_bounds__(kBX * kBY, S <= 2 ? 4 : 2)
    k_pass2_collide_tma(const mlbi_params p, const float *__restrict__ dg, const mlbi_entry *__restrict__ tab,
                        const float4 *__restrict__ pst, float *__restrict__ fout, unsigned int *__restrict__ flags,
                        const __grid_constant__ CUtensorMap map_f, const __grid_constant__ CUtensorMap map_mom,
                        const __grid_constant__ CUtensorMap map_rest)
{
    pass2_collide_tma_tile<S, R, DRAG>(p, dg, tab, pst, fout, flags, &map_f, &map_mom, &map_rest, blockIdx.x,
                                       blockIdx.y, blockIdx.z);
}

// every member of a group (block table entries {member, bx, by, bz}); odd:
// the members read f[cur ^ 1] and write f[cur]
template <int S, int R, bool DRAG>
__global__ void __launch_bounds__(kBX * kBY, S <= 2 ? 4 : 2)
    k_pass2_collide_group(const mlbi_member *__restrict__ mem, const int4 *__restrict__ blk, int odd)
{
    __shared__ mlbi_params sp;
    const int4 e = blk[blockIdx.x];
    const mlbi_member *m = mem + e.x;
    const int rd = m->cur ^ odd;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        tensormap_acquire(&m->map_f[rd]);
        tensormap_acquire(&m->map_mom);
        tensormap_acquire(&m->map_frest);
    }
    group_params(m, sp);
    const mlbi_buffers &b = m->b;
    pass2_collide_tma_tile<S, R, DRAG>(sp, b.dg, b.table, b.pst, b.f[rd ^ 1], b.flags, &m->map_f[rd], &m->map_mom,
                                       &m->map_frest, e.y, e.z, e.w);
}

template <int S, int R, bool DRAG>
cudaError_t launch_pass2_tiled(const mlbi_params &p, const mlbi_buffers &b, double *acc_out, cudaStream_t s)
{
    constexpr int TY = mlbi_tile_ty(S, R);
    if constexpr (TY == 0) {
        return cudaErrorInvalidValue;
    } else {
        using T = Tile<S, R, TY>;
        auto k = k_pass2_tiled<S, R, DRAG, TY>;
        const size_t bytes = T::bytes + staged_table_bytes<T, R>(p);
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        const dim3 g((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + TY - 1) / TY),
                     (unsigned)((p.nz + p.zchunk - 1) / p.zchunk));
        k<<<g, dim3(kBX, TY), bytes, s>>>(p, b.dg, b.table, b.frest, b.pst, b.acc, acc_out);
        return cudaGetLastError();
    }
}

template <int S, bool DRAG>
cudaError_t launch_pass2(const mlbi_params &p, const mlbi_buffers &b, double *acc_out, cudaStream_t s)
{
    if (p.tile_r == 1) return launch_pass2_tiled<S, 1, DRAG>(p, b, acc_out, s);
    if (p.tile_r == 2) return launch_pass2_tiled<S, 2, DRAG>(p, b, acc_out, s);
    if (p.tile_r == 3) return launch_pass2_tiled<S, 3, DRAG>(p, b, acc_out, s);
    k_pass2<S, DRAG><<<tiled_grid(p), dim3(kBX, kBY), 0, s>>>(p, b.dg, b.table, b.frest, b.pst, b.acc, acc_out);
    return cudaGetLastError();
}

constexpr size_t kMaxSharedPerBlock = 227 * 1024;

template <int S, int R, bool DRAG>
cudaError_t launch_pass2_collide_tiled(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s)
{
    using F = FusedTile<S, R>;
    if constexpr (F::bytes > kMaxSharedPerBlock) {
        return cudaErrorInvalidValue;
    } else {
    if constexpr (TmaTile<S, R>::bytes <= kMaxSharedPerBlock) {
        if (b.maps && b.maps->ok) {
            using G = TmaTile<S, R>;
            auto k = k_pass2_collide_tma<S, R, DRAG>;
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::bytes);
            if (e != cudaSuccess) return e;
            const dim3 g((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + kBY - 1) / kBY),
                         (unsigned)((p.nz + p.zchunk - 1) / p.zchunk));
            k<<<g, dim3(kBX, kBY), G::bytes, s>>>(p, b.dg, b.table, b.pst, b.f[cur ^ 1], b.flags, b.maps->f[cur],
                                                  b.maps->mom, b.maps->frest);
            return cudaGetLastError();
        }
    }
    auto k = k_pass2_collide<S, R, DRAG>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)F::bytes);
    if (e != cudaSuccess) return e;
    const dim3 g((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + kBY - 1) / kBY),
                 (unsigned)((p.nz + p.zchunk - 1) / p.zchunk));
    k<<<g, dim3(kBX, kBY), F::bytes, s>>>(p, b.dg, b.table, b.frest, b.pst, b.mom, b.f[cur], b.f[cur ^ 1]);
    return cudaGetLastError();
    }
}

template <int S>
bool collide_fits(int tile_r)
{
    if (tile_r == 1) return FusedTile<S, 1>::bytes <= kMaxSharedPerBlock;
    if (tile_r == 2) return FusedTile<S, 2>::bytes <= kMaxSharedPerBlock;
    return false;
}

template <int S, bool DRAG>
cudaError_t launch_pass2_collide(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s)
{
    if (p.tile_r == 1) return launch_pass2_collide_tiled<S, 1, DRAG>(p, b, cur, s);
    if (p.tile_r == 2) return launch_pass2_collide_tiled<S, 2, DRAG>(p, b, cur, s);
    return cudaErrorInvalidValue;          // the global-memory pass 2 is not fused
}

template <int S, int R, bool DRAG>
cudaError_t launch_pass2_collide_group(const mlbi_group &g, int odd, cudaStream_t s)
{
    using G = TmaTile<S, R>;
    if constexpr (G::bytes + sizeof(mlbi_params) > kMaxSharedPerBlock) {
        return cudaErrorInvalidValue;
    } else {
        auto k = k_pass2_collide_group<S, R, DRAG>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::bytes);
        if (e != cudaSuccess) return e;
        k<<<(unsigned)g.nblk[MLBI_GROUP_PASS2], dim3(kBX, kBY), G::bytes, s>>>(g.mem, g.blk[MLBI_GROUP_PASS2], odd);
        return cudaGetLastError();
    }
}

template <int S, int R>
cudaError_t launch_pass2_collide_group_r(const mlbi_group &g, int odd, cudaStream_t s)
{
    return g.drag ? launch_pass2_collide_group<S, R, true>(g, odd, s)
                  : launch_pass2_collide_group<S, R, false>(g, odd, s);
}

}  // namespace

cudaError_t mlbi_launch_group_pass2_collide(const mlbi_group &g, int odd, cudaStream_t s)
{
    if (g.nblk[MLBI_GROUP_PASS2] < 1) return cudaErrorInvalidValue;
    if (g.S == 1) return g.R == 1 ? launch_pass2_collide_group_r<1, 1>(g, odd, s)
                                  : launch_pass2_collide_group_r<1, 2>(g, odd, s);
    if (g.S == 2) return g.R == 1 ? launch_pass2_collide_group_r<2, 1>(g, odd, s)
                                  : launch_pass2_collide_group_r<2, 2>(g, odd, s);
    return cudaErrorInvalidValue;
}

bool mlbi_group_supported(const mlbi_params &p, const mlbi_buffers &b)
{
    if (p.S < 1 || p.S > 2 || !p.local_g || p.hc_from_attr || !b.maps || !b.maps->ok) return false;
    if (p.tile_r != 1 && p.tile_r != 2) return false;
    return mlbi_pass2_collide_supported(p);
}

void mlbi_group_grid(const mlbi_params &p, int stage, int grid[3])
{
    const int zc = (p.nz + p.zchunk - 1) / p.zchunk;
    if (stage == MLBI_GROUP_MOMENTS) {
        grid[0] = (int)grid_for(p.N);
        grid[1] = grid[2] = 1;
    } else {
        const int ty = stage == MLBI_GROUP_PASS1 ? mlbi_tile_ty(p.S, p.tile_r) : kBY;
        grid[0] = (p.nx + kBX - 1) / kBX;
        grid[1] = (p.ny + ty - 1) / ty;
        grid[2] = zc;
    }
}

cudaError_t mlbi_launch_pass2(const mlbi_params &p, const mlbi_buffers &b, double *acc_out, cudaStream_t s)
{
    if (p.drag_only) { MLBI_DISPATCH_S(return (launch_pass2<SS, true>(p, b, acc_out, s))); }
    MLBI_DISPATCH_S(return (launch_pass2<SS, false>(p, b, acc_out, s)));
    return cudaErrorInvalidValue;
}

bool mlbi_pass2_collide_supported(const mlbi_params &p)
{
    switch (p.S) {
    case 1: return collide_fits<1>(p.tile_r);
    case 2: return collide_fits<2>(p.tile_r);
    case 3: return collide_fits<3>(p.tile_r);
    case 4: return collide_fits<4>(p.tile_r);
    default: return false;
    }
}

cudaError_t mlbi_launch_pass2_collide(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s)
{
    if (p.drag_only) { MLBI_DISPATCH_S(return (launch_pass2_collide<SS, true>(p, b, cur, s))); }
    MLBI_DISPATCH_S(return (launch_pass2_collide<SS, false>(p, b, cur, s)));
    return cudaErrorInvalidValue;
}
