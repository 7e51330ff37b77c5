// mlb_passes.cuh -- device code shared by the two force passes of a time step
// (mlb_pass1.cu, mlb_pass2.cu): per-site pair weights, the arithmetic of one
// +-d pair of a contact shell, the shared-memory z-marching tiles and the
// compile-time offsets of the 3x3x3 cube.  Internal header.
#pragma once

#include "mlb_internal.h"
#include "mlb_device.cuh"

#include <type_traits>

namespace {

// ------------------------------------------------------------------ pair weights
// The midpoint contact value of Eqs. potmeanforce and gammaab between r and
// r + d is (g(r) + g(r+d))/2 = B + dg(r+d)/2 with B = g_ref + dg(r)/2 and
// dg = g - g_ref.  Per site and pair (a, b):
//   exchange weight  vx_ab (g(r) + g(r+d))/2 = kp + k1 dg(r+d),  kp = vx_ab B,  k1 = vx_ab / 2
//   hard core        -hc_ab [(g(r)+g(r+d))/2 n(r+d) - (g(r)+g(r-d))/2 n(r-d)]
//                    = h (n(r+d) - n(r-d)) + c (n(r+d) dg(r+d) - n(r-d) dg(r-d)),
//                    h = -hc_ab B,  c = -hc_ab / 2,
// with n(r+d) - n(r-d) formed from the deviations n - n_ref (exact to rounding).
template <int S>
struct PairW {
    static constexpr int NP = S * (S + 1) / 2;
    float kp[NP], h[NP];
};

template <int S>
__device__ __forceinline__ void pair_weights(const mlbi_params &p, const float *dgc, PairW<S> &w)
{
#pragma unroll
    for (int q = 0; q < PairW<S>::NP; ++q) {
        const float B = fmaf(0.5f, dgc[q], p.pair[q].g_ref);
        w.kp[q] = p.pair[q].vx_pre * B;
        w.h[q] = -p.pair[q].hc_pre * B;
    }
}

// ------------------------------------------------------------------ one +-d pair of a shell
// Pass 1 (inputs at r +- d: n, the n - n_ref difference dd, dg, and
// jp/jm = s.(u^b(r +- d) - u^a(r))):
//   t  = hard-core projection on s (Eq. potmeanforce),
//   wn = h+ + h-, the friction weight, h+- = weight(r +- d) n^b(r +- d),
//   sd = h+ jp + h- jm, the exchange projection (Eqs. gammaab, viscousforce);
//   drag only: sd = -wn s.(u^a - u^b)(r), with sdu = s.(u^a - u^b).
template <bool DRAG>
__device__ __forceinline__ void pass1_point(float np, float nm, float dd, float jp, float jm, float dgp, float dgm,
                                            float kp, float k1, float h, float c, float sdu, float &t, float &sd,
                                            float &wn)
{
    const float gp = fmaf(k1, dgp, kp), gm = fmaf(k1, dgm, kp);
    t = fmaf(h, dd, c * fmaf(np, dgp, -nm * dgm));
    const float hp = gp * np, hm = gm * nm;
    wn = hp + hm;
    sd = DRAG ? -wn * sdu : fmaf(hp, jp, hm * jm);
}

// Pass 2: the same exchange projection at u*, jp/jm = s.(u*^b(r +- d) - u*^a(r))
// (drag only: sdu = s.(u*^a - u*^b)(r)).
template <bool DRAG>
__device__ __forceinline__ float pass2_point(float np, float nm, float jp, float jm, float dgp, float dgm, float kp,
                                             float k1, float sdu)
{
    const float gp = fmaf(k1, dgp, kp), gm = fmaf(k1, dgm, kp);
    const float hp = gp * np, hm = gm * nm;
    return DRAG ? -(hp + hm) * sdu : fmaf(hp, jp, hm * jm);
}

// ------------------------------------------------------------------ packed FP32 pairs
// Pass 1 accumulates in lane pairs so that one packed instruction (two IEEE
// FP32 operations, each rounded as the scalar one) serves two sums:
//   hf[q] = (F^hc_q, F^v_q) per component q, and the friction matrix as
//   G[0] = (xx, yy), G[1] = (zz, xy), G[2] = (xz, yz).
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// accumulate one point with a unit vector s given at run time
__device__ __forceinline__ void add_pass1(float sx, float sy, float sz, float t, float sd, float wn, float2 (&hf)[3],
                                          float2 (&G)[3])
{
    const float2 tsd = f2(t, sd);
    hf[0] = fma2(f2(sx, sx), tsd, hf[0]);
    hf[1] = fma2(f2(sy, sy), tsd, hf[1]);
    hf[2] = fma2(f2(sz, sz), tsd, hf[2]);
    const float2 wxy = mul2(f2(wn, wn), f2(sx, sy));
    const float wz = wn * sz;
    G[0] = fma2(wxy, f2(sx, sy), G[0]);
    G[1] = fma2(f2(wz, wxy.x), f2(sz, sy), G[1]);
    G[2] = fma2(wxy, f2(sz, sz), G[2]);
}

// ------------------------------------------------------------------ neighbours from global memory
// species-b data at r + sign d (n = 0 and u = 0 beyond a wall): n, the
// deviation n - n_ref, the velocity, and the site index (-1 beyond a wall)
struct Nb {
    float dn, n, u0, u1, u2;
    long long q;
};

template <bool INTERIOR>
__device__ __forceinline__ Nb fetch_nb(const mlbi_params &p, const Loc &L, const float4 &e0, const float4 &e1,
                                       int sign, const float4 *__restrict__ fld, float nref)
{
    Nb o;
    o.q = INTERIOR ? L.r + sign * (long long)__float_as_int(e1.x) : nbr(p, L, e0, e1, sign);
    if (INTERIOR || o.q >= 0) {
        const float4 v = fld[o.q];
        o.dn = v.x; o.n = nref + v.x; o.u0 = v.y; o.u1 = v.z; o.u2 = v.w;
    } else {
        o.dn = -nref; o.n = 0.f; o.u0 = 0.f; o.u1 = 0.f; o.u2 = 0.f;
    }
    return o;
}

// ------------------------------------------------------------------ shared-memory tiles (z marching)
// A block of 32 x TY threads owns a 32 x TY column of sites and marches up z
// through `zchunk` planes.  The stencil field of every species (float4: the
// moments in pass 1, (n - n_ref, u*) in pass 2) and the contact-value
// deviations of every pair are staged in shared memory as a ring of planes
// of (32 + 2R) x (TY + 2R) sites: 2R + 1 planes in use and one more being
// filled by cp.async while the current plane is computed.  Every shell
// neighbour is then read from shared memory.
template <int S, int R, int TY_ = kBY>
struct Tile {
    static constexpr int TX = kBX, TY = TY_;
    static constexpr int TXH = TX + 2 * R, TYH = TY + 2 * R, PLANE = TXH * TYH;
    static constexpr int NSLOT = 2 * R + 2;
    static constexpr int NP = S * (S + 1) / 2;
    static constexpr int NT = kBX * TY;
    static constexpr int J = (PLANE + NT - 1) / NT;          // staging sites per thread and plane
    static constexpr size_t bytes = (size_t)NSLOT * PLANE * (S * sizeof(float4) + NP * sizeof(float));
    static_assert(bytes == (size_t)mlbi_tile_bytes(S, R, TY), "tile size formula");
};

// The shell entries of the table-driven reach-3 tiles, staged once per block
// into shared memory after the tile: the union shells' range of the table
// where it fits (one block per SM holds the tile anyway), read there instead
// of through the L1 on every shell point.  Host and device agree on the size.
constexpr int kMaxStagedEntries = 512;
__host__ __device__ inline int shell_entries(const mlbi_params &p, int &lo)
{
    lo = p.ushell_start[0];
    int hi = lo;
    for (int b = 0; b < p.S; ++b) {
        lo = p.ushell_start[b] < lo ? p.ushell_start[b] : lo;
        const int e = p.ushell_start[b] + p.ushell_count[b];
        hi = e > hi ? e : hi;
    }
    return hi - lo;
}
template <class T, int R>
__host__ __device__ inline size_t staged_table_bytes(const mlbi_params &p)
{
    if (R != 3) return 0;
    int lo;
    const int n = shell_entries(p, lo);
    const size_t b = (size_t)n * 2 * sizeof(mlbi_entry);
    return (n <= kMaxStagedEntries && T::bytes + b <= MLBI_MAX_TILE_BYTES) ? b : 0;
}
// copy the entries to dst (visible after the caller's next barrier); returns
// the table the shell loops read
template <class T, int R>
__device__ inline const mlbi_entry *stage_table(const mlbi_params &p, const mlbi_entry *tab, float4 *dst)
{
    if (staged_table_bytes<T, R>(p) == 0) return tab;
    int lo;
    const int n = shell_entries(p, lo);
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int e = tid; e < 2 * n; e += nt) dst[e] = __ldg(&tab[2 * lo + e]);
    return dst - 2 * lo;
}

// resident blocks per SM the tile's shared memory allows (at most `cap`)
constexpr int tile_blocks(size_t bytes, int cap)
{
    const int b = (int)((228 * 1024) / (bytes + 1024));
    return b < 1 ? 1 : (b > cap ? cap : b);
}

// (x, y) offsets x + nx y of this thread's staging sites, fixed while the
// block marches up z; -1 beyond a wall
template <int S, int R, int TY = kBY>
__device__ __forceinline__ void stage_sites(const mlbi_params &p, int x0, int y0, int (&xy)[Tile<S, R, TY>::J])
{
    using T = Tile<S, R, TY>;
    const int tid = threadIdx.y * kBX + threadIdx.x;
#pragma unroll
    for (int j = 0; j < T::J; ++j) {
        const int idx = tid + j * T::NT;
        const int hx = idx % T::TXH, hy = idx / T::TXH;
        const int x = wrap_or_out(x0 - R + hx, p.nx, p.wall_axis == 0);
        const int y = wrap_or_out(y0 - R + hy, p.ny, p.wall_axis == 1);
        xy[j] = (x < 0 || y < 0) ? -1 : x + p.nx * y;
    }
}

// plane index with one periodic wrap (|overhang| <= R < extent), or -1 beyond a wall
__device__ __forceinline__ int wrap_plane(int c, int L, bool wall)
{
    if (wall) return (c < 0 || c >= L) ? -1 : c;
    return c < 0 ? c + L : (c >= L ? c - L : c);
}

// Stage plane gz of the tile into ring slot `slot`.  Sites beyond a wall get
// n = 0 (n - n_ref = -n_ref) and zero velocity; their dg is never used (every
// term carries n(r+d) = 0) and is set to 0.
template <int S, int R, int TY = kBY>
__device__ __forceinline__ void stage_plane(const mlbi_params &p, const int (&xy)[Tile<S, R, TY>::J], int gz,
                                            int slot, const float4 *__restrict__ fld, const float *__restrict__ dg,
                                            float4 *sf, float *sg)
{
    using T = Tile<S, R, TY>;
    const long long N = p.N;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const int z = wrap_plane(gz, p.nz, p.wall_axis == 2);
    const long long zoff = (long long)p.nx * p.ny * z;
#pragma unroll
    for (int j = 0; j < T::J; ++j) {
        const int idx = tid + j * T::NT;
        if (j == T::J - 1 && idx >= T::PLANE) break;
        float4 *df = sf + (size_t)slot * S * T::PLANE + idx;
        float *dgs = sg + (size_t)slot * T::NP * T::PLANE + idx;
        if (xy[j] < 0 || z < 0) {
#pragma unroll
            for (int b = 0; b < S; ++b) df[b * T::PLANE] = make_float4(-p.nref[b], 0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < T::NP; ++q) dgs[q * T::PLANE] = 0.f;
        } else {
            const long long g = zoff + xy[j];
#pragma unroll
            for (int b = 0; b < S; ++b) cp_async16(df + b * T::PLANE, fld + b * N + g);
#pragma unroll
            for (int q = 0; q < T::NP; ++q) cp_async4(dgs + q * T::PLANE, dg + q * N + g);
        }
    }
}

// ------------------------------------------------------------------ the 3x3x3 cube
// The 13 canonical half offsets (first non-zero of (dz, dy, dx) positive).
// With reach 1 every contact shell is a union of the three classes |d|^2 = 1
// (axis), 2 (face diagonal), 3 (corner); the bit of class CL in cube_mask is
// the bit of its first offset.  All compile-time: the class loops unroll and
// the unit vectors become immediates.
__host__ __device__ constexpr int cube_kx(int k) { return k == 0 || k == 3 || k == 6 || k == 9 || k == 12 ? 1 : (k == 1 || k == 4 || k == 7 || k == 10 ? -1 : 0); }
__host__ __device__ constexpr int cube_ky(int k) { return k == 1 || k == 2 || k == 3 || k == 10 || k == 11 || k == 12 ? 1 : (k >= 4 && k <= 6 ? -1 : 0); }
__host__ __device__ constexpr int cube_kz(int k) { return k >= 4 ? 1 : 0; }
__host__ __device__ constexpr int cls_n(int cl) { return cl == 0 ? 3 : (cl == 1 ? 6 : 4); }
__host__ __device__ constexpr int cls_bit(int cl) { return cl == 0 ? 0 : (cl == 1 ? 1 : 4); }
__host__ __device__ constexpr int cls_k(int cl, int i)
{
    return cl == 0 ? (i == 0 ? 0 : (i == 1 ? 2 : 8)) : (cl == 1 ? 2 * i + 1 : (i < 2 ? 4 + 2 * i : 6 + 2 * i));
}
__host__ __device__ constexpr float cls_il(int cl)   // 1/|d|
{
    return cl == 0 ? 1.0f : (cl == 1 ? 0.70710678118654752f : 0.57735026918962576f);
}

// s . v for cube offset K (zero components drop out)
template <int K>
__device__ __forceinline__ float cube_dot(float il, float vx, float vy, float vz)
{
    float r = 0.f;
    if constexpr (cube_kx(K) != 0) r = fmaf(cube_kx(K) * il, vx, r);
    if constexpr (cube_ky(K) != 0) r = fmaf(cube_ky(K) * il, vy, r);
    if constexpr (cube_kz(K) != 0) r = fmaf(cube_kz(K) * il, vz, r);
    return r;
}

template <int K>
__device__ __forceinline__ void cube_add(float il, float t, float (&v)[3])
{
    if constexpr (cube_kx(K) != 0) v[0] = fmaf(cube_kx(K) * il, t, v[0]);
    if constexpr (cube_ky(K) != 0) v[1] = fmaf(cube_ky(K) * il, t, v[1]);
    if constexpr (cube_kz(K) != 0) v[2] = fmaf(cube_kz(K) * il, t, v[2]);
}

// (F^hc, F^v) += s (t, sd) for cube offset K, one packed FMA per non-zero component
template <int K>
__device__ __forceinline__ void cube_add2(float il, float2 tsd, float2 (&hf)[3])
{
    if constexpr (cube_kx(K) != 0) hf[0] = fma2(f2(cube_kx(K) * il, cube_kx(K) * il), tsd, hf[0]);
    if constexpr (cube_ky(K) != 0) hf[1] = fma2(f2(cube_ky(K) * il, cube_ky(K) * il), tsd, hf[1]);
    if constexpr (cube_kz(K) != 0) hf[2] = fma2(f2(cube_kz(K) * il, cube_kz(K) * il), tsd, hf[2]);
}

// G += wn s s^T for cube offset K, G packed as (xx, yy), (zz, xy), (xz, yz);
// a pair with one zero entry is a scalar FMA on the other lane
template <int K>
__device__ __forceinline__ void cube_add_ss(float il, float wn, float2 (&G)[3])
{
    constexpr int X = cube_kx(K), Y = cube_ky(K), Z = cube_kz(K);
    const float i2 = il * il;
    if constexpr (X != 0 && Y != 0) G[0] = fma2(f2(wn, wn), f2(i2, i2), G[0]);
    else if constexpr (X != 0) G[0].x = fmaf(wn, i2, G[0].x);
    else if constexpr (Y != 0) G[0].y = fmaf(wn, i2, G[0].y);
    if constexpr (Z != 0 && X * Y != 0) G[1] = fma2(f2(wn, wn), f2(i2, X * Y * i2), G[1]);
    else if constexpr (Z != 0) G[1].x = fmaf(wn, i2, G[1].x);
    else if constexpr (X * Y != 0) G[1].y = fmaf(wn, X * Y * i2, G[1].y);
    if constexpr (X * Z != 0 && Y * Z != 0) G[2] = fma2(f2(wn, wn), f2(X * Z * i2, Y * Z * i2), G[2]);
    else if constexpr (X * Z != 0) G[2].x = fmaf(wn, X * Z * i2, G[2].x);
    else if constexpr (Y * Z != 0) G[2].y = fmaf(wn, Y * Z * i2, G[2].y);
}

// compile-time loop: f(std::integral_constant<int, I>) for I = 0 .. N-1
template <int I, int N, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(f);
    }
}

}  // namespace

#define MLBI_DISPATCH_S(...)                                                                       \
    switch (p.S) {                                                                                 \
    case 1: { constexpr int SS = 1; __VA_ARGS__; } break;                                          \
    case 2: { constexpr int SS = 2; __VA_ARGS__; } break;                                          \
    case 3: { constexpr int SS = 3; __VA_ARGS__; } break;                                          \
    case 4: { constexpr int SS = 4; __VA_ARGS__; } break;                                          \
    default: return cudaErrorInvalidValue;                                                         \
    }
