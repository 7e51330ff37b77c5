// mlb_kernels.cu -- sm_103a kernels of the multispecies Enskog/RPA lattice
// Boltzmann step (arXiv:1105.3634, Secs. II-III and V).
//
// Storage (structure of arrays, x fastest, site r = x + nx (y + ny z)):
//   f[a][i][r]  FP32 populations minus w_i n_ref^a      (76 B per species-site)
//   mom[a][r]   float4 (n - n_ref, u_x, u_y, u_z)        (16 B per species-site)
//   dg[p][r]    g_ab - g_ab(reference densities)          (per unordered pair)
//   frest[a][r] F^hc + G + F_ext                          (pass 1 -> pass 2)
//   pst[a][r]   (n - n_ref, u* = u + du)                  (pass 1 -> pass 2)
//
// One step (all launches on one stream):
//   k_moments        f -> mom                                    (Eq. colonna)
//   k_gfield         mom -> dg: smoothed densities, BMCSL g       (Sec. II smoothing)
//   (k_moments_g     the two above in one pass when g is site-local)
//   k_pass1          mom, dg -> frest, pst: hard core + attraction  (Eqs. potmeanforce, gammaab,
//                    + velocity exchange at u, then the one-sweep    viscousforce)
//                    half-step predictor
//   k_pass2          velocity exchange at u* = u + du -> acc
//   k_collide        collision toward psi_perp at u + a/2 with      (Eqs. evolution, prefactor)
//                    (1 - omega/2) forcing, push streaming /
//                    halfway bounce-back
// Deviations from reference values (n - n_ref, g - g_ref) and velocities
// (rather than momenta) keep the FP32 differences that the contact sums take
// between neighbouring sites small and exact.
#include "mlb_internal.h"
#include "mlb_device.cuh"
#include "mlb_collide.cuh"
#include "mlb_popsum.cuh"

#include <math.h>

namespace {
// FP64 global sums of the state, taken while the moments are computed
// (SUMS, the monitored step): mass sum_r dn^a (n_ref N is added at the end)
// and momentum sum_a sum_r j^a of the step's own FP32 site moments.  A thread
// adds its sites in groups of 8 in FP32 and accumulates the groups in FP64,
// so the FP64 pipe, slow on this part, does an eighth of the additions.  A
// group's FP32 sum is off by at most 7 x 2^-24 times the sum of its terms'
// magnitudes, so the total is within 7 x 2^-24 sum_r |dn^a| (mass) and
// 7 x 2^-24 sum_a sum_r |j^a| (each momentum component) of the FP64 sum of
// the same site moments.  mlb_conservation sums the populations themselves
// in FP64 (mlb_popsum.cuh).  The block sums go to partial[block][S + 3] for
// k_conservation_final.
template <int S>
struct ConsSums {
    static constexpr int W = S + 3, G = 8;
    double acc[W];
    float part[W];
    int cnt = 0;
    bool bad = false;
    __device__ __forceinline__ ConsSums()
    {
#pragma unroll
        for (int k = 0; k < W; ++k) acc[k] = 0.0, part[k] = 0.f;
    }
    __device__ __forceinline__ void add(const float (&dn)[S], const float (&u)[S][3], const float (&j)[S][3])
    {
#pragma unroll
        for (int a = 0; a < S; ++a) {
            bad |= !isfinite(dn[a]) || !isfinite(u[a][0]) || !isfinite(u[a][1]) || !isfinite(u[a][2]);
            part[a] += dn[a];
            part[S + 0] += j[a][0];
            part[S + 1] += j[a][1];
            part[S + 2] += j[a][2];
        }
        if (++cnt == G) flush();
    }
    __device__ __forceinline__ void flush()
    {
#pragma unroll
        for (int k = 0; k < W; ++k) acc[k] += (double)part[k], part[k] = 0.f;
        cnt = 0;
    }
    // one tree over the block for all W sums at once (independent FP64 adds per level)
    __device__ __forceinline__ void store(double *__restrict__ partial, unsigned int *__restrict__ flags)
    {
        flush();
        if (bad) atomicOr(flags, MLBI_FLAG_NAN);
        __shared__ double sh[W][kBlock];
#pragma unroll
        for (int k = 0; k < W; ++k) sh[k][threadIdx.x] = acc[k];
        __syncthreads();
        for (int s = kBlock / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s)
#pragma unroll
                for (int k = 0; k < W; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x < W) partial[blockIdx.x * W + threadIdx.x] = sh[threadIdx.x][0];
    }
};

template <int S, bool SUMS>
__global__ void __launch_bounds__(kBlock) k_moments(const mlbi_params p, const float *__restrict__ f,
                                                    float4 *__restrict__ mom, double *__restrict__ partial,
                                                    unsigned int *__restrict__ flags)
{
    const long long N = p.N;
    ConsSums<S> cs;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        float dn[S], u[S][3], j[S][3];
        site_moments<S>(p, GlobalPops{f + r, N}, dn, u, j);
#pragma unroll
        for (int a = 0; a < S; ++a) mom[a * N + r] = make_float4(dn[a], u[a][0], u[a][1], u[a][2]);
        if constexpr (SUMS) cs.add(dn, u, j);
    }
    if constexpr (SUMS) cs.store(partial, flags);
}

// ------------------------------------------------------------------ contact values
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

// ------------------------------------------------------------------ moments with local contact values
// When every smoothing ball is the single site (kappa sigma < 1), g_ab at r
// depends on the moments at r only: one pass over f gives both.
// the sites of block `blk` of `nblk` (grid-stride)
template <int S, bool SUMS>
__device__ __forceinline__ void moments_g_blocks(const mlbi_params &p, const float *__restrict__ f,
                                                 float4 *__restrict__ mom, float *__restrict__ dg,
                                                 unsigned int *__restrict__ flags, double *__restrict__ partial,
                                                 long long blk, long long nblk)
{
    constexpr int NP = S * (S + 1) / 2;
    const long long N = p.N;
    ConsSums<S> cs;
    for (long long r = blk * blockDim.x + threadIdx.x; r < N; r += nblk * blockDim.x) {
        float dn[S], u[S][3], j[S][3], dgv[NP];
        site_moments<S>(p, GlobalPops{f + r, N}, dn, u, j);
#pragma unroll
        for (int a = 0; a < S; ++a) mom[a * N + r] = make_float4(dn[a], u[a][0], u[a][1], u[a][2]);
        if (!site_contact<S>(p, dn, dgv)) atomicOr(flags, MLBI_FLAG_XI3);
#pragma unroll
        for (int q = 0; q < NP; ++q) dg[q * N + r] = dgv[q];
        if constexpr (SUMS) cs.add(dn, u, j);
    }
    if constexpr (SUMS) cs.store(partial, flags);
}

template <int S, bool SUMS>
__global__ void __launch_bounds__(kBlock) k_moments_g(const mlbi_params p, const float *__restrict__ f,
                                                      float4 *__restrict__ mom, float *__restrict__ dg,
                                                      unsigned int *__restrict__ flags, double *__restrict__ partial)
{
    moments_g_blocks<S, SUMS>(p, f, mom, dg, flags, partial, blockIdx.x, gridDim.x);
}

// every member of a group: block table entries {member, block, blocks of the member, 0}
template <int S>
__global__ void __launch_bounds__(kBlock) k_moments_g_group(const mlbi_member *__restrict__ mem,
                                                            const int4 *__restrict__ blk, int odd)
{
    __shared__ mlbi_params sp;
    const int4 e = blk[blockIdx.x];
    const mlbi_member *m = mem + e.x;
    group_params(m, sp);
    const mlbi_buffers &b = m->b;
    moments_g_blocks<S, false>(sp, b.f[m->cur ^ odd], b.mom, b.dg, b.flags, nullptr, e.y, e.z);
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
    collide_push<S>(p, L.x, L.y, L.z, r, c, acc, GlobalPops{fin + r, N}, fout);
}

// ------------------------------------------------------------------ initial populations
// (one FP64 reciprocal per site: FP64 division is slow on this part)
template <int S>
__global__ void __launch_bounds__(kBlock) k_init(mlbi_params p, const double *__restrict__ nin,
                                                 const double *__restrict__ uin, float *__restrict__ f)
{
    const long long N = p.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < S; ++a) {
            double na = nin[a * N + r];
            rho += na;
            if (uin)
#pragma unroll
                for (int q = 0; q < 3; ++q) m[q] += na * uin[(a * 3 + q) * N + r];
        }
        const double irho = rho > 0.0 ? 1.0 / rho : 0.0;
        float ub[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) ub[q] = (float)(m[q] * irho);
        const float ubub = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
#pragma unroll
        for (int a = 0; a < S; ++a) {
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
// Sum of the block partials: two per thread, then one tree over 512 threads
// for all sums at once (FP64 adds are slow on this part: a 1024-long
// dependent chain costs ~0.25 ms, the tree 10 levels).
constexpr int kFinalThreads = 512;
__global__ void __launch_bounds__(kFinalThreads) k_conservation_final(mlbi_params p, const double *__restrict__ partial,
                                                                     int nblocks, double *__restrict__ sums)
{
    constexpr int WMAX = MLBI_MAXS + 3;
    const int W = p.S + 3;
    __shared__ double sh[WMAX][kFinalThreads];
    for (int k = 0; k < W; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += partial[b * W + k];
        sh[k][threadIdx.x] = v;
    }
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < W; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < W)       // mass = N n_ref + sum dn
        sums[threadIdx.x] = sh[threadIdx.x][0] + (threadIdx.x < p.S ? (double)p.nref[threadIdx.x] * (double)p.N : 0.0);
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

cudaError_t mlbi_launch_moments(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s, bool sums)
{
    if (sums) {
        MLBI_DISPATCH_S((k_moments<SS, true><<<MLBI_RED_BLOCKS, kBlock, 0, s>>>(p, b.f[cur], b.mom, b.partial,
                                                                                b.flags)));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_conservation_final<<<1, kFinalThreads, 0, s>>>(p, b.partial, MLBI_RED_BLOCKS, b.sums);
        return cudaGetLastError();
    }
    MLBI_DISPATCH_S((k_moments<SS, false><<<grid_for(p.N), kBlock, 0, s>>>(p, b.f[cur], b.mom, nullptr, nullptr)));
    return cudaGetLastError();
}


cudaError_t mlbi_launch_gfield(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    k_gfield<<<tiled_grid(p), dim3(kBX, kBY), 0, s>>>(p, b.mom, b.table, b.dg, b.flags);
    return cudaGetLastError();
}

namespace {
__global__ void __launch_bounds__(kBlock) k_export_vec(mlbi_params p, const float4 *__restrict__ src,
                                                       double *__restrict__ dst)
{
    const long long N = p.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x)
        for (int a = 0; a < p.S; ++a) {
            const float4 v = src[a * N + r];
            dst[(a * 3 + 0) * N + r] = v.x;
            dst[(a * 3 + 1) * N + r] = v.y;
            dst[(a * 3 + 2) * N + r] = v.z;
        }
}
}  // namespace

cudaError_t mlbi_launch_export_vec(const mlbi_params &p, const float4 *src, double *dst, cudaStream_t s)
{
    k_export_vec<<<grid_for(p.N), kBlock, 0, s>>>(p, src, dst);
    return cudaGetLastError();
}

cudaError_t mlbi_launch_moments_g(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s, bool sums)
{
    if (sums) {
        MLBI_DISPATCH_S((k_moments_g<SS, true><<<MLBI_RED_BLOCKS, kBlock, 0, s>>>(p, b.f[cur], b.mom, b.dg, b.flags,
                                                                                  b.partial)));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_conservation_final<<<1, kFinalThreads, 0, s>>>(p, b.partial, MLBI_RED_BLOCKS, b.sums);
        return cudaGetLastError();
    }
    MLBI_DISPATCH_S((k_moments_g<SS, false><<<grid_for(p.N), kBlock, 0, s>>>(p, b.f[cur], b.mom, b.dg, b.flags,
                                                                             nullptr)));
    return cudaGetLastError();
}

struct V3 {
    double v[MLBI_MAXS];
};

// the checks and sums of mlbi_launch_field_check; block sums to
// partial[block][S + 3] (the last three zero) for k_conservation_final
template <int S>
__global__ void __launch_bounds__(kBlock) k_field_check(long long N, const double *__restrict__ n,
                                                        const double *__restrict__ u, V3 v3,
                                                        double *__restrict__ partial,
                                                        unsigned long long *__restrict__ bad)
{
    constexpr int W = S + 3;
    constexpr unsigned long long kNone = ~0ull;
    double sum[S];
#pragma unroll
    for (int a = 0; a < S; ++a) sum[a] = 0.0;
    unsigned long long b_n = kNone, b_xi = kNone, b_u = kNone;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x) {
        double xi3 = 0.0;
#pragma unroll
        for (int a = 0; a < S; ++a) {
            const double v = n[a * N + r];
            if (!(isfinite(v) && v >= 0.0)) b_n = min(b_n, (unsigned long long)(a * N + r));
            sum[a] += v;
            xi3 += v3.v[a] * v;
        }
        if (!(xi3 < 1.0)) b_xi = min(b_xi, (unsigned long long)r);
        if (u) {
#pragma unroll
            for (int k = 0; k < 3 * S; ++k) {
                const double w = u[k * N + r];
                if (!(isfinite(w) && fabs(w) < 1.0)) b_u = min(b_u, (unsigned long long)(k * N + r));
            }
        }
    }
    if (b_n != kNone) atomicMin(&bad[0], b_n);
    if (b_xi != kNone) atomicMin(&bad[1], b_xi);
    if (b_u != kNone) atomicMin(&bad[2], b_u);
    __shared__ double sh[S][kBlock];
#pragma unroll
    for (int a = 0; a < S; ++a) sh[a][threadIdx.x] = sum[a];
    __syncthreads();
    for (int h = kBlock / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
#pragma unroll
            for (int a = 0; a < S; ++a) sh[a][threadIdx.x] += sh[a][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x < W) partial[blockIdx.x * W + threadIdx.x] = threadIdx.x < S ? sh[threadIdx.x][0] : 0.0;
}

__global__ void __launch_bounds__(kBlock) k_gather_flags(const unsigned int *const *__restrict__ flags, int n,
                                                         unsigned int *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = *flags[i];
}

cudaError_t mlbi_launch_gather_flags(const unsigned int *const *flags, int n, unsigned int *out, cudaStream_t s)
{
    if (n < 1) return cudaErrorInvalidValue;
    k_gather_flags<<<(n + kBlock - 1) / kBlock, kBlock, 0, s>>>(flags, n, out);
    return cudaGetLastError();
}

cudaError_t mlbi_launch_group_moments(const mlbi_group &g, int odd, cudaStream_t s)
{
    if (g.nblk[MLBI_GROUP_MOMENTS] < 1) return cudaErrorInvalidValue;
    const unsigned nb = (unsigned)g.nblk[MLBI_GROUP_MOMENTS];
    const int4 *blk = g.blk[MLBI_GROUP_MOMENTS];
    switch (g.S) {
    case 1: k_moments_g_group<1><<<nb, kBlock, 0, s>>>(g.mem, blk, odd); break;
    case 2: k_moments_g_group<2><<<nb, kBlock, 0, s>>>(g.mem, blk, odd); break;
    case 3: k_moments_g_group<3><<<nb, kBlock, 0, s>>>(g.mem, blk, odd); break;
    case 4: k_moments_g_group<4><<<nb, kBlock, 0, s>>>(g.mem, blk, odd); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t mlbi_launch_field_check(const mlbi_params &p, const mlbi_buffers &b, const double *n, const double *u,
                                    const double *v3, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(b.first_bad, 0xFF, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    V3 w{};
    for (int a = 0; a < p.S && a < MLBI_MAXS; ++a) w.v[a] = v3[a];
    MLBI_DISPATCH_S((k_field_check<SS><<<MLBI_RED_BLOCKS, kBlock, 0, s>>>(p.N, n, u, w, b.partial, b.first_bad)));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the partials are sums of n itself: no N n_ref term to add
    mlbi_params q = p;
    for (int a = 0; a < MLBI_MAXS; ++a) q.nref[a] = 0.f;
    k_conservation_final<<<1, kFinalThreads, 0, s>>>(q, b.partial, MLBI_RED_BLOCKS, b.sums);
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
    MLBI_DISPATCH_S((k_init<SS><<<grid_for(p.N), kBlock, 0, s>>>(p, n, u, b.f[cur])));
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


cudaError_t mlbi_launch_pop_sums(const mlbi_params &p, const mlbi_buffers &b, int cur, cudaStream_t s)
{
    mlbps::Nref nr{};
    for (int a = 0; a < p.S; ++a) nr.v[a] = (double)p.nref[a];
    return mlbps::launch_pop_sums(b.f[cur], p.S, p.N, nr, b.partial, b.sums, s);
}
