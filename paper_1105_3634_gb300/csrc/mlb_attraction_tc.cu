// mlb_attraction_tc.cu -- the attractive mean field of the RPA (Sec. III, G
// term of Eq. potmeanforce) as an implicit GEMM on the tcgen05 tensor cores,
// BF16 operands split hi + lo, FP32 accumulation in tensor memory.
//
// G^a(r) = sum_b sum_d K_ab(d) n^b(r + d),  K_ab(d) = 6 eps_ab sigma_ab^6 d / |d|^8
// on sigma_ab <= |d| <= lambda_c sigma_ab (n may be the deviation n - n_ref: K is odd).
//
// For one column shift (dx, dy) of the region the sum along z is a band
// (Toeplitz) matrix product.  A sub-tile is 128 consecutive x sites of one
// row y and 16 planes z0 .. z0 + 15:
//   D[x][(a, c, z)] += sum_{(b, z')} A_{dx,dy}[x][(b, z')] B_{dx,dy}[(b, z')][(a, c, z)]
//   A_{dx,dy}[x][(b, z')] = n^b(x + dx, y + dy, z'),   z' = z0 - 8 .. z0 + 23
//   B_{dx,dy}[(b, z')][(a, c, z)] = K_ab(dx, dy, z' - z)_c   (zero off the region)
// M = 128 sites, N = 3 S 16 outputs, K = 32 S.  B depends on z' - z only, so
// a tile holds kSub = 2 sub-tiles (32 planes) whose MMAs share every
// column's B; the second sub-tile's A is the same staged row 16 planes on.
// A is staged per row y + dy in a K-major layout [8-value chunk][x'][8 values]
// holding x' = x0 - 8 .. x0 + 135 and z' = z0 - 8 .. z0 + 39, so the x shift
// dx of a column is the same operand with its descriptor start moved by 16 dx
// bytes, and the sub-tile's z shift by two chunks.  B (hi and lo) is precomputed per column on the host
// (24 KB for S = 2) and streamed from L2 by bulk copies.  The compensated
// product is A_hi B_hi + A_hi B_lo + A_lo B_hi (three MMAs per K step; the
// single-product form A_hi B_hi is a flag).
//
// The densities are first copied (k_attraction_prep) into BF16 hi and lo
// arrays [yp][b][z / 8][xp][8 planes] padded by 8 sites on both sides in x
// and y (the periodic images, or -n_ref beyond a wall) and in x up to whole
// tiles, so one row's chunk (b, 8 planes) for the 144 staged sites is 2304
// contiguous bytes in exactly the staged layout: one in-bounds bulk copy.
//
// Warp roles (one CTA per SM, persistent over tiles):
//   warp 0      bulk-copies the columns' B into a ring of kStages slots
//   warp 1      issues the MMAs of a column once its B and its row's A are in,
//               commits them to the slot's and the row's "empty" barriers
//   warp 2      copies the A rows (2 S 6 bulk copies per row, hi and lo)
//   warps 3-10  after every dy row, read that row's accumulator (a lane
//               quarter of one sub-tile each) and add it to the sub-tile's
//               sums in registers (FP32, round to nearest), then store G
//               after the tile's last row
// Each dy row has an accumulator of its own per sub-tile (two rows in turn:
// all 512 tensor-memory columns): the tensor pipe's FP32 accumulation then
// runs over about 140 MMAs instead of the tile's ~2100, and the rows are
// added on the CUDA cores.
// Every wait is bounded; one that gives up sets an abort flag every role
// checks, and the kernel reports it through flags (MLB_ETIMEOUT).
#include "mlb_internal.h"
#include "mlb_device.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace {

constexpr int kTM = 128;                 // sites per tile (TMEM lanes)
constexpr int kTZ = 16;                  // planes per sub-tile (one accumulator, N = 48 S)
constexpr int kSub = 2;                  // z sub-tiles per tile: each column's B serves both
constexpr int kWin = 32;                 // planes of one sub-tile's window (K = 32 S)
constexpr int kAwin = kWin + (kSub - 1) * kTZ;   // staged planes z0 - 8 .. z0 + 39
constexpr int kXW = kTM + 16;            // staged sites x0 - 8 .. x0 + 135
constexpr int kStages = 4;               // B ring slots (the copies' look-ahead: 4 columns of MMAs)
constexpr int kEpiWarps = 4 * kSub;      // warps 3 .. 10: a lane quarter of one sub-tile each
constexpr int kThreads = 96 + 32 * kEpiWarps;
constexpr int kEpi = 32 * kEpiWarps;
constexpr int kPad = 8;                  // halo of the padded density copies
constexpr uint32_t kAccCols = 128;       // columns per accumulator (N <= 96 used)
constexpr int kMaxCols = 17 * 17;        // columns of a reach-8 region
constexpr int kMaxRows = 17;

struct TcArgs {
    int nx, ny, nz, S, wall_axis;
    int nxp, nyp;                        // padded extents of the density copies
    long long N;
    int ncols;                           // columns, sorted by dy then dx
    int nrows;                           // distinct dy among them
    int pass3;                           // 1: hi/lo compensated, 0: A_hi B_hi only
};

template <int S>
struct Shape {
    static constexpr int N = 3 * S * kTZ;                    // outputs per site
    static constexpr int K = kWin * S;                       // (species, plane) values
    static constexpr int KC = K / 8;                         // 16-byte chunks along K
    static constexpr int AC = kAwin / 8 * S;                 // staged 16-byte chunks of A (kAwin planes)
    static constexpr uint32_t a_bytes = (uint32_t)AC * kXW * 16;            // one staged row, hi or lo
    static constexpr uint32_t b_bytes = (uint32_t)KC * N * 16;              // one column's B, hi or lo
    static constexpr uint32_t col_bytes = 2 * b_bytes;                      // hi + lo
    // instruction descriptor (kind::f16): D FP32, A and B BF16, both K-major,
    // N >> 3 at bits 17-22, M >> 4 at bits 24-28
    static constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                                      ((uint32_t)(kTM >> 4) << 24);
    static constexpr size_t smem = 2 * 2 * (size_t)a_bytes + kStages * (size_t)col_bytes + 1024;
};

__device__ __forceinline__ uint64_t mdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    // start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4 (32-45), fixed 0b001 at
    // 46-48, base offset 0, no swizzle
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// bounded wait on phase `parity` of an mbarrier; false once `abort` is set or the limit is reached
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int *abort)
{
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(parity)
                     : "memory");
        if (done) return true;
        if (*abort) return false;
    }
    *abort = 1;
    return false;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                 : "memory");
}

__device__ __forceinline__ void commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// tile t -> (x0, y, z0)
__device__ __forceinline__ void tile_of(const TcArgs &g, long long t, int &x0, int &y, int &z0)
{
    const int nxt = (g.nx + kTM - 1) / kTM, nzt = (g.nz + kSub * kTZ - 1) / (kSub * kTZ);
    x0 = (int)(t % nxt) * kTM;
    const long long r = t / nxt;
    y = (int)(r % g.ny);
    z0 = (int)(r / g.ny % nzt) * (kSub * kTZ);
}

// Tensor-memory reads of the epilogue: 16 consecutive accumulator columns of
// the warp's 32 lanes into v, without waiting; tmem_wait waits for the
// thread's loads and only then lets v's registers be read (the empty asm
// statements order every later use of v after the wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait(uint32_t (&v)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) asm volatile("" : "+r"(v[i]));
}
// sum[c] += accumulator column c for the NC columns of one row (chunks of 16,
// the next chunk's load in flight while the current one is added)
template <int NC>
__device__ __forceinline__ void add_row(float (&sum)[NC], uint32_t taddr)
{
    constexpr int NCH = NC / 16;
    uint32_t v[2][16];
    tmem_ld16(taddr, v[0]);
    tmem_wait(v[0]);
#pragma unroll
    for (int i = 0; i < NCH; ++i) {
        if (i + 1 < NCH) tmem_ld16(taddr + 16 * (i + 1), v[(i + 1) & 1]);
#pragma unroll
        for (int k = 0; k < 16; ++k) sum[16 * i + k] += __uint_as_float(v[i & 1][k]);
        if (i + 1 < NCH) tmem_wait(v[(i + 1) & 1]);
    }
}

template <int S>
__global__ void __launch_bounds__(kThreads, 1)
    k_attraction_tc(const TcArgs g, const uint4 *__restrict__ qhi, const uint4 *__restrict__ qlo,
                    const uint4 *__restrict__ wts,
                    const int2 *__restrict__ cols, const int *__restrict__ row_start, float4 *__restrict__ attr,
                    unsigned int *__restrict__ flags)
{
    using Sh = Shape<S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[2 * kStages + 2 + 2 + 2 + 2 + 1];
    __shared__ uint32_t tmem_slot;
    __shared__ int s_abort;
    // the column table, read on the MMA thread's critical path: in shared memory
    __shared__ int s_dx[kMaxCols];
    __shared__ int s_rows[kMaxRows + 1], s_dy[kMaxRows];
    const uint32_t base = (smem_u32(smem_raw) + 127u) & ~127u;
    const uint32_t a_base = base;                                    // [2 slots][hi, lo][a_bytes]
    const uint32_t w_base = base + 4 * Sh::a_bytes;                  // [kStages][hi, lo][b_bytes]
    const uint32_t b_full = smem_u32(&bars[0]), b_empty = b_full + 8 * kStages;
    const uint32_t a_full = b_empty + 8 * kStages, a_empty = a_full + 16;
    const uint32_t d_full = a_empty + 16, d_empty = d_full + 16, drain = d_empty + 16;
    volatile int *abort = &s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int c = tid; c < g.ncols; c += kThreads) s_dx[c] = cols[c].x;
    for (int r = tid; r <= g.nrows; r += kThreads) {
        s_rows[r] = row_start[r];
        if (r < g.nrows) s_dy[r] = cols[row_start[r]].y;
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(b_full + 8 * s, 1);
            mbar_init(b_empty + 8 * s, 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(a_full + 8 * s, 1);
            mbar_init(a_empty + 8 * s, 1);
            mbar_init(d_full + 8 * s, 1);
            mbar_init(d_empty + 8 * s, kEpi);
        }
        mbar_init(drain, 1);
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(2 * kSub * kAccCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    const int nxt = (g.nx + kTM - 1) / kTM, nzt = (g.nz + kSub * kTZ - 1) / (kSub * kTZ);
    const long long ntiles = (long long)nxt * g.ny * nzt;

    if (warp == 0) {
        // ---- B producer
        if (lane == 0) {
            uint32_t k = 0;                                          // columns issued so far
            for (long long t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x)
                for (int c = 0; c < g.ncols && !*abort; ++c) {
                    const uint32_t s = k % kStages;
                    if (k >= kStages && !wait_or_abort(b_empty + 8 * s, ((k / kStages) - 1) & 1, abort)) break;
                    // the single-product form reads the hi half only
                    const uint32_t bytes = g.pass3 ? Sh::col_bytes : Sh::b_bytes;
                    mbar_expect_tx(b_full + 8 * s, bytes);
                    bulk_load(w_base + s * Sh::col_bytes, wts + (size_t)c * (Sh::col_bytes / 16), bytes,
                              b_full + 8 * s);
                    ++k;
                }
            // no copy may still be writing into this CTA's shared memory when it
            // exits: wait (bounded) for the last copy of every slot
            if (*abort)
                for (uint32_t j = k > kStages ? k - kStages : 0; j < k; ++j)
                    mbar_wait(b_full + 8 * (j % kStages), (j / kStages) & 1);
        }
    } else if (warp == 1) {
        // ---- MMA issuer
        if (lane == 0) {
            uint32_t k = 0, r = 0;
            for (long long t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
                for (int row = 0; row < g.nrows && !*abort; ++row, ++r) {
                    const uint32_t as = r & 1, buf = r & 1;
                    // the row's accumulator: free once the epilogue read it two rows ago
                    if (r >= 2 && !wait_or_abort(d_empty + 8 * buf, ((r / 2) - 1) & 1, abort)) break;
                    if (!wait_or_abort(a_full + 8 * as, (r / 2) & 1, abort)) break;
                    const uint32_t d = tmem + buf * kSub * kAccCols;      // sub-tile s at d + s kAccCols
                    uint32_t acc = 0;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a_hi = a_base + as * 2 * Sh::a_bytes, a_lo = a_hi + Sh::a_bytes;
                    for (int c = s_rows[row]; c < s_rows[row + 1]; ++c, ++k) {
                        const uint32_t s = k % kStages;
                        if (!wait_or_abort(b_full + 8 * s, (k / kStages) & 1, abort)) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const int dx = s_dx[c];
                        const uint32_t b_hi = w_base + s * Sh::col_bytes, b_lo = b_hi + Sh::b_bytes;
                        const uint64_t ah = mdesc(a_hi + (uint32_t)(8 + dx) * 16, kXW * 16, 128);
                        const uint64_t al = mdesc(a_lo + (uint32_t)(8 + dx) * 16, kXW * 16, 128);
                        const uint64_t bh = mdesc(b_hi, Sh::N * 16, 128), bl = mdesc(b_lo, Sh::N * 16, 128);
                        // K step q: species q / 2, planes 16 (q % 2) .. + 15 of the
                        // sub-tile's window, which starts 2 s chunks into the staged row
#pragma unroll
                        for (int q = 0; q < Sh::K / 16; ++q) {
                            const uint64_t bo = (uint64_t)((q * 2 * Sh::N * 16) >> 4);
#pragma unroll
                            for (int sub = 0; sub < kSub; ++sub) {
                                const int chunk = (q / 2) * (kAwin / 8) + 2 * (q % 2) + 2 * sub;
                                const uint64_t ao = (uint64_t)((chunk * kXW * 16) >> 4);
                                const uint32_t ds = d + sub * kAccCols;
                                mma(ds, ah + ao, bh + bo, Sh::idesc, acc);
                                if (g.pass3) {
                                    mma(ds, ah + ao, bl + bo, Sh::idesc, 1);
                                    mma(ds, al + ao, bh + bo, Sh::idesc, 1);
                                }
                            }
                            acc = 1;
                        }
                        commit(b_empty + 8 * s);                     // the slot is free once these finish
                    }
                    commit(a_empty + 8 * as);                        // the row is free once its MMAs finish
                    commit(d_full + 8 * buf);                        // the row's sum is ready
                }
            }
            // let every MMA issued so far finish before the teardown (bounded)
            if (*abort) {
                commit(drain);
                mbar_wait(drain, 0);
            }
        }
    } else if (warp == 2) {
        // ---- A producer: per row, 2 S 6 bulk copies of [144 sites][8 planes]
        if (lane == 0) {
            const uint32_t row_bytes = (g.pass3 ? 2u : 1u) * Sh::a_bytes;
            const int nzc = g.nz / 8;
            uint32_t r = 0;
            for (long long t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
                int x0, y, z0;
                tile_of(g, t, x0, y, z0);
                for (int row = 0; row < g.nrows && !*abort; ++row, ++r) {
                    const uint32_t as = r & 1;
                    if (r >= 2 && !wait_or_abort(a_empty + 8 * as, ((r / 2) - 1) & 1, abort)) break;
                    const uint32_t a_hi = a_base + as * 2 * Sh::a_bytes;
                    const int yp = y + s_dy[row] + kPad;
                    mbar_expect_tx(a_full + 8 * as, row_bytes);
                    for (int b = 0; b < S; ++b)
                        for (int j = 0; j < kAwin / 8; ++j) {
                            int zc = (z0 - 8) / 8 + j;                  // z0 is a multiple of 32, nz of 8
                            zc = ((zc % nzc) + nzc) % nzc;
                            const uint32_t dst = a_hi + (uint32_t)((b * (kAwin / 8) + j) * kXW) * 16;
                            const size_t e0 = (((size_t)yp * S + b) * nzc + zc) * g.nxp + x0;
                            bulk_load(dst, qhi + e0, kXW * 16, a_full + 8 * as);
                            if (g.pass3) bulk_load(dst + Sh::a_bytes, qlo + e0, kXW * 16, a_full + 8 * as);
                        }
                }
            }
            // no copy may still be writing into this CTA's shared memory when it exits
            if (*abort)
                for (uint32_t q = r > 2 ? r - 2 : 0; q < r; ++q) mbar_wait(a_full + 8 * (q & 1), (q / 2) & 1);
        }
    } else {
        // ---- epilogue (warps 3..10: TMEM lanes 32 (warp % 4) .. of sub-tile
        // (warp - 3) / 4); every decision is warp-uniform (__all_sync), so
        // the .sync.aligned tensor-memory loads always run with the whole warp
        uint32_t r = 0;
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
        const int sub = (warp - 3) / 4;
        bool stop = false;
        for (long long t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
            float sum[S * 3 * kTZ];
#pragma unroll
            for (int q = 0; q < S * 3 * kTZ; ++q) sum[q] = 0.f;
            for (int row = 0; row < g.nrows; ++row, ++r) {
                const uint32_t buf = r & 1;
                if (!__all_sync(0xffffffffu, wait_or_abort(d_full + 8 * buf, (r / 2) & 1, abort))) {
                    stop = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t taddr = tmem + (buf * kSub + sub) * kAccCols + lanes;
                add_row<S * 3 * kTZ>(sum, taddr);
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(d_empty + 8 * buf);
            }
            if (stop) break;
            int x0, y, z0;
            tile_of(g, t, x0, y, z0);
            z0 += sub * kTZ;
            const int x = x0 + (warp & 3) * 32 + lane;
            if (x < g.nx) {
#pragma unroll
                for (int a = 0; a < S; ++a)
#pragma unroll
                    for (int z = 0; z < kTZ; ++z)
                        if (z0 + z < g.nz)
                            attr[a * g.N + x + (long long)g.nx * (y + (long long)g.ny * (z0 + z))] =
                                make_float4(sum[(a * 3 + 0) * kTZ + z], sum[(a * 3 + 1) * kTZ + z],
                                            sum[(a * 3 + 2) * kTZ + z], 0.f);
            }
        }
    }
    __syncthreads();
    if (*abort && tid == 0) atomicOr(flags, MLBI_FLAG_TIMEOUT);
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kSub * kAccCols)
                     : "memory");
    }
}

// n - n_ref of every species as BF16 hi + lo (hi = RN(v), lo = RN(v - hi)) in
// the padded layout [yp][b][z / 8][xp][8 planes] the bulk copies read: site
// (xp - 8, yp - 8) wrapped periodically, or -n_ref beyond a wall; one thread
// per (xp, 8 planes, b, yp), consecutive threads at consecutive xp
__global__ void __launch_bounds__(256) k_attraction_prep(const mlbi_params p, int nxp, int nyp,
                                                         const float4 *__restrict__ mom, uint4 *__restrict__ qhi,
                                                         uint4 *__restrict__ qlo)
{
    const int nzc = p.nz / 8;
    const long long total = (long long)nxp * nyp * p.S * nzc;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int xp = (int)(e % nxp);
        long long rest = e / nxp;
        const int zc = (int)(rest % nzc);
        rest /= nzc;
        const int b = (int)(rest % p.S), yp = (int)(rest / p.S);
        const int xg = xp - kPad, yg = yp - kPad;
        const bool out = (p.wall_axis == 0 && (xg < 0 || xg >= p.nx)) || (p.wall_axis == 1 && (yg < 0 || yg >= p.ny));
        const int x = ((xg % p.nx) + p.nx) % p.nx, y = ((yg % p.ny) + p.ny) % p.ny;
        uint32_t h[4], l[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t hp = 0, lp = 0;
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int z = 8 * zc + 2 * k + m;
                const float v = out ? -p.nref[b] : mom[b * p.N + x + (long long)p.nx * (y + (long long)p.ny * z)].x;
                const __nv_bfloat16 hv = __float2bfloat16_rn(v);
                const __nv_bfloat16 lv = __float2bfloat16_rn(v - __bfloat162float(hv));
                hp |= (uint32_t)__bfloat16_as_ushort(hv) << (16 * m);
                lp |= (uint32_t)__bfloat16_as_ushort(lv) << (16 * m);
            }
            h[k] = hp;
            l[k] = lp;
        }
        qhi[e] = make_uint4(h[0], h[1], h[2], h[3]);
        qlo[e] = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

}  // namespace

bool mlbi_attraction_tc_supported(const mlbi_params &p)
{
    return p.S >= 1 && p.S <= 2 && p.attr_r >= 1 && p.attr_r <= 8 && p.wall_axis != 2 && p.nz % 8 == 0;
}

void mlbi_attraction_tc_padded(const mlbi_params &p, int *nxp, int *nyp)
{
    *nxp = (p.nx + kTM - 1) / kTM * kTM + 2 * kPad;
    *nyp = p.ny + 2 * kPad;
}

size_t mlbi_attraction_tc_column_bytes(int S)
{
    return S == 1 ? Shape<1>::col_bytes : Shape<2>::col_bytes;
}

cudaError_t mlbi_launch_attraction_tc(const mlbi_params &p, const mlbi_buffers &b, const mlbi_tc_tables &t,
                                      cudaStream_t s)
{
    if (!mlbi_attraction_tc_supported(p) || !t.weights || !t.qhi || !t.qlo) return cudaErrorInvalidValue;
    TcArgs g{};
    g.nx = p.nx; g.ny = p.ny; g.nz = p.nz; g.S = p.S; g.wall_axis = p.wall_axis; g.N = p.N;
    mlbi_attraction_tc_padded(p, &g.nxp, &g.nyp);
    g.ncols = t.ncols; g.nrows = t.nrows; g.pass3 = t.pass3;
    {
        const long long total = (long long)g.nxp * g.nyp * p.S * (p.nz / 8);
        const unsigned grid = (unsigned)std::min<long long>((total + 255) / 256, 152ll * 32);
        k_attraction_prep<<<grid, 256, 0, s>>>(p, g.nxp, g.nyp, b.mom, (uint4 *)t.qhi, (uint4 *)t.qlo);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const int nxt = (p.nx + kTM - 1) / kTM, nzt = (p.nz + kSub * kTZ - 1) / (kSub * kTZ);
    const long long ntiles = (long long)nxt * p.ny * nzt;
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(ntiles, nsm));
    cudaError_t e;
    if (p.S == 1) {
        auto k = k_attraction_tc<1>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Shape<1>::smem);
        if (e != cudaSuccess) return e;
        k<<<grid, kThreads, Shape<1>::smem, s>>>(g, (const uint4 *)t.qhi, (const uint4 *)t.qlo, (const uint4 *)t.weights, t.cols,
                                                 t.row_start, b.attr, b.flags);
    } else {
        auto k = k_attraction_tc<2>;
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Shape<2>::smem);
        if (e != cudaSuccess) return e;
        k<<<grid, kThreads, Shape<2>::smem, s>>>(g, (const uint4 *)t.qhi, (const uint4 *)t.qlo, (const uint4 *)t.weights, t.cols,
                                                 t.row_start, b.attr, b.flags);
    }
    return cudaGetLastError();
}
