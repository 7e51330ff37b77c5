// mlb_surrogate.cu -- a learned surrogate of the hard-core force (the F^hc
// term of Eq. potmeanforce) for binary mixtures on periodic lattices:
// a 3-layer 3D convolutional network, n - n_ref (2 channels) -> 32 -> 32 ->
// 6 force components, 3^3, 3^3 and 1^3 kernels (a 5^3 receptive field, the
// reach of the contact shells sigma_ab + 1/2 <= 2.5 of sigma <= 2 spheres),
// tanh activations and biases held at zero, so the network is odd in its
// input (F(-dn) = -F(dn), no force at rest, like the hard-core force at
// linear order).  Hidden activations are stored as BF16, site-major [N][C]
// (the 2-channel input stays FP32); every sum accumulates in FP32.  The 32 -> 32 layer and its input gradient run on
// the tensor cores (mma.sync m16n8k16 BF16); the small layers, the weight
// gradients, the loss and Adam on the FP32 pipes.  Training and inference
// kernels are both here; the host API is at the end.
#include "mlb.h"
#include "mlb_internal.h"

#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace {

constexpr int kCin = 2, kHid = 32, kOut = 6, kTaps = 27;
// parameter layout (FP32): W1[27][32 co][2 ci] b1[32] W2[27][32 co][32 ci] b2[32] W3[6][32] b3[6]
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kTaps * kCin * kHid, kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kTaps * kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid;
constexpr int kParams = kOffB3 + kOut;

struct Geo {
    int nx, ny, nz;
    long long N;
};

// periodic neighbour of site r at tap t = (dz+1)*9 + (dy+1)*3 + (dx+1)
__device__ __forceinline__ long long tap_nbr(const Geo &g, int x, int y, int z, int t)
{
    int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
    int xx = x + dx, yy = y + dy, zz = z + dz;
    xx += xx < 0 ? g.nx : 0; xx -= xx >= g.nx ? g.nx : 0;
    yy += yy < 0 ? g.ny : 0; yy -= yy >= g.ny ? g.ny : 0;
    zz += zz < 0 ? g.nz : 0; zz -= zz >= g.nz ? g.nz : 0;
    return xx + (long long)g.nx * (yy + (long long)g.ny * zz);
}

__device__ __forceinline__ void decode(const Geo &g, long long r, int &x, int &y, int &z)
{
    x = (int)(r % g.nx);
    const long long q = r / g.nx;
    y = (int)(q % g.ny);
    z = (int)(q / g.ny);
}

__device__ __forceinline__ float act_f(float v) { return tanhf(v); }
__device__ __forceinline__ float act_grad(float v)
{
    const float t = tanhf(v);
    return 1.f - t * t;
}

__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float to_f(float v) { return v; }

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    unsigned u;
    memcpy(&u, &h, 4);
    return u;
}

// ------------------------------------------------------------------ inputs
// x0[r][c] = (n^c - n_ref^c) in_scale_c in FP32, from the moments (float4 .x) or from FP64 host data.
// The input stays FP32: the force of a smooth field is a difference of
// neighbouring densities, and BF16's 8-bit significand on the densities
// themselves would cost several percent of it.
__global__ void k_input_from_mom(Geo g, const float4 *__restrict__ mom, float s0, float s1, float2 *__restrict__ x0)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < g.N; r += (long long)gridDim.x * blockDim.x)
        x0[r] = make_float2(mom[r].x * s0, mom[g.N + r].x * s1);
}

__global__ void k_input_from_f64(Geo g, const double *__restrict__ dn, float s0, float s1, float2 *__restrict__ x0)
{
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < g.N; r += (long long)gridDim.x * blockDim.x)
        x0[r] = make_float2((float)dn[r] * s0, (float)dn[g.N + r] * s1);
}

// ------------------------------------------------------------------ layer 1 (2 -> 32, 3^3), FP32 pipes
// pre1 = b1 + sum_{tap, ci} W1[tap][co][ci] x0[r + tap][ci];  act1 = act_f(pre1)
__global__ void __launch_bounds__(128) k_layer1(Geo g, const float2 *__restrict__ x0,
                                                const float *__restrict__ P, __nv_bfloat16 *__restrict__ pre1,
                                                __nv_bfloat16 *__restrict__ act1)
{
    __shared__ float w[kTaps * kCin * kHid + kHid];
    for (int i = threadIdx.x; i < kTaps * kCin * kHid + kHid; i += blockDim.x) w[i] = P[kOffW1 + i];
    __syncthreads();
    const float *b = w + kTaps * kCin * kHid;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < g.N; r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        decode(g, r, x, y, z);
        float acc[kHid];
#pragma unroll
        for (int c = 0; c < kHid; ++c) acc[c] = b[c];
        for (int t = 0; t < kTaps; ++t) {
            const float2 v = x0[tap_nbr(g, x, y, z, t)];
            const float *wt = w + t * kCin * kHid;
#pragma unroll
            for (int c = 0; c < kHid; ++c) acc[c] = fmaf(v.y, wt[2 * c + 1], fmaf(v.x, wt[2 * c], acc[c]));
        }
        unsigned *pp = reinterpret_cast<unsigned *>(pre1 + r * kHid);
        unsigned *pa = reinterpret_cast<unsigned *>(act1 + r * kHid);
#pragma unroll
        for (int c = 0; c < kHid; c += 2) {
            if (pre1) pp[c / 2] = pack_bf16(acc[c], acc[c + 1]);
            pa[c / 2] = pack_bf16(act_f(acc[c]), act_f(acc[c + 1]));
        }
    }
}

// ------------------------------------------------------------------ 32 -> 32, 3^3 on the tensor cores
// out[r][n] = sum_{tap} sum_k in[r + tap][k] B[tap][n][k]  (K = N = 32), then an epilogue:
//   FORWARD: + bias, store pre (optional) and tanh -> out
//   BACKDATA: multiply by tanh'(pre[r][n]) -> out (the input gradient of the previous layer)
// A warp computes 16 consecutive sites x 32 outputs: per tap two k-steps of
// four m16n8k16 MMAs.  B (BF16, [27][32][32], k innermost) sits in shared memory.
__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <bool FORWARD>
__global__ void __launch_bounds__(128) k_conv32_mma(Geo g, const __nv_bfloat16 *__restrict__ in,
                                                    const __nv_bfloat16 *__restrict__ B,
                                                    const float *__restrict__ bias,
                                                    const __nv_bfloat16 *__restrict__ pre_in,
                                                    __nv_bfloat16 *__restrict__ pre_out,
                                                    __nv_bfloat16 *__restrict__ out)
{
    extern __shared__ __align__(16) __nv_bfloat16 sB[];                // [27][32][32]
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(B);
        uint4 *dst = reinterpret_cast<uint4 *>(sB);
        for (int i = threadIdx.x; i < kTaps * kHid * kHid / 8; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gq = lane >> 2, tq = lane & 3;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long s0 = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * 16; s0 < g.N; s0 += nwarps * 16) {
        const long long r0 = min(s0 + gq, g.N - 1), r1 = min(s0 + gq + 8, g.N - 1);   // rows g and g + 8
        int x0, y0, z0, x1, y1, z1;
        decode(g, r0, x0, y0, z0);
        decode(g, r1, x1, y1, z1);
        float acc[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
        for (int t = 0; t < kTaps; ++t) {
            const unsigned *a_lo = reinterpret_cast<const unsigned *>(in + tap_nbr(g, x0, y0, z0, t) * kHid);
            const unsigned *a_hi = reinterpret_cast<const unsigned *>(in + tap_nbr(g, x1, y1, z1, t) * kHid);
            const unsigned *bt = reinterpret_cast<const unsigned *>(sB + t * kHid * kHid);
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const unsigned a0 = __ldg(a_lo + kk * 8 + tq), a1 = __ldg(a_hi + kk * 8 + tq);
                const unsigned a2 = __ldg(a_lo + kk * 8 + tq + 4), a3 = __ldg(a_hi + kk * 8 + tq + 4);
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const unsigned *bn = bt + (nt * 8 + gq) * (kHid / 2) + kk * 8;
                    mma_bf16(acc[nt], a0, a1, a2, a3, bn[tq], bn[tq + 4]);
                }
            }
        }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const long long r = s0 + gq + 8 * half;
            if (r >= g.N) continue;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int n = nt * 8 + 2 * tq;
                float v0 = acc[nt][2 * half], v1 = acc[nt][2 * half + 1];
                unsigned *po = reinterpret_cast<unsigned *>(out + r * kHid + n);
                if (FORWARD) {
                    v0 += bias[n];
                    v1 += bias[n + 1];
                    if (pre_out) *reinterpret_cast<unsigned *>(pre_out + r * kHid + n) = pack_bf16(v0, v1);
                    *po = pack_bf16(act_f(v0), act_f(v1));
                } else {
                    const float2 p = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(pre_in + r * kHid + n));
                    *po = pack_bf16(v0 * act_grad(p.x), v1 * act_grad(p.y));
                }
            }
        }
    }
}

// ------------------------------------------------------------------ layer 3 (32 -> 6, 1^3)
// out[r][o] = b3[o] + sum_c W3[o][c] act2[r][c], FP32; optionally the force
// field F^a = out[3a + i] / out_scale_a as float4 [2][N] for the step
__global__ void __launch_bounds__(128) k_layer3(Geo g, const __nv_bfloat16 *__restrict__ act2,
                                                const float *__restrict__ P, float *__restrict__ out,
                                                float4 *__restrict__ force, float inv0, float inv1)
{
    __shared__ float w[kOut * kHid + kOut];
    for (int i = threadIdx.x; i < kOut * kHid + kOut; i += blockDim.x) w[i] = P[kOffW3 + i];
    __syncthreads();
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < g.N; r += (long long)gridDim.x * blockDim.x) {
        float acc[kOut];
#pragma unroll
        for (int o = 0; o < kOut; ++o) acc[o] = w[kOut * kHid + o];
        const __nv_bfloat162 *a = reinterpret_cast<const __nv_bfloat162 *>(act2 + r * kHid);
#pragma unroll
        for (int c = 0; c < kHid; c += 2) {
            const float2 v = __bfloat1622float2(a[c / 2]);
#pragma unroll
            for (int o = 0; o < kOut; ++o) acc[o] = fmaf(v.y, w[o * kHid + c + 1], fmaf(v.x, w[o * kHid + c], acc[o]));
        }
        if (out)
#pragma unroll
            for (int o = 0; o < kOut; ++o) out[r * kOut + o] = acc[o];
        if (force) {
            force[r] = make_float4(acc[0] * inv0, acc[1] * inv0, acc[2] * inv0, 0.f);
            force[g.N + r] = make_float4(acc[3] * inv1, acc[4] * inv1, acc[5] * inv1, 0.f);
        }
    }
}

// ------------------------------------------------------------------ layers 2 + 3 on tcgen05 (inference)
// For lattices with nx a multiple of 128.  A tile is 128 consecutive sites
// x0 .. x0+127 of one (y, z) row: the 128 rows of the MMA's M dimension and
// the 128 TMEM lanes.  The 32 -> 32 3^3 convolution is an implicit GEMM
// D[m][n] = sum_{tap, ci} act1[nbr(m, tap)][ci] W2[tap][n][ci] with
// K = 27 x 32: per tap two MMAs of M128 N32 K16 (BF16 in, FP32 accumulate in
// TMEM).  The act1 rows a tile reads, (y+dy, z+dz) for sites x0-1 .. x0+128,
// sit in shared memory in the K-major layout without swizzle in which every
// K chunk of 8 channels keeps the sites at a 16-byte stride:
// [row][chunk][site][8 ch].  A core matrix (8 sites x 16 B) may then start at
// any site, so the x shift of a tap is only the start address of the A
// descriptor (LBO = the chunk stride, SBO = 8 sites = 128 B).  W2 is staged
// once per CTA as B = [tap][chunk][n][8 ch] (LBO 512 B, SBO 128 B).
//
// A CTA walks z along (segment, y) columns: its rows form a ring of five z
// planes (three y rows each).  While the MMAs of tile z (planes z-1 .. z+1)
// run, plane z+2 is in flight for tile z+1 and plane z+3 is requested for
// tile z+2, so the copies have two tiles' time to arrive.  The accumulators
// alternate between two 32-column TMEM buffers: one elected thread issues
// tile i+1's MMAs before the epilogue of tile i reads its buffer with
// tcgen05.ld.  The epilogue applies bias, tanh (the hardware approximation,
// relative error ~2^-11, below the BF16 rounding of the hidden layer) and
// the 1^3 layer 3 in FP32.  Persistent CTAs, one per SM, 8 warps: warps w
// and w + 4 read the same 32 TMEM lanes (tcgen05.ld reaches lanes
// 32 (w mod 4) ..), and each computes the force on one species.
constexpr int kTcM = 128;
constexpr int kTcRowSites = kTcM + 2;
constexpr int kTcLboA = kTcRowSites * 16;                   // bytes between K chunks of a staged row
constexpr int kTcRowBytes = 4 * kTcLboA;                    // one staged row, 4 chunks of 8 channels
constexpr int kTcPlaneBytes = 3 * kTcRowBytes;              // rows y-1, y, y+1 of one z plane
constexpr int kTcRing = 5;                                  // planes z-1 .. z+3 of a tile z
constexpr int kTcABytes = kTcRing * kTcPlaneBytes;
constexpr int kTcBBytes = kTaps * 4 * kHid * 16;            // 27 taps x 4 chunks x 32 outputs x 16 B
constexpr int kTcSmem = kTcBBytes + kTcABytes + 16;         // + mbarrier and the TMEM address
constexpr int kTcCols = 64;                                 // two accumulators of N = 32 FP32 columns
// instruction descriptor (kind::f16): D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kHid >> 3) << 17) |
                              ((uint32_t)(kTcM >> 4) << 24);
// spin limit of the mbarrier wait (each try_wait suspends for a while): far
// above the ~1 us the 54 MMAs of a tile take
constexpr unsigned kTcSpinLimit = 1u << 20;

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    // start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4 (32-45), fixed 0b001
    // at 46-48, base offset 0, absolute LBO mode, no swizzle (61-63 = 0)
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t phase)
{
    for (unsigned it = 0; it < kTcSpinLimit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(bar), "r"(phase)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ float tanh_fast(float v)
{
    float r;
    asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

__device__ __forceinline__ int tc_slot(int zp) { return (zp + kTcRing) % kTcRing; }   // zp >= -1

// cp.async the three rows (y-1, y, y+1) of plane zp (unwrapped, -1 .. nz) of
// the column (x0, y) into its ring slot, as one commit group
__device__ __forceinline__ void tc_stage_plane(const Geo &g, const __nv_bfloat16 *__restrict__ act1, uint32_t sA_a,
                                               int x0, int y, int zp)
{
    int zz = zp;
    zz += zz < 0 ? g.nz : 0; zz -= zz >= g.nz ? g.nz : 0;
    const uint32_t base = sA_a + (uint32_t)tc_slot(zp) * kTcPlaneBytes;
    for (int i = threadIdx.x; i < 3 * kTcRowSites * 4; i += blockDim.x) {
        const int row = i / (kTcRowSites * 4), rem = i % (kTcRowSites * 4), s = rem >> 2, j = rem & 3;
        int yy = y + row - 1, xx = x0 - 1 + s;
        yy += yy < 0 ? g.ny : 0; yy -= yy >= g.ny ? g.ny : 0;
        xx += xx < 0 ? g.nx : 0; xx -= xx >= g.nx ? g.nx : 0;
        const long long r = xx + (long long)g.nx * (yy + (long long)g.ny * zz);
        const uint32_t dst = base + row * kTcRowBytes + j * kTcLboA + s * 16;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(act1 + r * kHid + 8 * j) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// the 54 MMAs of tile z into accumulator columns tmem_d, then a commit to
// the mbarrier.  Descriptors are base descriptors plus compile-time offsets
// (in 16-byte units of the start-address field; every address stays below
// 256 KB, so the 14-bit field never carries).
__device__ __forceinline__ void tc_issue(uint32_t tmem_d, uint32_t sA_a, uint32_t sB_a, int z, uint32_t bar)
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint64_t aplane[3];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
        aplane[dz] = tc_desc(sA_a + (uint32_t)tc_slot(z + dz - 1) * kTcPlaneBytes, kTcLboA, 128);
    const uint64_t b0 = tc_desc(sB_a, kHid * 16, 128);
#pragma unroll
    for (int t = 0; t < kTaps; ++t) {
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const int dy = (t / 3) % 3, dx = t % 3;
            const uint64_t ad = aplane[t / 9] + (uint64_t)((dy * kTcRowBytes + dx * 16 + 2 * kk * kTcLboA) >> 4);
            const uint64_t bd = b0 + (uint64_t)((t * (4 * kHid * 16) + 2 * kk * (kHid * 16)) >> 4);
            const uint32_t acc = (t | kk) ? 1u : 0u;
            asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
                         "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(acc)
                         : "memory");
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

// Layer 1 for inference on lattices with nx % 128 == 0: a block computes
// act1 = tanh(b1 + W1 * x0) for 128 sites x0 .. x0+127 of four rows
// y0 .. y0+3 of one z plane.  The 18 input rows those read (y0-1 .. y0+4,
// z-1 .. z+1; sites x0-1 .. x0+128, FP32) are staged in shared memory.  A
// thread owns 8 channels of 8 sites (m, m+16, .., m+112 of one row), so a
// tap costs 8 + 4 shared loads for 128 FMAs; the four lanes of a site write
// its 64 bytes together (a warp stores 8 whole sites).  tanh is the hardware
// approximation.  Rows past ny (ny % 4 != 0) are computed and not stored.
constexpr int kL1Rows = 4;
__global__ void __launch_bounds__(256) k_layer1_rows(Geo g, const float2 *__restrict__ x0,
                                                     const float *__restrict__ P, __nv_bfloat16 *__restrict__ act1)
{
    __shared__ __align__(16) float w[kTaps * kHid * kCin];
    __shared__ float b[kHid];
    __shared__ float2 xs[3 * (kL1Rows + 2)][kTcRowSites];
    const int tid = threadIdx.x;
    for (int i = tid; i < kTaps * kHid * kCin; i += blockDim.x) w[i] = P[kOffW1 + i];
    for (int i = tid; i < kHid; i += blockDim.x) b[i] = P[kOffB1 + i];
    const int cg = tid & 3, q = tid >> 2, orow = q >> 4, sl = q & 15;   // channels 8cg.., row y0+orow, sites sl+16k
    const int nseg = g.nx / kTcM, nyb = (g.ny + kL1Rows - 1) / kL1Rows;
    const long long ntiles = (long long)nseg * nyb * g.nz;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int seg = (int)(tile % nseg);
        const long long rest = tile / nseg;
        const int y0 = (int)(rest % nyb) * kL1Rows, z = (int)(rest / nyb), xb = seg * kTcM;
        __syncthreads();
        // staged row (dz + 1) * (kL1Rows + 2) + (yy - y0 + 1)
        for (int i = tid; i < 3 * (kL1Rows + 2) * kTcRowSites; i += blockDim.x) {
            const int row = i / kTcRowSites, s = i % kTcRowSites;
            int yy = y0 + row % (kL1Rows + 2) - 1, zz = z + row / (kL1Rows + 2) - 1, xx = xb - 1 + s;
            yy = ((yy % g.ny) + g.ny) % g.ny;
            zz += zz < 0 ? g.nz : 0; zz -= zz >= g.nz ? g.nz : 0;
            xx += xx < 0 ? g.nx : 0; xx -= xx >= g.nx ? g.nx : 0;
            xs[row][s] = x0[xx + (long long)g.nx * (yy + (long long)g.ny * zz)];
        }
        __syncthreads();
        float acc[8][8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[k][c] = b[8 * cg + c];
#pragma unroll 1
        for (int t = 0; t < kTaps; ++t) {
            const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
            const float2 *xr = xs[dz * (kL1Rows + 2) + orow + dy] + sl + dx;
            const float4 *wt = reinterpret_cast<const float4 *>(w + (t * kHid + 8 * cg) * kCin);
            float4 ww[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) ww[h] = wt[h];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float2 v = xr[16 * k];
#pragma unroll
                for (int h = 0; h < 4; ++h) {    // channel 8cg+2h: (ww.x, ww.y); 8cg+2h+1: (ww.z, ww.w)
                    acc[k][2 * h] = fmaf(v.y, ww[h].y, fmaf(v.x, ww[h].x, acc[k][2 * h]));
                    acc[k][2 * h + 1] = fmaf(v.y, ww[h].w, fmaf(v.x, ww[h].z, acc[k][2 * h + 1]));
                }
            }
        }
        const int y = y0 + orow;
        if (y < g.ny) {
            const long long rb = xb + sl + (long long)g.nx * (y + (long long)g.ny * z);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                uint4 pk;
                pk.x = pack_bf16(tanh_fast(acc[k][0]), tanh_fast(acc[k][1]));
                pk.y = pack_bf16(tanh_fast(acc[k][2]), tanh_fast(acc[k][3]));
                pk.z = pack_bf16(tanh_fast(acc[k][4]), tanh_fast(acc[k][5]));
                pk.w = pack_bf16(tanh_fast(acc[k][6]), tanh_fast(acc[k][7]));
                *reinterpret_cast<uint4 *>(act1 + (rb + 16 * k) * kHid + 8 * cg) = pk;
            }
        }
    }
}

__global__ void __launch_bounds__(256, 1) k_conv23_tc(Geo g, const __nv_bfloat16 *__restrict__ act1,
                                                      const __nv_bfloat16 *__restrict__ W2f,
                                                      const float *__restrict__ P, float *__restrict__ out,
                                                      float4 *__restrict__ force, float inv0, float inv1,
                                                      int *__restrict__ flag)
{
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ float w3[kOut * kHid + kOut], b2[kHid];
    unsigned char *sB = smem;
    const uint32_t sB_a = (uint32_t)__cvta_generic_to_shared(sB);
    const uint32_t sA_a = sB_a + kTcBBytes;
    const uint32_t bar = sA_a + kTcABytes;
    const uint32_t slot = bar + 8;
    const uint32_t *slot_p = reinterpret_cast<const uint32_t *>(smem + kTcBBytes + kTcABytes + 8);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // B chunk (tap, j, n) = W2[tap][n][8j .. 8j+7]
    for (int i = tid; i < kTaps * 4 * kHid; i += blockDim.x) {
        const int t = i / (4 * kHid), j = (i / kHid) % 4, n = i % kHid;
        *reinterpret_cast<uint4 *>(sB + (size_t)i * 16) =
            *reinterpret_cast<const uint4 *>(W2f + ((size_t)t * kHid + n) * kHid + 8 * j);
    }
    for (int i = tid; i < kOut * kHid + kOut; i += blockDim.x) w3[i] = P[kOffW3 + i];
    for (int i = tid; i < kHid; i += blockDim.x) b2[i] = P[kOffB2 + i];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *slot_p;

    // this CTA's tiles: a contiguous range of tile = col * nz + z, col = seg + nseg * y
    const int nseg = g.nx / kTcM;
    const long long ntiles = (long long)nseg * g.ny * g.nz;
    const long long t_begin = ntiles * blockIdx.x / gridDim.x, t_end = ntiles * (blockIdx.x + 1) / gridDim.x;
    if (t_begin < t_end) {
        uint32_t phase = 0;
        auto coords = [&](long long t, int &x0, int &y, int &z) {
            const long long col = t / g.nz;
            z = (int)(t % g.nz);
            x0 = (int)(col % nseg) * kTcM;
            y = (int)(col / nseg);
        };
        // tiles a and b (> a) lie in one column: b's planes continue a's ring
        auto same_col = [&](long long a, long long b) { return b < t_end && a / g.nz == b / g.nz; };
        {
            int x0, y, z;
            coords(t_begin, x0, y, z);
            for (int dz = -1; dz <= 1; ++dz) tc_stage_plane(g, act1, sA_a, x0, y, z + dz);
            const bool more = same_col(t_begin, t_begin + 1);
            if (more) tc_stage_plane(g, act1, sA_a, x0, y, z + 2);
            if (more) asm volatile("cp.async.wait_group 1;" ::: "memory");
            else asm volatile("cp.async.wait_group 0;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) tc_issue(tmem, sA_a, sB_a, z, bar);
        }
        for (long long tile = t_begin; tile < t_end; ++tile) {
            int x0, y, z;
            coords(tile, x0, y, z);
            const uint32_t buf = (uint32_t)((tile - t_begin) & 1) * 32;
            const long long n1 = tile + 1;
            const bool has_n1 = n1 < t_end;
            // in flight: tile's MMAs (planes z-1 .. z+1) and, within the column, plane z+2
            bool newer = false;
            if (same_col(tile, tile + 2)) {
                tc_stage_plane(g, act1, sA_a, x0, y, z + 3);
                newer = true;
            }
            const bool ok = tc_wait(bar, phase);
            phase ^= 1u;
            if (__syncthreads_or(!ok)) {
                // give up on this call: record it, let the copies and MMAs drain (bounded), free TMEM below
                if (tid == 0) atomicExch(flag, 1);
                asm volatile("cp.async.wait_all;" ::: "memory");
                tc_wait(bar, phase ^ 1u);
                break;
            }
            int nx0 = 0, ny_ = 0, nz_ = 0;
            if (has_n1) coords(n1, nx0, ny_, nz_);
            if (has_n1 && !same_col(tile, n1)) {
                // a new column: nothing is in flight any more, stage its first planes
                for (int dz = -1; dz <= 1; ++dz) tc_stage_plane(g, act1, sA_a, nx0, ny_, nz_ + dz);
                newer = same_col(n1, n1 + 1);
                if (newer) tc_stage_plane(g, act1, sA_a, nx0, ny_, nz_ + 2);
            }
            if (newer) asm volatile("cp.async.wait_group 1;" ::: "memory");
            else asm volatile("cp.async.wait_group 0;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (has_n1 && tid == 0) tc_issue(tmem + (buf ^ 32u), sA_a, sB_a, nz_, bar);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            uint32_t v[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                "[%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(tmem + buf + ((uint32_t)((warp & 3) * 32) << 16)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int sp = warp >> 2;                         // species: outputs 3 sp .. 3 sp + 2
            const float *w3s = w3 + 3 * sp * kHid;
            float o[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) o[k] = w3[kOut * kHid + 3 * sp + k];
#pragma unroll
            for (int c = 0; c < kHid; ++c) {
                const float a = tanh_fast(__uint_as_float(v[c]) + b2[c]);
#pragma unroll
                for (int k = 0; k < 3; ++k) o[k] = fmaf(a, w3s[k * kHid + c], o[k]);
            }
            const long long r = x0 + (warp & 3) * 32 + lane + (long long)g.nx * (y + (long long)g.ny * z);
            if (out)
#pragma unroll
                for (int k = 0; k < 3; ++k) out[r * kOut + 3 * sp + k] = o[k];
            if (force) {
                const float inv = sp ? inv1 : inv0;
                force[sp * g.N + r] = make_float4(o[0] * inv, o[1] * inv, o[2] * inv, 0.f);
            }
            // the buffer just read is the next MMAs' target after this barrier
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
        }
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
}

// ------------------------------------------------------------------ training
// targets in the network's units: t[r][3a + i] = F^a_i(r) out_scale_a
// t = F out_scale in [N][6]; tnorm += sum t^2 (FP64 block sums)
__global__ void __launch_bounds__(256) k_target_from_f64(Geo g, const double *__restrict__ F, float s0, float s1,
                                                        float *__restrict__ t, double *__restrict__ tnorm)
{
    __shared__ double red[256];
    double s = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < g.N; r += (long long)gridDim.x * blockDim.x)
        for (int a = 0; a < 2; ++a)
            for (int i = 0; i < 3; ++i) {
                const float v = (float)F[(a * 3 + i) * g.N + r] * (a ? s1 : s0);
                t[r * kOut + 3 * a + i] = v;
                s += (double)v * v;
            }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(tnorm, red[0]);
}

// Relative squared error loss = sum (out - t)^2 / sum t^2 (the square of the
// relative force error the step's recheck bounds; every frame weighs the same
// whatever its amplitude); dout = d loss / d out.  tnorm = sum t^2 > 0.
__global__ void __launch_bounds__(256) k_loss(Geo g, const float *__restrict__ out, const float *__restrict__ t,
                                             const double *__restrict__ tnorm, float *__restrict__ dout,
                                             double *__restrict__ loss)
{
    __shared__ double red[256];
    double s = 0.0;
    const long long M = g.N * kOut;
    const double inv = 1.0 / fmax(*tnorm, 1e-300);
    const float scale = (float)(2.0 * inv);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < M; i += (long long)gridDim.x * blockDim.x) {
        const float e = out[i] - t[i];
        dout[i] = scale * e;
        s += (double)e * e;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] * inv);
}

// layer-3 input gradient: dpre2[r][c] = tanh'(pre2[r][c]) sum_o W3[o][c] dout[r][o]
__global__ void __launch_bounds__(128) k_back3(Geo g, const float *__restrict__ dout, const float *__restrict__ P,
                                               const __nv_bfloat16 *__restrict__ pre2,
                                               __nv_bfloat16 *__restrict__ dpre2)
{
    __shared__ float w[kOut * kHid];
    for (int i = threadIdx.x; i < kOut * kHid; i += blockDim.x) w[i] = P[kOffW3 + i];
    __syncthreads();
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < g.N; r += (long long)gridDim.x * blockDim.x) {
        float d[kOut];
#pragma unroll
        for (int o = 0; o < kOut; ++o) d[o] = dout[r * kOut + o];
        const __nv_bfloat162 *p = reinterpret_cast<const __nv_bfloat162 *>(pre2 + r * kHid);
        unsigned *q = reinterpret_cast<unsigned *>(dpre2 + r * kHid);
#pragma unroll
        for (int c = 0; c < kHid; c += 2) {
            float v0 = 0.f, v1 = 0.f;
#pragma unroll
            for (int o = 0; o < kOut; ++o) {
                v0 = fmaf(w[o * kHid + c], d[o], v0);
                v1 = fmaf(w[o * kHid + c + 1], d[o], v1);
            }
            const float2 pp = __bfloat1622float2(p[c / 2]);
            q[c / 2] = pack_bf16(v0 * act_grad(pp.x), v1 * act_grad(pp.y));
        }
    }
}

// weight gradient of a 3^3 layer: dW[tap][co][ci] += sum_r dy[r][co] x[r + tap][ci]
// (and db[co] += sum_r dy[r][co] at the centre tap).  One block per (tap,
// site chunk); the chunk's rows are staged in shared memory 32 sites at a
// time; per-block sums are added to the FP32 gradient with atomics.
template <int CI, int CO, class TX, class TY>
__global__ void __launch_bounds__(256) k_wgrad3(Geo g, const TX *__restrict__ xin, const TY *__restrict__ dy,
                                                long long chunk, float *__restrict__ dW, float *__restrict__ db,
                                                int w_tap_stride_co)
{
    constexpr int OUT = CI * CO, PER = (OUT + 255) / 256, TS = 32;
    __shared__ float sx[TS][CI], sd[TS][CO];
    const int t = blockIdx.y;
    const long long r_begin = blockIdx.x * chunk, r_end = min(r_begin + chunk, g.N);
    float acc[PER], bacc = 0.f;
#pragma unroll
    for (int k = 0; k < PER; ++k) acc[k] = 0.f;
    for (long long rb = r_begin; rb < r_end; rb += TS) {
        __syncthreads();
        for (int i = threadIdx.x; i < TS * (CI + CO); i += blockDim.x) {
            const int s = i / (CI + CO), c = i % (CI + CO);
            const long long r = rb + s;
            float v = 0.f;
            if (r < r_end) {
                if (c < CI) {
                    int x, y, z;
                    decode(g, r, x, y, z);
                    v = to_f(xin[tap_nbr(g, x, y, z, t) * CI + c]);
                } else {
                    v = to_f(dy[r * CO + (c - CI)]);
                }
            }
            if (c < CI) sx[s][c] = v;
            else sd[s][c - CI] = v;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int o = threadIdx.x + k * 256;
            if (o < OUT) {
                const int co = o / CI, ci = o % CI;
                float a = acc[k];
#pragma unroll 8
                for (int s = 0; s < TS; ++s) a = fmaf(sd[s][co], sx[s][ci], a);
                acc[k] = a;
            }
        }
        if (t == 13 && threadIdx.x < CO)
            for (int s = 0; s < TS; ++s) bacc += sd[s][threadIdx.x];
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int o = threadIdx.x + k * 256;
        if (o < OUT) {
            const int co = o / CI, ci = o % CI;
            atomicAdd(&dW[(size_t)t * w_tap_stride_co + (size_t)co * CI + ci], acc[k]);
        }
    }
    if (t == 13 && threadIdx.x < CO) atomicAdd(&db[threadIdx.x], bacc);
}

// layer-3 weight gradient: dW3[o][c] += sum_r dout[r][o] act2[r][c], db3[o] += sum_r dout[r][o]
__global__ void __launch_bounds__(256) k_wgrad_out(Geo g, const __nv_bfloat16 *__restrict__ act2,
                                                   const float *__restrict__ dout, long long chunk,
                                                   float *__restrict__ dW3, float *__restrict__ db3)
{
    constexpr int TS = 32;
    __shared__ float sx[TS][kHid], sd[TS][kOut];
    const long long r_begin = blockIdx.x * chunk, r_end = min(r_begin + chunk, g.N);
    const int o = threadIdx.x / kHid, c = threadIdx.x % kHid;          // 192 (o, c) pairs
    float acc = 0.f, bacc = 0.f;
    for (long long rb = r_begin; rb < r_end; rb += TS) {
        __syncthreads();
        for (int i = threadIdx.x; i < TS * (kHid + kOut); i += blockDim.x) {
            const int s = i / (kHid + kOut), k = i % (kHid + kOut);
            const long long r = rb + s;
            float v = 0.f;
            if (r < r_end) v = k < kHid ? __bfloat162float(act2[r * kHid + k]) : dout[r * kOut + (k - kHid)];
            if (k < kHid) sx[s][k] = v;
            else sd[s][k - kHid] = v;
        }
        __syncthreads();
        if (threadIdx.x < kOut * kHid)
            for (int s = 0; s < TS; ++s) acc = fmaf(sd[s][o], sx[s][c], acc);
        if (threadIdx.x < kOut)
            for (int s = 0; s < TS; ++s) bacc += sd[s][threadIdx.x];
    }
    if (threadIdx.x < kOut * kHid) atomicAdd(&dW3[o * kHid + c], acc);
    if (threadIdx.x < kOut) atomicAdd(&db3[threadIdx.x], bacc);
}

// the two BF16 copies of W2 the tensor-core kernels read: forward B[tap][co][ci]
// and input-gradient B[tap'][ci][co] with tap' the mirrored tap (26 - tap)
__global__ void k_w2_bf16(const float *__restrict__ P, __nv_bfloat16 *__restrict__ Bf, __nv_bfloat16 *__restrict__ Bb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kTaps * kHid * kHid) return;
    const int t = i / (kHid * kHid), co = (i / kHid) % kHid, ci = i % kHid;
    const float w = P[kOffW2 + i];
    Bf[i] = __float2bfloat16_rn(w);
    Bb[((26 - t) * kHid + ci) * kHid + co] = __float2bfloat16_rn(w);
}

__global__ void k_adam(int n, float *__restrict__ P, const float *__restrict__ G, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = G[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// the surrogate's error against the exact rest force: sums of |F_s - F_x|^2 and |F_x|^2
__global__ void __launch_bounds__(256) k_force_error(long long n4, const float4 *__restrict__ fs,
                                                     const float4 *__restrict__ fx, double *__restrict__ sums)
{
    __shared__ double r0[256], r1[256];
    double e = 0.0, t = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 a = fs[i], b = fx[i];
        const double dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
        e += dx * dx + dy * dy + dz * dz;
        t += (double)b.x * b.x + (double)b.y * b.y + (double)b.z * b.z;
    }
    r0[threadIdx.x] = e;
    r1[threadIdx.x] = t;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            r0[threadIdx.x] += r0[threadIdx.x + k];
            r1[threadIdx.x] += r1[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&sums[0], r0[0]);
        atomicAdd(&sums[1], r1[0]);
    }
}

constexpr int kConvSmem = kTaps * kHid * kHid * (int)sizeof(__nv_bfloat16);

unsigned grid_of(long long n, int block)
{
    long long b = (n + block - 1) / block;
    return (unsigned)(b < 1 ? 1 : (b > 8192 ? 8192 : b));
}

}  // namespace

// ------------------------------------------------------------------ the network object
struct mlb_net {
    Geo g{};
    float in_scale[2] = {1.f, 1.f}, out_scale[2] = {1.f, 1.f};
    float *P = nullptr, *G = nullptr, *m = nullptr, *v = nullptr;    // FP32 parameters, gradients, Adam moments
    __nv_bfloat16 *W2f = nullptr, *W2b = nullptr;                    // BF16 copies of W2
    float2 *x0 = nullptr;
    __nv_bfloat16 *pre1 = nullptr, *act1 = nullptr, *pre2 = nullptr, *act2 = nullptr, *dpre2 = nullptr,
                  *dpre1 = nullptr;
    float *out = nullptr, *tgt = nullptr, *dout = nullptr;
    double *dev_scalar = nullptr;                                    // [2] loss, sum of target^2
    double *stage = nullptr;                                         // FP64 host-transfer staging
    int *flag = nullptr;                                             // a bounded device wait gave up
    bool tc = false;                                                 // nx % 128 == 0: layers 2 + 3 on tcgen05
    int sms = 0;
    cudaError_t cuda_err = cudaSuccess;                              // the last CUDA error recorded
    cudaStream_t stream = nullptr;
    long long adam_t = 0;
    bool weights_dirty = true;
    std::string err;
};

namespace {

mlb_status net_fail(mlb_net *n, cudaError_t e, const char *what)
{
    n->err = std::string(what) + ": " + cudaGetErrorString(e);
    n->cuda_err = e;
    return MLB_ECUDA;
}

#define NET_CUDA(net, call)                                                                        \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return net_fail((net), e_, #call);                                  \
    } while (0)

mlb_status refresh_w2(mlb_net *n, cudaStream_t st)
{
    if (!n->weights_dirty) return MLB_OK;
    k_w2_bf16<<<(kTaps * kHid * kHid + 255) / 256, 256, 0, st>>>(n->P, n->W2f, n->W2b);
    NET_CUDA(n, cudaGetLastError());
    n->weights_dirty = false;
    return MLB_OK;
}

// forward from x0 (already staged); training keeps the pre-activations.
// Inference on lattices with nx % 128 == 0 runs layers 2 and 3 as one
// tcgen05 kernel (FP32 act2); otherwise, and in training, the mma.sync layer 2
// and layer 3 run separately (BF16 act2, kept for the backward pass).
mlb_status net_forward(mlb_net *n, bool keep, float *out, float4 *force, cudaStream_t cs)
{
    mlb_status st = refresh_w2(n, cs);
    if (st != MLB_OK) return st;
    const Geo &g = n->g;
    if (!keep && n->tc) {
        NET_CUDA(n, cudaFuncSetAttribute(k_conv23_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
        const long long tiles = (long long)(g.nx / kTcM) * g.ny * g.nz;
        const long long l1_tiles = (long long)(g.nx / kTcM) * ((g.ny + kL1Rows - 1) / kL1Rows) * g.nz;
        const long long l1_blocks = (long long)n->sms * 2;
        k_layer1_rows<<<(unsigned)(l1_tiles < l1_blocks ? l1_tiles : l1_blocks), 256, 0, cs>>>(g, n->x0,
                                                                                                      n->P, n->act1);
        NET_CUDA(n, cudaGetLastError());
        const unsigned grid = (unsigned)(tiles < n->sms ? tiles : n->sms);
        k_conv23_tc<<<grid, 256, kTcSmem, cs>>>(g, n->act1, n->W2f, n->P, out, force, 1.f / n->out_scale[0],
                                                        1.f / n->out_scale[1], n->flag);
        NET_CUDA(n, cudaGetLastError());
        return MLB_OK;
    }
    k_layer1<<<grid_of(g.N, 128), 128, 0, cs>>>(g, n->x0, n->P, keep ? n->pre1 : nullptr, n->act1);
    NET_CUDA(n, cudaGetLastError());
    NET_CUDA(n, cudaFuncSetAttribute(k_conv32_mma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem));
    k_conv32_mma<true><<<grid_of((g.N + 15) / 16 * 32, 128), 128, kConvSmem, cs>>>(
        g, n->act1, n->W2f, n->P + kOffB2, nullptr, keep ? n->pre2 : nullptr, n->act2);
    NET_CUDA(n, cudaGetLastError());
    k_layer3<<<grid_of(g.N, 128), 128, 0, cs>>>(g, n->act2, n->P, out, force, 1.f / n->out_scale[0],
                                                        1.f / n->out_scale[1]);
    NET_CUDA(n, cudaGetLastError());
    return MLB_OK;
}

// loss and parameter gradient for the staged input and target
mlb_status net_backward(mlb_net *n)
{
    const Geo &g = n->g;
    NET_CUDA(n, cudaMemsetAsync(n->G, 0, sizeof(float) * kParams, n->stream));
    NET_CUDA(n, cudaMemsetAsync(n->dev_scalar, 0, sizeof(double), n->stream));
    k_loss<<<grid_of(g.N * kOut, 256), 256, 0, n->stream>>>(g, n->out, n->tgt, n->dev_scalar + 1, n->dout,
                                                             n->dev_scalar);
    NET_CUDA(n, cudaGetLastError());
    const long long chunk = std::max<long long>(1024, (g.N + 1023) / 1024);
    const unsigned nch = (unsigned)((g.N + chunk - 1) / chunk);
    k_wgrad_out<<<nch, 256, 0, n->stream>>>(g, n->act2, n->dout, chunk, n->G + kOffW3, n->G + kOffB3);
    NET_CUDA(n, cudaGetLastError());
    k_back3<<<grid_of(g.N, 128), 128, 0, n->stream>>>(g, n->dout, n->P, n->pre2, n->dpre2);
    NET_CUDA(n, cudaGetLastError());
    k_wgrad3<kHid, kHid, __nv_bfloat16, __nv_bfloat16><<<dim3(nch, kTaps), 256, 0, n->stream>>>(
        g, n->act1, n->dpre2, chunk, n->G + kOffW2, n->G + kOffB2, kHid * kHid);
    NET_CUDA(n, cudaGetLastError());
    NET_CUDA(n, cudaFuncSetAttribute(k_conv32_mma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem));
    k_conv32_mma<false><<<grid_of((g.N + 15) / 16 * 32, 128), 128, kConvSmem, n->stream>>>(
        g, n->dpre2, n->W2b, nullptr, n->pre1, nullptr, n->dpre1);
    NET_CUDA(n, cudaGetLastError());
    k_wgrad3<kCin, kHid, float, __nv_bfloat16><<<dim3(nch, kTaps), 256, 0, n->stream>>>(
        g, reinterpret_cast<const float *>(n->x0), n->dpre1, chunk, n->G + kOffW1, n->G + kOffB1,
        kHid * kCin);
    NET_CUDA(n, cudaGetLastError());
    return MLB_OK;
}

mlb_status stage_frame(mlb_net *n, const double *dn, const double *F)
{
    const Geo &g = n->g;
    NET_CUDA(n, cudaMemcpyAsync(n->stage, dn, sizeof(double) * 2 * g.N, cudaMemcpyHostToDevice, n->stream));
    k_input_from_f64<<<grid_of(g.N, 256), 256, 0, n->stream>>>(g, n->stage, n->in_scale[0], n->in_scale[1], n->x0);
    NET_CUDA(n, cudaGetLastError());
    if (F) {
        NET_CUDA(n, cudaMemcpyAsync(n->stage, F, sizeof(double) * 6 * g.N, cudaMemcpyHostToDevice, n->stream));
        NET_CUDA(n, cudaMemsetAsync(n->dev_scalar + 1, 0, sizeof(double), n->stream));
        k_target_from_f64<<<grid_of(g.N, 256), 256, 0, n->stream>>>(g, n->stage, n->out_scale[0], n->out_scale[1],
                                                                     n->tgt, n->dev_scalar + 1);
        NET_CUDA(n, cudaGetLastError());
    }
    return MLB_OK;
}

}  // namespace

// ------------------------------------------------------------------ internal entry points for the step
cudaError_t mlbi_net_force_from_moments(mlb_net *n, const float4 *mom, float4 *force, cudaStream_t s)
{
    k_input_from_mom<<<grid_of(n->g.N, 256), 256, 0, s>>>(n->g, mom, n->in_scale[0], n->in_scale[1], n->x0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && net_forward(n, false, nullptr, force, s) != MLB_OK) e = n->cuda_err;
    return e;
}

cudaError_t mlbi_force_error(long long n4, const float4 *fs, const float4 *fx, double *sums, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    k_force_error<<<grid_of(n4, 256), 256, 0, s>>>(n4, fs, fx, sums);
    return cudaGetLastError();
}

bool mlbi_net_timed_out(mlb_net *n)
{
    int f = 0;
    if (cudaMemcpy(&f, n->flag, sizeof f, cudaMemcpyDeviceToHost) != cudaSuccess) return true;
    return f != 0;
}

bool mlbi_net_matches(const mlb_net *n, int nx, int ny, int nz)
{
    return n && n->g.nx == nx && n->g.ny == ny && n->g.nz == nz;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

int64_t mlb_net_param_count(void) { return kParams; }

mlb_status mlb_net_create(const int32_t *dims, mlb_net **out)
{
    if (!out) return MLB_EINVAL;
    *out = nullptr;
    if (!dims || dims[0] < 3 || dims[1] < 3 || dims[2] < 3) return MLB_EINVAL;
    mlb_net *n = new (std::nothrow) mlb_net();
    if (!n) return MLB_ENOMEM;
    n->g.nx = dims[0];
    n->g.ny = dims[1];
    n->g.nz = dims[2];
    n->g.N = (long long)dims[0] * dims[1] * dims[2];
    const long long N = n->g.N;
    cudaError_t e = cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking);
    auto al = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    al((void **)&n->P, sizeof(float) * kParams);
    al((void **)&n->G, sizeof(float) * kParams);
    al((void **)&n->m, sizeof(float) * kParams);
    al((void **)&n->v, sizeof(float) * kParams);
    al((void **)&n->W2f, sizeof(__nv_bfloat16) * kTaps * kHid * kHid);
    al((void **)&n->W2b, sizeof(__nv_bfloat16) * kTaps * kHid * kHid);
    al((void **)&n->x0, sizeof(float2) * N);
    for (__nv_bfloat16 **p : {&n->pre1, &n->act1, &n->pre2, &n->act2, &n->dpre2, &n->dpre1})
        al((void **)p, sizeof(__nv_bfloat16) * kHid * N);
    al((void **)&n->out, sizeof(float) * kOut * N);
    al((void **)&n->tgt, sizeof(float) * kOut * N);
    al((void **)&n->dout, sizeof(float) * kOut * N);
    al((void **)&n->dev_scalar, sizeof(double) * 2);
    al((void **)&n->stage, sizeof(double) * 6 * N);
    al((void **)&n->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(n->flag, 0, sizeof(int), n->stream);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, dev);
    n->tc = n->g.nx % kTcM == 0 && (long long)n->g.nx * n->g.ny * kHid < (1ll << 31);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->m, 0, sizeof(float) * kParams, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->v, 0, sizeof(float) * kParams, n->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->P, 0, sizeof(float) * kParams, n->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
    if (e != cudaSuccess) {
        mlb_net_destroy(n);
        return MLB_ENOMEM;
    }
    *out = n;
    return MLB_OK;
}

mlb_status mlb_net_set_params(mlb_net *n, const float *p)
{
    if (!n || !p) return MLB_EINVAL;
    for (int i = 0; i < kParams; ++i)
        if (!std::isfinite(p[i])) return MLB_EINVAL;
    NET_CUDA(n, cudaMemcpyAsync(n->P, p, sizeof(float) * kParams, cudaMemcpyHostToDevice, n->stream));
    NET_CUDA(n, cudaMemsetAsync(n->m, 0, sizeof(float) * kParams, n->stream));
    NET_CUDA(n, cudaMemsetAsync(n->v, 0, sizeof(float) * kParams, n->stream));
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
    n->adam_t = 0;
    n->weights_dirty = true;
    return MLB_OK;
}

mlb_status mlb_net_get_params(mlb_net *n, float *p)
{
    if (!n || !p) return MLB_EINVAL;
    NET_CUDA(n, cudaMemcpyAsync(p, n->P, sizeof(float) * kParams, cudaMemcpyDeviceToHost, n->stream));
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
    return MLB_OK;
}

mlb_status mlb_net_set_scales(mlb_net *n, const double *in_scale, const double *out_scale)
{
    if (!n || !in_scale || !out_scale) return MLB_EINVAL;
    for (int a = 0; a < 2; ++a) {
        if (!(in_scale[a] > 0.0) || !(out_scale[a] > 0.0) || !std::isfinite(in_scale[a]) ||
            !std::isfinite(out_scale[a]))
            return MLB_EINVAL;
        n->in_scale[a] = (float)in_scale[a];
        n->out_scale[a] = (float)out_scale[a];
    }
    return MLB_OK;
}

mlb_status mlb_net_forward(mlb_net *n, const double *dn, double *force)
{
    if (!n || !dn || !force) return MLB_EINVAL;
    const long long N = n->g.N;
    mlb_status st = stage_frame(n, dn, nullptr);
    if (st != MLB_OK) return st;
    st = net_forward(n, false, n->out, nullptr, n->stream);
    if (st != MLB_OK) return st;
    std::vector<float> o((size_t)kOut * N);
    NET_CUDA(n, cudaMemcpyAsync(o.data(), n->out, sizeof(float) * kOut * N, cudaMemcpyDeviceToHost, n->stream));
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
    if (mlbi_net_timed_out(n)) {
        n->err = "a bounded wait on the tensor-core MMAs gave up";
        return MLB_ETIMEOUT;
    }
    for (long long r = 0; r < N; ++r)
        for (int a = 0; a < 2; ++a)
            for (int i = 0; i < 3; ++i) force[(a * 3 + i) * N + r] = o[r * kOut + 3 * a + i] / n->out_scale[a];
    return MLB_OK;
}

mlb_status mlb_net_gradient(mlb_net *n, const double *dn, const double *F, float *grad, double *loss)
{
    if (!n || !dn || !F) return MLB_EINVAL;
    mlb_status st = stage_frame(n, dn, F);
    if (st == MLB_OK) st = net_forward(n, true, n->out, nullptr, n->stream);
    if (st == MLB_OK) st = net_backward(n);
    if (st != MLB_OK) return st;
    if (grad) NET_CUDA(n, cudaMemcpyAsync(grad, n->G, sizeof(float) * kParams, cudaMemcpyDeviceToHost, n->stream));
    if (loss) NET_CUDA(n, cudaMemcpyAsync(loss, n->dev_scalar, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
    return MLB_OK;
}

mlb_status mlb_net_train(mlb_net *n, const double *dn, const double *F, int32_t iters, double lr, double *loss)
{
    if (!n || !dn || !F || iters < 1 || !(lr > 0.0)) return MLB_EINVAL;
    mlb_status st = stage_frame(n, dn, F);
    if (st != MLB_OK) return st;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int it = 0; it < iters; ++it) {
        st = net_forward(n, true, n->out, nullptr, n->stream);
        if (st == MLB_OK) st = net_backward(n);
        if (st != MLB_OK) return st;
        // the biases keep their set values (zero: the network stays odd in its input)
        NET_CUDA(n, cudaMemsetAsync(n->G + kOffB1, 0, sizeof(float) * kHid, n->stream));
        NET_CUDA(n, cudaMemsetAsync(n->G + kOffB2, 0, sizeof(float) * kHid, n->stream));
        NET_CUDA(n, cudaMemsetAsync(n->G + kOffB3, 0, sizeof(float) * kOut, n->stream));
        ++n->adam_t;
        const float c1 = 1.f / (1.f - std::pow(b1, (float)n->adam_t)), c2 = 1.f / (1.f - std::pow(b2, (float)n->adam_t));
        k_adam<<<(kParams + 255) / 256, 256, 0, n->stream>>>(kParams, n->P, n->G, n->m, n->v, (float)lr, b1, b2, c1, c2,
                                                             1e-8f);
        NET_CUDA(n, cudaGetLastError());
        n->weights_dirty = true;
    }
    if (loss) NET_CUDA(n, cudaMemcpyAsync(loss, n->dev_scalar, sizeof(double), cudaMemcpyDeviceToHost, n->stream));
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
    return MLB_OK;
}

const char *mlb_net_last_error(const mlb_net *n) { return n ? n->err.c_str() : "null net"; }

void mlb_net_destroy(mlb_net *n)
{
    if (!n) return;
    if (n->stream) cudaStreamSynchronize(n->stream);
    for (void *p : {(void *)n->P, (void *)n->G, (void *)n->m, (void *)n->v, (void *)n->W2f, (void *)n->W2b,
                    (void *)n->x0, (void *)n->pre1, (void *)n->act1, (void *)n->pre2, (void *)n->act2,
                    (void *)n->dpre2, (void *)n->dpre1, (void *)n->out, (void *)n->tgt, (void *)n->dout,
                    (void *)n->dev_scalar, (void *)n->stage, (void *)n->flag})
        if (p) cudaFree(p);
    if (n->stream) cudaStreamDestroy(n->stream);
    delete n;
}

}  // extern "C"
