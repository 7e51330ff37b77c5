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
    cudaStream_t stream = nullptr;
    long long adam_t = 0;
    bool weights_dirty = true;
    std::string err;
};

namespace {

mlb_status net_fail(mlb_net *n, cudaError_t e, const char *what)
{
    n->err = std::string(what) + ": " + cudaGetErrorString(e);
    return MLB_ECUDA;
}

#define NET_CUDA(net, call)                                                                        \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return net_fail((net), e_, #call);                                  \
    } while (0)

mlb_status refresh_w2(mlb_net *n)
{
    if (!n->weights_dirty) return MLB_OK;
    k_w2_bf16<<<(kTaps * kHid * kHid + 255) / 256, 256, 0, n->stream>>>(n->P, n->W2f, n->W2b);
    NET_CUDA(n, cudaGetLastError());
    n->weights_dirty = false;
    return MLB_OK;
}

// forward from x0 (already staged); training keeps the pre-activations
mlb_status net_forward(mlb_net *n, bool keep, float *out, float4 *force)
{
    mlb_status st = refresh_w2(n);
    if (st != MLB_OK) return st;
    const Geo &g = n->g;
    k_layer1<<<grid_of(g.N, 128), 128, 0, n->stream>>>(g, n->x0, n->P, keep ? n->pre1 : nullptr, n->act1);
    NET_CUDA(n, cudaGetLastError());
    NET_CUDA(n, cudaFuncSetAttribute(k_conv32_mma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kConvSmem));
    k_conv32_mma<true><<<grid_of((g.N + 15) / 16 * 32, 128), 128, kConvSmem, n->stream>>>(
        g, n->act1, n->W2f, n->P + kOffB2, nullptr, keep ? n->pre2 : nullptr, n->act2);
    NET_CUDA(n, cudaGetLastError());
    k_layer3<<<grid_of(g.N, 128), 128, 0, n->stream>>>(g, n->act2, n->P, out, force, 1.f / n->out_scale[0],
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
    cudaStream_t keep = n->stream;
    n->stream = s;
    k_input_from_mom<<<grid_of(n->g.N, 256), 256, 0, s>>>(n->g, mom, n->in_scale[0], n->in_scale[1], n->x0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && net_forward(n, false, nullptr, force) != MLB_OK) e = cudaErrorLaunchFailure;
    n->stream = keep;
    return e;
}

cudaError_t mlbi_force_error(long long n4, const float4 *fs, const float4 *fx, double *sums, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    k_force_error<<<grid_of(n4, 256), 256, 0, s>>>(n4, fs, fx, sums);
    return cudaGetLastError();
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
    st = net_forward(n, false, n->out, nullptr);
    if (st != MLB_OK) return st;
    std::vector<float> o((size_t)kOut * N);
    NET_CUDA(n, cudaMemcpyAsync(o.data(), n->out, sizeof(float) * kOut * N, cudaMemcpyDeviceToHost, n->stream));
    NET_CUDA(n, cudaStreamSynchronize(n->stream));
    for (long long r = 0; r < N; ++r)
        for (int a = 0; a < 2; ++a)
            for (int i = 0; i < 3; ++i) force[(a * 3 + i) * N + r] = o[r * kOut + 3 * a + i] / n->out_scale[a];
    return MLB_OK;
}

mlb_status mlb_net_gradient(mlb_net *n, const double *dn, const double *F, float *grad, double *loss)
{
    if (!n || !dn || !F) return MLB_EINVAL;
    mlb_status st = stage_frame(n, dn, F);
    if (st == MLB_OK) st = net_forward(n, true, n->out, nullptr);
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
        st = net_forward(n, true, n->out, nullptr);
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
                    (void *)n->dev_scalar, (void *)n->stage})
        if (p) cudaFree(p);
    if (n->stream) cudaStreamDestroy(n->stream);
    delete n;
}

}  // extern "C"
