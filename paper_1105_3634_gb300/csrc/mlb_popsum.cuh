// mlb_popsum.cuh -- FP64 mass and momentum sums taken from the populations
// themselves (the conservation laws of Eqs. continuity and momentcomponent:
// sum_r n^a and sum_a sum_r j^a with n^a = sum_i f_i^a, j^a = sum_i c_i f_i^a,
// masses 1).  Every population is converted to FP64 before any addition, so
// the sums carry no FP32 rounding beyond that of the stored populations.
// Shared by mlb_conservation (the context's buffers) and
// mlb_conservation_noalloc (a fixed device array), which therefore agree bit
// for bit.  Internal header.
#pragma once

#include <cuda_runtime.h>

namespace mlbps {
namespace {          // each including unit gets its own kernels

constexpr int kBlocks = 512;          // blocks of the first pass; partial holds kBlocks x (S + 3) doubles
constexpr int kThreads = 256;
constexpr int kMaxWidth = 4 + 3;      // MLB_MAX_SPECIES masses + 3 momentum components

// D3Q19 velocities in the order of mlb_velocity_set
__device__ constexpr int PX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__device__ constexpr int PY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__device__ constexpr int PZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

// Block b sums the sites r = b * kThreads + t (grid-strided) in a fixed
// order: per site and species sum_i f_i and sum_i c_i f_i in FP64; then a
// fixed-order tree over the block.  Every block writes all S + 3 of its
// partials, so nothing from an earlier call is read.  f: [S][19][N] FP32
// populations minus w_i n_ref.
template <int S>
__global__ void __launch_bounds__(kThreads) k_pop_sums(const float *__restrict__ f, long long N,
                                                       double *__restrict__ partial)
{
    constexpr int W = S + 3;
    double acc[W];
#pragma unroll
    for (int k = 0; k < W; ++k) acc[k] = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < S; ++a) {
            const float *fa = f + (long long)a * 19 * N + r;
            double m0 = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                const double v = (double)__ldg(fa + i * N);
                m0 += v;
                if (PX[i]) mx += PX[i] * v;
                if (PY[i]) my += PY[i] * v;
                if (PZ[i]) mz += PZ[i] * v;
            }
            acc[a] += m0;
            acc[S + 0] += mx;
            acc[S + 1] += my;
            acc[S + 2] += mz;
        }
    }
    __shared__ double sh[W][kThreads];
#pragma unroll
    for (int k = 0; k < W; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < W; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < W) partial[blockIdx.x * W + threadIdx.x] = sh[threadIdx.x][0];
}

struct Nref {
    double v[kMaxWidth - 3];
};

// Sum of the kBlocks partials of each of the W = S + 3 sums: two per thread,
// then one fixed-order tree; mass[a] gets n_ref^a N back (the populations are
// stored minus w_i n_ref and sum_i w_i = 1).  One block of kBlocks / 2 threads.
__global__ void __launch_bounds__(kBlocks / 2) k_pop_sums_final(const double *__restrict__ partial, int S,
                                                                long long N, Nref nref, double *__restrict__ out)
{
    const int W = S + 3;
    __shared__ double sh[kMaxWidth][kBlocks / 2];
    for (int k = 0; k < W; ++k)
        sh[k][threadIdx.x] = partial[threadIdx.x * W + k] + partial[(threadIdx.x + kBlocks / 2) * W + k];
    __syncthreads();
    for (int s = kBlocks / 4; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < W; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x < W) out[threadIdx.x] = sh[threadIdx.x][0] + (threadIdx.x < S ? nref.v[threadIdx.x] * (double)N : 0.0);
}

// Both launches on stream s; partial must hold kBlocks * (S + 3) doubles.
inline cudaError_t launch_pop_sums(const float *f, int S, long long N, const Nref &nref, double *partial,
                                   double *out, cudaStream_t s)
{
    switch (S) {
    case 1: k_pop_sums<1><<<kBlocks, kThreads, 0, s>>>(f, N, partial); break;
    case 2: k_pop_sums<2><<<kBlocks, kThreads, 0, s>>>(f, N, partial); break;
    case 3: k_pop_sums<3><<<kBlocks, kThreads, 0, s>>>(f, N, partial); break;
    case 4: k_pop_sums<4><<<kBlocks, kThreads, 0, s>>>(f, N, partial); break;
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_pop_sums_final<<<1, kBlocks / 2, 0, s>>>(partial, S, N, nref, out);
    return cudaGetLastError();
}

}  // namespace
}  // namespace mlbps
