// mlb_noalloc.cu -- mlb_conservation_noalloc: FP64 mass and momentum sums of
// a population array the caller holds on the device, without allocating.
//
// Some callers cannot let the library allocate device memory: a host
// application whose memory manager owns every device byte (its own pool or a
// stream-ordered allocator that must not be mixed with cudaMalloc), or code
// that must not allocate once a run is under way.  Such callers cannot create
// an mlb context (mlb_create obtains all of a context's memory at once).  This
// entry point gives them the conservation check of the method's state: the
// caller passes the populations and an output buffer, both on the device,
// and the block partial sums of the reduction live in the fixed array
// below, which every GPU that loads this library holds until the process
// exits.
#include "mlb.h"

#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

namespace {

constexpr int kBlocks = 512;                        // blocks of the first reduction pass
constexpr int kThreads = 256;
constexpr int kWidth = MLB_MAX_SPECIES + 3;         // mass per species + 3 momentum components

// Block partial sums: kBlocks x kWidth doubles = 28 KiB per device.
static __device__ __align__(256) double g_noalloc_partials[kBlocks * kWidth];

// D3Q19 velocities in the order of mlb_velocity_set
__device__ constexpr int NX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__device__ constexpr int NY[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__device__ constexpr int NZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

struct NrefArg {
    double v[MLB_MAX_SPECIES];
};

// Per block: sums over its sites, in a fixed order, of sum_i f and
// sum_i c_i f; then a fixed-order tree over the block's threads.  Every block
// writes all kWidth of its partials, so no call reads a previous call's data.
__global__ void __launch_bounds__(kThreads) k_conservation_pop(const float *__restrict__ f, int S, long long N,
                                                               double *__restrict__ partial)
{
    const int W = S + 3;
    double acc[kWidth];
    for (int k = 0; k < kWidth; ++k) acc[k] = 0.0;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        for (int a = 0; a < S; ++a) {
            const float *fa = f + (long long)a * 19 * N + r;
            double m0 = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
#pragma unroll
            for (int i = 0; i < 19; ++i) {
                const double v = (double)fa[i * N];
                m0 += v;
                mx += NX[i] * v;
                my += NY[i] * v;
                mz += NZ[i] * v;
            }
            acc[a] += m0;
            acc[S + 0] += mx;
            acc[S + 1] += my;
            acc[S + 2] += mz;
        }
    }
    __shared__ double sh[kThreads];
    for (int k = 0; k < W; ++k) {
        sh[threadIdx.x] = acc[k];
        __syncthreads();
        for (int s = kThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[blockIdx.x * W + k] = sh[0];
        __syncthreads();
    }
}

__global__ void k_conservation_pop_final(const double *__restrict__ partial, int S, long long N, NrefArg nref,
                                         double *__restrict__ out)
{
    const int W = S + 3;
    if (threadIdx.x < W) {
        double s = 0.0;
        for (int b = 0; b < kBlocks; ++b) s += partial[b * W + threadIdx.x];
        if (threadIdx.x < S) s += nref.v[threadIdx.x] * (double)N;   // populations are stored minus w_i n_ref
        out[threadIdx.x] = s;
    }
}

// Device address of g_noalloc_partials, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_lock;
double *g_scratch[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(double **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> guard(g_lock);
    if (!g_scratch[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = (double *)p;
    }
    *ptr = g_scratch[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" mlb_status mlb_conservation_noalloc(const float *fdev, const double *nref, int32_t nspecies,
                                               int64_t nsites, double *out, void *stream)
{
    if (!fdev || !nref || !out) return MLB_EINVAL;
    if (nspecies < 1 || nspecies > MLB_MAX_SPECIES) return MLB_EINVAL;   // beyond the fixed scratch
    if (nsites < 1 || nsites > (1ll << 34)) return MLB_EINVAL;
    NrefArg nr{};
    for (int a = 0; a < nspecies; ++a) {
        if (!std::isfinite(nref[a])) return MLB_EINVAL;
        nr.v[a] = nref[a];
    }
    double *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return MLB_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    k_conservation_pop<<<kBlocks, kThreads, 0, s>>>(fdev, nspecies, (long long)nsites, scratch);
    if (cudaGetLastError() != cudaSuccess) return MLB_ECUDA;
    k_conservation_pop_final<<<1, 32, 0, s>>>(scratch, nspecies, (long long)nsites, nr, out);
    if (cudaGetLastError() != cudaSuccess) return MLB_ECUDA;
    return MLB_OK;
}
