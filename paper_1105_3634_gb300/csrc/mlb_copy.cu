// mlb_copy.cu -- the measured peaks the kernels' roofline fractions are
// quoted against: the device-to-device copy bandwidth (a grid-stride float4
// copy between two buffers larger than L2) and the FP32 FMA throughput (16
// independent dependent-FMA chains per thread, as packed pairs), each timed
// with CUDA events over `reps` launches.
#include "mlb.h"

#include <cuda_runtime.h>

namespace {

__global__ void __launch_bounds__(256) k_copy(const float4 *__restrict__ a, float4 *__restrict__ b, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = a[i];
}

// 8 packed pairs = 16 FP32 chains per thread, `iters` rounds of one FMA on
// each; the result is written only if a chain ends on an impossible value,
// so the work cannot be dropped and nothing is stored
__global__ void __launch_bounds__(256) k_fma(int iters, float x, float y, float *__restrict__ out)
{
    float2 c[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) c[k] = make_float2((float)(threadIdx.x + k), (float)(blockIdx.x - k));
    const float2 x2 = make_float2(x, x), y2 = make_float2(y, y);
    for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int k = 0; k < 8; ++k) c[k] = __ffma2_rn(c[k], x2, y2);
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += c[k].x + c[k].y;
    if (sum == -1.2345e38f) out[0] = sum;
}

}  // namespace

extern "C" mlb_status mlb_fma_throughput(int32_t iters, int32_t reps, double *tflops)
{
    if (!tflops || iters < 1 || reps < 1) return MLB_EINVAL;
    *tflops = 0.0;
    float *out = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms = 0.f;
    const unsigned grid = (unsigned)sms * 8;              // 2048 threads per SM
    if (e == cudaSuccess) {
        // x slightly below 1 keeps the chains finite for any iteration count
        k_fma<<<grid, 256, 0, s>>>(iters, 0.999999f, 1e-7f, out);
        cudaEventRecord(e0, s);
        for (int k = 0; k < reps; ++k) k_fma<<<grid, 256, 0, s>>>(iters, 0.999999f, 1e-7f, out);
        cudaEventRecord(e1, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e == cudaSuccess && ms > 0.f)
        *tflops = 2.0 * 16.0 * (double)iters * grid * 256.0 * reps / (ms * 1e-3) / 1e12;
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    if (out) cudaFree(out);
    if (e == cudaErrorMemoryAllocation) return MLB_ENOMEM;
    return e == cudaSuccess ? MLB_OK : MLB_ECUDA;
}

extern "C" mlb_status mlb_copy_bandwidth(int64_t bytes, int32_t reps, double *gbs)
{
    if (!gbs || bytes < (int64_t)1 << 20 || reps < 1) return MLB_EINVAL;
    *gbs = 0.0;
    const long long n4 = bytes / 16;
    float4 *a = nullptr, *b = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaMalloc(&a, (size_t)n4 * 16);
    if (e == cudaSuccess) e = cudaMalloc(&b, (size_t)n4 * 16);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemsetAsync(a, 0, (size_t)n4 * 16, s);
    float ms = 0.f;
    if (e == cudaSuccess) {
        const unsigned grid = (unsigned)sms * 8;          // 8 blocks of 256 threads: 2048 threads per SM
        for (int k = 0; k < 2; ++k) k_copy<<<grid, 256, 0, s>>>(a, b, n4);
        cudaEventRecord(e0, s);
        for (int k = 0; k < reps; ++k) k_copy<<<grid, 256, 0, s>>>(a, b, n4);
        cudaEventRecord(e1, s);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e == cudaSuccess && ms > 0.f) *gbs = 2.0 * (double)n4 * 16.0 * reps / (ms * 1e-3) / 1e9;
    if (e1) cudaEventDestroy(e1);
    if (e0) cudaEventDestroy(e0);
    if (s) cudaStreamDestroy(s);
    if (b) cudaFree(b);
    if (a) cudaFree(a);
    if (e == cudaErrorMemoryAllocation) return MLB_ENOMEM;
    return e == cudaSuccess ? MLB_OK : MLB_ECUDA;
}
