// mlb_attraction.cu -- the attractive mean field of the RPA (Sec. III, G term
// of Eq. potmeanforce) as a shared-memory z-marching stencil on sm_103a.
#include "mlb_internal.h"
#include "mlb_device.cuh"

namespace {

// ------------------------------------------------------------------ attraction (tiled)
// G^a = sum_b sum_{+d} K_ab(d) (n^b(r+d) - n^b(r-d))  (G term of Eq. potmeanforce, RPA),
// K_ab(d) = 6 eps_ab sigma_ab^6 d / |d|^8 on sigma_ab <= |d| <= lambda_c sigma_ab.
// z-marching like the force passes, staging only n - n_ref of every species:
// a ring of 2R + 2 planes of (32 + 2R) x (4 + 2R) sites, R = attraction reach.
template <int S, int R>
struct ATile {
    static constexpr int TXH = kBX + 2 * R, TYH = kBY + 2 * R, PLANE = TXH * TYH;
    static constexpr int NSLOT = 2 * R + 2;
    static constexpr size_t bytes = (size_t)NSLOT * S * PLANE * sizeof(float);
};

template <int S, int R>
__device__ __forceinline__ void stage_density_plane(const mlbi_params &p, int x0, int y0, int gz, int slot,
                                                    const float4 *__restrict__ mom, float *sa)
{
    using T = ATile<S, R>;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const int z = wrap_or_out(gz, p.nz, p.wall_axis == 2);
    for (int idx = tid; idx < T::PLANE; idx += kBX * kBY) {
        const int hx = idx % T::TXH, hy = idx / T::TXH;
        const int x = wrap_or_out(x0 - R + hx, p.nx, p.wall_axis == 0);
        const int y = wrap_or_out(y0 - R + hy, p.ny, p.wall_axis == 1);
        float *d = sa + slot * S * T::PLANE + idx;
        if (x < 0 || y < 0 || z < 0) {
#pragma unroll
            for (int b = 0; b < S; ++b) d[b * T::PLANE] = -p.nref[b];     // no particles beyond a wall
        } else {
            const long long g = x + (long long)p.nx * (y + (long long)p.ny * z);
#pragma unroll
            for (int b = 0; b < S; ++b) cp_async4(d + b * T::PLANE, reinterpret_cast<const float *>(mom + b * p.N + g));
        }
    }
}

template <int S, int R>
__global__ void __launch_bounds__(kBX * kBY) k_attraction_tiled(const mlbi_params p, const float4 *__restrict__ mom,
                                                                const mlbi_entry *__restrict__ tab,
                                                                float4 *__restrict__ attr)
{
    using T = ATile<S, R>;
    extern __shared__ float sa[];                  // [NSLOT][S][PLANE]
    const long long N = p.N;
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * kBY, z0 = blockIdx.z * p.zchunk;
    const int z1 = min(z0 + p.zchunk, p.nz);
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const bool active = x < p.nx && y < p.ny;
    const int cidx = (threadIdx.y + R) * T::TXH + threadIdx.x + R;
    for (int k = 0; k < 2 * R + 1; ++k) stage_density_plane<S, R>(p, x0, y0, z0 - R + k, ring(k, T::NSLOT), mom, sa);
    cp_async_commit();
    for (int z = z0; z < z1; ++z) {
        cp_async_wait_all();
        __syncthreads();
        const int kz = z - z0 + R;
        if (z + 1 < z1) {
            stage_density_plane<S, R>(p, x0, y0, z + R + 1, ring(kz + R + 1, T::NSLOT), mom, sa);
            cp_async_commit();
        }
        if (!active) continue;
        const long long r = x + (long long)p.nx * (y + (long long)p.ny * z);
#pragma unroll
        for (int a = 0; a < S; ++a) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int b = 0; b < S; ++b) {
                const mlbi_pair &pr = p.pair[pair_of(a, b, S)];
                const float *sb = sa + b * T::PLANE + cidx;
#pragma unroll 4
                for (int k = pr.attr_start; k < pr.attr_start + pr.attr_count; ++k) {
                    const float4 e0 = __ldg(&tab[2 * k]);
                    const float4 e1 = __ldg(&tab[2 * k + 1]);
                    const int off = __float_as_int(e1.z), dz = __float_as_int(e1.w);
                    const float vp = sb[ring(kz + dz, T::NSLOT) * S * T::PLANE + off];
                    const float vm = sb[ring(kz - dz, T::NSLOT) * S * T::PLANE - off];
                    const float d = vp - vm;          // deviations: n_ref cancels exactly
                    s0 += e0.x * d; s1 += e0.y * d; s2 += e0.z * d;
                }
            }
            attr[a * N + r] = make_float4(s0, s1, s2, 0.f);
        }
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

template <int S, int R>
cudaError_t launch_attraction_tiled(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    using T = ATile<S, R>;
    auto k = k_attraction_tiled<S, R>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::bytes);
    if (e != cudaSuccess) return e;
    const dim3 g((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + kBY - 1) / kBY),
                 (unsigned)((p.nz + p.zchunk - 1) / p.zchunk));
    k<<<g, dim3(kBX, kBY), T::bytes, s>>>(p, b.mom, b.table, b.attr);
    return cudaGetLastError();
}

// tile reach tiers: the smallest tier >= the attraction reach (a wider halo
// than needed is harmless); tiles above 200 KiB of shared memory are not built
template <int S, int R>
cudaError_t launch_tier(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    if constexpr (ATile<S, R>::bytes <= 200 * 1024) return launch_attraction_tiled<S, R>(p, b, s);
    return cudaErrorInvalidValue;
}

template <int S>
cudaError_t attraction_for_reach(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    if (p.attr_r <= 3) return launch_tier<S, 3>(p, b, s);
    if (p.attr_r <= 5) return launch_tier<S, 5>(p, b, s);
    if (p.attr_r <= 7) return launch_tier<S, 7>(p, b, s);
    if (p.attr_r <= 8) return launch_tier<S, 8>(p, b, s);
    return cudaErrorInvalidValue;
}

cudaError_t mlbi_launch_attraction(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    MLBI_DISPATCH_S(return attraction_for_reach<SS>(p, b, s));
    return cudaErrorInvalidValue;
}

