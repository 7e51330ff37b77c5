// mlb_attraction.cu -- the attractive mean field of the RPA (Sec. III, G term
// of Eq. potmeanforce) as a column stencil on sm_103a.
//
// G^a(r) = sum_b sum_d K_ab(d) n^b(r + d), K_ab(d) = 6 eps_ab sigma_ab^6 d / |d|^8
// on sigma_ab <= |d| <= lambda_c sigma_ab.  K is odd, so n may be replaced by
// the deviation n - n_ref (the constant part sums to zero over the region).
//
// The region is cut into columns c = (dx, dy) of the half plane.  A column and
// its mirror -c hold, along z, the windows w+ = n(x + c, .) and w- = n(x - c, .);
// with D = w+ - w- and P = w+ + w- the oddness of K gives, per output plane z,
//   (G_x, G_y) += (dx, dy) [k(0) D(z) + sum_{dz>0} k(dz) (D(z+dz) + D(z-dz))]
//   G_z        +=          sum_{dz>0} dz k(dz) (P(z+dz) - P(z-dz))
// with k(dz) = 6 eps sigma^6 / (dx^2 + dy^2 + dz^2)^4 on the region, else 0.
// Each thread owns Z consecutive planes of one (x, y) site; a block stages the
// deviations of one neighbour species over its (32 + 2R) x (TY + 2R) x (Z + 2R)
// slab in shared memory, and every column window is read once into registers
// and reused by all Z outputs and every output species of the group.
#include "mlb_internal.h"
#include "mlb_device.cuh"

namespace {

template <int S, int R, int TY, int Z>
struct CTile {
    static constexpr int TXH = kBX + 2 * R, TYH = TY + 2 * R, TZH = Z + 2 * R;
    static constexpr int PL = TXH * TYH;                   // one slab plane
    static constexpr int NT = kBX * TY;                    // threads
    static constexpr int AG = (S % 2 == 0) ? 2 : 1;        // output species per pass
    static constexpr size_t bytes = (size_t)PL * TZH * sizeof(float);
};

// stage n^b - n_ref^b of the block's slab; beyond a wall there are no particles (n = 0)
template <int S, int R, int TY, int Z>
__device__ __forceinline__ void stage_slab(const mlbi_params &p, int x0, int y0, int z0,
                                           const float4 *__restrict__ momb, float nrefb, float *slab)
{
    using T = CTile<S, R, TY, Z>;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    for (int idx = tid; idx < T::PL; idx += T::NT) {
        const int hx = idx % T::TXH, hy = idx / T::TXH;
        const int x = wrap_or_out(x0 - R + hx, p.nx, p.wall_axis == 0);
        const int y = wrap_or_out(y0 - R + hy, p.ny, p.wall_axis == 1);
        const long long xy = (x < 0 || y < 0) ? -1 : x + (long long)p.nx * y;
        const long long nxy = (long long)p.nx * p.ny;
        for (int hz = 0; hz < T::TZH; ++hz) {
            const int z = wrap_or_out(z0 - R + hz, p.nz, p.wall_axis == 2);
            float *d = slab + hz * T::PL + idx;
            if (xy < 0 || z < 0) *d = -nrefb;
            else cp_async4(d, reinterpret_cast<const float *>(momb + xy + nxy * z));
        }
    }
    cp_async_commit();
}

template <int S, int R, int TY, int Z>
__global__ void __launch_bounds__(kBX * TY, 2) k_attraction_columns(const mlbi_params p,
                                                                    const float4 *__restrict__ mom,
                                                                    const float4 *__restrict__ cols,
                                                                    const float2 *__restrict__ wts,
                                                                    float4 *__restrict__ attr)
{
    using T = CTile<S, R, TY, Z>;
    constexpr int AG = T::AG, W = T::TZH;
    extern __shared__ float slab[];                         // [TZH][TYH][TXH]
    const int x0 = blockIdx.x * kBX, y0 = blockIdx.y * TY, z0 = blockIdx.z * Z;
    const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
    const float *centre = slab + (threadIdx.y + R) * T::TXH + threadIdx.x + R;
    const int stride = p.attr_r + 1;
    for (int a0 = 0; a0 < S; a0 += AG) {
        float acc[AG][Z][3];
#pragma unroll
        for (int g = 0; g < AG; ++g)
#pragma unroll
            for (int i = 0; i < Z; ++i) acc[g][i][0] = acc[g][i][1] = acc[g][i][2] = 0.f;
        for (int b = 0; b < S; ++b) {
            __syncthreads();                                 // the previous slab is consumed
            stage_slab<S, R, TY, Z>(p, x0, y0, z0, mom + b * p.N, p.nref[b], slab);
            cp_async_wait_all();
            __syncthreads();
            int pr[AG];
#pragma unroll
            for (int g = 0; g < AG; ++g) pr[g] = pair_of(a0 + g, b, S);
            for (int c = 0; c < p.acol_count; ++c) {
                const float4 cc = __ldg(&cols[c]);
                const int dx = __float_as_int(cc.x), dy = __float_as_int(cc.y), E = __float_as_int(cc.z);
                const int off = dy * T::TXH + dx;
                float D[W], P[W];
#pragma unroll
                for (int j = 0; j < W; ++j) {
                    const float vp = centre[j * T::PL + off], vm = centre[j * T::PL - off];
                    D[j] = vp - vm;
                    P[j] = vp + vm;
                }
                const float2 *wc = wts + (size_t)c * p.npairs * stride;
                float Tt[AG][Z];
#pragma unroll
                for (int g = 0; g < AG; ++g) {
                    const float k0 = __ldg(&wc[pr[g] * stride]).x;
#pragma unroll
                    for (int i = 0; i < Z; ++i) Tt[g][i] = k0 * D[i + R];
                }
#pragma unroll
                for (int dz = 1; dz <= R; ++dz) {
                    if (dz > E) break;
                    float2 k[AG];
#pragma unroll
                    for (int g = 0; g < AG; ++g) k[g] = __ldg(&wc[pr[g] * stride + dz]);
#pragma unroll
                    for (int i = 0; i < Z; ++i) {
                        const float sd = D[i + R + dz] + D[i + R - dz];
                        const float sp = P[i + R + dz] - P[i + R - dz];
#pragma unroll
                        for (int g = 0; g < AG; ++g) {
                            Tt[g][i] = fmaf(k[g].x, sd, Tt[g][i]);
                            acc[g][i][2] = fmaf(k[g].y, sp, acc[g][i][2]);
                        }
                    }
                }
                const float fx = (float)dx, fy = (float)dy;
#pragma unroll
                for (int g = 0; g < AG; ++g)
#pragma unroll
                    for (int i = 0; i < Z; ++i) {
                        acc[g][i][0] = fmaf(fx, Tt[g][i], acc[g][i][0]);
                        acc[g][i][1] = fmaf(fy, Tt[g][i], acc[g][i][1]);
                    }
            }
        }
        if (x < p.nx && y < p.ny) {
#pragma unroll
            for (int g = 0; g < AG; ++g)
#pragma unroll
                for (int i = 0; i < Z; ++i) {
                    const int z = z0 + i;
                    if (z < p.nz) {
                        const long long r = x + (long long)p.nx * (y + (long long)p.ny * z);
                        attr[(a0 + g) * p.N + r] = make_float4(acc[g][i][0], acc[g][i][1], acc[g][i][2], 0.f);
                    }
                }
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

constexpr int kAttrTY = 8, kAttrZ = 8;

template <int S, int R>
cudaError_t launch_columns(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    using T = CTile<S, R, kAttrTY, kAttrZ>;
    auto k = k_attraction_columns<S, R, kAttrTY, kAttrZ>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::bytes);
    if (e != cudaSuccess) return e;
    const dim3 g((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + kAttrTY - 1) / kAttrTY),
                 (unsigned)((p.nz + kAttrZ - 1) / kAttrZ));
    const float4 *cols = reinterpret_cast<const float4 *>(b.table) + p.acol_start;
    const float2 *wts = reinterpret_cast<const float2 *>(reinterpret_cast<const float4 *>(b.table) + p.aw_start);
    k<<<g, dim3(kBX, kAttrTY), T::bytes, s>>>(p, b.mom, cols, wts, b.attr);
    return cudaGetLastError();
}

// reach tiers: the smallest tier >= the attraction reach (a wider halo than
// needed is harmless: columns and weights stop at the true reach)
template <int S>
cudaError_t attraction_for_reach(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    if (p.attr_r <= 3) return launch_columns<S, 3>(p, b, s);
    if (p.attr_r <= 5) return launch_columns<S, 5>(p, b, s);
    if (p.attr_r <= 7) return launch_columns<S, 7>(p, b, s);
    if (p.attr_r <= 8) return launch_columns<S, 8>(p, b, s);
    return cudaErrorInvalidValue;
}

cudaError_t mlbi_launch_attraction(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    if (p.acol_count <= 0) return cudaErrorInvalidValue;
    MLBI_DISPATCH_S(return attraction_for_reach<SS>(p, b, s));
    return cudaErrorInvalidValue;
}
