// mlb_device.cuh -- device helpers shared by the kernel translation units:
// the D3Q19 velocity set, lattice addressing with periodic wrap and walls,
// the 32 x 4 site tiles, and cp.async staging.  Internal header.
#pragma once

#include "mlb_internal.h"

namespace {

// D3Q19 velocities: rest, 6 axis links, 12 face diagonals; opposite of i >= 1 is i^1 shifted
__device__ constexpr int CX[MLBI_Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
__device__ constexpr int CY[MLBI_Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
__device__ constexpr int CZ[MLBI_Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
__device__ constexpr float WQ[MLBI_Q] = {1.f / 3.f,
                                         1.f / 18.f, 1.f / 18.f, 1.f / 18.f, 1.f / 18.f, 1.f / 18.f, 1.f / 18.f,
                                         1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f,
                                         1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};

__device__ __forceinline__ int opposite(int i) { return i == 0 ? 0 : (((i - 1) ^ 1) + 1); }

// the same velocity set for a runtime index, from bit tables (no memory access):
// component = (bit of "plus" mask) - (bit of "minus" mask)
__device__ __forceinline__ int comp_of(int i, unsigned plus, unsigned minus)
{
    return (int)((plus >> i) & 1u) - (int)((minus >> i) & 1u);
}
__device__ __forceinline__ int CXv(int i) { return comp_of(i, 0x2A82u, 0x5504u); }
__device__ __forceinline__ int CYv(int i) { return comp_of(i, 0x28488u, 0x50310u); }
__device__ __forceinline__ int CZv(int i) { return comp_of(i, 0x4C820u, 0x33040u); }
__device__ __forceinline__ float WQv(int i) { return i == 0 ? 1.f / 3.f : (i < 7 ? 1.f / 18.f : 1.f / 36.f); }

constexpr int kBlock = 256;
constexpr float kTinyDensity = 1e-12f;

inline unsigned grid_for(long long N)
{
    long long g = (N + kBlock - 1) / kBlock;
    if (g < 1) g = 1;
    if (g > (1ll << 30)) g = 1ll << 30;
    return (unsigned)g;
}

// r + d with periodic wrap (|d| < extent is guaranteed by the host) or -1 beyond a wall
__device__ __forceinline__ long long neighbour(const mlbi_params &p, int x, int y, int z, int dx, int dy, int dz)
{
    int c0 = x + dx, c1 = y + dy, c2 = z + dz;
    if (p.wall_axis == 0) { if (c0 < 0 || c0 >= p.nx) return -1; }
    else { c0 += (c0 < 0) ? p.nx : 0; c0 -= (c0 >= p.nx) ? p.nx : 0; }
    if (p.wall_axis == 1) { if (c1 < 0 || c1 >= p.ny) return -1; }
    else { c1 += (c1 < 0) ? p.ny : 0; c1 -= (c1 >= p.ny) ? p.ny : 0; }
    if (p.wall_axis == 2) { if (c2 < 0 || c2 >= p.nz) return -1; }
    else { c2 += (c2 < 0) ? p.nz : 0; c2 -= (c2 >= p.nz) ? p.nz : 0; }
    return c0 + (long long)p.nx * (c1 + (long long)p.ny * c2);
}

// ------------------------------------------------------------------ site mapping of the stencil kernels
// Blocks of 32 x 4 sites (x fastest): a warp covers 32 consecutive x, so
// every stream of the structure of arrays is read in 128-byte rows.  Sites
// farther than `reach` from every face (the interior) address neighbours by
// the precomputed linear offset of each stencil entry; the others wrap or
// stop at walls through `neighbour`.
constexpr int kBX = 32, kBY = 4;

struct Loc {
    int x, y, z;
    long long r;
    bool interior;
};

__device__ __forceinline__ bool locate(const mlbi_params &p, Loc &L)
{
    L.x = blockIdx.x * kBX + threadIdx.x;
    L.y = blockIdx.y * kBY + threadIdx.y;
    L.z = blockIdx.z;
    if (L.x >= p.nx || L.y >= p.ny) return false;
    L.r = L.x + (long long)p.nx * (L.y + (long long)p.ny * L.z);
    const int R = p.reach;
    L.interior = L.x >= R && L.x < p.nx - R && L.y >= R && L.y < p.ny - R && L.z >= R && L.z < p.nz - R;
    return true;
}

// index of r + sign*d for table entry (e0, e1), or -1 beyond a wall
__device__ __forceinline__ long long nbr(const mlbi_params &p, const Loc &L, const float4 &e0, const float4 &e1,
                                         int sign)
{
    if (L.interior) return L.r + sign * (long long)__float_as_int(e1.x);
    int dx, dy, dz;
    mlbi_unpack(__float_as_int(e0.w), dx, dy, dz);
    return neighbour(p, L.x, L.y, L.z, sign * dx, sign * dy, sign * dz);
}

__host__ __device__ constexpr int pair_of(int a, int b, int S)
{
    return a <= b ? a * S - a * (a - 1) / 2 + (b - a) : b * S - b * (b - 1) / 2 + (a - b);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ------------------------------------------------------------------ TMA and mbarriers
// One mbarrier per CTA tracks the bulk tensor copies of a z plane; waits are
// bounded (kSpinLimit tries) so that a copy that never lands turns into an
// error flag instead of a hang.
constexpr unsigned kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase)
{
    for (unsigned it = 0; it < kSpinLimit; ++it) {
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
// tiled bulk tensor copies global -> shared, completing on mbarrier `bar`;
// `map` is the address of a __grid_constant__ CUtensorMap kernel parameter
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const void *map, uint32_t bar, int c0, int c1, int c2, int c3)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%3, %4, %5, %6}], [%2];"
                 ::"r"(dst), "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const void *map, uint32_t bar, int c0, int c1, int c2, int c3,
                                            int c4)
{
    asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];"
                 ::"r"(dst), "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
                 : "memory");
}

__device__ __forceinline__ int wrap_or_out(int c, int L, bool wall)
{
    if (wall) return (c < 0 || c >= L) ? -1 : c;
    c %= L;
    return c < 0 ? c + L : c;
}


// ring slot of plane z0 - R + k
__device__ __forceinline__ int ring(int k, int nslot) { return k % nslot; }

// ------------------------------------------------------------------ centre moments
template <int S>
struct Centre {
    float n[S], dn[S], u[S][3];
};

template <int S>
__device__ __forceinline__ void load_centre(const mlbi_params &p, const float4 *__restrict__ mom, long long r,
                                            Centre<S> &c)
{
#pragma unroll
    for (int a = 0; a < S; ++a) {
        const float4 v = mom[a * p.N + r];
        c.dn[a] = v.x;
        c.n[a] = p.nref[a] + v.x;
        c.u[a][0] = v.y; c.u[a][1] = v.z; c.u[a][2] = v.w;
    }
}

// ------------------------------------------------------------------ grouped launches
// The block's member parameters, copied from global into shared memory by the
// whole block (ends with a barrier).
__device__ __forceinline__ void group_params(const mlbi_member *__restrict__ m, mlbi_params &sp)
{
    static_assert(sizeof(mlbi_params) % 4 == 0, "parameters copied as words");
    const int *src = reinterpret_cast<const int *>(&m->p);
    int *dst = reinterpret_cast<int *>(&sp);
    const int nt = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int k = tid; k < (int)(sizeof(mlbi_params) / 4); k += nt) dst[k] = __ldg(src + k);
    __syncthreads();
}

// make a tensor map that the host wrote to global memory visible to the bulk
// copies of this thread (the tensormap proxy's acquire of its 128 bytes)
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

inline dim3 tiled_grid(const mlbi_params &p)
{
    return dim3((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + kBY - 1) / kBY), (unsigned)p.nz);
}

}  // namespace
