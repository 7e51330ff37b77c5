// mlb_pass1.cu -- launchers of pass 1 of a time step (device code in
// mlb_pass1.cuh): the exact pass and the learned surrogate's variant.
#include "mlb_pass1.cuh"

namespace {

template <int S, int R, bool DRAG, int MODE = kExact>
cudaError_t launch_pass1_tiled(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    constexpr int TY = mlbi_tile_ty(S, R);
    if constexpr (TY == 0) {
        return cudaErrorInvalidValue;
    } else {
        using T = Tile<S, R, TY>;
        auto k = k_pass1_tiled<S, R, DRAG, TY, MODE>;
        const size_t bytes = T::bytes + staged_table_bytes<T, R>(p);
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        const dim3 g((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + TY - 1) / TY),
                     (unsigned)((p.nz + p.zchunk - 1) / p.zchunk));
        k<<<g, dim3(kBX, TY), bytes, s>>>(p, b.mom, b.dg, b.table, b.fext, b.attr, b.mom, b.frest, b.pst);
        return cudaGetLastError();
    }
}

template <int S, bool DRAG>
cudaError_t launch_pass1(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    if (p.hc_from_attr) {
        // the surrogate's case only: binary, no drag-only mode, reach 1 or 2
        if constexpr (S == 2 && !DRAG) {
            if (p.tile_r == 1) return launch_pass1_tiled<S, 1, DRAG, kSurrogate>(p, b, s);
            if (p.tile_r == 2) return launch_pass1_tiled<S, 2, DRAG, kSurrogate>(p, b, s);
        }
        return cudaErrorInvalidValue;
    }
    if (p.tile_r == 1) return launch_pass1_tiled<S, 1, DRAG>(p, b, s);
    if (p.tile_r == 2) return launch_pass1_tiled<S, 2, DRAG>(p, b, s);
    if (p.tile_r == 3) return launch_pass1_tiled<S, 3, DRAG>(p, b, s);
    k_pass1<S, DRAG, kExact><<<tiled_grid(p), dim3(kBX, kBY), 0, s>>>(p, b.mom, b.dg, b.table, b.fext, b.attr, b.mom,
                                                                        b.frest, b.pst);
    return cudaGetLastError();
}

template <int S, int R, bool DRAG>
cudaError_t launch_pass1_group(const mlbi_group &g, cudaStream_t s)
{
    constexpr int TY = mlbi_tile_ty(S, R);
    if constexpr (TY == 0) {
        return cudaErrorInvalidValue;
    } else {
        using T = Tile<S, R, TY>;
        auto k = k_pass1_group<S, R, DRAG, TY>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)T::bytes);
        if (e != cudaSuccess) return e;
        k<<<(unsigned)g.nblk[MLBI_GROUP_PASS1], dim3(kBX, TY), T::bytes, s>>>(g.mem, g.blk[MLBI_GROUP_PASS1]);
        return cudaGetLastError();
    }
}

template <int S, int R>
cudaError_t launch_pass1_group_r(const mlbi_group &g, cudaStream_t s)
{
    return g.drag ? launch_pass1_group<S, R, true>(g, s) : launch_pass1_group<S, R, false>(g, s);
}

}  // namespace

cudaError_t mlbi_launch_group_pass1(const mlbi_group &g, cudaStream_t s)
{
    if (g.nblk[MLBI_GROUP_PASS1] < 1) return cudaErrorInvalidValue;
    if (g.S == 1) return g.R == 1 ? launch_pass1_group_r<1, 1>(g, s) : launch_pass1_group_r<1, 2>(g, s);
    if (g.S == 2) return g.R == 1 ? launch_pass1_group_r<2, 1>(g, s) : launch_pass1_group_r<2, 2>(g, s);
    return cudaErrorInvalidValue;
}

cudaError_t mlbi_launch_pass1(const mlbi_params &p, const mlbi_buffers &b, cudaStream_t s)
{
    if (p.drag_only) { MLBI_DISPATCH_S(return launch_pass1<SS, true>(p, b, s)); }
    MLBI_DISPATCH_S(return launch_pass1<SS, false>(p, b, s));
    return cudaErrorInvalidValue;
}
