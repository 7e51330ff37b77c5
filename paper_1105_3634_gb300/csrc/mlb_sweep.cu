// mlb_sweep.cu -- further Jacobi sweeps of the half step of the semi-implicit
// forcing (Eq. evolution with the half-force shift): u* = u + a(u*)/2 solved
// at every site as (I + Gamma/2) du = (F^hc + G + F_ext + F^v)/2, where the
// velocity exchange F^v (Eqs. gammaab, viscousforce) now takes the partners'
// velocities from the previous sweep's u*.  Pass 1 is the first sweep; each
// further sweep is one more pass over the contact shells (device code in
// mlb_pass1.cuh, mode kSweep).
#include "mlb_pass1.cuh"

namespace {

template <int S, int R, bool DRAG>
cudaError_t launch_sweep_tiled(const mlbi_params &p, const mlbi_buffers &b, const float4 *prev, float4 *next,
                               cudaStream_t s)
{
    constexpr int TY = mlbi_tile_ty(S, R);
    if constexpr (TY == 0) {
        return cudaErrorInvalidValue;
    } else {
        using T = Tile<S, R, TY>;
        auto k = k_pass1_tiled<S, R, DRAG, TY, kSweep>;
        const size_t bytes = T::bytes + staged_table_bytes<T, R>(p);
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        const dim3 g((unsigned)((p.nx + kBX - 1) / kBX), (unsigned)((p.ny + TY - 1) / TY),
                     (unsigned)((p.nz + p.zchunk - 1) / p.zchunk));
        k<<<g, dim3(kBX, TY), bytes, s>>>(p, prev, b.dg, b.table, b.fext, b.attr, b.mom, b.frest, next);
        return cudaGetLastError();
    }
}

template <int S, bool DRAG>
cudaError_t launch_sweep(const mlbi_params &p, const mlbi_buffers &b, const float4 *prev, float4 *next, cudaStream_t s)
{
    if (p.tile_r == 1) return launch_sweep_tiled<S, 1, DRAG>(p, b, prev, next, s);
    if (p.tile_r == 2) return launch_sweep_tiled<S, 2, DRAG>(p, b, prev, next, s);
    if (p.tile_r == 3) return launch_sweep_tiled<S, 3, DRAG>(p, b, prev, next, s);
    k_pass1<S, DRAG, kSweep><<<tiled_grid(p), dim3(kBX, kBY), 0, s>>>(p, prev, b.dg, b.table, b.fext, b.attr, b.mom,
                                                                        b.frest, next);
    return cudaGetLastError();
}

}  // namespace

cudaError_t mlbi_launch_sweep(const mlbi_params &p, const mlbi_buffers &b, const float4 *prev, float4 *next,
                              cudaStream_t s)
{
    if (p.drag_only) { MLBI_DISPATCH_S(return (launch_sweep<SS, true>(p, b, prev, next, s))); }
    MLBI_DISPATCH_S(return (launch_sweep<SS, false>(p, b, prev, next, s)));
    return cudaErrorInvalidValue;
}
