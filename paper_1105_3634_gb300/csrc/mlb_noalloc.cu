// mlb_noalloc.cu -- mlb_conservation_noalloc: FP64 mass and momentum sums of
// a population array the caller holds on the device, without allocating.
// The sums are those of mlb_conservation (the same kernels, mlb_popsum.cuh).
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
#include "mlb_popsum.cuh"

#include <cuda_runtime.h>

#include <cmath>

namespace {

// Block partial sums of the reduction: 512 blocks x (MLB_MAX_SPECIES + 3)
// doubles = 28 KiB per device.
static __device__ __align__(256) double g_noalloc_partials[mlbps::kBlocks * mlbps::kMaxWidth];

static_assert(mlbps::kMaxWidth == MLB_MAX_SPECIES + 3, "scratch width");

}  // namespace

extern "C" mlb_status mlb_conservation_noalloc(const float *fdev, const double *nref, int32_t nspecies,
                                               int64_t nsites, double *out, void *stream)
{
    if (!fdev || !nref || !out) return MLB_EINVAL;
    if (nspecies < 1 || nspecies > MLB_MAX_SPECIES) return MLB_EINVAL;   // beyond the fixed scratch
    if (nsites < 1 || nsites > (1ll << 34)) return MLB_EINVAL;
    mlbps::Nref nr{};
    for (int a = 0; a < nspecies; ++a) {
        if (!std::isfinite(nref[a])) return MLB_EINVAL;
        nr.v[a] = nref[a];
    }
    // The array's device address on the current device.  Looked up on every
    // call (a host-side query that allocates nothing), so that a device reset
    // or a new context between calls cannot leave a stale address behind.
    void *scratch = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_noalloc_partials) != cudaSuccess) return MLB_ECUDA;
    if (mlbps::launch_pop_sums(fdev, nspecies, (long long)nsites, nr, (double *)scratch, out,
                               (cudaStream_t)stream) != cudaSuccess)
        return MLB_ECUDA;
    return MLB_OK;
}
