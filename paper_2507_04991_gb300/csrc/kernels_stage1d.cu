// Instantiations of the P-ERK stage kernel for 1D meshes (split per dimension
// so that the translation units compile in parallel).
#include <cuda_runtime.h>

#include "stage.cuh"

namespace perrk {

template <int EQ, typename Real, bool CURVED>
static cudaError_t go(const StageParams &P, int epb, int grid, cudaStream_t st) {
    if (epb == 16) {
        if constexpr (stage_smem_bytes<1, EQ, Real, CURVED, 16>() <= 48 * 1024) {
            k_stage<1, EQ, Real, CURVED, 16><<<grid, 16 * ipow4(1), 0, st>>>(P);
            return cudaGetLastError();
        }
        return cudaErrorInvalidConfiguration;
    }
    if (epb == 32) {
        if constexpr (stage_smem_bytes<1, EQ, Real, CURVED, 32>() <= 48 * 1024) {
            k_stage<1, EQ, Real, CURVED, 32><<<grid, 32 * ipow4(1), 0, st>>>(P);
            return cudaGetLastError();
        }
        return cudaErrorInvalidConfiguration;
    }
    return cudaErrorInvalidValue;
}

cudaError_t stage_launch_1d(const StageParams &P, bool burgers, bool mixed, bool curved, int epb, int grid, cudaStream_t st) {
    if (burgers) { if (mixed) return go<EQ_BURGERS, float, false>(P, epb, grid, st); return go<EQ_BURGERS, double, false>(P, epb, grid, st); }
    if (mixed) return go<EQ_EULER, float, false>(P, epb, grid, st);
    return go<EQ_EULER, double, false>(P, epb, grid, st);
}

}  // namespace perrk
