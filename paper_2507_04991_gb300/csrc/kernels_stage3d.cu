// Instantiations of the P-ERK stage kernel for 3D meshes (split per dimension
// so that the translation units compile in parallel).
#include <cuda_runtime.h>

#include "stage.cuh"

namespace perrk {

template <int EQ, typename Real, bool CURVED>
static cudaError_t go(const StageParams &P, int epb, int grid, cudaStream_t st) {
    if (epb == 1) {
        if constexpr (stage_smem_bytes<3, EQ, Real, CURVED, 1>() <= 48 * 1024) {
            k_stage<3, EQ, Real, CURVED, 1><<<grid, 1 * ipow4(3), 0, st>>>(P);
            return cudaGetLastError();
        }
        return cudaErrorInvalidConfiguration;
    }
    if (epb == 2) {
        if constexpr (stage_smem_bytes<3, EQ, Real, CURVED, 2>() <= 48 * 1024) {
            k_stage<3, EQ, Real, CURVED, 2><<<grid, 2 * ipow4(3), 0, st>>>(P);
            return cudaGetLastError();
        }
        return cudaErrorInvalidConfiguration;
    }
    if (epb == 4) {
        if constexpr (stage_smem_bytes<3, EQ, Real, CURVED, 4>() <= 48 * 1024) {
            k_stage<3, EQ, Real, CURVED, 4><<<grid, 4 * ipow4(3), 0, st>>>(P);
            return cudaGetLastError();
        }
        return cudaErrorInvalidConfiguration;
    }
    return cudaErrorInvalidValue;
}

cudaError_t stage_launch_3d(const StageParams &P, bool burgers, bool mixed, bool curved, int epb, int grid, cudaStream_t st) {
    (void)burgers; (void)curved;
    if (mixed) return go<EQ_EULER, float, false>(P, epb, grid, st);
    return go<EQ_EULER, double, false>(P, epb, grid, st);
}

}  // namespace perrk
