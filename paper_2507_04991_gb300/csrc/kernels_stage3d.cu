// Instantiations of the P-ERK stage kernel for 3D meshes (split per dimension
// so that the translation units compile in parallel).
#include <cuda_runtime.h>

#include "stage_box.cuh"

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

// mixed form on axis-aligned box elements; pipe: stage the next group's data with cp.async
template <int EPB, bool PIPE>
static cudaError_t box_go(const StageParams &P, int grid, cudaStream_t st) {
    if constexpr (stage_box_smem_bytes<3, EPB, PIPE>() <= 48 * 1024) {
        if (P.visc_kv) k_stage_box<3, EPB, PIPE, true><<<grid, EPB * ipow4(3), 0, st>>>(P);
        else k_stage_box<3, EPB, PIPE, false><<<grid, EPB * ipow4(3), 0, st>>>(P);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidConfiguration;
    }
}

cudaError_t stage_launch_box_3d(const StageParams &P, int epb, bool pipe, int grid, cudaStream_t st) {
    if (epb == 1) return pipe ? box_go<1, true>(P, grid, st) : box_go<1, false>(P, grid, st);
    if (epb == 2) return pipe ? box_go<2, true>(P, grid, st) : box_go<2, false>(P, grid, st);
    if (epb == 4) return pipe ? box_go<4, true>(P, grid, st) : box_go<4, false>(P, grid, st);
    return cudaErrorInvalidValue;
}

// Per-node work table of the 3D box kernels, built on the host from the
// same function the kernels were written against; bytes written to out (if
// non-null), returns the table size.
size_t box_node_table_3d(const float *Df, void *out) {
    constexpr int NP = ipow4(3);
    if (out) {
        NodeTable<3> *T = reinterpret_cast<NodeTable<3> *>(out);
        for (int q = 0; q < NP; ++q) build_node_table<3>(T[q], q, Df);
    }
    return sizeof(NodeTable<3>) * NP;
}
}  // namespace perrk
