// Instantiations of the P-ERK stage kernel for 2D meshes (split per dimension
// so that the translation units compile in parallel).
#include <cuda_runtime.h>

#include "stage_box.cuh"

namespace perrk {

template <int EQ, typename Real, bool CURVED>
static cudaError_t go(const StageParams &P, int epb, int grid, cudaStream_t st) {
    if (epb == 4) {
        if constexpr (stage_smem_bytes<2, EQ, Real, CURVED, 4>() <= 48 * 1024) {
            k_stage<2, EQ, Real, CURVED, 4><<<grid, 4 * ipow4(2), 0, st>>>(P);
            return cudaGetLastError();
        }
        return cudaErrorInvalidConfiguration;
    }
    if (epb == 8) {
        if constexpr (stage_smem_bytes<2, EQ, Real, CURVED, 8>() <= 48 * 1024) {
            k_stage<2, EQ, Real, CURVED, 8><<<grid, 8 * ipow4(2), 0, st>>>(P);
            return cudaGetLastError();
        }
        return cudaErrorInvalidConfiguration;
    }
    if (epb == 16) {
        if constexpr (stage_smem_bytes<2, EQ, Real, CURVED, 16>() <= 48 * 1024) {
            k_stage<2, EQ, Real, CURVED, 16><<<grid, 16 * ipow4(2), 0, st>>>(P);
            return cudaGetLastError();
        }
        return cudaErrorInvalidConfiguration;
    }
    return cudaErrorInvalidValue;
}

cudaError_t stage_launch_2d(const StageParams &P, bool burgers, bool mixed, bool curved, int epb, int grid, cudaStream_t st) {
    (void)burgers;
    if (curved) { if (mixed) return go<EQ_EULER, float, true>(P, epb, grid, st); return go<EQ_EULER, double, true>(P, epb, grid, st); }
    if (mixed) return go<EQ_EULER, float, false>(P, epb, grid, st);
    return go<EQ_EULER, double, false>(P, epb, grid, st);
}

// mixed form on axis-aligned box elements; pipe: stage the next group's data with cp.async
template <int EPB, bool PIPE>
static cudaError_t box_go(const StageParams &P, int grid, cudaStream_t st) {
    if constexpr (stage_box_smem_bytes<2, EPB, PIPE>() <= 48 * 1024) {
        if (P.visc_kv) k_stage_box<2, EPB, PIPE, true><<<grid, EPB * ipow4(2), 0, st>>>(P);
        else k_stage_box<2, EPB, PIPE, false><<<grid, EPB * ipow4(2), 0, st>>>(P);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidConfiguration;
    }
}

cudaError_t stage_launch_box_2d(const StageParams &P, int epb, bool pipe, int grid, cudaStream_t st) {
    if (epb == 4) return pipe ? box_go<4, true>(P, grid, st) : box_go<4, false>(P, grid, st);
    if (epb == 8) return pipe ? box_go<8, true>(P, grid, st) : box_go<8, false>(P, grid, st);
    if (epb == 16) return pipe ? box_go<16, true>(P, grid, st) : box_go<16, false>(P, grid, st);
    return cudaErrorInvalidValue;
}

// Per-node work table of the 2D box kernels, built on the host from the
// same function the kernels were written against; bytes written to out (if
// non-null), returns the table size.
size_t box_node_table_2d(const float *Df, void *out) {
    constexpr int NP = ipow4(2);
    if (out) {
        NodeTable<2> *T = reinterpret_cast<NodeTable<2> *>(out);
        for (int q = 0; q < NP; ++q) build_node_table<2>(T[q], q, Df);
    }
    return sizeof(NodeTable<2>) * NP;
}
}  // namespace perrk
