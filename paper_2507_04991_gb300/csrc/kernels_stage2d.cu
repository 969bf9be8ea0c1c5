// Instantiations of the P-ERK stage kernel for 2D meshes (split per dimension
// so that the translation units compile in parallel).
#include <cuda_runtime.h>

#include "stage_box.cuh"
#include "stage_ws.cuh"

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
        if (P.face_mortar) {
            // meshes with mortars (inviscid, no staging: the only combination
            // the context accepts with mortars)
            if constexpr (!PIPE) {
                if (!P.visc_kv) {
                    k_stage_box<2, EPB, false, false, true><<<grid, EPB * ipow4(2), 0, st>>>(P);
                    return cudaGetLastError();
                }
            }
            return cudaErrorNotSupported;
        }
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

// Staged (warp-specialised) box kernel: elements per group 8 (two consumer
// groups, four staging buffers) or 4 (four groups, eight buffers); both use
// about 85 KB of shared memory, so two CTAs fit an SM.  bulk: the own rows by
// bulk copies (TMA), else by 16-byte cp.async.
namespace {
constexpr int kWsMaxDevices = 64;
int g_ws_per_sm[kWsMaxDevices][2][2][2] = {};   // [device][epb 4 / 8][viscous][bulk]: resident CTAs per SM

template <int EPB, int NCG, int NBUF, bool VISC, bool BULK>
cudaError_t ws_prepare_one(int dev) {
    constexpr size_t smem = stage_ws_smem_bytes<EPB, NCG, NBUF>();
    auto kern = k_stage_ws<EPB, NCG, NBUF, VISC, BULK>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, ws_threads<EPB, NCG>(), smem);
    if (e != cudaSuccess) return e;
    g_ws_per_sm[dev][EPB == 8 ? 1 : 0][VISC ? 1 : 0][BULK ? 1 : 0] = per_sm;
    return cudaSuccess;
}

template <int EPB, int NCG, int NBUF>
cudaError_t ws_prepare_epb(int dev) {
    cudaError_t e;
    if ((e = ws_prepare_one<EPB, NCG, NBUF, false, false>(dev)) != cudaSuccess) return e;
    if ((e = ws_prepare_one<EPB, NCG, NBUF, false, true>(dev)) != cudaSuccess) return e;
    if ((e = ws_prepare_one<EPB, NCG, NBUF, true, false>(dev)) != cudaSuccess) return e;
    return ws_prepare_one<EPB, NCG, NBUF, true, true>(dev);
}
bool g_ws_ready[kWsMaxDevices] = {};
}  // namespace

// Opt the staged kernels in to their dynamic shared memory on the current
// device and record their occupancy (host calls that must not run inside a
// stream capture: called when a context is created).
cudaError_t stage_ws_prepare_2d() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kWsMaxDevices) return cudaErrorInvalidDevice;
    if (g_ws_ready[dev]) return cudaSuccess;
    if ((e = ws_prepare_epb<4, 4, 8>(dev)) != cudaSuccess) return e;
    if ((e = ws_prepare_epb<8, 2, 4>(dev)) != cudaSuccess) return e;
    g_ws_ready[dev] = true;
    return cudaSuccess;
}

template <int EPB, int NCG, int NBUF, bool BULK>
static cudaError_t ws_go(const StageParams &P, int grid_req, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kWsMaxDevices) return cudaErrorInvalidDevice;
    const bool visc = P.visc_kv != nullptr;
    const int per_sm = g_ws_per_sm[dev][EPB == 8 ? 1 : 0][visc ? 1 : 0][BULK ? 1 : 0];
    if (per_sm < 1) return cudaErrorInvalidConfiguration;   // not prepared on this device, or does not fit
    const int groups = (P.n_active + EPB - 1) / EPB;
    int grid = grid_req > 0 ? grid_req : per_sm * sms;
    grid = grid < groups ? grid : groups;
    constexpr size_t smem = stage_ws_smem_bytes<EPB, NCG, NBUF>();
    if (visc) k_stage_ws<EPB, NCG, NBUF, true, BULK><<<grid, ws_threads<EPB, NCG>(), smem, st>>>(P);
    else k_stage_ws<EPB, NCG, NBUF, false, BULK><<<grid, ws_threads<EPB, NCG>(), smem, st>>>(P);
    return cudaGetLastError();
}

cudaError_t stage_launch_ws_2d(const StageParams &P, int epb, bool bulk, int grid, cudaStream_t st) {
    if (epb == 8) return bulk ? ws_go<8, 2, 4, true>(P, grid, st) : ws_go<8, 2, 4, false>(P, grid, st);
    if (epb == 4) return bulk ? ws_go<4, 4, 8, true>(P, grid, st) : ws_go<4, 4, 8, false>(P, grid, st);
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
