// Allocation-free evaluation of the entropy functional H(U) = sum omega J s(U)
// (the library's float64 entropy reduction, with its cross-block scratch in a
// file-scope device array instead of memory owned by a context).
//
// Why: some callers cannot call cudaMalloc at the point where they need the
// entropy -- e.g. code that hands all device memory to its own pool
// allocator up front, or a latency-critical loop in which an allocation (which
// may synchronise the device and can fail under memory pressure) is not
// allowed.  Such a caller passes its state, its quadrature weights and an
// output buffer; this entry point allocates nothing.
//
// The scratch array is shared by every call in the process and keeps the
// last call's contents; the ticket counter is cleared at the start of each
// call.  Calls whose work overlaps on the GPU race on the scratch.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>

#include "physics.cuh"

namespace perrk {

namespace {

constexpr int kStaticMaxChunks = 4096;             // blocks per call
constexpr int kStaticThreads = 256;
constexpr int kStaticNodesPerChunk = 16 * kStaticThreads;
constexpr long long kStaticMaxNodes = (long long)kStaticMaxChunks * kStaticNodesPerChunk;   // 16,777,216

struct StaticScratch {
    double partial[kStaticMaxChunks][4];            // per block: H sum, H compensation, A sum, A compensation
    unsigned int counter;                           // ticket of the finishing block
};

static __device__ __align__(256) StaticScratch g_static_scratch;   // ~128 KiB per device, held until exit

template <int DIM, int EQ>
__global__ void __launch_bounds__(kStaticThreads) k_entropy_static(const double *__restrict__ u,
                                                                   const double *__restrict__ wJ, long long n,
                                                                   double gam, StaticScratch *scr, double *out) {
    constexpr int V = EQ == EQ_BURGERS ? 1 : DIM + 2;
    const long long n0 = (long long)blockIdx.x * kStaticNodesPerChunk;
    const long long n1 = n0 + kStaticNodesPerChunk < n ? n0 + kStaticNodesPerChunk : n;
    double s[2] = {0.0, 0.0}, c[2] = {0.0, 0.0};
    uint32_t bad = 0;
    for (long long j = n0 + threadIdx.x; j < n1; j += blockDim.x) {
        double uv[V], sv;
#pragma unroll
        for (int v = 0; v < V; ++v) uv[v] = __ldg(u + v * n + j);
        if constexpr (EQ == EQ_BURGERS) {
            sv = 0.5 * uv[0] * uv[0];
        } else {
            uint32_t node_bad = 0;
            euler_entropy<DIM>(uv, gam, sv, nullptr, node_bad);
            // rho <= 0 or p <= 0: the entropy is undefined there (p = 0 alone
            // would give +inf); report NaN in both sums
            if (node_bad) sv = NAN;
            bad |= node_bad;
        }
        const double w = __ldg(wJ + j);
        comp_add(s[0], c[0], w * sv);
        comp_add(s[1], c[1], w * fabs(sv));
    }
    (void)bad;   // a non-physical node gives a NaN entropy, which reaches out[0] and out[1]
    __shared__ double sm[2 * 2 * 32];
    __shared__ int s_last;
    block_sum<2>(s, c, sm);
    if (threadIdx.x == 0) {
        scr->partial[blockIdx.x][0] = s[0];
        scr->partial[blockIdx.x][1] = c[0];
        scr->partial[blockIdx.x][2] = s[1];
        scr->partial[blockIdx.x][3] = c[1];
        __threadfence();
        const unsigned ticket = atomicAdd(&scr->counter, 1u);
        s_last = (ticket == gridDim.x - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double ss[2] = {0.0, 0.0}, cc[2] = {0.0, 0.0};
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
        for (int k = 0; k < 2; ++k) {
            comp_add(ss[k], cc[k], __ldcg(&scr->partial[b][2 * k]));
            cc[k] += __ldcg(&scr->partial[b][2 * k + 1]);
        }
    block_sum<2>(ss, cc, sm);
    if (threadIdx.x == 0) {
        out[0] = ss[0] + cc[0];
        out[1] = ss[1] + cc[1];
        scr->counter = 0u;
    }
}

// Device address of the scratch array, looked up once per device (with that
// device current) and cached.  The slots are atomic: two host threads making
// their first call on one device at the same time both look the address up
// (the same value) and store it, without a data race.  The cache is not
// refreshed: after cudaDeviceReset the module, and with it the array, may
// move, so a process that resets a device must not call this entry point on
// it again.
constexpr int kMaxDevices = 64;
std::atomic<StaticScratch *> g_scratch_addr[kMaxDevices] = {};

perrk_status scratch_for_current_device(StaticScratch **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_check((int)e, "entropy_static: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("entropy_static: device index beyond the supported range");
        return PERRK_NOT_SUPPORTED;
    }
    StaticScratch *addr = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!addr) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_check((int)e, "entropy_static: cudaGetSymbolAddress");
        addr = (StaticScratch *)p;
        g_scratch_addr[dev].store(addr, std::memory_order_release);
    }
    *out = addr;
    return PERRK_OK;
}

}  // namespace

}  // namespace perrk

using namespace perrk;

extern "C" perrk_status perrk_entropy_static(int equation, double gamma_gas, const double *u, const double *wJ,
                                            long long n_nodes, double *out, void *stream) {
    if (!u || !wJ || !out) {
        set_error("entropy_static: null pointer");
        return PERRK_INVALID_ARG;
    }
    if (n_nodes < 1 || n_nodes > kStaticMaxNodes) {
        char buf[160];
        snprintf(buf, sizeof buf, "entropy_static: n_nodes = %lld outside [1, %lld] (the static scratch holds %d blocks)",
                 n_nodes, kStaticMaxNodes, kStaticMaxChunks);
        set_error(buf);
        return PERRK_INVALID_ARG;
    }
    if (equation != PERRK_BURGERS_1D && !(gamma_gas > 1.0)) {
        set_error("entropy_static: gamma_gas must be > 1");
        return PERRK_INVALID_ARG;
    }
    StaticScratch *scr = nullptr;
    perrk_status st = scratch_for_current_device(&scr);
    if (st != PERRK_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_check((int)e, "entropy_static: counter clear");
    const unsigned blocks = (unsigned)((n_nodes + kStaticNodesPerChunk - 1) / kStaticNodesPerChunk);
    switch (equation) {
        case PERRK_BURGERS_1D:
            k_entropy_static<1, EQ_BURGERS><<<blocks, kStaticThreads, 0, s>>>(u, wJ, n_nodes, gamma_gas, scr, out);
            break;
        case PERRK_EULER_1D:
            k_entropy_static<1, EQ_EULER><<<blocks, kStaticThreads, 0, s>>>(u, wJ, n_nodes, gamma_gas, scr, out);
            break;
        case PERRK_EULER_2D:
            k_entropy_static<2, EQ_EULER><<<blocks, kStaticThreads, 0, s>>>(u, wJ, n_nodes, gamma_gas, scr, out);
            break;
        case PERRK_EULER_3D:
            k_entropy_static<3, EQ_EULER><<<blocks, kStaticThreads, 0, s>>>(u, wJ, n_nodes, gamma_gas, scr, out);
            break;
        default:
            set_error("entropy_static: unknown equation");
            return PERRK_INVALID_ARG;
    }
    return cuda_check((int)cudaGetLastError(), "entropy_static launch");
}
