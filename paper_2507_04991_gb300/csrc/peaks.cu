// FMA throughput of this GPU in FP32 and FP64: the denominator of the
// roofline of kernels bound by plain ALU arithmetic (the float64 form's stage
// and Newton kernels, whose per-node logarithms and divisions run on the FP64
// pipe).  The paper has no counterpart; this is a measurement helper.
//
// Every thread runs kChains independent FMA chains a <- a * b + c for `iters`
// rounds (independent chains hide the pipe latency), over a grid of
// kBlocksPerSM CTAs per SM; b and c come from kernel arguments so the compiler
// cannot fold the chains, and the chains' sum is stored so they are not
// removed.  Timed with CUDA events on the caller's stream; one FMA counts two
// flops.
#include <cuda_runtime.h>

#include "perrk_internal.h"

namespace perrk {

namespace {
constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(T b, T c, int iters, T *out) {
    T a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename T>
perrk_status run(int iters, double *tflops, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_check((int)e, "fma_peak: device query");
    const int blocks = sms * kBlocksPerSM;
    T *out = nullptr;
    e = cudaMalloc((void **)&out, (size_t)blocks * kThreads * sizeof(T));
    if (e != cudaSuccess) return cuda_check((int)e, "fma_peak: alloc");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // b slightly below 1 keeps the chains finite for any iteration count
    const T b = (T)0.999999, c = (T)1e-7;
    k_fma_chains<T><<<blocks, kThreads, 0, st>>>(b, c, iters / 10 + 1, out);   // warm-up
    cudaEventRecord(e0, st);
    k_fma_chains<T><<<blocks, kThreads, 0, st>>>(b, c, iters, out);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return cuda_check((int)e, "fma_peak: timing");
    const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return PERRK_OK;
}
}  // namespace

}  // namespace perrk

using namespace perrk;

extern "C" perrk_status perrk_fma_peak(int fp64, int iters, double *tflops, void *stream) {
    if (!tflops || iters < 1) {
        set_error("fma_peak: null output or iters < 1");
        return PERRK_INVALID_ARG;
    }
    return fp64 ? run<double>(iters, tflops, (cudaStream_t)stream) : run<float>(iters, tflops, (cudaStream_t)stream);
}
