// Learned Newton initial guess: a 2 x 64 tanh MLP (float32).
//   features x = (g_{n-1}-1, g_{n-2}-1, g_{n-3}-1, dH_n/A_n, (dH/A)_{n-1}, (dH/A)_{n-2})
//   x^ = (x - mean) / scale,  h1 = tanh(W1 x^ + b1),  h2 = tanh(W2 h1 + b2),
//   y = W3 . h2 + b3,  guess gamma_0 = gamma_{n-1} + out_scale * y.
// The Newton iteration that follows is unchanged, so the converged gamma does
// not depend on the guess; a non-finite or far-off prediction falls back to
// gamma_{n-1}.  Training: per-sample forward/backward (one thread per sample,
// gradients written parameter-major), a deterministic per-parameter reduction
// and an Adam step (Kingma & Ba 2015) per epoch.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "perrk_internal.h"

namespace perrk {

namespace {
constexpr int F = kMlpFeatures, H = kMlpHidden;
constexpr int oW1 = 0, ob1 = oW1 + H * F, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + H;
constexpr int oMean = ob3 + 1, oScale = oMean + F, oOut = oScale + F, NW = oOut + 1;
constexpr int NPARAM = ob3 + 1;  // trainable entries
}  // namespace

__global__ void k_mlp_guess(const float *__restrict__ W, InstScalars *scal, int n_inst) {
    __shared__ float x[F], h1[H], h2[H], red[H];
    const int inst = blockIdx.x, j = threadIdx.x;
    if (inst >= n_inst) return;
    InstScalars &S = scal[inst];
    if (j == 0) {
        for (int f = 0; f < F; ++f) x[f] = (float)((S.feat[f] - (double)W[oMean + f]) / (double)W[oScale + f]);
    }
    __syncthreads();
    float z = W[ob1 + j];
    for (int f = 0; f < F; ++f) z = fmaf(W[oW1 + j * F + f], x[f], z);
    h1[j] = tanhf(z);
    __syncthreads();
    z = W[ob2 + j];
    for (int k = 0; k < H; ++k) z = fmaf(W[oW2 + j * H + k], h1[k], z);
    h2[j] = tanhf(z);
    red[j] = W[oW3 + j] * h2[j];
    __syncthreads();
    if (j == 0) {
        float y = W[ob3];
        for (int k = 0; k < H; ++k) y += red[k];
        // trust region: the learned increment may move the guess from
        // gamma_{n-1} by at most twice the larger of the last two observed
        // step-to-step changes (a poorly trained network cannot push Newton,
        // whose residual test is loose where r(gamma) is flat, to a distant
        // gamma); no history yet: the method's own guess
        const double tau = 2.0 * fmax(fabs(S.hist_gamma[0] - S.hist_gamma[1]), fabs(S.hist_gamma[1] - S.hist_gamma[2]));
        const double raw = (double)W[oOut] * (double)y;
        // fmax / fmin drop a NaN operand, so a non-finite output is caught
        // before the clamp: the guess stays gamma_{n-1}
        const double inc = fmin(fmax(raw, -tau), tau);
        const double g0 = S.hist_gamma[0] + inc;
        if (isfinite(raw) && isfinite(g0) && fabs(g0 - 1.0) < 0.5) {
            S.gamma = g0;
            S.gamma_guess = g0;
        }
    }
}

// One thread per sample: forward, backward, gradient column written to g[p * n + i].
__global__ void k_mlp_fwd_bwd(const float *__restrict__ W, const float *__restrict__ X, const float *__restrict__ T,
                              int n, float *__restrict__ g, float *__restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[F], h1[H], h2[H], dz2[H];
    for (int f = 0; f < F; ++f) x[f] = (X[(size_t)i * F + f] - W[oMean + f]) / W[oScale + f];
    for (int j = 0; j < H; ++j) {
        float z = W[ob1 + j];
        for (int f = 0; f < F; ++f) z = fmaf(W[oW1 + j * F + f], x[f], z);
        h1[j] = tanhf(z);
    }
    float y = W[ob3];
    for (int j = 0; j < H; ++j) {
        float z = W[ob2 + j];
        for (int k = 0; k < H; ++k) z = fmaf(W[oW2 + j * H + k], h1[k], z);
        h2[j] = tanhf(z);
        y = fmaf(W[oW3 + j], h2[j], y);
    }
    const float err = y - T[i];
    loss[i] = err * err;
    const float dy = 2.0f * err / (float)n;
    const size_t N = (size_t)n;
    g[(size_t)ob3 * N + i] = dy;
    for (int j = 0; j < H; ++j) {
        g[(size_t)(oW3 + j) * N + i] = dy * h2[j];
        dz2[j] = dy * W[oW3 + j] * (1.0f - h2[j] * h2[j]);
        g[(size_t)(ob2 + j) * N + i] = dz2[j];
    }
    for (int k = 0; k < H; ++k) {
        float dh1 = 0.0f;
        for (int j = 0; j < H; ++j) {
            g[(size_t)(oW2 + j * H + k) * N + i] = dz2[j] * h1[k];
            dh1 = fmaf(W[oW2 + j * H + k], dz2[j], dh1);
        }
        const float dz1 = dh1 * (1.0f - h1[k] * h1[k]);
        g[(size_t)(ob1 + k) * N + i] = dz1;
        for (int f = 0; f < F; ++f) g[(size_t)(oW1 + k * F + f) * N + i] = dz1 * x[f];
    }
}

// One block per parameter (plus block NPARAM for the loss): fixed-order sum
// over samples, then an Adam step when lr > 0.
__global__ void k_mlp_reduce_adam(float *W, const float *__restrict__ g, const float *__restrict__ loss, int n,
                                  float *m, float *v, float *grad_out, float *loss_out, int step, float lr) {
    __shared__ float sm[256];
    const int p = blockIdx.x;
    const float *src = (p < NPARAM) ? g + (size_t)p * n : loss;
    float acc = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += src[i];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const float tot = sm[0];
    if (p == NPARAM) {
        if (loss_out) *loss_out = tot / (float)n;
        return;
    }
    if (grad_out) grad_out[p] = tot;
    if (lr > 0.0f) {
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        m[p] = b1 * m[p] + (1.0f - b1) * tot;
        v[p] = b2 * v[p] + (1.0f - b2) * tot * tot;
        const float mh = m[p] / (1.0f - powf(b1, (float)step));
        const float vh = v[p] / (1.0f - powf(b2, (float)step));
        W[p] -= lr * mh / (sqrtf(vh) + eps);
    }
}

perrk_status launch_mlp_guess(Ctx &c, void *stream) {
    k_mlp_guess<<<c.n_inst, H, 0, (cudaStream_t)stream>>>(c.g_mlp, c.g_scal, c.n_inst);
    return cuda_check((int)cudaGetLastError(), "mlp guess launch");
}

perrk_status mlp_train_device(const float *feats, const float *target, int n, float *weights, int epochs, float lr,
                              float *loss, float *grad_out, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    float *dW = nullptr, *dX = nullptr, *dT = nullptr, *dg = nullptr, *dl = nullptr, *dm = nullptr, *dv = nullptr,
          *dgo = nullptr, *dlo = nullptr;
    perrk_status s = PERRK_OK;
    auto ck = [&](cudaError_t e, const char *w) {
        if (s == PERRK_OK && e != cudaSuccess) s = cuda_check((int)e, w);
    };
    ck(cudaMalloc((void **)&dW, NW * sizeof(float)), "mlp alloc");
    ck(cudaMalloc((void **)&dX, (size_t)n * F * sizeof(float)), "mlp alloc");
    ck(cudaMalloc((void **)&dT, (size_t)n * sizeof(float)), "mlp alloc");
    ck(cudaMalloc((void **)&dg, (size_t)NPARAM * n * sizeof(float)), "mlp alloc");
    ck(cudaMalloc((void **)&dl, (size_t)n * sizeof(float)), "mlp alloc");
    ck(cudaMalloc((void **)&dm, NPARAM * sizeof(float)), "mlp alloc");
    ck(cudaMalloc((void **)&dv, NPARAM * sizeof(float)), "mlp alloc");
    ck(cudaMalloc((void **)&dgo, NW * sizeof(float)), "mlp alloc");
    ck(cudaMalloc((void **)&dlo, sizeof(float)), "mlp alloc");
    if (s == PERRK_OK) {
        ck(cudaMemcpyAsync(dW, weights, NW * sizeof(float), cudaMemcpyHostToDevice, st), "mlp copy");
        ck(cudaMemcpyAsync(dX, feats, (size_t)n * F * sizeof(float), cudaMemcpyHostToDevice, st), "mlp copy");
        ck(cudaMemcpyAsync(dT, target, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st), "mlp copy");
        ck(cudaMemsetAsync(dm, 0, NPARAM * sizeof(float), st), "mlp clear");
        ck(cudaMemsetAsync(dv, 0, NPARAM * sizeof(float), st), "mlp clear");
        ck(cudaMemsetAsync(dgo, 0, NW * sizeof(float), st), "mlp clear");
        const int tb = 128, nb = (n + tb - 1) / tb;
        const int passes = epochs > 0 ? epochs : 1;
        for (int ep = 0; ep < passes && s == PERRK_OK; ++ep) {
            k_mlp_fwd_bwd<<<nb, tb, 0, st>>>(dW, dX, dT, n, dg, dl);
            k_mlp_reduce_adam<<<NPARAM + 1, 256, 0, st>>>(dW, dg, dl, n, dm, dv, dgo, dlo, ep + 1,
                                                          epochs > 0 ? lr : 0.0f);
            ck(cudaGetLastError(), "mlp launch");
        }
        if (epochs > 0) {
            // loss of the final weights
            k_mlp_fwd_bwd<<<nb, tb, 0, st>>>(dW, dX, dT, n, dg, dl);
            k_mlp_reduce_adam<<<NPARAM + 1, 256, 0, st>>>(dW, dg, dl, n, dm, dv, nullptr, dlo, 1, 0.0f);
            ck(cudaGetLastError(), "mlp launch");
        }
        ck(cudaMemcpyAsync(weights, dW, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st), "mlp copy back");
        if (grad_out) ck(cudaMemcpyAsync(grad_out, dgo, NW * sizeof(float), cudaMemcpyDeviceToHost, st), "mlp copy back");
        float lh = 0.0f;
        ck(cudaMemcpyAsync(&lh, dlo, sizeof(float), cudaMemcpyDeviceToHost, st), "mlp copy back");
        ck(cudaStreamSynchronize(st), "mlp sync");
        if (loss) *loss = lh;
    }
    float *all[] = {dW, dX, dT, dg, dl, dm, dv, dgo, dlo};
    for (float *p : all)
        if (p) cudaFree(p);
    return s;
}

}  // namespace perrk
