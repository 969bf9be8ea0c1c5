// Adaptive mesh refinement on quadtree meshes of 2D boxes: the refinement
// indicator and the solution transfer to a new mesh (the paper's adaptive
// runs refine where the shock-capturing indicator of Hennemann et al. (2021)
// on the density is large, Sec. 3.2.2, and re-derive the partitions from the
// new element sizes, Sec. 2.2).  Both kernels work in float64 (the mixed
// form's state is read as its float pair hi + lo).
//
// Indicator of an element (N = 3): the density in the orthonormal Legendre
// basis, m = (Vinv (x) Vinv) rho; the energies E_N, E_{N-1}, E_{N-2} of the
// modes up to degree N, N-1, N-2 in each direction;
//   e = max((E_N - E_{N-1}) / E_N, (E_{N-1} - E_{N-2}) / E_{N-1}),
//   alpha = 1 / (1 + exp(-(s / T)(e - T))), T = 0.5 10^(-1.8 (N+1)^(1/4)),
//   s = log((1 - 1e-4) / 1e-4).
// Transfer, per new element, from a map row (kind, a0, a1, a2, a3):
//   0: the old element a0 unchanged;
//   1: child a1 = a + 2 b of old element a0, u = (P_b (x) P_a) u_old
//      (the parent polynomial at the child's nodes);
//   2: parent of the old children a0..a3 (child order a + 2 b), the L2
//      projection u = 1/4 sum (R_b (x) R_a) u_child.
// P_m, R_m are the half-interval interpolation and projection operators of
// the mortars, so refinement is exact for the parent polynomial and
// coarsening keeps every integral sum omega J u.
#include <cuda_runtime.h>

#include <cmath>

#include "perrk_internal.h"

namespace perrk {

namespace {

__device__ __forceinline__ double state_at(const double *U, const float *Uf, const float *Ul, size_t i) {
    return U ? U[i] : (double)Uf[i] + (double)Ul[i];
}

__global__ void k_amr_indicator(const double *U, const float *Uf, const float *Ul, int NE, AmrIndicatorConsts K,
                                double *alpha) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NE) return;
    double r[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) r[q] = state_at(U, Uf, Ul, (size_t)e * 16 + q);   // variable 0: density
    // t[j][a] = sum_i Vinv[a][i] r[j][i]; m[b][a] = sum_j Vinv[b][j] t[j][a]
    double t[4][4], m2[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            double v = 0.0;
#pragma unroll
            for (int i = 0; i < 4; ++i) v = fma(K.Vinv[a * 4 + i], r[j * 4 + i], v);
            t[j][a] = v;
        }
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            double v = 0.0;
#pragma unroll
            for (int j = 0; j < 4; ++j) v = fma(K.Vinv[b * 4 + j], t[j][a], v);
            m2[b][a] = v * v;
        }
    double EN = 0.0, E1 = 0.0, E2 = 0.0;
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            EN += m2[b][a];
            if (a < 3 && b < 3) E1 += m2[b][a];
            if (a < 2 && b < 2) E2 += m2[b][a];
        }
    const double en = fmax((EN - E1) / EN, (E1 - E2) / E1);
    alpha[e] = 1.0 / (1.0 + exp(-(K.s / K.T) * (en - K.T)));
}

__global__ void k_amr_transfer(const double *U, const float *Uf, const float *Ul, int NEs, const int32_t *map, int NEd,
                               int V, AmrOps O, double *Ud) {
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= NEd * 16) return;
    const int e = gi >> 4, q = gi & 15, jq = q >> 2, iq = q & 3;
    const int kind = map[5 * e], a0 = map[5 * e + 1];
    const size_t ns = (size_t)NEs * 16, nd = (size_t)NEd * 16;
    for (int v = 0; v < V; ++v) {
        double val;
        if (kind == 0) {
            val = state_at(U, Uf, Ul, v * ns + (size_t)a0 * 16 + q);
        } else if (kind == 1) {
            const int child = map[5 * e + 2], a = child & 1, b = child >> 1;
            val = 0.0;
            for (int l = 0; l < 4; ++l) {
                double row = 0.0;
                for (int k = 0; k < 4; ++k)
                    row = fma(O.P[(a * 4 + iq) * 4 + k], state_at(U, Uf, Ul, v * ns + (size_t)a0 * 16 + l * 4 + k), row);
                val = fma(O.P[(b * 4 + jq) * 4 + l], row, val);
            }
        } else {
            val = 0.0;
            for (int c = 0; c < 4; ++c) {
                const int ec = map[5 * e + 1 + c], a = c & 1, b = c >> 1;
                double sc = 0.0;
                for (int l = 0; l < 4; ++l) {
                    double row = 0.0;
                    for (int k = 0; k < 4; ++k)
                        row = fma(O.R[(a * 4 + iq) * 4 + k], state_at(U, Uf, Ul, v * ns + (size_t)ec * 16 + l * 4 + k), row);
                    sc = fma(O.R[(b * 4 + jq) * 4 + l], row, sc);
                }
                val = fma(0.25, sc, val);
            }
        }
        Ud[v * nd + (size_t)e * 16 + q] = val;
    }
}

// the relaxation history carries over to the new mesh: time, the last
// gamma and Delta H / A values (Newton warm start, learned-guess features)
// and the step count
__global__ void k_amr_history(const InstScalars *src, InstScalars *dst) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    dst->t = src->t;
    for (int k = 0; k < 3; ++k) {
        dst->hist_gamma[k] = src->hist_gamma[k];
        dst->hist_dh[k] = src->hist_dh[k];
    }
    dst->nsteps_done = src->nsteps_done;
}

}  // namespace

// Orthonormal Legendre Vandermonde matrix V_ik = sqrt((2k+1)/2) P_k(x_i) on
// the LGL nodes, inverted (extended precision), and the indicator constants.
void amr_indicator_consts(const std::vector<double> &x, AmrIndicatorConsts &K) {
    long double V[4][8];
    for (int i = 0; i < 4; ++i) {
        const long double xi = (long double)x[i];
        long double p0 = 1.0L, p1 = xi;
        long double P[4] = {p0, p1, 0, 0};
        for (int k = 1; k < 3; ++k) {
            const long double p2 = ((2 * k + 1) * xi * p1 - k * p0) / (k + 1);
            P[k + 1] = p2;
            p0 = p1;
            p1 = p2;
        }
        for (int k = 0; k < 4; ++k) V[i][k] = sqrtl((2.0L * k + 1.0L) / 2.0L) * P[k];
        for (int k = 0; k < 4; ++k) V[i][4 + k] = i == k ? 1.0L : 0.0L;
    }
    for (int c = 0; c < 4; ++c) {   // Gauss-Jordan with partial pivoting
        int piv = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabsl(V[r][c]) > fabsl(V[piv][c])) piv = r;
        for (int j = 0; j < 8; ++j) {
            const long double tmp = V[c][j];
            V[c][j] = V[piv][j];
            V[piv][j] = tmp;
        }
        const long double d = V[c][c];
        for (int j = 0; j < 8; ++j) V[c][j] /= d;
        for (int r = 0; r < 4; ++r)
            if (r != c) {
                const long double f = V[r][c];
                for (int j = 0; j < 8; ++j) V[r][j] -= f * V[c][j];
            }
    }
    for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 4; ++i) K.Vinv[a * 4 + i] = (double)V[a][4 + i];
    K.T = 0.5 * pow(10.0, -1.8 * pow(4.0, 0.25));
    K.s = log((1.0 - 1e-4) / 1e-4);
}

perrk_status launch_amr_indicator(const Ctx &c, const AmrIndicatorConsts &K, double *alpha, void *stream) {
    const int nb = (c.n_elem + 127) / 128;
    k_amr_indicator<<<nb, 128, 0, (cudaStream_t)stream>>>(c.Uf ? nullptr : c.U, c.Uf, c.Ul, c.n_elem, K, alpha);
    return cuda_check((int)cudaGetLastError(), "amr indicator launch");
}

perrk_status launch_amr_transfer(const Ctx &src, Ctx &dst, const int32_t *map_dev, const AmrOps &O, void *stream) {
    const int n = dst.n_elem * 16;
    k_amr_transfer<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(src.Uf ? nullptr : src.U, src.Uf, src.Ul,
                                                                       src.n_elem, map_dev, dst.n_elem, dst.V, O, dst.U);
    return cuda_check((int)cudaGetLastError(), "amr transfer launch");
}

perrk_status launch_amr_history(const Ctx &src, Ctx &dst, void *stream) {
    k_amr_history<<<1, 32, 0, (cudaStream_t)stream>>>(src.g_scal, dst.g_scal);
    return cuda_check((int)cudaGetLastError(), "amr history launch");
}

}  // namespace perrk
