// 2:1 non-conforming interfaces by L2 projection mortars (Kopriva 1996), the
// interface treatment of the paper's adaptive meshes (Sec. 4.2 notes that it
// is not entropy-conservative), for 2D meshes of axis-aligned boxes.
//
// A coarse face s in [-1, 1] is split at s = 0 into mortar 0 (lower half) and
// mortar 1 (upper half), each the face of one fine element.  At every stage,
// for each mortar that touches an active element:
//   1. the stage rows U_{n,i} of the coarse face nodes and of each fine face
//      node (an inactive element's row is its cheap update, as for
//      conforming neighbours);
//   2. the coarse face state at mortar m's nodes, u_m = P_m u_coarse, with
//      P_m[j][i] = l_i((x_j -+ 1) / 2);
//   3. the numerical flux g_m = f*(U_plus, U_minus; nu_m) at mortar m's
//      nodes, the '+' side first and nu_m the fine face's scaled normal;
//   4. the coarse face's flux G = R_0 g_0 + R_1 g_1 with R_m = M^-1 P_m^T M
//      (M the exact mass matrix of the face basis; the factor 1/2 of the
//      half-length cancels the halved normal).
// The fluxes are written as traces (kernel precision, [slot][NFP][V], slot
// 3 m + 0 coarse, 1 lower, 2 upper), which the stage kernel takes for those
// faces in place of a conforming flux; the lift is then the usual one.
#include <cuda_runtime.h>

#include "stage.cuh"

namespace perrk {

namespace {
constexpr int kMortarsPerBlock = 16;   // 8 threads per mortar (2 halves x 4 nodes)
}

template <typename Real>
__global__ void __launch_bounds__(8 * kMortarsPerBlock) k_mortar(const StageParams P) {
    constexpr int V = 4, NP = 16, NFP = 4;
    __shared__ Real sC[kMortarsPerBlock][NFP][V];      // coarse face states
    __shared__ Real sG[kMortarsPerBlock][2][NFP][V];   // mortar fluxes
    const int lm = threadIdx.x >> 3, m = (threadIdx.x >> 2) & 1, j = threadIdx.x & 3;
    const int mi = blockIdx.x * kMortarsPerBlock + lm;
    const bool live = mi < P.n_mortar;
    const int4 row = reinterpret_cast<const int4 *>(P.mortars)[live ? mi : P.n_mortar - 1];   // (ec, fc, elo, ehi)
    const int ec = row.x, fc = row.y, ef = m ? row.w : row.z;
    const int k = fc >> 1;
    const bool cplus = (fc & 1) != 0;
    const size_t NPtot = P.NE * NP;
    Real gm1, inv_gm1, gam;
    if constexpr (sizeof(Real) == 8) {
        gm1 = P.gamma_gas - 1.0;
        inv_gm1 = 1.0 / (P.gamma_gas - 1.0);
        gam = P.gamma_gas;
    } else {
        gm1 = P.gm1_f;
        inv_gm1 = P.inv_gm1_f;
        gam = P.gam_f;
    }
    const Real *Pm = sizeof(Real) == 8 ? (const Real *)P.mortar_P : (const Real *)P.mortar_Pf;
    const Real *Rm = sizeof(Real) == 8 ? (const Real *)P.mortar_R : (const Real *)P.mortar_Rf;
    uint32_t bad = 0;
    double t0[V], t1[V], t2[V];
    if (m == 0) {
        Real uc[V];
        stage_state<V, Real>(P, NPtot, (size_t)ec * NP + face_node_dev<2>(fc, j), P.gp[ec], uc, t0, t1, t2);
#pragma unroll
        for (int v = 0; v < V; ++v) sC[lm][j][v] = uc[v];
    }
    Real uf[V];
    stage_state<V, Real>(P, NPtot, (size_t)ef * NP + face_node_dev<2>(fc ^ 1, j), P.gp[ef], uf, t0, t1, t2);
    __syncthreads();
    Real um[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
        Real a = 0;
#pragma unroll
        for (int i = 0; i < NFP; ++i) a = dfma(Pm[(m * NFP + j) * NFP + i], sC[lm][i][v], a);
        um[v] = a;
    }
    const Real nf = Geo<Real>::elem(P, (size_t)ef, k);   // the fine face's scaled normal (+ direction)
    Real nv[2];
    nv[0] = k == 0 ? nf : Real(0);
    nv[1] = k == 1 ? nf : Real(0);
    const Real *uL = cplus ? um : uf;
    const Real *uR = cplus ? uf : um;
    const Prim<Real, 2> pL = make_prim<Real, 2>(uL, gm1, bad);
    const Prim<Real, 2> pR = make_prim<Real, 2>(uR, gm1, bad);
    Real fs[V];
    ranocha<Real, 2, -1>(pL, pR, nv, inv_gm1, fs);
    if (P.es) {
        const Real lam = max_speed_nn<Real, 2>(pL, pR, nv, fabs(nf), gam);
#pragma unroll
        for (int v = 0; v < V; ++v) fs[v] -= Real(0.5) * lam * (uR[v] - uL[v]);
    }
    Real *tr = static_cast<Real *>(P.mtrace);
    if (live) {
#pragma unroll
        for (int v = 0; v < V; ++v) tr[((size_t)(3 * mi + 1 + m) * NFP + j) * V + v] = fs[v];
    }
#pragma unroll
    for (int v = 0; v < V; ++v) sG[lm][m][j][v] = fs[v];
    __syncthreads();
    if (m == 0 && live) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            Real G = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int i = 0; i < NFP; ++i) G = dfma(Rm[(h * NFP + j) * NFP + i], sG[lm][h][i][v], G);
            tr[((size_t)(3 * mi) * NFP + j) * V + v] = G;
        }
    }
    if (bad) atomicOr(P.flags, bad);
}

cudaError_t mortar_launch(const StageParams &P, bool mixed, cudaStream_t st) {
    if (P.n_mortar <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((P.n_mortar + kMortarsPerBlock - 1) / kMortarsPerBlock);
    if (mixed) k_mortar<float><<<blocks, 8 * kMortarsPerBlock, 0, st>>>(P);
    else k_mortar<double><<<blocks, 8 * kMortarsPerBlock, 0, st>>>(P);
    return cudaGetLastError();
}

}  // namespace perrk
