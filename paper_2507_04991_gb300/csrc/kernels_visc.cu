// Viscous terms of the compressible Navier-Stokes-Fourier equations (the
// paper's viscous test, Sec. 4.3.2) by BR1 (Bassi & Rebay 1997) with the
// gradients taken of the entropy variables, for one P-ERK stage:
//
//   k_visc_flux  over the stage's gradient set (active prefix + the ring of
//                inactive face neighbours): stage state, entropy variables
//                w_m = (gamma-1) beta v, w_E = -(gamma-1) beta (beta = rho / p;
//                the density component's gradient is not needed), the BR1
//                gradient
//                  J q_l = sum_k Ja^k_l D_k w + sum_faces (1/omega) (w* - w) nu_out,l
//                with the central trace w* = (w^- + w^+)/2, then the viscous
//                flux at the node (Stokes' hypothesis, Fourier heat flux,
//                kappa = mu gamma / ((gamma-1) Pr)) into visc_fv;
//   k_visc_div   over the active prefix: the divergence
//                  J div f_v = sum_k D_k (sum_l Ja^k_l f_v,l) + sum_faces (1/omega) (f_v* - f_v) . nu_out
//                with the central flux f_v* = (f_v^- + f_v^+)/2, into visc_kv,
//                which the stage kernel adds to K_i before its entropy
//                integrand and direction epilogue.
//
// An inactive element's stage state is U_n + dt c_i K_1 (its partition's
// row), so the gradient of a ring element is formed like any other; its
// neighbours' face states come from the same rows.  One thread per node,
// elements in groups of 128 / NP per CTA.
#include <cuda_runtime.h>

#include "stage.cuh"

namespace perrk {

// entropy-variable components 1..V-1 (momentum, energy) of a state
template <int DIM, typename Real>
__device__ __forceinline__ void visc_wvars(const Real *u, Real gm1, Real *w, Real &beta, Real *vel) {
    const Real rho = u[0];
    const Real ir = Real(1) / rho;
    Real v2 = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        vel[a] = u[1 + a] * ir;
        v2 += vel[a] * u[1 + a];
    }
    const Real p = gm1 * (u[DIM + 1] - Real(0.5) * v2);
    beta = rho / p;
#pragma unroll
    for (int a = 0; a < DIM; ++a) w[a] = gm1 * beta * vel[a];
    w[DIM] = -gm1 * beta;
}

template <int DIM, typename Real, bool CURVED>
__device__ __forceinline__ Real ja_comp(const StageParams &P, size_t NPtot, size_t idx, size_t e, int k, int l) {
    // Ja^k_l at a node: curved 2D node tables (Ja^1_x, Ja^1_y, Ja^2_x, Ja^2_y), boxes diagonal
    if constexpr (CURVED) return Geo<Real>::node(P, 2 * k + l, NPtot, idx);
    else return k == l ? Geo<Real>::elem(P, e, k) : Real(0);
}

template <int DIM, typename Real, bool CURVED>
__device__ __forceinline__ Real normal_comp(const StageParams &P, size_t e, int f, int kk, int l) {
    constexpr int NF = 2 * DIM, NFP = ipow4(DIM - 1);
    const int k = f >> 1;
    if constexpr (CURVED) return Geo<Real>::fn(P, (((size_t)e * NF + f) * NFP + kk) * 2 + l);
    else return l == k ? Geo<Real>::fn(P, (size_t)e * NF + f) : Real(0);
}

// Occupancy bound of the 3D mixed-form kernels (registers per thread <= 56,
// nine CTAs of 128 threads per SM): the neighbour prefetch otherwise raises
// them to 72 / 64 and costs resident warps.
template <int DIM, typename Real, int EPB>
constexpr int visc_min_blocks() {
    return (DIM == 3 && sizeof(Real) == 4 && EPB * ipow4(DIM) == 128) ? 9 : 1;
}

template <int DIM, typename Real, bool CURVED, int EPB>
__global__ void __launch_bounds__(EPB * ipow4(DIM), visc_min_blocks<DIM, Real, EPB>()) k_visc_flux(const StageParams P) {
    constexpr int NP = ipow4(DIM), NF = 2 * DIM, NFP = ipow4(DIM - 1), V = DIM + 2, VW = DIM + 1;
    __shared__ Real s_w[EPB][VW][NP];
    __shared__ Real s_jump[EPB][NF * NFP][VW];
    const int el = threadIdx.x / NP, q = threadIdx.x % NP;
    const size_t NPtot = P.NE * NP;
    Real gm1, mu, kappa, inv_w;
    if constexpr (sizeof(Real) == 8) {
        gm1 = P.gamma_gas - 1.0;
        mu = P.mu;
        kappa = P.kappa;
        inv_w = 1.0 / P.w_end;
    } else {
        gm1 = P.gm1_f;
        mu = P.mu_f;
        kappa = P.kappa_f;
        inv_w = P.inv_w_f;
    }
    Real *fv = static_cast<Real *>(P.visc_fv);
    const int n_items = P.n_active + P.n_ring;
    const int ngroups = (n_items + EPB - 1) / EPB;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int slot = grp * EPB + el;
        const bool valid = slot < n_items;
        const int item = valid ? slot : n_items - 1;
        const int e = item < P.n_active ? P.elist[item] : P.ring[item - P.n_active];
        const size_t idx = (size_t)e * NP + q;

        // the neighbour face states this thread needs are formed first, so
        // that their loads overlap the element's own
        constexpr int NSLOT = (NF * NFP + NP - 1) / NP;
        Real wpre[NSLOT][VW];
#pragma unroll
        for (int t = 0; t < NSLOT; ++t) {
            const int sl = q + t * NP;
            if (sl < NF * NFP) {
                const int f = sl / NFP, kk = sl % NFP;
                const int nb = P.nbr[(size_t)e * NF + f];
                const int qn = face_node_dev<DIM>(f ^ 1, kk);
                Real un[V], bn, vn[DIM];
                double t0[V], t1[V], t2[V];
                stage_state<V, Real>(P, NPtot, (size_t)nb * NP + qn, P.gp[nb], un, t0, t1, t2);
                visc_wvars<DIM, Real>(un, gm1, wpre[t], bn, vn);
            }
        }
        Real u[V], w[VW], beta, vel[DIM];
        {
            double t0[V], t1[V], t2[V];
            stage_state<V, Real>(P, NPtot, idx, P.gp[e], u, t0, t1, t2);
        }
        visc_wvars<DIM, Real>(u, gm1, w, beta, vel);
#pragma unroll
        for (int c = 0; c < VW; ++c) s_w[el][c][q] = w[c];
        __syncthreads();

        // face slots of this element: half jumps (w_nb - w_self) / 2
#pragma unroll
        for (int t = 0; t < NSLOT; ++t) {
            const int sl = q + t * NP;
            if (sl < NF * NFP) {
                const int f = sl / NFP, kk = sl % NFP;
                const int qs = face_node_dev<DIM>(f, kk);
#pragma unroll
                for (int c = 0; c < VW; ++c) s_jump[el][sl][c] = Real(0.5) * (wpre[t][c] - s_w[el][c][qs]);
            }
        }
        __syncthreads();

        // J q_l: volume part
        const int id[3] = {q & 3, (q >> 2) & 3, (q >> 4) & 3};
        Real jq[DIM][VW];
#pragma unroll
        for (int l = 0; l < DIM; ++l)
#pragma unroll
            for (int c = 0; c < VW; ++c) jq[l][c] = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int ik = id[k];
            const int stride = k == 0 ? 1 : (k == 1 ? 4 : 16);
            const int q0 = q - ik * stride;
            Real dw[VW];
#pragma unroll
            for (int c = 0; c < VW; ++c) dw[c] = 0;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const Real Dv = Geo<Real>::D(P, ik * 4 + m);
#pragma unroll
                for (int c = 0; c < VW; ++c) dw[c] += Dv * s_w[el][c][q0 + m * stride];
            }
#pragma unroll
            for (int l = 0; l < DIM; ++l) {
                const Real ja = ja_comp<DIM, Real, CURVED>(P, NPtot, idx, (size_t)e, k, l);
#pragma unroll
                for (int c = 0; c < VW; ++c) jq[l][c] += ja * dw[c];
            }
        }
        // surface part at face nodes: (1/omega) (w* - w) nu_out
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int ik = id[k];
            if (ik == 0 || ik == 3) {
                const int f = 2 * k + (ik == 3 ? 1 : 0);
                const int kk = face_pos<DIM>(q, k);
                const int sl = f * NFP + kk;
                const Real sg = (f & 1) ? Real(1) : Real(-1);
#pragma unroll
                for (int l = 0; l < DIM; ++l) {
                    const Real nu = sg * normal_comp<DIM, Real, CURVED>(P, (size_t)e, f, kk, l) * inv_w;
#pragma unroll
                    for (int c = 0; c < VW; ++c) jq[l][c] += nu * s_jump[el][sl][c];
                }
            }
        }
        const Real invJ = CURVED ? Geo<Real>::node(P, 4, NPtot, idx) : Geo<Real>::elem(P, (size_t)e, 3);

        // primitive gradients by the chain rule: T = 1 / beta,
        // d T = d w_E / ((gamma-1) beta^2), d v_a = (d w_a + v_a d w_E) / ((gamma-1) beta)
        const Real igb = Real(1) / (gm1 * beta);
        Real dv[DIM][DIM], dT[DIM];
#pragma unroll
        for (int l = 0; l < DIM; ++l) {
            const Real qE = jq[l][DIM] * invJ;
            dT[l] = qE * igb / beta;
#pragma unroll
            for (int a = 0; a < DIM; ++a) dv[l][a] = (jq[l][a] * invJ + vel[a] * qE) * igb;
        }
        Real div = 0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) div += dv[a][a];
        if (valid) {
#pragma unroll
            for (int l = 0; l < DIM; ++l) {
                Real fe = kappa * dT[l];
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    Real tau = mu * (dv[l][a] + dv[a][l]);
                    if (a == l) tau -= Real(2.0 / 3.0) * mu * div;
                    fv[(size_t)(l * VW + a) * NPtot + idx] = tau;
                    fe += tau * vel[a];
                }
                fv[(size_t)(l * VW + DIM) * NPtot + idx] = fe;
            }
        }
        __syncthreads();
    }
}

template <int DIM, typename Real, bool CURVED, int EPB>
__global__ void __launch_bounds__(EPB * ipow4(DIM), visc_min_blocks<DIM, Real, EPB>()) k_visc_div(const StageParams P) {
    constexpr int NP = ipow4(DIM), NF = 2 * DIM, NFP = ipow4(DIM - 1), VW = DIM + 1;
    __shared__ Real s_F[EPB][DIM][VW][NP];
    const int el = threadIdx.x / NP, q = threadIdx.x % NP;
    const size_t NPtot = P.NE * NP;
    const Real inv_w = sizeof(Real) == 8 ? Real(1.0 / P.w_end) : Real(P.inv_w_f);
    const Real *fv = static_cast<const Real *>(P.visc_fv);
    Real *kv = static_cast<Real *>(P.visc_kv);
    const int ngroups = (P.n_active + EPB - 1) / EPB;
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int slot = grp * EPB + el;
        const bool valid = slot < P.n_active;
        const int e = P.elist[valid ? slot : P.n_active - 1];
        const size_t idx = (size_t)e * NP + q;
        const int id[3] = {q & 3, (q >> 2) & 3, (q >> 4) & 3};
        // neighbours' flux traces at this node's faces, loaded first (boxes
        // need only the normal component, curved elements all of them)
        constexpr int NL = CURVED ? DIM : 1;
        Real fnb[DIM][NL][VW];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int ik = id[k];
            if (ik == 0 || ik == 3) {
                const int fc = 2 * k + (ik == 3 ? 1 : 0);
                const int nb = P.nbr[(size_t)e * NF + fc];
                const size_t in = (size_t)nb * NP + face_node_dev<DIM>(fc ^ 1, face_pos<DIM>(q, k));
#pragma unroll
                for (int li = 0; li < NL; ++li) {
                    const int l = CURVED ? li : k;
#pragma unroll
                    for (int c = 0; c < VW; ++c) fnb[k][li][c] = fv[(size_t)(l * VW + c) * NPtot + in];
                }
            }
        }
        Real f[DIM][VW];
#pragma unroll
        for (int l = 0; l < DIM; ++l)
#pragma unroll
            for (int c = 0; c < VW; ++c) f[l][c] = fv[(size_t)(l * VW + c) * NPtot + idx];
        // contravariant fluxes sum_l Ja^k_l f_l
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
#pragma unroll
            for (int c = 0; c < VW; ++c) {
                Real s = 0;
#pragma unroll
                for (int l = 0; l < DIM; ++l) s += ja_comp<DIM, Real, CURVED>(P, NPtot, idx, (size_t)e, k, l) * f[l][c];
                s_F[el][k][c][q] = s;
            }
        }
        __syncthreads();
        Real acc[VW];
#pragma unroll
        for (int c = 0; c < VW; ++c) acc[c] = 0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int ik = id[k];
            const int stride = k == 0 ? 1 : (k == 1 ? 4 : 16);
            const int q0 = q - ik * stride;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const Real Dv = Geo<Real>::D(P, ik * 4 + m);
#pragma unroll
                for (int c = 0; c < VW; ++c) acc[c] += Dv * s_F[el][k][c][q0 + m * stride];
            }
        }
        // interface terms (1/omega) (f* - f) . nu_out = (1/omega) (f_nb - f) . nu_out / 2
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int ik = id[k];
            if (ik == 0 || ik == 3) {
                const int fc = 2 * k + (ik == 3 ? 1 : 0);
                const int kk = face_pos<DIM>(q, k);
                const Real sg = (fc & 1) ? Real(0.5) : Real(-0.5);
#pragma unroll
                for (int li = 0; li < NL; ++li) {
                    const int l = CURVED ? li : k;
                    const Real nu = sg * normal_comp<DIM, Real, CURVED>(P, (size_t)e, fc, kk, l) * inv_w;
#pragma unroll
                    for (int c = 0; c < VW; ++c) acc[c] += nu * (fnb[k][li][c] - f[l][c]);
                }
            }
        }
        const Real invJ = CURVED ? Geo<Real>::node(P, 4, NPtot, idx) : Geo<Real>::elem(P, (size_t)e, 3);
        if (valid) {
#pragma unroll
            for (int c = 0; c < VW; ++c) kv[(size_t)c * NPtot + idx] = acc[c] * invJ;
        }
        __syncthreads();
    }
}

template <int DIM, typename Real, bool CURVED>
static cudaError_t visc_go(const StageParams &P, cudaStream_t st) {
    constexpr int EPB = 128 / ipow4(DIM);
    const int n_items = P.n_active + P.n_ring;
    if (n_items > 0) {
        k_visc_flux<DIM, Real, CURVED, EPB><<<(n_items + EPB - 1) / EPB, EPB * ipow4(DIM), 0, st>>>(P);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (P.n_active > 0) k_visc_div<DIM, Real, CURVED, EPB><<<(P.n_active + EPB - 1) / EPB, EPB * ipow4(DIM), 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t visc_launch(const StageParams &P, int dim, bool mixed, bool curved, cudaStream_t st) {
    if (dim == 2) {
        if (curved) return mixed ? visc_go<2, float, true>(P, st) : visc_go<2, double, true>(P, st);
        return mixed ? visc_go<2, float, false>(P, st) : visc_go<2, double, false>(P, st);
    }
    if (dim == 3 && !curved) return mixed ? visc_go<3, float, false>(P, st) : visc_go<3, double, false>(P, st);
    return cudaErrorInvalidValue;
}

}  // namespace perrk
