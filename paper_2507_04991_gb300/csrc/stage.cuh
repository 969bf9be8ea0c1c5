// P-ERK stage kernel: for the elements active at stage i (a prefix of the
// partition-major element list) evaluate
//   U_{n,i} = U_n + a1 K_1 + asub K_{i-1}              (low-storage stage row, dt folded in)
//   J_q K_{i,q} = - sum_k sum_m 2 D_{qm} f#(U_q, U_m; avg Ja^k)     (flux differencing)
//                 - sum_{faces} (1/omega) (f*(U-, U+; nu) - f(U_q).nu)  (surface lift)
// (Sec. 2.1-2.2, eq. PartitionedRKSystem; DGSEM with EC volume flux and EC/ES
// surface flux) and, at stages with b_i != 0, the per-element entropy
// integrand b_i sum_q omega_q J_q <w(U_{n,i,q}), K_{i,q}> (eq.
// EntropyChange_EntropyVariables_ReArranged) and d += b_i K_i (Sec. 3).
//
// Layout: one thread per node, EPB elements per CTA; state SoA [V][NE][NP]
// float64.  Neighbour face traces are recomputed from the neighbour's U_n,
// K_1, K_{i-1} with the neighbour's own stage row (an inactive neighbour has
// the row (c_i dt, 0): the cheap update of eq. InternalConsistency).  An
// interface flux is always evaluated as f*(U_plus_side, U_minus_side; nu of
// the '+' side), so both elements compute bit-identical values.
#pragma once

#include "dfloat.cuh"
#include "physics.cuh"

namespace perrk {

struct StageParams {
    const double *U, *K1, *Kprev;              // float64 form
    double *Kout;
    const float *Uf, *K1f, *Kprevf;            // mixed form: FP32 copy of U_n, FP32 stage registers
    float *Koutf;
    double *d, *e_dh;
    float *dh, *dl, *e_dhf;                    // mixed form: d and the element Delta H sums as float pairs
    const int32_t *elist, *nbr, *gp;
    const StageCoef *coef;      // [n_gp] rows of this stage
    const StageCoefF *coef_f;
    const double *g_node, *g_elem, *fnorm, *wJ;
    size_t NE;
    int n_active;
    int stage1;                 // U_{n,1} = U_n: no K loads
    int do_b;                   // some element has b_i != 0 at this stage
    int d_read;                 // some element adds to an existing direction d at this stage
    int d_fused;                // d = b_1 K_1 + b_m K_{S-1} + b_S K_S written once at the last stage
    int es;                     // Rusanov dissipation on the surface flux
    const float *g_node_f, *g_elem_f, *fnorm_f, *wJ_f;   // FP32 geometry (mixed form)
    const void *box_tab;        // box kernels: per-node work table (NodeTable rows, built on the host)
    double gamma_gas;
    // viscous (Navier-Stokes-Fourier, BR1): the gradient set of a stage is
    // the active prefix plus ring[0 .. n_ring); node fluxes in visc_fv
    // [dim][V-1][NE NP], + div f_v of the active elements in visc_kv
    // [V-1][NE NP] (kernel precision), added by the stage kernel when set
    const int32_t *ring;
    int n_ring;
    void *visc_fv, *visc_kv;
    double mu, kappa;           // kappa = mu gamma / ((gamma - 1) Pr)
    float mu_f, kappa_f;
    double D[16];
    double w_end;
    float Df[16];               // FP32 copies of the tables and constants (mixed form)
    float inv_w_f, gm1_f, inv_gm1_f, gam_f;
    uint32_t *flags;
    int ws_stall;               // test hook of the staged 2D box kernel: its producer fills no buffer
    int k_store;                // store K_i (0 at a step's last stage: K_S enters d from registers and is
                                // read by no later launch)
    // 2:1 mortars: rows (coarse, face, fine lower, fine upper) of this stage's
    // n_mortar mortars, the trace slot of each element face (or -1; null
    // without mortars), the traces [slot][NFP][V] in kernel precision and the
    // operators P_m[j][i], R_m[j][i] (index (m NFP + j) NFP + i)
    const int32_t *mortars, *face_mortar;
    void *mtrace;
    int n_mortar;
    double mortar_P[32], mortar_R[32];
    float mortar_Pf[32], mortar_Rf[32];
};

// Geometry and constants in the kernel's arithmetic type, without per-use
// float64 -> float conversions in the mixed form.
template <typename Real>
struct Geo {
    __device__ static Real node(const StageParams &P, int c, size_t NPtot, size_t idx) {
        if constexpr (sizeof(Real) == 8) return __ldg(P.g_node + c * NPtot + idx);
        else return __ldg(P.g_node_f + c * NPtot + idx);
    }
    __device__ static Real elem(const StageParams &P, size_t e, int c) {
        if constexpr (sizeof(Real) == 8) return __ldg(P.g_elem + e * 8 + c);
        else return __ldg(P.g_elem_f + e * 8 + c);
    }
    __device__ static Real fn(const StageParams &P, size_t i) {
        if constexpr (sizeof(Real) == 8) return __ldg(P.fnorm + i);
        else return __ldg(P.fnorm_f + i);
    }
    __device__ static Real D(const StageParams &P, int i) {
        if constexpr (sizeof(Real) == 8) return P.D[i];
        else return P.Df[i];
    }
};

template <int DIM>
__host__ __device__ __forceinline__ int face_pos(int q, int k) {
    const int i0 = q & 3, i1 = (q >> 2) & 3, i2 = (q >> 4) & 3;
    if (DIM == 1) return 0;
    if (DIM == 2) return k == 0 ? i1 : i0;
    return k == 0 ? (i1 + 4 * i2) : (k == 1 ? (i0 + 4 * i2) : (i0 + 4 * i1));
}

template <int DIM>
__host__ __device__ __forceinline__ int face_node_dev(int f, int kk) {
    const int k = f >> 1, ed = (f & 1) ? 3 : 0;
    if (DIM == 1) return ed;
    if (DIM == 2) return k == 0 ? ed + 4 * kk : kk + 4 * ed;
    const int a = kk & 3, b = kk >> 2;
    return k == 0 ? ed + 4 * a + 16 * b : (k == 1 ? a + 4 * ed + 16 * b : a + 4 * b + 16 * ed);
}

// Stage-row combination at one node; the same instruction sequence is used
// for an element's own nodes and for its neighbours' face nodes.  The float64
// form also returns the float64 inputs (for the entropy integrand).
template <int V, typename Real>
__device__ __forceinline__ void stage_state(const StageParams &P, size_t NPtot, size_t idx, int g, Real *u, double *Ud,
                                            double *K1d, double *Kpd) {
    if constexpr (sizeof(Real) == 8) {
        if (P.stage1) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                Ud[v] = __ldg(P.U + v * NPtot + idx);
                K1d[v] = 0.0;
                Kpd[v] = 0.0;
                u[v] = (Real)Ud[v];
            }
            return;
        }
        const StageCoef c = P.coef[g];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            Ud[v] = __ldg(P.U + v * NPtot + idx);
            K1d[v] = __ldg(P.K1 + v * NPtot + idx);
            Kpd[v] = (c.asub != 0.0 || c.bm != 0.0) ? __ldg(P.Kprev + v * NPtot + idx) : 0.0;
        }
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = (Real)fma(c.asub, Kpd[v], fma(c.a1, K1d[v], Ud[v]));
    } else {
        if (P.stage1) {
#pragma unroll
            for (int v = 0; v < V; ++v) u[v] = __ldg(P.Uf + v * NPtot + idx);
            return;
        }
        const StageCoefF cf = P.coef_f[g];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float k1 = __ldg(P.K1f + v * NPtot + idx);
            const float kp = (cf.asub != 0.0f) ? __ldg(P.Kprevf + v * NPtot + idx) : 0.0f;
            u[v] = fmaf(cf.asub, kp, fmaf(cf.a1, k1, __ldg(P.Uf + v * NPtot + idx)));
        }
    }
}

// Static shared memory of k_stage (must stay within the 48 KiB static limit).
template <int DIM, int EQ, typename Real, bool CURVED, int EPB>
constexpr size_t stage_smem_bytes() {
    constexpr int NP = ipow4(DIM), NF = 2 * DIM, NFP = ipow4(DIM - 1);
    constexpr int V = EQ == EQ_BURGERS ? 1 : DIM + 2;
    constexpr int NPR = EQ == EQ_BURGERS ? 1 : DIM + 5;
    constexpr int NPAIR = DIM * ipow4(DIM - 1) * 6;
    return sizeof(Real) * (size_t)EPB * (V * NP + NPR * NP + NF * NFP * V + (CURVED ? 4 : 1) * NP + NPAIR * V) +
           sizeof(double) * (size_t)EPB * NP;
}

// Occupancy of the 2D mixed-form kernel: <= 40 registers per thread (12 CTAs
// of 128 threads per SM hide the global-load latency); other forms unbounded.
template <int DIM, typename Real, int EPB>
constexpr int stage_min_blocks() {
    return (DIM == 2 && sizeof(Real) == 4 && EPB >= 8) ? 1536 / (EPB * ipow4(DIM)) : 1;
}

template <int DIM, int EQ, typename Real, bool CURVED, int EPB>
__global__ void __launch_bounds__(EPB * ipow4(DIM), stage_min_blocks<DIM, Real, EPB>()) k_stage(const StageParams P) {
    constexpr int NP = ipow4(DIM), NF = 2 * DIM, NFP = ipow4(DIM - 1);
    constexpr int V = EQ == EQ_BURGERS ? 1 : DIM + 2;
    constexpr int NPR = EQ == EQ_BURGERS ? 1 : DIM + 5;
    __shared__ Real s_u[EPB][V][NP];
    __shared__ Real s_pr[EPB][NPR][NP];
    __shared__ Real s_sf[EPB][NF * NFP][V];
    __shared__ Real s_ja[EPB][CURVED ? 4 : 1][NP];
    __shared__ double s_red[EPB][NP];
    constexpr int NLINE = DIM * ipow4(DIM - 1);       // reference lines per element
    constexpr int NPAIR = NLINE * 6;                  // node pairs (q < m) on those lines
    __shared__ Real s_pf[EPB][NPAIR][V];              // two-point volume fluxes, one per pair


    constexpr bool MIX = sizeof(Real) == 4;           // mixed form: no float64 instruction per node
    const int el = threadIdx.x / NP, q = threadIdx.x % NP;
    const size_t NPtot = P.NE * NP;
    Real gm1, inv_gm1, gam, inv_w;
    if constexpr (sizeof(Real) == 8) {
        gm1 = P.gamma_gas - 1.0;
        inv_gm1 = 1.0 / (P.gamma_gas - 1.0);
        gam = P.gamma_gas;
        inv_w = 1.0 / P.w_end;
    } else {
        gm1 = P.gm1_f;
        inv_gm1 = P.inv_gm1_f;
        gam = P.gam_f;
        inv_w = P.inv_w_f;
    }
    uint32_t bad = 0;
    const int ngroups = (P.n_active + EPB - 1) / EPB;

    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int slot = grp * EPB + el;
        const bool valid = slot < P.n_active;
        const int e = P.elist[valid ? slot : P.n_active - 1];
        const int g = P.gp[e];
        const size_t idx = (size_t)e * NP + q;

        // ---- A: own stage state; the neighbour face states this thread needs
        // in phase B are loaded first so that their latency overlaps phase A
        constexpr int NSLOT = (NF * NFP + NP - 1) / NP;
        Real un_pre[NSLOT][V];
#pragma unroll
        for (int t = 0; t < NSLOT; ++t) {
            const int sl = q + t * NP;
            if (sl < NF * NFP) {
                const int f = sl / NFP, kk = sl % NFP;
                const int nb = P.nbr[(size_t)e * NF + f];
                const int qn = face_node_dev<DIM>(f ^ 1, kk);
                double t0[V], t1[V], t2[V];
                stage_state<V, Real>(P, NPtot, (size_t)nb * NP + qn, P.gp[nb], un_pre[t], t0, t1, t2);
            }
        }
        Real u[V];
        double Ud[V], K1d[V], Kpd[V];
        stage_state<V, Real>(P, NPtot, idx, g, u, Ud, K1d, Kpd);

#pragma unroll
        for (int v = 0; v < V; ++v) s_u[el][v][q] = u[v];
        if constexpr (EQ == EQ_EULER) {
            Prim<Real, (EQ == EQ_EULER ? DIM : 1)> pr = make_prim<Real, (EQ == EQ_EULER ? DIM : 1)>(u, gm1, bad);
            s_pr[el][0][q] = pr.rho;
#pragma unroll
            for (int a = 0; a < DIM; ++a) s_pr[el][1 + a][q] = pr.v[a];
            s_pr[el][DIM + 1][q] = pr.p;
            s_pr[el][DIM + 2][q] = pr.beta;
            s_pr[el][DIM + 3][q] = pr.lrho;
            s_pr[el][DIM + 4][q] = pr.lbeta;
        }
        Real invJ, Jak_box[DIM > 0 ? DIM : 1];
        if constexpr (CURVED) {
#pragma unroll
            for (int c = 0; c < 4; ++c) s_ja[el][c][q] = Geo<Real>::node(P, c, NPtot, idx);
            invJ = Geo<Real>::node(P, 4, NPtot, idx);
        } else {
#pragma unroll
            for (int a = 0; a < DIM; ++a) Jak_box[a] = Geo<Real>::elem(P, (size_t)e, a);
            invJ = Geo<Real>::elem(P, (size_t)e, 3);
        }
        __syncthreads();

        // ---- B: interface fluxes at this element's face nodes
#pragma unroll
        for (int t = 0; t < NSLOT; ++t) {
            const int sl = q + t * NP;
            if (sl >= NF * NFP) break;
            const int f = sl / NFP, kk = sl % NFP;
            const int qs = face_node_dev<DIM>(f, kk);
            const Real *un = un_pre[t];
            Real us[V];
#pragma unroll
            for (int v = 0; v < V; ++v) us[v] = s_u[el][v][qs];
            Real nrm[DIM];
            if constexpr (CURVED) {
                nrm[0] = Geo<Real>::fn(P, (((size_t)e * NF + f) * NFP + kk) * 2 + 0);
                nrm[1 % DIM] = Geo<Real>::fn(P, (((size_t)e * NF + f) * NFP + kk) * 2 + 1);
            } else {
                nrm[0] = Geo<Real>::fn(P, (size_t)e * NF + f);
            }
            const bool self_plus = (f & 1);
            const Real *uL = self_plus ? us : un;
            const Real *uR = self_plus ? un : us;
            Real fs[V], fp[V];
            if constexpr (EQ == EQ_BURGERS) {
                const Real a = uL[0], b = uR[0];
                fs[0] = (a * a + a * b + b * b) * Real(1.0 / 6.0) * nrm[0];
                if (P.es) {
                    Real lam = fmax(fabs(a), fabs(b)) * fabs(nrm[0]);
                    fs[0] -= Real(0.5) * lam * (b - a);
                }
                fp[0] = Real(0.5) * us[0] * us[0] * nrm[0];
            } else {
                constexpr int DD = EQ == EQ_EULER ? DIM : 1;
                Prim<Real, DD> ps, pn;
                ps.rho = s_pr[el][0][qs];
#pragma unroll
                for (int a = 0; a < DD; ++a) ps.v[a] = s_pr[el][1 + a][qs];
                ps.p = s_pr[el][DD + 1][qs];
                ps.beta = s_pr[el][DD + 2][qs];
                ps.lrho = s_pr[el][DD + 3][qs];
                ps.lbeta = s_pr[el][DD + 4][qs];
                pn = make_prim<Real, DD>(un, gm1, bad);
                const Prim<Real, DD> &PL = self_plus ? ps : pn;
                const Prim<Real, DD> &PR = self_plus ? pn : ps;
                const int k = f >> 1;
                if constexpr (MIX && !CURVED) {
                    // axis normal as a full vector (zeros off the axis): one
                    // instruction stream for every face direction
                    Real nv[DD];
#pragma unroll
                    for (int a = 0; a < DD; ++a) nv[a] = (a == k) ? nrm[0] : Real(0);
                    ranocha<Real, DD, -1>(PL, PR, nv, inv_gm1, fs);
                    if (P.es) {
                        Real lam = max_speed_nn<Real, DD>(PL, PR, nv, fabs(nrm[0]), gam);
#pragma unroll
                        for (int v = 0; v < V; ++v) fs[v] -= Real(0.5) * lam * (uR[v] - uL[v]);
                    }
                } else if constexpr (MIX) {
                    ranocha<Real, DD, -1>(PL, PR, nrm, inv_gm1, fs);
                    if (P.es) {
                        Real lam = max_speed<Real, DD, -1>(PL, PR, nrm, gam);
#pragma unroll
                        for (int v = 0; v < V; ++v) fs[v] -= Real(0.5) * lam * (uR[v] - uL[v]);
                    }
                } else if constexpr (CURVED) {
                    ranocha<Real, DD, -1>(PL, PR, nrm, inv_gm1, fs);
                    euler_flux<Real, DD, -1>(us, ps, nrm, fp);
                    if (P.es) {
                        Real lam = max_speed<Real, DD, -1>(PL, PR, nrm, gam);
#pragma unroll
                        for (int v = 0; v < V; ++v) fs[v] -= Real(0.5) * lam * (uR[v] - uL[v]);
                    }
                } else {
#define PERRK_AXIS_CASE(KK)                                                                   \
    if (k == KK) {                                                                            \
        ranocha<Real, DD, (KK < DD ? KK : 0)>(PL, PR, nrm, inv_gm1, fs);                      \
        euler_flux<Real, DD, (KK < DD ? KK : 0)>(us, ps, nrm, fp);                            \
        if (P.es) {                                                                           \
            Real lam = max_speed<Real, DD, (KK < DD ? KK : 0)>(PL, PR, nrm, gam);            \
            for (int v = 0; v < V; ++v) fs[v] -= Real(0.5) * lam * (uR[v] - uL[v]);           \
        }                                                                                     \
    }
                    PERRK_AXIS_CASE(0)
                    if (DIM > 1) PERRK_AXIS_CASE(1)
                    if (DIM > 2) PERRK_AXIS_CASE(2)
#undef PERRK_AXIS_CASE
                }
            }
            if (P.face_mortar) {
                // a 2:1 mortar face: the mortar kernel's flux for this element face
                const int ms = P.face_mortar[(size_t)e * NF + f];
                if (ms >= 0) {
#pragma unroll
                    for (int v = 0; v < V; ++v) fs[v] = static_cast<const Real *>(P.mtrace)[((size_t)ms * NFP + kk) * V + v];
                }
            }
            const Real sg = self_plus ? Real(1) : Real(-1);
            if constexpr (MIX) {
                // LGL SBP: 2 D_NN = 1/omega_N and 2 D_00 = -1/omega_0, so the
                // diagonal volume term 2 D_qq f(U_q).Ja and the -f(U_q).nu part
                // of the lift cancel at end nodes; only f* remains
#pragma unroll
                for (int v = 0; v < V; ++v) s_sf[el][sl][v] = sg * fs[v] * inv_w;
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) s_sf[el][sl][v] = sg * (fs[v] - fp[v]) * inv_w;
            }
        }

        // ---- C: volume flux differencing.  The two-point flux is symmetric,
        // so each pair (q, m) on a reference line is evaluated once (pairs
        // spread over the element's threads) and used by both nodes.
        for (int pp = q; pp < NPAIR; pp += NP) {
            const int k = pp / (NPAIR / DIM), line = (pp % (NPAIR / DIM)) / 6, lp = pp % 6;
            const int a = lp < 3 ? 0 : (lp < 5 ? 1 : 2);
            const int b = lp < 3 ? lp + 1 : (lp < 5 ? lp - 1 : 3);
            // nodes with index a / b along direction k on this line
            int qa, qb;
            if (DIM == 1) {
                qa = a;
                qb = b;
            } else if (DIM == 2) {
                qa = k == 0 ? a + 4 * line : line + 4 * a;
                qb = k == 0 ? b + 4 * line : line + 4 * b;
            } else {
                const int l0 = line & 3, l1 = line >> 2;
                qa = k == 0 ? a + 4 * l0 + 16 * l1 : (k == 1 ? l0 + 4 * a + 16 * l1 : l0 + 4 * l1 + 16 * a);
                qb = k == 0 ? b + 4 * l0 + 16 * l1 : (k == 1 ? l0 + 4 * b + 16 * l1 : l0 + 4 * l1 + 16 * b);
            }
            Real F[V];
            if constexpr (EQ == EQ_BURGERS) {
                const Real ua = s_u[el][0][qa], ub = s_u[el][0][qb];
                F[0] = (ua * ua + ua * ub + ub * ub) * Real(1.0 / 6.0) * Jak_box[0];
            } else {
                constexpr int DD = EQ == EQ_EULER ? DIM : 1;
                Prim<Real, DD> pa, pb;
                pa.rho = s_pr[el][0][qa];
                pb.rho = s_pr[el][0][qb];
#pragma unroll
                for (int c = 0; c < DD; ++c) {
                    pa.v[c] = s_pr[el][1 + c][qa];
                    pb.v[c] = s_pr[el][1 + c][qb];
                }
                pa.p = s_pr[el][DD + 1][qa];
                pb.p = s_pr[el][DD + 1][qb];
                pa.beta = s_pr[el][DD + 2][qa];
                pb.beta = s_pr[el][DD + 2][qb];
                pa.lrho = s_pr[el][DD + 3][qa];
                pb.lrho = s_pr[el][DD + 3][qb];
                pa.lbeta = s_pr[el][DD + 4][qa];
                pb.lbeta = s_pr[el][DD + 4][qb];
                Real nv[DD];
                if constexpr (CURVED) {
                    nv[0] = Real(0.5) * (s_ja[el][2 * k][qa] + s_ja[el][2 * k][qb]);
                    nv[1 % DD] = Real(0.5) * (s_ja[el][2 * k + 1][qa] + s_ja[el][2 * k + 1][qb]);
                    ranocha<Real, DD, -1>(pa, pb, nv, inv_gm1, F);
                } else if constexpr (MIX) {
                    Real jk = Jak_box[0];
#pragma unroll
                    for (int a = 1; a < DD; ++a) jk = (k == a) ? Jak_box[a] : jk;
#pragma unroll
                    for (int a = 0; a < DD; ++a) nv[a] = (a == k) ? jk : Real(0);
                    ranocha<Real, DD, -1>(pa, pb, nv, inv_gm1, F);
                } else {
                    nv[0] = Jak_box[k];
                    if (k == 0) ranocha<Real, DD, 0>(pa, pb, nv, inv_gm1, F);
                    else if (k == 1) ranocha<Real, DD, (1 < DD ? 1 : 0)>(pa, pb, nv, inv_gm1, F);
                    else ranocha<Real, DD, (2 < DD ? 2 : 0)>(pa, pb, nv, inv_gm1, F);
                }
            }
#pragma unroll
            for (int v = 0; v < V; ++v) s_pf[el][pp][v] = F[v];
        }
        __syncthreads();
        Real acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0;
        const int id[3] = {q & 3, (q >> 2) & 3, (q >> 4) & 3};
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int ik = id[k];
            const int line = DIM == 1 ? 0 : (DIM == 2 ? (k == 0 ? id[1] : id[0])
                                                      : (k == 0 ? id[1] + 4 * id[2] : (k == 1 ? id[0] + 4 * id[2] : id[0] + 4 * id[1])));
            const int base = k * (NPAIR / DIM) + line * 6;
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (m == ik) continue;
                const int lo = m < ik ? m : ik, hi = m < ik ? ik : m;
                const int lp = lo == 0 ? hi - 1 : (lo == 1 ? hi + 1 : 5);
                const Real Dv = Real(2.0) * Geo<Real>::D(P, ik * 4 + m);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = dfma(Dv, s_pf[el][base + lp][v], acc[v]);
            }
            if (!MIX && (ik == 0 || ik == 3)) {
                // diagonal term 2 D_qq f(U_q) . Ja^k_q (consistency of the two-point flux);
                // the mixed form folds it into the lift (see phase B)
                const Real Dv = Real(2.0) * Geo<Real>::D(P, ik * 4 + ik);
                Real F[V];
                if constexpr (EQ == EQ_BURGERS) {
                    F[0] = Real(0.5) * u[0] * u[0] * Jak_box[0];
                } else {
                    constexpr int DD = EQ == EQ_EULER ? DIM : 1;
                    Prim<Real, DD> pq;
                    pq.rho = s_pr[el][0][q];
#pragma unroll
                    for (int c = 0; c < DD; ++c) pq.v[c] = s_pr[el][1 + c][q];
                    pq.p = s_pr[el][DD + 1][q];
                    Real nv[DD];
                    if constexpr (CURVED) {
                        nv[0] = s_ja[el][2 * k][q];
                        nv[1 % DD] = s_ja[el][2 * k + 1][q];
                        euler_flux<Real, DD, -1>(u, pq, nv, F);
                    } else {
                        nv[0] = Jak_box[k];
                        if (k == 0) euler_flux<Real, DD, 0>(u, pq, nv, F);
                        else if (k == 1) euler_flux<Real, DD, (1 < DD ? 1 : 0)>(u, pq, nv, F);
                        else euler_flux<Real, DD, (2 < DD ? 2 : 0)>(u, pq, nv, F);
                    }
                }
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = dfma(Dv, F[v], acc[v]);
            }
        }
        __syncthreads();

        // ---- D: surface terms, then K = -acc / J
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int ik = id[k];
            if (ik == 0 || ik == 3) {
                const int f = 2 * k + (ik == 3 ? 1 : 0);
                const int sl = f * NFP + face_pos<DIM>(q, k);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] += s_sf[el][sl][v];
            }
        }
        Real Kr[V];
        const Real *kv = static_cast<const Real *>(P.visc_kv);
#pragma unroll
        for (int v = 0; v < V; ++v) {
            // with viscous terms one rounding: fma(-acc, 1/J, div f_v), as in the box kernels
            if (EQ == EQ_EULER && v > 0 && kv) Kr[v] = dfma(-acc[v], invJ, kv[(size_t)(v - 1) * NPtot + idx]);
            else Kr[v] = -acc[v] * invJ;
            if (!isfinite(Kr[v])) bad |= PERRK_FLAG_NONFINITE;
            if (valid && P.k_store) {
                if constexpr (sizeof(Real) == 8) P.Kout[v * NPtot + idx] = Kr[v];
                else P.Koutf[v * NPtot + idx] = Kr[v];
            }
        }

        // ---- E: stages with b_i != 0: entropy integrand and direction
        if constexpr (MIX) {
            if (P.do_b) {
                // Mixed form, FP32 pipe only: K_i carries FP32 rounding, so the
                // integrand <w(U_{n,i}), K_i> is evaluated from the FP32 stage
                // state and primitives (log p = log rho - log beta: no extra
                // logs) and summed over the element in FP32; the direction
                // d += b_i K_i and the element's running sum are float pairs.
                const StageCoefF cf = P.coef_f[g];
                float wdf = 0.0f;
                if (cf.has_b) {
                    if constexpr (EQ == EQ_BURGERS) {
                        wdf = u[0] * Kr[0];
                    } else {
                        constexpr int DD = EQ == EQ_EULER ? DIM : 1;
                        const Real rho = s_pr[el][0][q], p = s_pr[el][DD + 1][q];
                        const Real lr = s_pr[el][DD + 3][q], lb = s_pr[el][DD + 4][q];
                        const Real S = (Real(1) - gam) * lr - lb;        // log p - gamma log rho
                        const Real ip = rcp(p);
                        Real v2 = 0, mk = 0;
#pragma unroll
                        for (int a = 0; a < DD; ++a) {
                            const Real va = s_pr[el][1 + a][q];
                            v2 = dfma(va, va, v2);
                            mk = dfma(va, Kr[1 + a], mk);
                        }
                        const Real k0 = Kr[0], kE = Kr[DD + 1];
                        const Real w0 = gam - S - gm1 * Real(0.5) * rho * v2 * ip;
                        // w_m . K_m + w_E K_E = (gamma-1) rho / p (v . K_m - K_E)
                        wdf = dfma(w0, k0, gm1 * rho * ip * (mk - kE));
                    }
                    wdf *= __ldg(P.wJ_f + idx);
                    if (valid && (!P.d_fused || cf.d_final)) {
                        const df bb{cf.b_hi, cf.b_lo};
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            const size_t j = v * NPtot + idx;
                            df dn;
                            if (P.d_fused) {
                                // d = b_1 K_1 + b_m K_{S-1} + b_S K_S (the sums of the stage-by-stage form)
                                dn = df_mul_f(df{cf.b1_hi, cf.b1_lo}, __ldg(P.K1f + j));   // L2-resident: read by the stage row
                                dn = df_fma_f(dn, df{cf.bm_hi, cf.bm_lo}, __ldg(P.Kprevf + j));
                                dn = df_fma_f(dn, bb, Kr[v]);
                            } else {
                                dn = cf.first_b ? df_mul_f(bb, Kr[v]) : df_fma_f(df{P.dh[j], P.dl[j]}, bb, Kr[v]);
                            }
                            P.dh[j] = dn.hi;
                            P.dl[j] = dn.lo;
                        }
                    }
                }
                // element sum over its NP consecutive threads (fixed shuffle tree)
                constexpr int W = NP < 32 ? NP : 32;
#pragma unroll
                for (int off = W / 2; off > 0; off >>= 1) wdf += __shfl_xor_sync(0xffffffffu, wdf, off);
                if constexpr (NP > 32) {
                    float *sr = reinterpret_cast<float *>(&s_red[el][0]);
                    if ((q & 31) == 0) sr[q >> 5] = wdf;
                    __syncthreads();
                    if (q == 0)
                        for (int w = 1; w < NP / 32; ++w) wdf += sr[w];
                }
                if (q == 0 && valid && cf.has_b) {
                    const df bs = df_mul_f(df{cf.b_hi, cf.b_lo}, wdf);
                    const df en = cf.first_b ? bs : df_add(df{P.e_dhf[2 * e], P.e_dhf[2 * e + 1]}, bs);
                    P.e_dhf[2 * e] = en.hi;
                    P.e_dhf[2 * e + 1] = en.lo;
                }
            }
        } else if (P.do_b) {
            const StageCoef c = P.coef[g];
            double wdot = 0.0;
            if (c.b != 0.0) {
                double Ui[V];
#pragma unroll
                for (int v = 0; v < V; ++v) Ui[v] = P.stage1 ? Ud[v] : fma(c.asub, Kpd[v], fma(c.a1, K1d[v], Ud[v]));
                if constexpr (EQ == EQ_BURGERS) {
                    wdot = Ui[0] * (double)Kr[0];
                } else {
                    constexpr int DD = EQ == EQ_EULER ? DIM : 1;
                    double s, w[DD + 2];
                    euler_entropy<DD>(Ui, P.gamma_gas, s, w, bad);
#pragma unroll
                    for (int v = 0; v < V; ++v) wdot = fma(w[v], (double)Kr[v], wdot);
                }
                wdot *= __ldg(P.wJ + idx);
                if (valid && P.d_fused) {
                    // d = b_1 K_1 + b_m K_{S-1} + b_S K_S at the last stage (the
                    // stage-by-stage sums in the same order)
                    if (c.d_final != 0.0) {
#pragma unroll
                        for (int v = 0; v < V; ++v)
                            P.d[v * NPtot + idx] = fma(c.b, (double)Kr[v], fma(c.bm, Kpd[v], c.b1 * K1d[v]));
                    }
                } else if (valid) {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        double dold = (c.first_b != 0.0) ? 0.0 : P.d[v * NPtot + idx];
                        P.d[v * NPtot + idx] = fma(c.b, (double)Kr[v], dold);
                    }
                }
            }
            s_red[el][q] = wdot;
            __syncthreads();
            if (q == 0 && valid && c.b != 0.0) {
                double sacc = 0.0;
                for (int j = 0; j < NP; ++j) sacc += s_red[el][j];
                double old = (c.first_b != 0.0) ? 0.0 : P.e_dh[e];
                P.e_dh[e] = fma(c.b, sacc, old);
            }
        }
        __syncthreads();
    }
    if (__syncthreads_or(bad != 0)) {
        if (bad) atomicOr(P.flags, bad);
    }
}

}  // namespace perrk
