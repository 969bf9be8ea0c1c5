// Launch of one P-ERK stage (or one plain RHS evaluation) over the active
// element prefix of the partition-major element list.
#include <cuda_runtime.h>

#include <algorithm>

#include "stage.cuh"

namespace perrk {

cudaError_t stage_launch_1d(const StageParams &, bool, bool, bool, int, int, cudaStream_t);
cudaError_t stage_launch_2d(const StageParams &, bool, bool, bool, int, int, cudaStream_t);
cudaError_t stage_launch_3d(const StageParams &, bool, bool, bool, int, int, cudaStream_t);
cudaError_t stage_launch_box_2d(const StageParams &, int, bool, int, cudaStream_t);
cudaError_t stage_launch_box_3d(const StageParams &, int, bool, int, cudaStream_t);
cudaError_t stage_launch_ws_2d(const StageParams &, int, bool, int, cudaStream_t);
cudaError_t visc_launch(const StageParams &, int, bool, bool, cudaStream_t);
cudaError_t mortar_launch(const StageParams &, bool, cudaStream_t);

int default_epb(int dim) { return dim == 1 ? 32 : (dim == 2 ? 8 : 2); }

__global__ void k_convert(const double *sd, float *df_, const float *sf, double *dd, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (sd) df_[i] = __double2float_rn(sd[i]);
    else dd[i] = (double)sf[i];
}

perrk_status launch_convert(const double *src_d, float *dst_f, const float *src_f, double *dst_d, size_t n,
                            void *stream) {
    if (n == 0) return PERRK_OK;
    k_convert<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(src_d, dst_f, src_f, dst_d, n);
    return cuda_check((int)cudaGetLastError(), "convert launch");
}

__global__ void k_join(const float *hi, const float *lo, double *dst, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dst[i] = (double)hi[i] + (double)lo[i];
}

perrk_status launch_join(const float *hi, const float *lo, double *dst, size_t n, void *stream) {
    if (n == 0) return PERRK_OK;
    k_join<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(hi, lo, dst, n);
    return cuda_check((int)cudaGetLastError(), "join launch");
}

perrk_status launch_stage(Ctx &c, int stage, bool rhs_only, const double *in_u, const float *in_uf, double *out_k,
                          float *out_kf, void *stream) {
    StageParams P{};
    const bool mixed = c.opt.precision == PERRK_MIXED;
    P.U = rhs_only ? in_u : c.U;
    P.Uf = rhs_only ? in_uf : c.Uf;
    P.K1 = c.K1;
    P.K1f = c.K1f;
    P.Kprev = (stage <= 1) ? c.K1 : (((stage - 1) % 2) ? c.Ka : c.Kb);
    P.Kprevf = (stage <= 1) ? c.K1f : (((stage - 1) % 2) ? c.Kaf : c.Kbf);
    P.Kout = rhs_only ? out_k : ((stage == 0) ? c.K1 : ((stage % 2) ? c.Ka : c.Kb));
    P.Koutf = rhs_only ? out_kf : ((stage == 0) ? c.K1f : ((stage % 2) ? c.Kaf : c.Kbf));
    if (mixed ? (!P.Uf || !P.Koutf) : (!P.U || !P.Kout)) {
        set_error("stage buffers missing for the selected precision");
        return PERRK_INVALID_ARG;
    }
    P.d = c.d;
    P.e_dh = c.e_dh;
    P.dh = c.dh;
    P.dl = c.dl;
    P.e_dhf = c.e_dhf;
    P.elist = c.g_elist;
    P.nbr = c.g_nbr;
    P.gp = c.g_gp;
    P.coef = c.g_coef + (size_t)stage * c.n_gp;
    P.coef_f = c.g_coef_f + (size_t)stage * c.n_gp;
    P.g_node = c.g_node;
    P.g_elem = c.g_elem;
    P.fnorm = c.g_fnorm;
    P.wJ = c.g_wJ;
    P.NE = (size_t)c.n_elem;
    P.n_active = rhs_only ? c.n_elem : c.n_active[stage];
    P.stage1 = (stage == 0 || rhs_only) ? 1 : 0;
    // K_S of a step's last stage enters d from registers and no later launch
    // reads it (the next step starts from K_1): not stored
    P.k_store = (rhs_only || stage != c.S - 1) ? 1 : 0;
    P.do_b = (!rhs_only && c.any_b[stage]) ? 1 : 0;
    P.d_read = (!rhs_only && c.d_read[stage]) ? 1 : 0;
    P.d_fused = c.d_fused ? 1 : 0;
    P.es = c.surface == PERRK_SURFACE_ES_RUSANOV ? 1 : 0;
    P.gamma_gas = c.gamma_gas;
    for (int i = 0; i < 16; ++i) {
        P.D[i] = c.lgl_D[i];
        P.Df[i] = (float)c.lgl_D[i];
    }
    P.w_end = c.lgl_w[0];
    P.inv_w_f = (float)(1.0 / c.lgl_w[0]);
    P.gm1_f = (float)(c.gamma_gas - 1.0);
    P.inv_gm1_f = (float)(1.0 / (c.gamma_gas - 1.0));
    P.gam_f = (float)c.gamma_gas;
    P.g_node_f = c.g_node_f;
    P.g_elem_f = c.g_elem_f;
    P.fnorm_f = c.g_fnorm_f;
    P.wJ_f = c.g_wJ_f;
    P.box_tab = c.g_box_tab;
    P.flags = c.g_flags;
    P.ws_stall = c.ws_stall;
    if (c.n_mortars > 0) {
        P.mortars = c.g_mortars;
        P.face_mortar = c.g_face_mortar;
        P.mtrace = c.g_mtrace;
        P.n_mortar = rhs_only ? c.n_mortars : c.mortar_active[stage];
        for (int i = 0; i < 32; ++i) {
            P.mortar_P[i] = c.mortar_P[i];
            P.mortar_R[i] = c.mortar_R[i];
            P.mortar_Pf[i] = (float)c.mortar_P[i];
            P.mortar_Rf[i] = (float)c.mortar_R[i];
        }
    }
    if (c.viscous) {
        P.ring = c.g_ring ? c.g_ring + (rhs_only ? 0 : c.ring_off[stage]) : nullptr;
        P.n_ring = rhs_only ? 0 : c.ring_off[stage + 1] - c.ring_off[stage];
        P.visc_fv = c.visc_fv;
        P.visc_kv = c.visc_kv;
        P.mu = c.mu;
        P.kappa = c.mu * c.gamma_gas / ((c.gamma_gas - 1.0) * c.prandtl);
        P.mu_f = (float)P.mu;
        P.kappa_f = (float)P.kappa;
        if (!P.visc_fv || !P.visc_kv || (P.n_ring > 0 && !P.ring)) {
            set_error("viscous buffers missing");
            return PERRK_INVALID_ARG;
        }
    }
    if (P.n_active <= 0) return PERRK_OK;
    if (c.curved && c.dim != 2) {
        set_error("curved geometry is only implemented in 2D");
        return PERRK_NOT_SUPPORTED;
    }
    if ((c.curved && (!c.g_node || !c.g_fnorm)) || (!c.curved && (!c.g_elem || !c.g_fnorm)) ||
        (mixed && (!c.g_wJ_f || !c.g_fnorm_f || (c.curved ? !c.g_node_f : !c.g_elem_f)))) {
        set_error("geometry tables missing for the selected geometry mode");
        return PERRK_INVALID_ARG;
    }
    const bool burgers = c.equation == PERRK_BURGERS_1D;
    // mixed form on box elements: kernel variant 0 = the generic stage kernel,
    // 1 = the float4 box kernel, 2 = the box kernel with cp.async staging,
    // 3 (2D) = the box kernel fed by a producer warp (own rows by bulk copies,
    // neighbour face nodes by cp.async, into a ring of shared-memory buffers),
    // 4 (2D) = the same with the own rows by 16-byte cp.async; their grid is
    // persistent (stage_persistent CTAs, or as many as are resident)
    const bool box = mixed && !burgers && !c.curved && c.dim >= 2 && c.stage_variant > 0;
    if (box && !c.g_box_tab) {
        set_error("box stage kernel: node table missing");
        return PERRK_INVALID_ARG;
    }
    if (c.n_mortars > 0) {
        // the stage kernels that take mortar traces: the generic kernel and the box kernel (variant 1)
        if (box && c.stage_variant >= 2) {
            set_error("mortars: stage kernel variants 2-4 do not take mortar traces (use 0 or 1)");
            return PERRK_NOT_SUPPORTED;
        }
        cudaError_t em = mortar_launch(P, mixed, (cudaStream_t)stream);
        if (em != cudaSuccess) return cuda_check((int)em, "mortar launch");
    }
    if (c.viscous) {
        // viscous fluxes over the gradient set, their divergence over the
        // active prefix; the stage kernel then adds it to K_i
        cudaError_t ev = visc_launch(P, c.dim, mixed, c.curved, (cudaStream_t)stream);
        if (ev != cudaSuccess) return cuda_check((int)ev, "viscous launch");
    }
    const int epb = c.stage_epb > 0 ? c.stage_epb : default_epb(c.dim);
    const int groups = (P.n_active + epb - 1) / epb;
    int grid = groups;
    if (c.stage_persistent > 0) grid = std::min(groups, c.stage_persistent);
    cudaError_t e;
    if (box && c.dim == 2 && c.stage_variant >= 3)
        e = stage_launch_ws_2d(P, epb, c.stage_variant == 3, c.stage_persistent, (cudaStream_t)stream);
    else if (box && c.dim == 2) e = stage_launch_box_2d(P, epb, c.stage_variant == 2, grid, (cudaStream_t)stream);
    else if (box && c.dim == 3) e = stage_launch_box_3d(P, epb, c.stage_variant == 2, grid, (cudaStream_t)stream);
    else if (c.dim == 1) e = stage_launch_1d(P, burgers, mixed, c.curved, epb, grid, (cudaStream_t)stream);
    else if (c.dim == 2) e = stage_launch_2d(P, burgers, mixed, c.curved, epb, grid, (cudaStream_t)stream);
    else e = stage_launch_3d(P, burgers, mixed, c.curved, epb, grid, (cudaStream_t)stream);
    return cuda_check((int)e, "stage launch");
}

}  // namespace perrk
