// Internal types of libperrk shared by the host setup and the CUDA translation units.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/perrk.h"

namespace perrk {

constexpr int kMaxDim = 3;
constexpr int kNodes1D = 4;                 // N + 1 with N = 3
constexpr int kMaxR = 64;                   // partitions per instance
constexpr int kMlpHidden = 64;
constexpr int kMlpFeatures = 6;

#ifdef __CUDACC__
#define PERRK_HD __host__ __device__
#else
#define PERRK_HD
#endif

PERRK_HD inline constexpr int ipow4(int d) { return d == 0 ? 1 : 4 * ipow4(d - 1); }

// Per (stage, global partition) coefficients of the low-storage stage row,
// already multiplied by the instance's dt: U_{n,i} = U_n + a1 K_1 + asub K_{i-1}.
struct StageCoef {
    double a1;
    double asub;
    double b;        // b_i of the instance (the direction d += b K_i)
    double first_b;  // 1.0 at the instance's first stage with b != 0
    // fused direction (all b_i != 0 at the first, penultimate and last stage):
    // at the last stage d = b_1 K_1 + b_m K_{S-1} + b_S K_S in one write
    double b1, bm;   // b of the first and of the penultimate stage (bm = 0 if S = 2)
    double d_final;  // 1.0 at the last stage when the direction is fused
};

// FP32 twin for the mixed form; b_i as a float pair (b_hi + b_lo) for the
// double-float direction d += b_i K_i.
struct alignas(16) StageCoefF {
    float a1;
    float asub;
    float b_hi;
    float b_lo;
    int32_t has_b;    // b_i != 0
    int32_t first_b;  // first stage of the instance with b_i != 0
    int32_t d_final;  // last stage of a fused direction (see StageCoef)
    int32_t pad0;
    float b1_hi, b1_lo, bm_hi, bm_lo;   // b_1 and b_m as float pairs
};
static_assert(sizeof(StageCoefF) == 48, "StageCoefF is read as float4 + int4 + float4");

// Per-instance relaxation scalars, resident in device memory.
struct InstScalars {
    double dt;
    double t;
    double H_n;        // H(U_n)
    double A_n;        // sum omega J |s(U_n)| (tolerance scale)
    double H0;         // H(U_0)
    double dH;         // Delta H of the current step
    double gamma;      // current Newton iterate / accepted gamma
    double gamma_eval; // gamma of the last full-state pass
    double R_last;     // H(U_n + gamma_eval dt d)
    double G_last;     // <w(U_n + gamma_eval dt d), dt d>
    double A_last;     // sum omega J |s| at gamma_eval
    double gamma_guess;
    double hist_gamma[3];  // gamma_{n-1}, gamma_{n-2}, gamma_{n-3}
    double hist_dh[3];     // (Delta H / A)_{n}, _{n-1}, _{n-2} after the step
    double H_next;
    double feat[6];        // learned-guess features of the current step
    double br_lo, br_hi;   // bisection bracket
    double r_lo, r_hi;     // residuals at the bracket ends (r_hi unset until the second pass)
    double g_prev, r_prev; // secant: previous iterate and residual
    int32_t iters;
    int32_t done;
    int32_t converged;
    int32_t need_H;
    uint32_t flags;
    int32_t nsteps_done;
};

struct HostMesh {
    int dim = 0, n_elem = 0;
    std::vector<double> coords;      // [n_elem][NP][dim]
    std::vector<int32_t> faces;      // [n_faces][4]
    std::vector<int32_t> part;       // local partition id
};

struct Instance {
    int elem0 = 0, n_elem = 0;       // element range in the concatenated numbering
    int gp0 = 0, R = 0;              // global partition ids gp0 .. gp0+R-1
    int S = 0, p = 0;
    std::vector<int> E;
    std::vector<double> c, b, a1, asub;  // local tableau, a1/asub [R][S]
    double dt = 0.0;
    int chunk0 = 0, n_chunks = 0;    // relaxation work chunks
};

struct Ctx {
    // shape
    int dim = 0, NP = 0, V = 0, n_elem = 0, n_inst = 0, S = 0, p = 0, n_gp = 0;
    int equation = 0, surface = 0;
    double gamma_gas = 1.4;
    bool viscous = false;                     // Navier-Stokes-Fourier viscous terms (BR1)
    double mu = 0.0, prandtl = 0.75;
    bool curved = false;
    perrk_options opt{};
    std::vector<Instance> inst;
    std::vector<int32_t> gp_of_elem;          // [n_elem]
    std::vector<int32_t> E_of_gp;             // [n_gp]
    std::vector<int32_t> elist;               // elements sorted by E descending
    std::vector<int32_t> n_active;            // [S] active prefix length per stage
    std::vector<int32_t> ring, ring_off;      // viscous: per stage the inactive face neighbours of the active
                                              // prefix (their gradients enter the active viscous fluxes)
    std::vector<int32_t> any_b;               // [S] 1 if some instance has b_i != 0
    std::vector<int32_t> d_read;              // [S] 1 if some instance adds to an existing d at this stage
    bool d_fused = false;                     // every instance: b_i != 0 only at its first, penultimate, last stage
    std::vector<int32_t> chunk_inst, chunk_e0, chunk_e1;
    int chunk_elems = 0;
    // host geometry (double)
    std::vector<double> lgl_w;                // [4]
    std::vector<double> lgl_D;                // [4][4]
    std::vector<double> geo_node;             // curved: [6][n_elem][NP] = Ja11 Ja12 Ja21 Ja22 invJ wJ
    std::vector<double> geo_elem;             // box: [n_elem][8] = Ja_kk (dim) , invJ, J
    std::vector<double> fnorm;                // curved: [n_elem][4][4][2]; box: [n_elem][2 dim]
    std::vector<double> wJ;                   // [n_elem][NP] omega_q J_q (always)
    std::vector<int32_t> nbr;                 // [n_elem][2 dim] (a mortar face points to its own element)
    // 2:1 mortars (2D boxes): rows (coarse, face, fine lower, fine upper) in
    // global element ids, sorted by the largest E of their three elements
    // (descending) so that each stage's mortars form a prefix; the trace
    // slot of mortar m's element j (0 coarse, 1 lower, 2 upper) is 3 m + j
    int n_mortars = 0;
    std::vector<int32_t> mortars;             // [n_mortars][4]
    std::vector<int32_t> face_mortar;         // [n_elem][2 dim]: trace slot or -1
    std::vector<int32_t> mortar_active;       // [S] mortars to evaluate at each stage (prefix length)
    double mortar_P[32] = {0}, mortar_R[32] = {0};   // interpolation to / projection from the two mortars

    // device buffers
    double *U = nullptr, *K1 = nullptr, *Ka = nullptr, *Kb = nullptr, *d = nullptr;
    float *Uf = nullptr, *K1f = nullptr, *Kaf = nullptr, *Kbf = nullptr;   // mixed form
    // mixed form: the state and the direction as float pairs, U = Uf + Ul and
    // d = dh + dl (double-float, ~48 bits); U (float64) is then only the
    // staging buffer of set_state / get_state
    float *Ul = nullptr, *dh = nullptr, *dl = nullptr;
    double *e_dh = nullptr;                   // [n_elem] per-element b-weighted <w, K> sums
    float *e_dhf = nullptr;                   // mixed form: the same as float pairs [n_elem][2]
    double *g_node = nullptr, *g_elem = nullptr, *g_fnorm = nullptr, *g_wJ = nullptr;
    float *g_node_f = nullptr, *g_elem_f = nullptr, *g_fnorm_f = nullptr, *g_wJ_f = nullptr;
    float *g_wJ_lo = nullptr;                 // mixed form: omega J = g_wJ_f + g_wJ_lo
    int32_t *g_nbr = nullptr, *g_gp = nullptr, *g_elist = nullptr, *g_ring = nullptr;
    int32_t *g_mortars = nullptr, *g_face_mortar = nullptr;
    void *g_mtrace = nullptr;                 // mortar traces [3 n_mortars][NFP][V], kernel precision: the
                                              // numerical flux of each mortar element face (+ direction normal)
    void *visc_fv = nullptr;                  // viscous: node fluxes [dim][V-1][n_elem * NP] (kernel precision)
    void *visc_kv = nullptr;                  // viscous: + div f_v of the active elements [V-1][n_elem * NP]
    int32_t *g_chunk_inst = nullptr, *g_chunk_e0 = nullptr, *g_chunk_e1 = nullptr;
    int32_t *g_inst_chunk0 = nullptr, *g_inst_nchunks = nullptr;
    StageCoef *g_coef = nullptr;              // [S][n_gp]
    StageCoefF *g_coef_f = nullptr;           // [S][n_gp]
    InstScalars *g_scal = nullptr;            // [n_inst]
    double *g_partials = nullptr;             // [n_chunks][8]
    uint32_t *g_counters = nullptr;           // [n_inst]
    uint32_t *g_flags = nullptr;              // [1]
    perrk_step_info *g_records = nullptr;     // [rec_cap][n_inst]
    int rec_cap = 0;
    float *g_mlp = nullptr;                   // weights (nullptr: no MLP)
    float *g_dftab = nullptr;                 // double-float log table [129][4]
    void *g_box_tab = nullptr;                // box stage kernels: per-node work table
    float df_consts[8] = {0};                 // log 2, (unused), gamma-1, gamma (float pairs)
    int sm_count = 0;                         // SMs of the device the context was created on
    void *arena = nullptr;                    // one device allocation holding the buffers sized at create
    size_t arena_bytes = 0;
    int mlp_on = 0;

    // launch configuration (autotuned)
    int stage_epb = 0;                        // elements per CTA in the stage kernel
    int stage_persistent = 0;                 // grid = min(groups, persistent blocks)
    int relax_threads = 128;
    int stage_variant = 1;                    // mixed box: 0 generic kernel, 1 box kernel, 2 box kernel + cp.async staging,
                                              // 3 (2D) box kernel fed by a producer warp
    int ws_stall = 0;                         // test hook: the staged kernel's producer fills nothing
    bool tuned = false;

    // CUDA graph of one step
    void *graph_exec = nullptr;               // cudaGraphExec_t
    void *graph = nullptr;                    // cudaGraph_t
    bool graph_dirty = true;
};

// host setup (setup.cpp)
void lgl_tables(std::vector<double> &x, std::vector<double> &w, std::vector<double> &D);
perrk_status build_ctx(Ctx &c, int n, const perrk_mesh_desc *mesh, const perrk_scheme_desc *scheme,
                       const perrk_options *opts, std::string &err);
void stage_coefficients(const Ctx &c, std::vector<StageCoef> &coef, std::vector<StageCoefF> &coef_f);
void make_chunks(Ctx &c, int sm_count);
void df_tables(double gamma_gas, std::vector<float> &tab, std::vector<float> &consts);

// device side (kernels_*.cu)
// One stage over its active prefix (rhs_only: F on all elements of the state
// in_u / in_uf into out_k / out_kf instead of the step buffers).
perrk_status launch_stage(Ctx &c, int stage, bool rhs_only, const double *in_u, const float *in_uf, double *out_k,
                          float *out_kf, void *stream);
void mortar_operators(const std::vector<double> &x, double *P, double *R);

// AMR (kernels_amr.cu): indicator constants, transfer operators
struct AmrIndicatorConsts {
    double Vinv[16];   // Vinv[a * 4 + i]: orthonormal Legendre coefficient a from nodal value i (one direction)
    double T, s;       // threshold and sharpness of the indicator
};
struct AmrOps {
    double P[32], R[32];   // the mortars' half-interval interpolation / projection, index (m 4 + j) 4 + i
};
void amr_indicator_consts(const std::vector<double> &x, AmrIndicatorConsts &K);
perrk_status launch_amr_indicator(const Ctx &c, const AmrIndicatorConsts &K, double *alpha, void *stream);
perrk_status launch_amr_transfer(const Ctx &src, Ctx &dst, const int32_t *map_dev, const AmrOps &O, void *stream);
perrk_status launch_amr_history(const Ctx &src, Ctx &dst, void *stream);
perrk_status launch_convert(const double *src_d, float *dst_f, const float *src_f, double *dst_d, size_t n,
                            void *stream);
// float pair -> float64 (hi + lo); the split (hi = round(x), lo = round(x - hi))
// is part of launch_split_entropy_set
perrk_status launch_join(const float *hi, const float *lo, double *dst, size_t n, void *stream);
perrk_status launch_relax_init(Ctx &c, void *stream);
perrk_status launch_newton_pass(Ctx &c, void *stream);
perrk_status launch_update(Ctx &c, int rec_slot, void *stream);
perrk_status launch_entropy_set(Ctx &c, void *stream);
// mixed form: split U into the float pair and set the entropy scalars in one pass
perrk_status launch_split_entropy_set(Ctx &c, void *stream);
perrk_status launch_entropy(Ctx &c, int query, void *stream);
perrk_status launch_mlp_guess(Ctx &c, void *stream);
size_t box_node_table_2d(const float *Df, void *out);
size_t box_node_table_3d(const float *Df, void *out);
perrk_status launch_df_log(const float *tab, const float *consts, const double *x, double *y, int n, void *stream);
perrk_status mlp_train_device(const float *feats, const float *target, int n, float *weights, int epochs,
                              float lr, float *loss, float *grad_out, void *stream);

void set_error(const std::string &e);
perrk_status cuda_check(int err, const char *what);

}  // namespace perrk
