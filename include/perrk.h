/*
 * perrk.h -- C ABI of the GB300 P-ERRK multirate stage-loop library (libperrk.so).
 *
 * The library advances a DGSEM semidiscretisation U' = F(U) (Sec. 2.1 of
 * arXiv 2507.04991, eq. SemidiscretizationODE) with a Paired Explicit
 * Relaxation Runge-Kutta (P-ERRK) method:
 *   - partitioned P-ERK stage loop, F evaluated only on the elements of the
 *     partitions active at each stage (Sec. 2.2, eq. PartitionedRKSystem and
 *     the example after eq. PERK_ButcherTableauClassic_p2_E36);
 *   - direction d = sum_i b_i K_i and entropy change
 *     Delta H = dt sum_i b_i <w(U_{n,i}), K_i>_M (Sec. 3, eq.
 *     EntropyChange_EntropyVariables_ReArranged);
 *   - Newton solve of r(gamma) = H(U_n + gamma dt d) - H_n - gamma Delta H = 0
 *     (eq. RelaxationEquation, Sec. 3.1) and the relaxed update
 *     U_{n+1} = U_n + gamma dt d, t_{n+1} = t_n + gamma dt (eq. RRKM_Update);
 *   - optionally the Navier-Stokes-Fourier viscous terms in F (BR1 on
 *     entropy-variable gradients, the paper's viscous test, Sec. 4.3.2);
 *   - bisection and secant as alternatives to Newton (Sec. 3.1), checkpoint
 *     and bit-identical resume.
 *
 * Conventions shared by all calls
 *   - polynomial degree N = 3 on Legendre-Gauss-Lobatto nodes; NP = 4^dim
 *     nodes per element, node index q = i + 4 j + 16 k (i along xi fastest);
 *   - state layout SoA [V][n_elem][NP] float64, V = 1 (Burgers) or dim + 2
 *     (Euler: rho, rho v, rho E);
 *   - faces of an element: 0 = -xi, 1 = +xi, 2 = -eta, 3 = +eta, 4 = -zeta,
 *     5 = +zeta; a face row (eL, fL, eR, fR) pairs the '+' face fL of eL with
 *     the '-' face fR = fL - 1 of eR, face nodes in the same order on both
 *     sides (logically structured, possibly periodic, conforming meshes);
 *   - every device call is enqueued on the caller's CUDA stream (a
 *     cudaStream_t passed as void*, NULL = legacy default stream);
 *   - all entry points return perrk_status; nothing is thrown across the ABI.
 *
 * Ownership: the library allocates and frees its own device buffers
 * (perrk_create*, perrk_destroy).  Caller pointers are only read or written
 * during the call (or the work it enqueues) and are never retained.
 */
#ifndef PERRK_H
#define PERRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PERRK_OK = 0,
    PERRK_INVALID_ARG = 1,       /* malformed mesh / tableau / options; nothing allocated */
    PERRK_CUDA_ERROR = 2,        /* a CUDA runtime call failed; see perrk_last_error() */
    PERRK_NONPHYSICAL_STATE = 3, /* rho <= 0, p <= 0 or non-finite values were met */
    PERRK_TIMEOUT = 4,           /* a bounded device wait expired */
    PERRK_OUT_OF_MEMORY = 5,
    PERRK_NOT_SUPPORTED = 6
} perrk_status;

typedef enum { PERRK_BURGERS_1D = 0, PERRK_EULER_1D = 1, PERRK_EULER_2D = 2, PERRK_EULER_3D = 3 } perrk_equation;
typedef enum { PERRK_VOLUME_EC = 0 } perrk_volume_flux;          /* Burgers (a^2+ab+b^2)/6 or Ranocha's EC/KEP flux */
typedef enum { PERRK_SURFACE_EC = 0, PERRK_SURFACE_ES_RUSANOV = 1 } perrk_surface_flux;
typedef enum { PERRK_FP64 = 0, PERRK_MIXED = 1 } perrk_precision;
typedef enum { PERRK_GUESS_ONE = 0, PERRK_GUESS_PREV = 1, PERRK_GUESS_MLP = 2 } perrk_guess;
typedef enum { PERRK_TARGET_DELTA_H = 0, PERRK_TARGET_PREV = 1, PERRK_TARGET_INITIAL = 2 } perrk_target;
/* Root finder for the relaxation equation (Sec. 3.1): Newton-Raphson with
 * unit step from the guess; bisection on [bracket_lo, bracket_hi] (r at both
 * ends, which must differ in sign, then midpoints; stop on |r| <= tol_r A_n,
 * a bracket of length <= tol_g, or max_it passes); secant from the two
 * guesses bracket_lo, bracket_hi (stop on |r| <= tol_r A_n or a step
 * <= tol_g).  One full-state pass per evaluation of r. */
typedef enum { PERRK_SOLVER_NEWTON = 0, PERRK_SOLVER_BISECTION = 1, PERRK_SOLVER_SECANT = 2 } perrk_solver;

/* Step-status flags (perrk_step_info.flags), OR-ed over the steps of a call. */
#define PERRK_FLAG_NEWTON_FALLBACK 0x1u   /* Newton did not converge: gamma = 1 taken (Sec. 3.2.1) */
#define PERRK_FLAG_NONPHYSICAL     0x2u   /* rho <= 0 or p <= 0 met at some node */
#define PERRK_FLAG_NONFINITE       0x4u   /* NaN / Inf met */
#define PERRK_FLAG_TIMEOUT         0x8u   /* a bounded device wait gave up (the step's results are not valid) */

/* Mesh (Sec. 2.2: elements carry a partition id r in 0..R-1). */
typedef struct {
    int dim;                      /* 1, 2 or 3 */
    int N;                        /* polynomial degree; must be 3 */
    int n_elem;
    const double *node_coords;    /* host, [n_elem][NP][dim]: physical LGL node positions */
    int n_faces;                  /* conforming interfaces; n_elem * dim when n_mortars = 0 */
    const int32_t *faces;         /* host, [n_faces][4] = (eL, fL, eR, fR) as above */
    const int32_t *partition_id;  /* host, [n_elem], values in 0..R-1 */
    /* 2:1 non-conforming interfaces (2D meshes of axis-aligned boxes, inviscid):
     * L2 projection mortars, the treatment of the paper's adaptive runs (Sec.
     * 4.2 notes that they are not entropy-conservative).  Row (ec, fc, elo,
     * ehi): face fc of the coarse element ec is split at its midpoint into
     * two halves matched by face fc ^ 1 of the fine elements elo (the half at
     * the face's lower tangential coordinate) and ehi; face nodes in the same
     * tangential order on all three.  Every element face is then covered
     * exactly once, by a conforming row or by a mortar row.  NULL / 0: none. */
    int n_mortars;
    const int32_t *mortars;       /* host, [n_mortars][4] */
} perrk_mesh_desc;

/* P-ERK family in low-storage form (Sec. 2.2, appendix A archetypes): the
 * stage-i row of partition r is U_{n,i} = U_n + dt (a1[r][i] K_1 + asub[r][i] K_{i-1}).
 * Member r evaluates F at stage 1 and at stages S - E[r] + 2 .. S; at every other
 * stage its row must be (c_i, 0), and at its first active stage after stage 1
 * asub must be 0.  c and b are shared by all members (eq. InternalConsistency:
 * a1 + asub = c_i; eq. Conservation: one b).  b_i != 0 only at stages where all
 * members are active. */
typedef struct {
    int order;                    /* p: 2, 3 or 4 (minimum E: 2, 3, 5) */
    int S;                        /* stages, = max E */
    int R;                        /* partitions */
    const int32_t *E;             /* host, [R] stage evaluations per member */
    const double *c;              /* host, [S] */
    const double *b;              /* host, [S] */
    const double *a1;             /* host, [R][S] coefficient of K_1 (row i = index i, 0-based) */
    const double *asub;           /* host, [R][S] coefficient of K_{i-1} */
    int equation;                 /* perrk_equation */
    double gamma_gas;             /* ratio of specific heats (Euler), e.g. 1.4 */
    int volume_flux;              /* perrk_volume_flux */
    int surface_flux;             /* perrk_surface_flux */
    double mu;                    /* dynamic viscosity: 0 = Euler; > 0 adds the Navier-Stokes-Fourier viscous
                                     terms (Euler 2D / 3D only), BR1 on entropy-variable gradients (Sec. 4.3.2) */
    double prandtl;               /* Prandtl number Pr = c_p mu / kappa (> 0 when mu > 0), gas constant 1 */
} perrk_scheme_desc;

typedef struct {
    int precision;                /* perrk_precision.  PERRK_FP64: every node operation in float64.
                                     PERRK_MIXED: flux differencing, surface fluxes and the stage
                                     registers K_i in FP32; the state U and the direction d as float
                                     pairs (hi + lo, ~48-bit significand), with the entropy passes,
                                     the Newton residuals and the update evaluated in double-float on
                                     the FP32 pipe; Delta H, the Newton scalars and the step records in
                                     float64.  No float64 instruction runs per node.  Delta H then
                                     carries the FP32 rounding of the K_i (noise of ~1e-7 relative to
                                     its terms): EC runs in this form take PERRK_TARGET_PREV to keep
                                     H_{n+1} = H_n to round-off. */
    int relaxation;               /* 1: P-ERRK (relaxed), 0: plain P-ERK (gamma = 1) */
    int newton_max_it;            /* maximum Newton passes per step (>= 0) */
    double newton_tol_r;          /* stop when |r| <= tol_r * sum omega J |s(U_n)| */
    double newton_tol_g;          /* stop when |gamma update| <= tol_g */
    int guess;                    /* perrk_guess: initial Newton guess */
    int target;                   /* perrk_target: which entropy equality is enforced */
    int use_graph;                /* 1: capture one step in a CUDA graph and replay it */
    int fuse_direction;           /* 1 (default): when every b_i != 0 sits at a first, penultimate or last
                                     stage (all archetypes), form d = sum b_i K_i once at the last stage
                                     from K_1, K_{S-1}, K_S; 0: accumulate d at every stage with b_i != 0.
                                     Same sums in the same order either way. */
    int solver;                   /* a perrk_solver value, Newton by default */
    double bracket_lo, bracket_hi; /* bisection bracket / secant initial guesses (default 0.8, 1.2, Sec. 4.3.2) */
} perrk_options;

/* Per-step record (perrk_step fills one per step when info != NULL). */
typedef struct {
    double gamma;                 /* relaxation parameter taken */
    double H_n;                   /* H(U_n) */
    double dH;                    /* Delta H (eq. EntropyChangeDefinition) */
    double H_next;                /* H(U_{n+1}) */
    double t;                     /* time after the step, t_n + gamma dt */
    double gamma_guess;           /* initial Newton guess used */
    double gamma_prev;            /* gamma_{n-1}: the last converged gamma before this step (1 at the start) */
    int32_t newton_iters;         /* full-state Newton passes */
    uint32_t flags;               /* PERRK_FLAG_* */
    float features[6];            /* learned-guess features of this step (see perrk_mlp_features) */
} perrk_step_info;

typedef struct perrk_ctx perrk_ctx;

/* Fill opts with defaults: FP64, relaxed, max_it 10, tol_r 1e-14, tol_g 1e-14,
 * guess PREV (Sec. 3.1: gamma_{n-1}, 1 at the first step), target DELTA_H, no
 * graph, fused direction, Newton with bracket [0.8, 1.2] for the others. */
void perrk_default_options(perrk_options *opts);

/* Validate and copy mesh and scheme, compute LGL tables and metric terms,
 * allocate device storage on the current device.  Returns INVALID_ARG (and
 * *out = NULL) for: N != 3, bad dims, face rows not pairing '+' with the
 * matching '-' face, faces whose nodes do not coincide up to a translation,
 * non-positive Jacobians, partition ids out of range, a1 + asub != c,
 * E below the order's minimum or above S, b_i != 0 where some member is
 * inactive, nonzero asub at inactive or first-active rows. */
perrk_status perrk_create(const perrk_mesh_desc *mesh, const perrk_scheme_desc *scheme,
                          const perrk_options *opts, perrk_ctx **out);

/* n independent instances advanced together (one launch per stage covers all
 * instances' active elements; the Newton solves run per instance in one
 * launch per pass).  Instance k has its own mesh[k], scheme[k] and time step;
 * all schemes share equation, fluxes and order p.  States are concatenated in
 * instance order: [V][sum n_elem][NP]. */
perrk_status perrk_create_batched(int n, const perrk_mesh_desc *mesh, const perrk_scheme_desc *scheme,
                                  const perrk_options *opts, perrk_ctx **out);

void perrk_destroy(perrk_ctx *ctx);

/* Build a P-ERK family of order p (2, 3, 4) with members E[0..R-1] and
 * S = max E in the low-storage form above (host only, no GPU needed).
 * Archetypes of appendix A: p = 2 eq. PERK_ButcherTableauClassic_p2_E36 with
 * c_i = (i-1)/(2(S-1)); p = 3 eq. PERK_ButcherTableauOwn_p3 with
 * c_i = (i-1)/(S-3), row S read as (1/2 - a, a) and a_{S,S-1} = (1 - a_{S-1,S-2})/4;
 * p = 4 eq. PERK_ButcherTableau_p4 with eq. 4thOrderPERK_BaseCoeffs and c_2..c_{S-3} = 1.
 * The paper's optimised free coefficients are not printed; here p = 2 matches
 * the Taylor coefficients 1/j! of exp up to degree E, p = 3/4 take
 * a_{i,i-1} = c_i/8 on free rows and a_{S-1,S-2} = 1/4 (p = 3).
 * Outputs (caller-allocated): c[S], b[S], a1[R][S], asub[R][S]; *S_out = S. */
perrk_status perrk_build_tableau(int p, int R, const int32_t *E, int S_cap, int *S_out, double *c, double *b,
                                 double *a1, double *asub);

/* Total elements, variables, nodes per element and instances of ctx. */
perrk_status perrk_shape(const perrk_ctx *ctx, int *n_elem, int *nvar, int *np, int *n_inst);

/* Copy a state (SoA, float64, n_elem*NP*V values) in or out.  on_device:
 *   0  host memory; the call returns when the copy is complete;
 *   1  device memory (ordered on the stream);
 *   2  host memory, asynchronous: the copy is enqueued on the stream and the
 *      call returns at once; the caller keeps the buffer unchanged (set) or
 *      unread (get) until the stream is synchronised.  With page-locked
 *      buffers the copies of one context overlap the kernels of another.
 * set_state resets t = 0, gamma_{n-1} = 1 and sets H_n = H(U_0) = H(u),
 * A_n = sum omega J |s(u)| for every instance.  INVALID_ARG for any other
 * on_device value. */
perrk_status perrk_set_state(perrk_ctx *ctx, const double *u, int on_device, void *stream);
perrk_status perrk_get_state(perrk_ctx *ctx, double *u, int on_device, void *stream);

/* Set the time step of instance inst (-1: all).  Coefficients dt * a are
 * recomputed; a captured graph is re-instantiated on the next step. */
perrk_status perrk_set_dt(perrk_ctx *ctx, int inst, double dt);

/* Advance nsteps steps.  info: NULL (asynchronous) or host array of
 * nsteps * n_inst records (step-major), which forces a stream sync; then
 * PERRK_TIMEOUT if a bounded device wait gave up (PERRK_FLAG_TIMEOUT) and
 * PERRK_NONPHYSICAL_STATE if a non-physical or non-finite value was met. */
perrk_status perrk_step(perrk_ctx *ctx, int nsteps, perrk_step_info *info, void *stream);

/* Checkpoint / resume.  A checkpoint is a host byte buffer holding everything
 * a resumed run needs to continue bit-identically to an uninterrupted one:
 *
 *   perrk_checkpoint_header
 *   perrk_resume_info[n_inst]     the relaxation history of each instance
 *   the state in the context's own representation: float64 [V][n_elem][NP]
 *   (float64 form) or the float pair hi[V][n_elem][NP] then lo[...] (mixed
 *   form; a float64 round trip through perrk_get_state would round lo).
 *
 * The history carries the Newton warm start gamma_{n-1} (Sec. 3.1), H(U_n)
 * as the previous step left it, the tolerance scale A_n, H(U_0) for
 * TARGET_INITIAL, the learned-guess history, dt, time and step count.  The
 * mesh, tableaux, options and guess weights are the caller's: load a
 * checkpoint into a context created with the same inputs. */
typedef struct {
    uint32_t magic;               /* PERRK_CHECKPOINT_MAGIC */
    uint32_t version;             /* 1 */
    int32_t precision, n_inst, n_elem, nvar, np, reserved;
    uint64_t state_bytes;         /* bytes of the state section */
} perrk_checkpoint_header;

#define PERRK_CHECKPOINT_MAGIC 0x4b435250u   /* "PRCK" */

typedef struct {
    double t;                     /* time */
    double dt;                    /* step size of the instance */
    double H_n;                   /* H(U_n) carried from the previous step */
    double A_n;                   /* sum omega J |s(U_n)| (tolerance scale) */
    double H0;                    /* H(U_0) */
    double gamma_hist[3];         /* gamma_{n-1}, gamma_{n-2}, gamma_{n-3} */
    double dh_hist[3];            /* (Delta H / A) of the last three steps */
    int64_t steps;                /* steps since the state was set */
} perrk_resume_info;

/* Size in bytes of a checkpoint of this context (0 for a null context). */
size_t perrk_checkpoint_size(const perrk_ctx *ctx);
/* Write a checkpoint into buf (host, at least perrk_checkpoint_size bytes);
 * syncs the stream.  INVALID_ARG if buf is null or too small. */
perrk_status perrk_checkpoint_save(perrk_ctx *ctx, void *buf, size_t size, void *stream);
/* Restore state and history from a checkpoint; syncs.  INVALID_ARG if the
 * header does not match this context (precision, shapes) or the buffer is
 * short; the context is unchanged then. */
perrk_status perrk_checkpoint_load(perrk_ctx *ctx, const void *buf, size_t size, void *stream);

/* Autotune the launch mapping of ctx on the current device: times the stage
 * kernels of a whole step (every stage in order, as the step runs them) for
 * every valid elements-per-CTA choice, grid mapping (one CTA per element
 * group, or a persistent grid of k CTAs per SM, k = 2, 4, 8 and, for the box
 * kernels, the k of exactly one resident wave)
 * and, for the mixed form on box elements, stage kernel variant (generic;
 * float4 box kernel; box kernel staging the next element group with
 * cp.async; in 2D the box kernel fed by a producer warp, two ways), then the
 * relaxation block size; keeps the fastest and
 * re-captures the step graph.  Results do not depend on the choice (same
 * per-element arithmetic in the same order).  Overwrites the stage registers
 * and d (call between steps).  best_ms_out (nullable): mean time per stage
 * launch of the chosen mapping.  Synchronises the stream. */
perrk_status perrk_autotune(perrk_ctx *ctx, void *stream, float *best_ms_out);

/* Current launch mapping (elements per CTA, persistent grid size or 0,
 * relaxation block size, stage kernel variant 0/1/2 as above); each output
 * pointer is nullable. */
perrk_status perrk_tuning(const perrk_ctx *ctx, int *elems_per_cta, int *persistent_grid, int *relax_threads,
                          int *stage_variant);

/* Set the launch mapping explicitly (reproducible timing, or a mapping found
 * on another run): elements per CTA (1D: 16, 32; 2D: 4, 8, 16; 3D: 1, 2, 4),
 * persistent grid size (0: one CTA per element group), relaxation block size
 * (128, 256), stage kernel variant (0/1/2 for the mixed form on box elements;
 * 3 and 4 for the mixed form on 2D box elements: a producer warp stages
 * each element group into a ring of shared-memory buffers while consumer
 * warps compute, the own rows by bulk asynchronous copies (3) or by 16-byte
 * cp.async (4), the neighbour face nodes by cp.async, with 4 or 8 elements
 * per group and always a persistent grid, of the given size or, for 0, as
 * many CTAs as are resident; other contexts keep theirs).  Values outside these sets:
 * PERRK_INVALID_ARG.
 * A mapping whose shared memory does not fit is reported by the next launch
 * (PERRK_CUDA_ERROR, invalid configuration).  The step graph is re-captured. */
perrk_status perrk_set_tuning(perrk_ctx *ctx, int elems_per_cta, int persistent_grid, int relax_threads,
                              int stage_variant);

/* Adaptive mesh refinement (the paper's adaptive runs, Sec. 3.2.2 and Sec.
 * 5.3: refine where the shock-capturing indicator of Hennemann et al. on the
 * density is large, change the mesh every few steps, re-derive the
 * partitions from the element sizes, Sec. 2.2).  The mesh adaptation itself
 * (a 2:1-balanced quadtree) is host logic of the caller (the Python
 * package's amr module); these calls run its two device parts, for
 * single-instance 2D Euler contexts on box elements, in float64 (the mixed
 * form's state read as its float pair).
 *
 * perrk_amr_indicator: alpha (host, [n_elem]) = 1 / (1 + exp(-(s/T)(e - T)))
 * per element, e the relative energy of the highest Legendre modes of the
 * density (orthonormal basis; e = max((E_N - E_{N-1}) / E_N,
 * (E_{N-1} - E_{N-2}) / E_{N-1}), E_k the energy of the modes up to degree k
 * in each direction), T = 0.5 10^(-1.8 (N+1)^(1/4)), s = log((1-1e-4)/1e-4).
 * Synchronises the stream.
 *
 * perrk_amr_transfer: the state of src carried to the context dst of the
 * adapted mesh.  map (host, [dst n_elem][5]) row (kind, a0, a1, a2, a3):
 * kind 0 = dst element is src element a0; 1 = child a1 (a + 2 b: a the half
 * in xi, b in eta) of src element a0, by interpolation of the parent
 * polynomial; 2 = parent of src elements a0..a3 (child order a + 2 b), by L2
 * projection.  Element integrals sum omega J u are kept up to rounding.  dst
 * then holds the new state as after perrk_set_state, except that the time,
 * the relaxation history (gamma and Delta H / A of the last steps) and the
 * step count carry over from src.  INVALID_ARG for map rows out of range.
 * Synchronises the stream. */
perrk_status perrk_amr_indicator(perrk_ctx *ctx, double *alpha, void *stream);
perrk_status perrk_amr_transfer(const perrk_ctx *src, perrk_ctx *dst, const int32_t *map, void *stream);

/* The adaptive runs' mesh (host only, no GPU): a 2:1-balanced periodic
 * quadtree of square cells on [-L, L]^2 over an n x n base grid.  A leaf is
 * (level, ix, iy), 0 <= ix, iy < n 2^level, with the cell
 * [-L + ix h, -L + (ix+1) h] x [-L + iy h, -L + (iy+1) h], h = 2L / (n 2^level);
 * leaves are kept in the canonical order of (level, ix, iy).
 *
 * perrk_quadtree_create: the uniform tree (n x n leaves at level 0).
 * perrk_quadtree_leaves: out[n_leaves][3] = (level, ix, iy).
 * perrk_quadtree_adapt: marks[n_leaves] (+1 refine, -1 coarsen, 0 keep).
 * Families whose four leaves are all marked -1 (and none +1) merge, in
 * descending (level, ix, iy) order of the parent, unless a face neighbour
 * of the parent would then be two levels finer; leaves marked +1 split;
 * then leaves are split until every face neighbour differs by at most one
 * level.  The tree is replaced by the new one; map (caller-allocated,
 * map_cap rows of 5; 4 x the old leaf count always suffices) receives the
 * rows of perrk_amr_transfer for the new leaves, *n_new their count.
 * perrk_quadtree_mesh: the mesh arrays of perrk_mesh_desc for the current
 * leaves: coords [n_leaves][16][2] (LGL nodes), faces [n_faces][4]
 * (conforming pairs), mortars [n_mortars][4] (2:1 rows), levels [n_leaves];
 * any output may be NULL (call once with NULLs to get n_faces, n_mortars:
 * at most 2 and 4 per leaf).  INVALID_ARG for null arguments, a map
 * capacity below the new count, or a refinement beyond n 2^level = 2^29
 * cells per direction. */
typedef struct perrk_quadtree perrk_quadtree;
perrk_status perrk_quadtree_create(int n, double L, perrk_quadtree **out);
void perrk_quadtree_destroy(perrk_quadtree *tree);
int perrk_quadtree_size(const perrk_quadtree *tree);
perrk_status perrk_quadtree_leaves(const perrk_quadtree *tree, int32_t *out);
perrk_status perrk_quadtree_adapt(perrk_quadtree *tree, const int8_t *marks, int32_t *map, int map_cap, int *n_new);
perrk_status perrk_quadtree_mesh(const perrk_quadtree *tree, double *coords, int32_t *faces, int *n_faces,
                                 int32_t *mortars, int *n_mortars, int32_t *levels);

/* Test hook (the paper has no counterpart): with on != 0, the producer warp
 * of stage kernel variants 3 and 4 fills no staging buffer, so that its consumer
 * warps' bounded waits run out after about one second each; the next
 * perrk_step with records then returns PERRK_TIMEOUT (PERRK_FLAG_TIMEOUT),
 * with nothing left in flight on the GPU.  on = 0 restores normal launches;
 * the context stays usable.  Other stage kernels ignore it. */
perrk_status perrk_test_stall_producer(perrk_ctx *ctx, int on);

/* H(U) = sum omega J s(U) of the current state per instance (host array [n_inst]); syncs. */
perrk_status perrk_entropy(perrk_ctx *ctx, double *H, void *stream);

/* Enqueue exactly one stage kernel (stage index 0..S-1, 0-based) of the
 * step on the context's current buffers (for timing and profiling; the
 * result is the stage's K_i, which the last stage keeps in registers only:
 * it enters d there and nothing reads it later).  Asynchronous on stream. */
perrk_status perrk_launch_stage(perrk_ctx *ctx, int stage, void *stream);

/* Static facts of one stage launch: elements evaluated and the algorithmic
 * bytes it must move (own-element reads of U_n, K_1, K_{i-1} as the stage
 * rows require, the K_i write (not at the last stage), the d read/write at
 * stages with b_i != 0,
 * geometry and index data; neighbour face reads are not counted; with
 * viscous terms also the BR1 node fluxes of the gradient set and their
 * divergence).  Also the
 * stages per step, the number of kernels one step launches and the DOF-stage
 * updates (sum_r E^(r) M^(r), eq. RHSEvals) of one step. */
perrk_status perrk_stage_info(const perrk_ctx *ctx, int stage, int64_t *n_active, int64_t *bytes, int *n_stages,
                              int *kernels_per_step, int64_t *dof_stage_per_step);

/* Allocation-free entropy functional (the paper has no counterpart; this is
 * an interface for callers that cannot allocate device memory when they need
 * the value, e.g. because they hand all device memory to their own pool
 * allocator up front, or run a loop in which cudaMalloc -- which may
 * synchronise the device and can fail under memory pressure -- is not
 * allowed).  out[0] = sum_q wJ[q] s(u_q), out[1] = sum_q wJ[q] |s(u_q)|, with
 * s the entropy of `equation` (u^2/2 for Burgers, -rho log(p rho^-gamma) for
 * Euler), in float64 with compensated sums.  u: device, SoA [V][n_nodes];
 * wJ: device [n_nodes] (quadrature weight times Jacobian per node); out:
 * device double[2].  No context is used and nothing is allocated: the
 * cross-block scratch is a file-scope device array of ~128 KiB that every
 * device which loads the library holds until process exit.  n_nodes must lie
 * in [1, 16777216]; larger inputs are rejected with PERRK_INVALID_ARG.  The
 * first call on a device looks up the array's device address (with that
 * device current); make that first call before any stream capture.  All
 * calls share the array (it keeps the last call's contents; its counter is
 * cleared at the start of each call), so calls whose work overlaps on the
 * GPU race.  A non-physical node (rho <= 0 or p <= 0) yields NaN in out[0]
 * and out[1].  The cached array address is not refreshed after
 * cudaDeviceReset: do not call this again on a device that was reset.
 * Asynchronous on stream. */
perrk_status perrk_entropy_static(int equation, double gamma_gas, const double *u, const double *wJ, long long n_nodes,
                                  double *out, void *stream);

/* One evaluation of F on all elements: u_in, k_out device arrays [V][n_elem][NP]. */
perrk_status perrk_rhs(perrk_ctx *ctx, const double *u_in, double *k_out, void *stream);

/* Learned Newton guess: a 2x64 tanh MLP on F = 6 features
 * available before the first Newton pass of step n, all from quantities the
 * step has already computed: (gamma_{n-1} - 1, gamma_{n-2} - 1, gamma_{n-3} - 1,
 * Delta H_n / A_n, (Delta H / A)_{n-1}, (Delta H / A)_{n-2}) with
 * A = sum omega J |s(U)|; it predicts gamma_n - gamma_{n-1} and the guess is
 * gamma_{n-1} + prediction.  The Newton iteration then runs unchanged, so the
 * converged gamma does not depend on the guess.  weights: host float32 array of perrk_mlp_size() values
 * laid out W1[64][F], b1[64], W2[64][64], b2[64], W3[64], b3, then F input
 * means, F input scales, an output scale; NULL disables it. */
int perrk_mlp_size(void);
int perrk_mlp_features(void);
perrk_status perrk_set_mlp(perrk_ctx *ctx, const float *weights, int n);

/* Train the MLP on the device with the library's own forward/backward/Adam
 * kernels: feats [n][F], target [n] (host float32), in/out weights as above
 * (updated in place), epochs of full-batch Adam with learning rate lr.
 * loss_out (nullable): final mean squared error. */
perrk_status perrk_mlp_train(const float *feats, const float *target, int n, float *weights,
                             int epochs, float lr, float *loss_out, void *stream);

/* Full-batch gradient of the mean squared error of the MLP (same layout as
 * weights; only the network parameters, the normalisation entries are 0):
 * grad_out host float32 [perrk_mlp_size()], loss_out host float32 (nullable).
 * Used to check the device backward pass against an independent one. */
perrk_status perrk_mlp_grad(const float *feats, const float *target, int n, const float *weights, float *grad_out,
                            float *loss_out, void *stream);

/* Diagnostic: y[i] = log(x[i]) evaluated by the library's double-float
 * logarithm (the one the mixed form uses for the entropy functional); x, y
 * device arrays of n float64 values, x > 0.  Synchronises the stream. */
perrk_status perrk_df_log(const double *x, double *y, int n, void *stream);

/* Diagnostic (the paper has no counterpart): FMA throughput of the current
 * device in TFLOP/s, FP32 (fp64 = 0) or FP64 (fp64 = 1), from independent FMA
 * chains over 8 CTAs of 256 threads per SM, `iters` rounds of 8 chains per
 * thread, timed with CUDA events on the stream (one FMA = 2 flops).  It is
 * the peak against which kernels bound by plain ALU arithmetic (the float64
 * form's stage and Newton kernels) are reported.  Allocates and frees a
 * small output buffer; synchronises the stream.  INVALID_ARG for a null
 * output or iters < 1. */
perrk_status perrk_fma_peak(int fp64, int iters, double *tflops, void *stream);

/* Last CUDA error string seen by this thread (static storage). */
const char *perrk_last_error(void);
const char *perrk_status_string(perrk_status s);

#ifdef __cplusplus
}
#endif
#endif /* PERRK_H */
