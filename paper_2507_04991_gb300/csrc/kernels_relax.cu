// Relaxation kernels (Sec. 3 and Sec. 3.1 of the paper), float64:
//   k_relax_init   Delta H = dt sum_e e_dh[e] per instance; initial Newton guess
//   k_newton_pass  one full-state pass at the current gamma:
//                  R = sum omega J s(U_n + gamma dt d), G = sum omega J <w(.), dt d>,
//                  then (last block of the instance) one Newton update of
//                  r(gamma) = R - H_target(gamma) (eq. RelaxationEquation)
//   k_update       U_{n+1} = U_n + gamma dt d (eq. RRKM_Update), t += gamma dt,
//                  step record; H(U_{n+1}) recomputed only after a fallback
//   k_entropy      H(U) and sum omega J |s(U)| per instance
// Work is split into chunks of contiguous elements of one instance; each
// chunk writes a compensated partial, and the last chunk of an instance to
// finish (atomic ticket, no waiting) sums the partials in chunk order, so the
// result is deterministic.  Passes of an instance whose Newton solve is done
// return immediately, so a fixed number of launches (graph-capturable)
// realises the data-dependent iteration count.
#include <cuda_runtime.h>

#include <cmath>

#include "dfloat.cuh"
#include "physics.cuh"

namespace perrk {

struct RelaxParams {
    double *U;
    float *Uf, *Ul;        // mixed form: the state as a float pair U = Uf + Ul
    const float *dh, *dl;  // mixed form: the direction as a float pair
    const float *e_dhf;    // mixed form: element Delta H sums as float pairs [n_elem][2]
    const float *wJf, *wJl;  // mixed form: omega J as a float pair
    const double *d, *e_dh, *wJ;
    const int32_t *chunk_inst, *chunk_e0, *chunk_e1, *inst_chunk0, *inst_nchunks;
    InstScalars *scal;
    double *partials;      // [n_chunks][8]
    uint32_t *counters;    // [n_inst]
    uint32_t *flags;
    perrk_step_info *rec;
    const float *mlp;
    int rec_slot, rec_cap, n_inst;
    size_t NE;
    double gamma_gas;
    int max_it, guess, target, relax, query, mixed, solver;
    int split;             // mixed form, k_entropy: split U (float64) into Uf, Ul first (set_state)
    double tol_r, tol_g, br_lo, br_hi;
    const float4 *dftab;    // double-float log table (mixed form)
    DfConst K;
};

// Entropy of one node in double-float (mixed form) from the state as float
// pairs: returns s and, when dv != nullptr (the direction, float), the float
// value of <w(u), dv>.  s = -rho (log p - gamma log rho).
template <int DIM, int EQ>
__device__ __forceinline__ df df_entropy(const df *x, const float *dv, const RelaxParams &P, float &wd, uint32_t &bad) {
    if constexpr (EQ == EQ_BURGERS) {
        df sq = df_mul(x[0], x[0]);
        if (dv) wd = x[0].hi * dv[0];
        return df{0.5f * sq.hi, 0.5f * sq.lo};
    } else {
        const df ir = df_rcp(x[0]);
        df m2 = df_mul(x[1], x[1]);
#pragma unroll
        for (int a = 1; a < DIM; ++a) m2 = df_add(m2, df_mul(x[1 + a], x[1 + a]));
        df ke = df_mul(m2, ir);
        ke.hi *= 0.5f;
        ke.lo *= 0.5f;
        const df p = df_mul(P.K.gm1, df_sub(x[DIM + 1], ke));
        if (!(x[0].hi > 0.0f) || !(p.hi > 0.0f) || !isfinite(p.hi)) {
            bad |= PERRK_FLAG_NONPHYSICAL;
            wd = 0.0f;
            return df{0.0f, 0.0f};
        }
        const df lp = df_log(p, P.dftab, P.K), lr = df_log(x[0], P.dftab, P.K);
        const df S = df_sub(lp, df_mul(P.K.gam, lr));
        if (dv) {
            // w in float: (gamma - S - (gamma-1) |m|^2/(2 rho p), (gamma-1) m/p, -(gamma-1) rho/p)
            float ip;   // w only needs float accuracy
            asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(ip) : "f"(p.hi));
            const float gm1 = P.K.gm1.hi;
            const float w0 = P.K.gam.hi - S.hi - gm1 * ke.hi * ip;
            float md = 0.0f;
#pragma unroll
            for (int a = 0; a < DIM; ++a) md = fmaf(x[1 + a].hi, dv[1 + a], md);
            wd = fmaf(w0, dv[0], gm1 * ip * (md - x[0].hi * dv[DIM + 1]));
        }
        return df_neg(df_mul(x[0], S));
    }
}

template <int DIM, int EQ>
__device__ __forceinline__ void node_entropy(const double *u, double gam, double &s, double *w, uint32_t &bad) {
    if constexpr (EQ == EQ_BURGERS) {
        s = 0.5 * u[0] * u[0];
        if (w) w[0] = u[0];
    } else {
        euler_entropy<DIM>(u, gam, s, w, bad);
    }
}

// Write this block's NQ compensated sums and take a ticket.  The instance's
// last block then reduces all chunk partials with all of its threads (fixed
// strided assignment and fixed tree: deterministic); returns true in its
// thread 0, where tot[] holds the instance totals.
template <int NQ>
__device__ __forceinline__ bool chunk_publish(const RelaxParams &P, int chunk, int inst, double (&s)[NQ],
                                              double (&c)[NQ], double (&tot)[NQ]);

template <int NQ>
__device__ __forceinline__ bool chunk_finish(const RelaxParams &P, int chunk, int inst, double (&s)[NQ], double (&c)[NQ],
                                             double (&tot)[NQ]) {
    __shared__ double sm0[2 * NQ * 32];
    block_sum<NQ>(s, c, sm0);
    return chunk_publish<NQ>(P, chunk, inst, s, c, tot);
}

// Block sum of a per-thread double-float value and two floats on the FP32
// pipe (fixed shuffle tree); the block's result is valid in thread 0.
__device__ __forceinline__ void block_sum_df(df &r, float &g, float &a) {
    __shared__ float sm[4][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int off = 16; off > 0; off >>= 1) {
        df o{__shfl_down_sync(0xffffffffu, r.hi, off), __shfl_down_sync(0xffffffffu, r.lo, off)};
        r = df_add(r, o);
        g += __shfl_down_sync(0xffffffffu, g, off);
        a += __shfl_down_sync(0xffffffffu, a, off);
    }
    if (lane == 0) {
        sm[0][warp] = r.hi;
        sm[1][warp] = r.lo;
        sm[2][warp] = g;
        sm[3][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < nw; ++w) {
            r = df_add(r, df{sm[0][w], sm[1][w]});
            g += sm[2][w];
            a += sm[3][w];
        }
    }
    __syncthreads();
}

// Publish thread 0's block sums as the chunk's partial and take a ticket; the
// instance's last block reduces all partials (see chunk_finish).
template <int NQ>
__device__ __forceinline__ bool chunk_publish(const RelaxParams &P, int chunk, int inst, double (&s)[NQ],
                                              double (&c)[NQ], double (&tot)[NQ]) {
    __shared__ double sm[2 * NQ * 32];
    __shared__ int s_last;
    if (threadIdx.x == 0) {
        for (int k = 0; k < NQ; ++k) {
            P.partials[(size_t)chunk * 8 + 2 * k] = s[k];
            P.partials[(size_t)chunk * 8 + 2 * k + 1] = c[k];
        }
        __threadfence();
        unsigned ticket = atomicAdd(P.counters + inst, 1u);
        s_last = (ticket == (unsigned)P.inst_nchunks[inst] - 1u);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    const int c0 = P.inst_chunk0[inst], nc = P.inst_nchunks[inst];
    double ss[NQ], cc[NQ];
    for (int k = 0; k < NQ; ++k) {
        ss[k] = 0.0;
        cc[k] = 0.0;
    }
    for (int j = threadIdx.x; j < nc; j += blockDim.x)
        for (int k = 0; k < NQ; ++k) {
            comp_add(ss[k], cc[k], __ldcg(P.partials + (size_t)(c0 + j) * 8 + 2 * k));
            cc[k] += __ldcg(P.partials + (size_t)(c0 + j) * 8 + 2 * k + 1);
        }
    block_sum<NQ>(ss, cc, sm);
    if (threadIdx.x != 0) return false;
    for (int k = 0; k < NQ; ++k) tot[k] = ss[k] + cc[k];
    P.counters[inst] = 0u;
    return true;
}

__device__ void accept_gamma(InstScalars &s) {
    // Sec. 3.2.1: a non-converged Newton solve falls back to gamma = 1;
    // roots outside (0.5, 1.5) are rejected as spurious (r(0) = 0 always).
    if (!s.converged || !isfinite(s.gamma) || !(s.gamma > 0.5 && s.gamma < 1.5)) {
        s.gamma = 1.0;
        s.converged = 0;
        s.flags |= PERRK_FLAG_NEWTON_FALLBACK;
        s.need_H = !(s.iters > 0 && s.gamma_eval == 1.0);
        if (!s.need_H) s.H_next = s.R_last;
    } else {
        s.need_H = 0;
        s.H_next = (s.gamma == s.gamma_eval) ? s.R_last : fma(s.G_last, s.gamma - s.gamma_eval, s.R_last);
    }
}

// The instance's Delta H, the features of the learned guess and the initial
// gamma of its root solve, from the total of its element Delta H sums
// (thread 0 of the block that holds the total)
__device__ void init_instance(const RelaxParams &P, int inst, double tot) {
    InstScalars &S = P.scal[inst];
    S.dH = S.dt * tot;
    S.feat[0] = S.hist_gamma[0] - 1.0;
    S.feat[1] = S.hist_gamma[1] - 1.0;
    S.feat[2] = S.hist_gamma[2] - 1.0;
    S.feat[3] = S.A_n > 0.0 ? S.dH / S.A_n : 0.0;
    S.feat[4] = S.hist_dh[0];
    S.feat[5] = S.hist_dh[1];
    S.iters = 0;
    S.flags = 0;
    S.converged = 0;
    S.need_H = 0;
    if (!P.relax) {
        S.gamma = 1.0;
        S.done = 1;
        S.converged = 1;
        S.gamma_guess = 1.0;
        return;
    }
    S.gamma = (P.guess == PERRK_GUESS_ONE) ? 1.0 : S.hist_gamma[0];
    if (P.solver != PERRK_SOLVER_NEWTON) {
        // bisection: first pass at the bracket's lower end; secant: first guess
        S.br_lo = P.br_lo;
        S.br_hi = P.br_hi;
        S.gamma = P.br_lo;
    }
    S.gamma_guess = S.gamma;
    S.gamma_eval = NAN;
    S.done = 0;
    if (P.max_it == 0) {
        S.done = 1;
        accept_gamma(S);
    }
}

template <int DIM, int EQ>
__global__ void k_relax_init(const RelaxParams P) {
    const int chunk = blockIdx.x;
    const int inst = P.chunk_inst[chunk];
    double s[1] = {0.0}, c[1] = {0.0}, tot[1];
    if (P.mixed) {
        // mixed form: Delta H carries FP32 rounding; double-float block sum on the FP32 pipe
        df r = {0.0f, 0.0f};
        float g = 0.0f, a = 0.0f;
        for (int e = P.chunk_e0[chunk] + threadIdx.x; e < P.chunk_e1[chunk]; e += blockDim.x)
            r = df_add(r, df{P.e_dhf[2 * e], P.e_dhf[2 * e + 1]});
        block_sum_df(r, g, a);
        s[0] = (double)r.hi;
        c[0] = (double)r.lo;
        if (!chunk_publish<1>(P, chunk, inst, s, c, tot)) return;
    } else {
        for (int e = P.chunk_e0[chunk] + threadIdx.x; e < P.chunk_e1[chunk]; e += blockDim.x) comp_add(s[0], c[0], P.e_dh[e]);
        if (!chunk_finish<1>(P, chunk, inst, s, c, tot)) return;
    }
    init_instance(P, inst, tot[0]);
}

// One block per instance (contexts with at least as many instances as SMs,
// where one block per work chunk is mostly launch overhead): the block sums
// all element Delta H values of its instance in a fixed order, with no
// cross-block partials, and sets the instance up.
__global__ void __launch_bounds__(256) k_relax_init_inst(const RelaxParams P) {
    const int inst = blockIdx.x;
    const int c0 = P.inst_chunk0[inst], nc = P.inst_nchunks[inst];
    const int e0 = P.chunk_e0[c0], e1 = P.chunk_e1[c0 + nc - 1];
    double tot;
    if (P.mixed) {
        df r = {0.0f, 0.0f};
        float g = 0.0f, a = 0.0f;
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) r = df_add(r, df{P.e_dhf[2 * e], P.e_dhf[2 * e + 1]});
        block_sum_df(r, g, a);
        tot = (double)r.hi + (double)r.lo;
    } else {
        double sc[1] = {0.0}, cc[1] = {0.0};
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) comp_add(sc[0], cc[0], P.e_dh[e]);
        __shared__ double sm0[2 * 32];
        block_sum<1>(sc, cc, sm0);
        tot = sc[0] + cc[0];
    }
    if (threadIdx.x == 0) init_instance(P, inst, tot);
}

template <int DIM, int EQ, bool DF>
__global__ void __launch_bounds__(256) k_newton_pass(const RelaxParams P) {
    constexpr int NP = ipow4(DIM);
    constexpr int V = EQ == EQ_BURGERS ? 1 : DIM + 2;
    const int chunk = blockIdx.x;
    const int inst = P.chunk_inst[chunk];
    if (P.scal[inst].done) return;       // uniform per block
    const double gam = P.scal[inst].gamma, dt = P.scal[inst].dt, gdt = gam * dt;
    const size_t NPtot = P.NE * NP;
    const size_t n0 = (size_t)P.chunk_e0[chunk] * NP, n1 = (size_t)P.chunk_e1[chunk] * NP;
    double s[3] = {0, 0, 0}, c[3] = {0, 0, 0}, tot[3];
    uint32_t bad = 0;
    if constexpr (DF) {
        // U_n + gamma dt d and the entropy in double-float on the FP32 pipe
        const df gdtf = df_from(gdt);
        df R = {0.0f, 0.0f};
        float G = 0.0f, A = 0.0f;
        for (size_t j = n0 + threadIdx.x; j < n1; j += blockDim.x) {
            df x[V];
            float dv[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const size_t i = v * NPtot + j;
                const df dd{__ldg(P.dh + i), __ldg(P.dl + i)};
                dv[v] = dd.hi;
                x[v] = df_add(df{__ldg(P.Uf + i), __ldg(P.Ul + i)}, df_mul(gdtf, dd));
            }
            float wd;
            const df sv = df_entropy<DIM, EQ>(x, dv, P, wd, bad);
            const df wj{__ldg(P.wJf + j), __ldg(P.wJl + j)};
            R = df_add(R, df_mul(sv, wj));
            G = fmaf(wj.hi, wd, G);
            A = fmaf(wj.hi, fabsf(sv.hi), A);
        }
        block_sum_df(R, G, A);
        s[0] = (double)R.hi;
        c[0] = (double)R.lo;
        s[1] = (double)G * dt;
        s[2] = (double)A;
        if (bad) atomicOr(P.flags, bad);
        if (!chunk_publish<3>(P, chunk, inst, s, c, tot)) return;
    } else {
        for (size_t j = n0 + threadIdx.x; j < n1; j += blockDim.x) {
            double u[V], dv[V], w[V], sv;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                dv[v] = __ldg(P.d + v * NPtot + j);
                u[v] = fma(gdt, dv[v], __ldg(P.U + v * NPtot + j));
            }
            node_entropy<DIM, EQ>(u, P.gamma_gas, sv, w, bad);
            double wd = 0.0;
#pragma unroll
            for (int v = 0; v < V; ++v) wd = fma(w[v], dv[v], wd);
            const double wj = __ldg(P.wJ + j);
            comp_add(s[0], c[0], wj * sv);
            comp_add(s[1], c[1], wj * dt * wd);
            comp_add(s[2], c[2], wj * fabs(sv));
        }
        if (bad) atomicOr(P.flags, bad);
        if (!chunk_finish<3>(P, chunk, inst, s, c, tot)) return;
    }
    InstScalars &S = P.scal[inst];
    const double R = tot[0], G = tot[1], A = tot[2];
    double T, dT;
    if (P.target == PERRK_TARGET_DELTA_H) {
        T = fma(S.gamma, S.dH, S.H_n);
        dT = S.dH;
    } else if (P.target == PERRK_TARGET_PREV) {
        T = S.H_n;
        dT = 0.0;
    } else {
        T = S.H0;
        dT = 0.0;
    }
    const double r = R - T, rp = G - dT;
    S.iters += 1;
    S.gamma_eval = S.gamma;
    S.R_last = R;
    S.G_last = G;
    S.A_last = A;
    if (P.solver == PERRK_SOLVER_BISECTION) {
        // Sec. 3.1 bisection: r at lo, at hi (must differ in sign), then midpoints
        const double g = S.gamma;
        if (!isfinite(r)) {
            S.done = 1;
        } else if (fabs(r) <= P.tol_r * S.A_n) {
            S.converged = 1;
            S.done = 1;
        } else if (S.iters == 1) {
            S.r_lo = r;
            S.gamma = S.br_hi;
        } else if (S.iters == 2) {
            S.r_hi = r;
            if (!(S.r_lo * r < 0.0)) S.done = 1;   // no sign change: no bracketed root
            else S.gamma = 0.5 * (S.br_lo + S.br_hi);
        } else {
            if (r * S.r_lo < 0.0) {
                S.br_hi = g;
                S.r_hi = r;
            } else {
                S.br_lo = g;
                S.r_lo = r;
            }
            if (S.br_hi - S.br_lo <= P.tol_g) {
                S.converged = 1;                    // take the evaluated midpoint
                S.done = 1;
            } else {
                S.gamma = 0.5 * (S.br_lo + S.br_hi);
            }
        }
    } else if (P.solver == PERRK_SOLVER_SECANT) {
        // Sec. 3.1 secant from the two guesses br_lo, br_hi
        const double g = S.gamma;
        if (!isfinite(r)) {
            S.done = 1;
        } else if (fabs(r) <= P.tol_r * S.A_n) {
            S.converged = 1;
            S.done = 1;
        } else if (S.iters == 1) {
            S.g_prev = g;
            S.r_prev = r;
            S.gamma = S.br_hi;
        } else {
            const double den = r - S.r_prev;
            if (den == 0.0) {
                S.done = 1;
            } else {
                const double g_new = g - r * (g - S.g_prev) / den;
                if (fabs(g_new - g) <= P.tol_g) {
                    S.converged = 1;                // take the evaluated g
                    S.done = 1;
                } else {
                    S.g_prev = g;
                    S.r_prev = r;
                    S.gamma = g_new;
                }
            }
        }
        if (!S.done && S.iters >= P.max_it) S.done = 1;
        if (S.done) accept_gamma(S);
        return;
    } else if (fabs(r) <= P.tol_r * S.A_n) {
        // no further pass; the correction from this pass is still applied
        if (isfinite(r) && isfinite(rp) && rp != 0.0) S.gamma = S.gamma - r / rp;
        S.converged = 1;
        S.done = 1;
    } else if (!isfinite(r) || !isfinite(rp) || rp == 0.0) {
        S.done = 1;
    } else {
        const double dg = -r / rp;
        S.gamma = S.gamma + dg;
        if (fabs(dg) <= P.tol_g) {
            S.converged = 1;
            S.done = 1;
        }
    }
    if (!S.done && S.iters >= P.max_it) S.done = 1;
    if (S.done) accept_gamma(S);
}

template <int DIM, int EQ, bool DF>
__global__ void __launch_bounds__(256) k_update(const RelaxParams P) {
    constexpr int NP = ipow4(DIM);
    constexpr int V = EQ == EQ_BURGERS ? 1 : DIM + 2;
    const int chunk = blockIdx.x;
    const int inst = P.chunk_inst[chunk];
    const double gdt = P.scal[inst].gamma * P.scal[inst].dt;
    const int needH = P.scal[inst].need_H;   // uniform per block
    const size_t NPtot = P.NE * NP;
    const size_t n0 = (size_t)P.chunk_e0[chunk] * NP, n1 = (size_t)P.chunk_e1[chunk] * NP;
    double s[2] = {0, 0}, c[2] = {0, 0}, tot[2];
    uint32_t bad = 0;
    df R = {0.0f, 0.0f};
    float A = 0.0f, G = 0.0f;
    const df gdtf = df_from(gdt);
    if constexpr (DF) {
        if (!needH) {
            // the common case: a pure stream over the float pairs, four
            // consecutive nodes per thread and 16-byte accesses (chunk bounds
            // and array offsets are multiples of NP >= 4 nodes)
            const size_t j0 = n0 / 4, j1 = n1 / 4, NP4 = NPtot / 4;
            float4 *Uf4 = reinterpret_cast<float4 *>(P.Uf), *Ul4 = reinterpret_cast<float4 *>(P.Ul);
            const float4 *dh4 = reinterpret_cast<const float4 *>(P.dh), *dl4 = reinterpret_cast<const float4 *>(P.dl);
            for (size_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const size_t i = v * NP4 + j;
                    const float4 uh = Uf4[i], ul = Ul4[i], dh = __ldg(dh4 + i), dl = __ldg(dl4 + i);
                    const df x0 = df_add(df{uh.x, ul.x}, df_mul(gdtf, df{dh.x, dl.x}));
                    const df x1 = df_add(df{uh.y, ul.y}, df_mul(gdtf, df{dh.y, dl.y}));
                    const df x2 = df_add(df{uh.z, ul.z}, df_mul(gdtf, df{dh.z, dl.z}));
                    const df x3 = df_add(df{uh.w, ul.w}, df_mul(gdtf, df{dh.w, dl.w}));
                    Uf4[i] = make_float4(x0.hi, x1.hi, x2.hi, x3.hi);
                    Ul4[i] = make_float4(x0.lo, x1.lo, x2.lo, x3.lo);
                    if (!isfinite(x0.hi) || !isfinite(x1.hi) || !isfinite(x2.hi) || !isfinite(x3.hi))
                        bad |= PERRK_FLAG_NONFINITE;
                }
            }
        }
    }
    for (size_t j = n0 + threadIdx.x; j < n1; j += blockDim.x) {
        if constexpr (DF) {
            if (!needH) break;
            // U_{n+1} = U_n + gamma dt d in double-float (FP32 pipe)
            df x[V];
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const size_t i = v * NPtot + j;
                x[v] = df_add(df{P.Uf[i], P.Ul[i]}, df_mul(gdtf, df{__ldg(P.dh + i), __ldg(P.dl + i)}));
                P.Uf[i] = x[v].hi;
                P.Ul[i] = x[v].lo;
                if (!isfinite(x[v].hi)) bad |= PERRK_FLAG_NONFINITE;
            }
            if (needH) {
                float wd;
                const df sv = df_entropy<DIM, EQ>(x, nullptr, P, wd, bad);
                const df t = df_mul(sv, df{__ldg(P.wJf + j), __ldg(P.wJl + j)});
                R = df_add(R, t);
                A += fabsf(t.hi);
            }
            continue;
        } else {
        double u[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
            u[v] = fma(gdt, __ldg(P.d + v * NPtot + j), P.U[v * NPtot + j]);
            P.U[v * NPtot + j] = u[v];
            if (!isfinite(u[v])) bad |= PERRK_FLAG_NONFINITE;
        }
        if (needH) {
            {
                double sv;
                node_entropy<DIM, EQ>(u, P.gamma_gas, sv, nullptr, bad);
                const double wj = __ldg(P.wJ + j);
                comp_add(s[0], c[0], wj * sv);
                comp_add(s[1], c[1], wj * fabs(sv));
            }
        }
        }
    }
    if (bad) atomicOr(P.flags, bad);
    if (needH) {
        if constexpr (DF) {
            block_sum_df(R, G, A);
            s[0] = (double)R.hi;
            c[0] = (double)R.lo;
            s[1] = (double)A;
            if (!chunk_publish<2>(P, chunk, inst, s, c, tot)) return;
        } else {
            if (!chunk_finish<2>(P, chunk, inst, s, c, tot)) return;
        }
    } else {
        // no reduction: only the instance's last block does the bookkeeping
        __shared__ int s_last;
        if (threadIdx.x == 0) {
            __threadfence();
            const unsigned ticket = atomicAdd(P.counters + inst, 1u);
            s_last = (ticket == (unsigned)P.inst_nchunks[inst] - 1u);
        }
        __syncthreads();
        if (!s_last || threadIdx.x != 0) return;
        __threadfence();
        P.counters[inst] = 0u;
    }
    InstScalars &S = P.scal[inst];
    double Hn1, An1;
    if (needH) {
        Hn1 = tot[0];
        An1 = tot[1];
    } else if (P.relax) {
        Hn1 = S.H_next;
        An1 = S.A_last;
    } else {
        Hn1 = NAN;
        An1 = S.A_n;
    }
    S.t += S.gamma * S.dt;
    const uint32_t fl = S.flags | (*(volatile uint32_t *)P.flags);
    if (P.rec) {
        perrk_step_info &R = P.rec[(size_t)(S.nsteps_done % P.rec_cap) * P.n_inst + inst];
        R.gamma = S.gamma;
        R.H_n = S.H_n;
        R.dH = S.dH;
        R.H_next = Hn1;
        R.t = S.t;
        R.gamma_guess = S.gamma_guess;
        R.gamma_prev = S.hist_gamma[0];
        R.newton_iters = S.iters;
        R.flags = fl;
        for (int k = 0; k < 6; ++k) R.features[k] = (float)S.feat[k];
    }
    if (P.relax) {
        if (S.converged) {
            S.hist_gamma[2] = S.hist_gamma[1];
            S.hist_gamma[1] = S.hist_gamma[0];
            S.hist_gamma[0] = S.gamma;
        }
        S.hist_dh[2] = S.hist_dh[1];
        S.hist_dh[1] = S.hist_dh[0];
        S.hist_dh[0] = S.A_n > 0.0 ? S.dH / S.A_n : 0.0;
    }
    S.H_n = Hn1;
    if (isfinite(An1)) S.A_n = An1;
    S.nsteps_done += 1;
}

template <int DIM, int EQ, bool DF>
__global__ void __launch_bounds__(256) k_entropy(const RelaxParams P) {
    constexpr int NP = ipow4(DIM);
    constexpr int V = EQ == EQ_BURGERS ? 1 : DIM + 2;
    const int chunk = blockIdx.x;
    const int inst = P.chunk_inst[chunk];
    const size_t NPtot = P.NE * NP;
    const size_t n0 = (size_t)P.chunk_e0[chunk] * NP, n1 = (size_t)P.chunk_e1[chunk] * NP;
    double s[2] = {0, 0}, c[2] = {0, 0}, tot[2];
    uint32_t bad = 0;
    df R = {0.0f, 0.0f};
    float A = 0.0f, G = 0.0f;
    for (size_t j = n0 + threadIdx.x; j < n1; j += blockDim.x) {
        if constexpr (DF) {
            df x[V];
            if (P.split) {
                // hi = round(u), lo = round(u - hi): the float pair set_state stores
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const size_t i = v * NPtot + j;
                    const double u = P.U[i];
                    const float hi = __double2float_rn(u);
                    const float lo = __double2float_rn(u - (double)hi);
                    P.Uf[i] = hi;
                    P.Ul[i] = lo;
                    x[v] = df{hi, lo};
                }
            } else {
#pragma unroll
                for (int v = 0; v < V; ++v) x[v] = df{__ldg(P.Uf + v * NPtot + j), __ldg(P.Ul + v * NPtot + j)};
            }
            float wd;
            const df sv = df_entropy<DIM, EQ>(x, nullptr, P, wd, bad);
            const df t = df_mul(sv, df{__ldg(P.wJf + j), __ldg(P.wJl + j)});
            R = df_add(R, t);
            A += fabsf(t.hi);
        } else {
            double u[V];
#pragma unroll
            for (int v = 0; v < V; ++v) u[v] = __ldg(P.U + v * NPtot + j);
            double sv;
            node_entropy<DIM, EQ>(u, P.gamma_gas, sv, nullptr, bad);
            const double wj = __ldg(P.wJ + j);
            comp_add(s[0], c[0], wj * sv);
            comp_add(s[1], c[1], wj * fabs(sv));
        }
    }
    if (bad) atomicOr(P.flags, bad);
    if constexpr (DF) {
        block_sum_df(R, G, A);
        s[0] = (double)R.hi;
        c[0] = (double)R.lo;
        s[1] = (double)A;
        if (!chunk_publish<2>(P, chunk, inst, s, c, tot)) return;
    } else {
        if (!chunk_finish<2>(P, chunk, inst, s, c, tot)) return;
    }
    InstScalars &S = P.scal[inst];
    if (P.query) {
        S.H_next = tot[0];
        return;
    }
    S.H_n = tot[0];
    S.H0 = tot[0];
    S.A_n = tot[1];
    S.t = 0.0;
    S.gamma = 1.0;
    for (int k = 0; k < 3; ++k) {
        S.hist_gamma[k] = 1.0;
        S.hist_dh[k] = 0.0;
    }
    S.nsteps_done = 0;
}

// ------------------------------------------------------------------ launchers

static RelaxParams relax_params(Ctx &c) {
    RelaxParams P{};
    P.U = c.U;
    P.Uf = c.Uf;
    P.Ul = c.Ul;
    P.dh = c.dh;
    P.dl = c.dl;
    P.e_dhf = c.e_dhf;
    P.wJf = c.g_wJ_f;
    P.wJl = c.g_wJ_lo;
    P.d = c.d;
    P.e_dh = c.e_dh;
    P.wJ = c.g_wJ;
    P.chunk_inst = c.g_chunk_inst;
    P.chunk_e0 = c.g_chunk_e0;
    P.chunk_e1 = c.g_chunk_e1;
    P.inst_chunk0 = c.g_inst_chunk0;
    P.inst_nchunks = c.g_inst_nchunks;
    P.scal = c.g_scal;
    P.partials = c.g_partials;
    P.counters = c.g_counters;
    P.flags = c.g_flags;
    P.rec = nullptr;
    P.mlp = c.g_mlp;
    P.n_inst = c.n_inst;
    P.NE = (size_t)c.n_elem;
    P.gamma_gas = c.gamma_gas;
    P.max_it = c.opt.newton_max_it;
    P.guess = c.opt.guess;
    P.target = c.opt.target;
    P.relax = c.opt.relaxation;
    P.mixed = c.opt.precision == PERRK_MIXED ? 1 : 0;
    P.tol_r = c.opt.newton_tol_r;
    P.tol_g = c.opt.newton_tol_g;
    P.solver = c.opt.solver;
    P.br_lo = c.opt.bracket_lo;
    P.br_hi = c.opt.bracket_hi;
    P.dftab = (const float4 *)c.g_dftab;
    P.K.ln2 = df{c.df_consts[0], c.df_consts[1]};
    P.K.gm1 = df{c.df_consts[4], c.df_consts[5]};
    P.K.gam = df{c.df_consts[6], c.df_consts[7]};
    return P;
}

#define PERRK_RELAX_DISPATCH(NAME, KERNEL, TPL)                                                  \
    static void NAME(Ctx &c, const RelaxParams &P, cudaStream_t st, int threads) {                 \
        const int nb = (int)c.chunk_inst.size();                                                    \
        const bool df = c.opt.precision == PERRK_MIXED;                                             \
        if (c.equation == PERRK_BURGERS_1D) {                                                       \
            if (df) KERNEL<1, EQ_BURGERS TPL(true)><<<nb, threads, 0, st>>>(P);                    \
            else KERNEL<1, EQ_BURGERS TPL(false)><<<nb, threads, 0, st>>>(P);                      \
        } else if (c.dim == 1) {                                                                    \
            if (df) KERNEL<1, EQ_EULER TPL(true)><<<nb, threads, 0, st>>>(P);                      \
            else KERNEL<1, EQ_EULER TPL(false)><<<nb, threads, 0, st>>>(P);                        \
        } else if (c.dim == 2) {                                                                    \
            if (df) KERNEL<2, EQ_EULER TPL(true)><<<nb, threads, 0, st>>>(P);                      \
            else KERNEL<2, EQ_EULER TPL(false)><<<nb, threads, 0, st>>>(P);                        \
        } else {                                                                                    \
            if (df) KERNEL<3, EQ_EULER TPL(true)><<<nb, threads, 0, st>>>(P);                      \
            else KERNEL<3, EQ_EULER TPL(false)><<<nb, threads, 0, st>>>(P);                        \
        }                                                                                           \
    }
#define PERRK_WITH_DF(x) , x
#define PERRK_NO_DF(x)
PERRK_RELAX_DISPATCH(run_init, k_relax_init, PERRK_NO_DF)
PERRK_RELAX_DISPATCH(run_pass, k_newton_pass, PERRK_WITH_DF)
PERRK_RELAX_DISPATCH(run_update, k_update, PERRK_WITH_DF)
PERRK_RELAX_DISPATCH(run_entropy, k_entropy, PERRK_WITH_DF)
#undef PERRK_RELAX_DISPATCH

__global__ void k_df_log(const float4 *tab, const float *kc, const double *x, double *y, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    DfConst K;
    K.ln2 = df{kc[0], kc[1]};
    y[i] = df_to(df_log(df_from(x[i]), tab, K));
}

perrk_status launch_df_log(const float *tab, const float *consts, const double *x, double *y, int n, void *stream) {
    if (n == 0) return PERRK_OK;
    k_df_log<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>((const float4 *)tab, consts, x, y, n);
    return cuda_check((int)cudaGetLastError(), "df_log launch");
}

perrk_status launch_relax_init(Ctx &c, void *stream) {
    RelaxParams P = relax_params(c);
    if (c.n_inst >= c.sm_count && c.sm_count > 0)
        k_relax_init_inst<<<c.n_inst, 256, 0, (cudaStream_t)stream>>>(P);
    else
        run_init(c, P, (cudaStream_t)stream, 256);
    return cuda_check((int)cudaGetLastError(), "relax_init launch");
}

perrk_status launch_newton_pass(Ctx &c, void *stream) {
    RelaxParams P = relax_params(c);
    run_pass(c, P, (cudaStream_t)stream, c.relax_threads);
    return cuda_check((int)cudaGetLastError(), "newton_pass launch");
}

perrk_status launch_update(Ctx &c, int rec_slot, void *stream) {
    RelaxParams P = relax_params(c);
    P.rec = c.g_records;
    P.rec_slot = rec_slot;
    P.rec_cap = c.rec_cap;
    run_update(c, P, (cudaStream_t)stream, c.relax_threads);
    return cuda_check((int)cudaGetLastError(), "update launch");
}

perrk_status launch_entropy(Ctx &c, int query, void *stream) {
    RelaxParams P = relax_params(c);
    P.query = query;
    P.split = (query == 2 && c.Uf) ? 1 : 0;
    if (query == 2) P.query = 0;
    run_entropy(c, P, (cudaStream_t)stream, c.relax_threads);
    return cuda_check((int)cudaGetLastError(), "entropy launch");
}

perrk_status launch_entropy_set(Ctx &c, void *stream) { return launch_entropy(c, 0, stream); }
perrk_status launch_split_entropy_set(Ctx &c, void *stream) { return launch_entropy(c, 2, stream); }

}  // namespace perrk
