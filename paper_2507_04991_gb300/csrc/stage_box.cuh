// Mixed-form P-ERK stage kernel for axis-aligned box elements (2D and 3D
// Euler): the same computation as k_stage<DIM, EQ_EULER, float, false, EPB>
// (stage row, flux differencing with Ranocha's two-point flux, EC/ES surface
// flux and lift, b-stage epilogue; Sec. 2.1-2.2 and Sec. 3 of the paper), laid
// out for fewer instructions per node:
//
//  * shared-memory records are float4: a node's primitives (rho, v, p, beta,
//    log rho, log beta) are two float4, its state one float4 (+1 float in 3D),
//    a two-point or face flux one float4 (+1 float in 3D);
//  * the work lists of a node (the node pairs whose symmetric flux its
//    thread evaluates, the pair fluxes and D entries that it accumulates, its
//    face slots) depend only on the node and are built once per CTA into a
//    shared table;
//  * every face and line direction runs the same instruction stream (the
//    axis normal as a full vector), the log means select instead of branch,
//    and the end-node diagonal term is folded into the lift (2 D_NN = 1/w_N);
//  * optionally (PIPE, an autotuned choice) the per-node global data of the
//    next element group (own U_n, K_1, K_{i-1}, at b-stages d and omega J;
//    the neighbour face nodes' U_n, K_1, K_{i-1}) is copied into shared
//    memory with cp.async while the current group computes its fluxes (the
//    staging columns are thread-private and free once the stage rows are
//    formed), so the loads' latency overlaps the flux arithmetic.
#pragma once

#include "dfloat.cuh"
#include "stage.cuh"

namespace perrk {

template <int DIM>
struct BoxShape {
    static constexpr int NP = ipow4(DIM);
    static constexpr int NF = 2 * DIM;
    static constexpr int NFP = ipow4(DIM - 1);
    static constexpr int V = DIM + 2;
    static constexpr int NPAIR = DIM * ipow4(DIM - 1) * 6;   // node pairs (a < b) on all reference lines
    static constexpr int PPT = (NPAIR + NP - 1) / NP;         // pairs per thread
    static constexpr int NSF = NF * NFP;                      // face nodes of an element
    static constexpr int FPT = (NSF + NP - 1) / NP;           // face nodes per thread
    static constexpr int X = DIM == 3 ? 1 : 0;                // 3D: fifth component beside a float4
};

// Face slot that thread q takes in face iteration t (or -1): iterations
// 0 .. FPT - 2 take slot q + NP t; a partial last iteration (3D: 96 face
// slots over 64 threads) goes to the upper threads, so that it does not fall
// on the same warps as the partial last iteration of node pairs (pairs
// q + NP t go to the lower threads).
template <int DIM>
__host__ __device__ constexpr int box_face_slot(int q, int t) {
    using B = BoxShape<DIM>;
    return (B::NSF % B::NP == 0 || t < B::FPT - 1) ? q + B::NP * t
                                                   : (q >= B::FPT * B::NP - B::NSF ? q + B::NSF - B::NP : -1);
}

// primitives <-> two float4: 2D (rho, v0, v1, p) (beta, lrho, lbeta, -);
// 3D (rho, v0, v1, v2) (p, beta, lrho, lbeta)
// Shared-memory slots.  A warp's 16-byte loads are served eight threads at a
// time, without conflict when the eight addresses fall in distinct 16-byte
// bank groups (address / 16 mod 8) or coincide.  2D: the node and pair-flux
// slots below are permutations found by exhaustive local search over the
// kernel's access pattern (each quarter warp is a row pair of one element):
// every float4 access of the primitives, states and pair fluxes is then
// conflict-free.  3D: the permutations below.
constexpr unsigned long long kNodeSlot2 = 0x71a86c5320f9dbe4ull;   // 4 bits per node
// pair slots: 8 bits per pair, eight pairs per word
constexpr unsigned long long kPairSlot2_0 = 0x0c221b2916002d07ull;
constexpr unsigned long long kPairSlot2_1 = 0x120b2521042f1026ull;
constexpr unsigned long long kPairSlot2_2 = 0x27242b2e202a0d19ull;
constexpr unsigned long long kPairSlot2_3 = 0x281c0215011e230full;
constexpr unsigned long long kPairSlot2_4 = 0x0e091d1803141f1aull;
constexpr unsigned long long kPairSlot2_5 = 0x06080a172c110513ull;   // 8 bits per pair

// 3D: permutations from the same search (quarter-warp conflicts within 2% and
// 9% of the minimum; an XOR swizzle and the identity were 22% and 52% above)
constexpr unsigned char kNodeSlot3[64] = {
    3, 48, 12, 6, 9, 21, 26, 55, 38, 59, 33, 37, 52, 7, 40, 42, 18, 62, 29, 51, 31, 44, 49, 0,
    24, 58, 47, 36, 13, 46, 35, 57, 61, 23, 41, 50, 14, 32, 19, 20, 4, 53, 22, 17, 43, 34, 15, 8,
    16, 11, 28, 54, 1, 2, 45, 39, 63, 56, 10, 27, 60, 25, 30, 5,
};
constexpr unsigned short kPairSlot3[288] = {
    114, 275, 205, 176, 249, 7, 206, 252, 208, 101, 278, 259, 119, 233, 66, 284, 231, 160, 157, 59, 228, 178, 134, 73,
    182, 27, 236, 192, 185, 106, 247, 69, 88, 204, 110, 39, 57, 269, 42, 283, 255, 45, 235, 164, 232, 210, 238, 177,
    22, 122, 17, 195, 191, 212, 112, 37, 187, 145, 32, 246, 74, 229, 287, 276, 131, 133, 6, 281, 36, 151, 138, 272,
    211, 128, 223, 50, 60, 214, 189, 65, 10, 87, 261, 115, 188, 262, 40, 81, 44, 41, 250, 5, 179, 48, 95, 190,
    70, 171, 56, 245, 143, 153, 240, 241, 130, 146, 270, 136, 125, 23, 253, 116, 163, 58, 227, 222, 108, 264, 89, 230,
    82, 277, 9, 244, 126, 167, 168, 219, 172, 271, 197, 194, 140, 62, 175, 104, 251, 165, 221, 242, 8, 97, 258, 28,
    19, 256, 201, 20, 279, 54, 285, 34, 76, 193, 24, 135, 266, 102, 237, 67, 86, 68, 96, 103, 11, 149, 18, 137,
    220, 121, 218, 38, 93, 55, 216, 35, 158, 26, 120, 129, 267, 109, 12, 15, 107, 170, 141, 72, 71, 180, 265, 46,
    29, 91, 209, 132, 47, 234, 152, 78, 53, 203, 90, 4, 94, 273, 111, 248, 99, 33, 25, 100, 243, 183, 142, 215,
    84, 169, 254, 162, 184, 173, 263, 75, 156, 30, 213, 43, 154, 127, 64, 49, 260, 16, 51, 31, 282, 117, 1, 166,
    198, 217, 200, 21, 2, 124, 147, 199, 3, 80, 159, 85, 161, 196, 186, 286, 150, 79, 224, 155, 52, 98, 61, 257,
    207, 226, 113, 139, 148, 118, 77, 280, 63, 105, 83, 144, 268, 13, 14, 92, 225, 274, 202, 174, 181, 239, 0, 123,
};

// slot maps, used by the host-side table builder
template <int DIM>
inline int node_slot(int n) {
    if constexpr (DIM == 2) return (int)((kNodeSlot2 >> (4 * n)) & 15u);
    else return kNodeSlot3[n];
}
template <int DIM>
inline int pair_slot(int pp) {
    if constexpr (DIM == 3) {
        return kPairSlot3[pp];
    } else {
        const int w = pp >> 3;
        unsigned long long x = kPairSlot2_0;
        x = (w == 1) ? kPairSlot2_1 : x;
        x = (w == 2) ? kPairSlot2_2 : x;
        x = (w == 3) ? kPairSlot2_3 : x;
        x = (w == 4) ? kPairSlot2_4 : x;
        x = (w == 5) ? kPairSlot2_5 : x;
        return (int)((x >> (8 * (pp & 7))) & 255u);
    }
}

template <int DIM>
__device__ __forceinline__ void prim_store(float4 *pa, float4 *pb, const Prim<float, DIM> &P) {
    if constexpr (DIM == 2) {
        *pa = make_float4(P.rho, P.v[0], P.v[1], P.p);
        *pb = make_float4(P.beta, P.lrho, P.lbeta, 0.0f);
    } else {
        *pa = make_float4(P.rho, P.v[0], P.v[1], P.v[2]);
        *pb = make_float4(P.p, P.beta, P.lrho, P.lbeta);
    }
}

template <int DIM>
__device__ __forceinline__ Prim<float, DIM> prim_load(const float4 *pa, const float4 *pb) {
    Prim<float, DIM> P;
    const float4 a = *pa, b = *pb;
    P.rho = a.x;
    P.v[0] = a.y;
    P.v[1] = a.z;
    if constexpr (DIM == 2) {
        P.p = a.w;
        P.beta = b.x;
        P.lrho = b.y;
        P.lbeta = b.z;
    } else {
        P.v[2] = a.w;
        P.p = b.x;
        P.beta = b.y;
        P.lrho = b.z;
        P.lbeta = b.w;
    }
    return P;
}

template <int DIM>
__device__ __forceinline__ Prim<float, DIM> prim_select(bool first, const Prim<float, DIM> &a, const Prim<float, DIM> &b) {
    Prim<float, DIM> r;
    r.rho = first ? a.rho : b.rho;
#pragma unroll
    for (int d = 0; d < DIM; ++d) r.v[d] = first ? a.v[d] : b.v[d];
    r.p = first ? a.p : b.p;
    r.beta = first ? a.beta : b.beta;
    r.lrho = first ? a.lrho : b.lrho;
    r.lbeta = first ? a.lbeta : b.lbeta;
    return r;
}

template <int V>
__device__ __forceinline__ void vec_store(float4 *a, float *x, const float *f) {
    *a = make_float4(f[0], f[1], f[2], f[3]);
    if constexpr (V == 5) *x = f[4];
}

template <int V>
__device__ __forceinline__ void vec_load(const float4 *a, const float *x, float *f) {
    const float4 t = *a;
    f[0] = t.x;
    f[1] = t.y;
    f[2] = t.z;
    f[3] = t.w;
    if constexpr (V == 5) f[4] = *x;
}

// 4-byte asynchronous global -> shared copy (cached in L1), its commit and wait
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Node work table (shared, one row per node q of the element):
//   pd[t]    pair t of this thread: slot(qa) | slot(qb) << 8 | k << 16
//   pw[t]    pair-flux slot that pair t is written to
//   aslot[k] three 10-bit pair-flux slots accumulated by node q along k
//   fslot[k] face slot of node q along k, or -1
//   sfd[t]   face slot t of this thread: face | slot(own face node) << 8 | neighbour's node << 16
//   qsl      slot of node q
//   acoef    2 D_{q m} for the three other nodes m of each line
template <int DIM>
struct NodeTable {
    int pd[BoxShape<DIM>::PPT];
    int pw[BoxShape<DIM>::PPT];
    int aslot[DIM];
    int fslot[DIM];
    int sfd[BoxShape<DIM>::FPT];
    int qsl;
    float acoef[DIM][3];
};

template <int DIM>
inline void build_node_table(NodeTable<DIM> &T, int q, const float *Df) {   // host
    using B = BoxShape<DIM>;
    constexpr int NP = B::NP, NFP = B::NFP, LPD = B::NPAIR / DIM;
    const int id[3] = {q & 3, (q >> 2) & 3, (q >> 4) & 3};
#pragma unroll
    for (int t = 0; t < B::PPT; ++t) {
        const int pp = q + NP * t;
        const int k = pp / LPD, rem = pp % LPD, line = rem / 6, lp = rem % 6;
        const int a = lp < 3 ? 0 : (lp < 5 ? 1 : 2);
        const int b = lp < 3 ? lp + 1 : (lp < 5 ? lp - 1 : 3);
        int qa, qb;
        if constexpr (DIM == 2) {
            qa = k == 0 ? a + 4 * line : line + 4 * a;
            qb = k == 0 ? b + 4 * line : line + 4 * b;
        } else {
            const int l0 = line & 3, l1 = line >> 2;
            qa = k == 0 ? a + 4 * l0 + 16 * l1 : (k == 1 ? l0 + 4 * a + 16 * l1 : l0 + 4 * l1 + 16 * a);
            qb = k == 0 ? b + 4 * l0 + 16 * l1 : (k == 1 ? l0 + 4 * b + 16 * l1 : l0 + 4 * l1 + 16 * b);
        }
        T.pd[t] = node_slot<DIM>(qa) | (node_slot<DIM>(qb) << 8) | (k << 16);
        T.pw[t] = pair_slot<DIM>(pp < B::NPAIR ? pp : 0);
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
        const int ik = id[k];
        const int line = DIM == 2 ? (k == 0 ? id[1] : id[0])
                                  : (k == 0 ? id[1] + 4 * id[2] : (k == 1 ? id[0] + 4 * id[2] : id[0] + 4 * id[1]));
        int sl = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int m = c < ik ? c : c + 1;   // the c-th node of the line other than q
            const int lo = m < ik ? m : ik, hi = m < ik ? ik : m;
            const int lp = lo == 0 ? hi - 1 : (lo == 1 ? hi + 1 : 5);
            sl |= pair_slot<DIM>(k * LPD + line * 6 + lp) << (10 * c);
            T.acoef[k][c] = 2.0f * Df[ik * 4 + m];
        }
        T.aslot[k] = sl;
        T.fslot[k] = (ik == 0 || ik == 3) ? (2 * k + (ik == 3 ? 1 : 0)) * NFP + face_pos<DIM>(q, k) : -1;
    }
#pragma unroll
    for (int t = 0; t < B::FPT; ++t) {
        const int sl = box_face_slot<DIM>(q, t);
        if (sl < 0) {
            T.sfd[t] = 0;
            continue;
        }
        const int f = sl / NFP, kk = sl % NFP;
        T.sfd[t] = f | (node_slot<DIM>(face_node_dev<DIM>(f, kk)) << 8) | (face_node_dev<DIM>(f ^ 1, kk) << 16);
    }
    T.qsl = node_slot<DIM>(q);
}

// FP32 stage row U_n + a1 K_1 + asub K_{i-1} at one node, from global memory
template <int V>
__device__ __forceinline__ void stage_row_f(const StageParams &P, size_t NPtot, size_t idx, int g, float *u) {
    if (P.stage1) {
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = __ldg(P.Uf + v * NPtot + idx);
        return;
    }
    const float2 c = __ldg(reinterpret_cast<const float2 *>(P.coef_f + g));   // (a1, asub)
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float k1 = __ldg(P.K1f + v * NPtot + idx);
        const float kp = (c.y != 0.0f) ? __ldg(P.Kprevf + v * NPtot + idx) : 0.0f;
        u[v] = fmaf(c.y, kp, fmaf(c.x, k1, __ldg(P.Uf + v * NPtot + idx)));
    }
}

template <int DIM, int EPB, bool PIPE>
struct BoxSmem {
    using B = BoxShape<DIM>;
    static constexpr int NP = B::NP, V = B::V, X = B::X;
    static constexpr int NOWN = PIPE ? 5 * V + 1 : 1;   // staging: own [U | K_1 | K_{i-1} | d hi | d lo] x V, omega J
    static constexpr int NNB = PIPE ? 3 * V : 1;        // staging: neighbour face node [U | K_1 | K_{i-1}] x V
    float4 pa[EPB][NP], pb[EPB][NP];   // primitives, node n at node_slot(n)
    float4 u[EPB][NP];                 // state, node n at node_slot(n)
    // (pair fluxes: pair pp at pair_slot(pp))
    float u5[EPB][X ? NP : 1];
    float4 pf[EPB][B::NPAIR];
    float pf5[EPB][X ? B::NPAIR : 1];
    float4 sf[EPB][B::NSF];
    float sf5[EPB][X ? B::NSF : 1];
    float red[EPB][NP > 32 ? NP / 32 : 1];
    NodeTable<DIM> tab[NP];
    float st_own[NOWN][PIPE ? EPB * NP : 1];
    float st_nb[B::FPT][NNB][PIPE ? EPB * NP : 1];
};

template <int DIM, int EPB, bool PIPE>
constexpr size_t stage_box_smem_bytes() {
    return sizeof(BoxSmem<DIM, EPB, PIPE>);
}

// Register budget per thread: 48 in 2D without staging (10 CTAs of 128
// threads per SM; at 40 the kernel spills, A/B 5% slower per step), ~72 with
// staging, 80 in 3D (A/B on TGV 64^3: 3% faster per step than unbounded).
template <int DIM, int EPB, bool PIPE>
constexpr int box_min_blocks() {
    return DIM == 2 ? ((PIPE ? 896 : 1280) / (EPB * ipow4(DIM)) > 0 ? (PIPE ? 896 : 1280) / (EPB * ipow4(DIM)) : 1)
                    : (EPB * ipow4(DIM) <= 128 ? 768 / (EPB * ipow4(DIM)) : 3);
}

// VISC: add the viscous divergence visc_kv (Navier-Stokes-Fourier runs); the
// inviscid instantiation carries no trace of it.  MORT: meshes with 2:1
// mortars, whose element faces on a mortar take the mortar kernel's flux (a
// separate instantiation, so that conforming meshes run without the extra
// registers it needs).
template <int DIM, int EPB, bool PIPE, bool VISC, bool MORT = false>
__global__ void __launch_bounds__(EPB * ipow4(DIM), box_min_blocks<DIM, EPB, PIPE>()) k_stage_box(const StageParams P) {
    using B = BoxShape<DIM>;
    constexpr int NP = B::NP, NF = B::NF, V = B::V, NPAIR = B::NPAIR, PPT = B::PPT;
    constexpr int NSF = B::NSF, FPT = B::FPT, X = B::X;
    __shared__ __align__(16) BoxSmem<DIM, EPB, PIPE> S;

    const int el = threadIdx.x / NP, q = threadIdx.x % NP, tid = threadIdx.x;
    const size_t NPtot = P.NE * NP;
    const float gm1 = P.gm1_f, inv_gm1 = P.inv_gm1_f, gam = P.gam_f, inv_w = P.inv_w_f;
    // the table is built once on the host (build_node_table) and copied per CTA
    if (el == 0) S.tab[q] = reinterpret_cast<const NodeTable<DIM> *>(P.box_tab)[q];
    __syncthreads();
    const NodeTable<DIM> &T = S.tab[q];

    uint32_t bad = 0;
    const int ngroups = (P.n_active + EPB - 1) / EPB;
    const bool need_k = !P.stage1;

    // element and neighbour ids of a group (clamped past the active prefix)
    auto group_ids = [&](int grp, int &e_out, int (&nb_out)[FPT]) {
        const int slot = grp * EPB + el;
        e_out = __ldg(P.elist + (slot < P.n_active ? slot : P.n_active - 1));
#pragma unroll
        for (int t = 0; t < FPT; ++t)
            nb_out[t] = (box_face_slot<DIM>(q, t) >= 0) ? __ldg(P.nbr + (size_t)e_out * NF + (T.sfd[t] & 0xff)) : e_out;
    };
    // PIPE: asynchronous copies of a group's per-node data into the staging columns
    auto issue = [&](int e_i, const int (&nb_i)[FPT]) {
        if constexpr (PIPE) {
            const size_t ix = (size_t)e_i * NP + q;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                cp_async4(&S.st_own[v][tid], P.Uf + v * NPtot + ix);
                if (need_k) {
                    cp_async4(&S.st_own[V + v][tid], P.K1f + v * NPtot + ix);
                    cp_async4(&S.st_own[2 * V + v][tid], P.Kprevf + v * NPtot + ix);
                }
                if (P.d_read) {
                    cp_async4(&S.st_own[3 * V + v][tid], P.dh + v * NPtot + ix);
                    cp_async4(&S.st_own[4 * V + v][tid], P.dl + v * NPtot + ix);
                }
            }
            if (P.do_b) cp_async4(&S.st_own[5 * V][tid], P.wJ_f + ix);
#pragma unroll
            for (int t = 0; t < FPT; ++t) {
                if (box_face_slot<DIM>(q, t) >= 0) {
                    const size_t jn = (size_t)nb_i[t] * NP + (T.sfd[t] >> 16);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        cp_async4(&S.st_nb[t][v][tid], P.Uf + v * NPtot + jn);
                        if (need_k) {
                            cp_async4(&S.st_nb[t][V + v][tid], P.K1f + v * NPtot + jn);
                            cp_async4(&S.st_nb[t][2 * V + v][tid], P.Kprevf + v * NPtot + jn);
                        }
                    }
                }
            }
            cp_async_commit();
        }
    };
    // PIPE: stage row from staging columns (rows 0..V-1: U_n, V..: K_1, 2V..: K_{i-1})
    auto row_staged = [&](const float (*col)[PIPE ? EPB * NP : 1], int g_i, float *u) {
        if (!need_k) {
#pragma unroll
            for (int v = 0; v < V; ++v) u[v] = col[v][PIPE ? tid : 0];
            return;
        }
        const float2 c = __ldg(reinterpret_cast<const float2 *>(P.coef_f + g_i));   // (a1, asub)
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const float kp = (c.y != 0.0f) ? col[2 * V + v][PIPE ? tid : 0] : 0.0f;
            u[v] = fmaf(c.y, kp, fmaf(c.x, col[V + v][PIPE ? tid : 0], col[v][PIPE ? tid : 0]));
        }
    };

    int e_c = 0, nb_c[FPT];
    if ((int)blockIdx.x < ngroups) {
        group_ids(blockIdx.x, e_c, nb_c);
        issue(e_c, nb_c);
    }
    for (int grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        const int slot = grp * EPB + el;
        const bool valid = slot < P.n_active;
        const int e = e_c;
        const size_t idx = (size_t)e * NP + q;
        const int g = __ldg(P.gp + e);
        const int gn = grp + gridDim.x;
        int e_n = e_c, nb_n[FPT];
#pragma unroll
        for (int t = 0; t < FPT; ++t) nb_n[t] = nb_c[t];

        // ---- A: stage rows of the own node and of the neighbour face nodes
        float un[FPT][V], u[V], dprev[2 * V], wj = 0.0f;
#pragma unroll
        for (int v = 0; v < 2 * V; ++v) dprev[v] = 0.0f;
        if constexpr (PIPE) {
            int gnb[FPT];
#pragma unroll
            for (int t = 0; t < FPT; ++t) gnb[t] = __ldg(P.gp + nb_c[t]);
            if (gn < ngroups) group_ids(gn, e_n, nb_n);   // ids of the next group: loads overlap the wait
            cp_async_wait_all();                          // staging columns are thread-private: no barrier
#pragma unroll
            for (int t = 0; t < FPT; ++t)
                if (box_face_slot<DIM>(q, t) >= 0) row_staged(S.st_nb[t], gnb[t], un[t]);
            row_staged(S.st_own, g, u);
            if (P.d_read) {
#pragma unroll
                for (int v = 0; v < 2 * V; ++v) dprev[v] = S.st_own[3 * V + v][tid];
            }
            if (P.do_b) wj = S.st_own[5 * V][tid];
        } else {
#pragma unroll
            for (int t = 0; t < FPT; ++t)
                if (box_face_slot<DIM>(q, t) >= 0)
                    stage_row_f<V>(P, NPtot, (size_t)nb_c[t] * NP + (T.sfd[t] >> 16), __ldg(P.gp + nb_c[t]), un[t]);
            stage_row_f<V>(P, NPtot, idx, g, u);
            if (gn < ngroups) group_ids(gn, e_n, nb_n);
        }
        const float4 geo = __ldg(reinterpret_cast<const float4 *>(P.g_elem_f + (size_t)e * 8));   // Ja_kk, invJ
        const float jak[3] = {geo.x, geo.y, geo.z};
        const float invJ = geo.w;
        const Prim<float, DIM> pr = make_prim<float, DIM>(u, gm1, bad);
        const int qsl = T.qsl;
        prim_store<DIM>(&S.pa[el][qsl], &S.pb[el][qsl], pr);
        vec_store<V>(&S.u[el][qsl], &S.u5[el][X ? qsl : 0], u);
        __syncthreads();
        if constexpr (PIPE) {
            if (gn < ngroups) issue(e_n, nb_n);   // the staging columns are free
        }
        e_c = e_n;
#pragma unroll
        for (int t = 0; t < FPT; ++t) nb_c[t] = nb_n[t];

        // ---- B: interface fluxes at this element's face nodes
#pragma unroll
        for (int t = 0; t < FPT; ++t) {
            const int sl = box_face_slot<DIM>(q, t);
            if (sl >= 0) {
                const int sfd = T.sfd[t];
                const int f = sfd & 0xff, k = f >> 1, qs = (sfd >> 8) & 0xff;
                const int qss = qs;   // already a slot
                const Prim<float, DIM> ps = prim_load<DIM>(&S.pa[el][qss], &S.pb[el][qss]);
                float us[V];
                vec_load<V>(&S.u[el][qss], &S.u5[el][X ? qss : 0], us);
                const Prim<float, DIM> pn = make_prim<float, DIM>(un[t], gm1, bad);
                const float fnv = __ldg(P.fnorm_f + (size_t)e * NF + f);
                // canonical order f*(U_plus_side, U_minus_side): both elements of
                // the face evaluate the identical instruction sequence on the
                // identical operands (conservation to round-off)
                const bool self_plus = (f & 1);
                const Prim<float, DIM> PL = prim_select<DIM>(self_plus, ps, pn);
                const Prim<float, DIM> PR = prim_select<DIM>(self_plus, pn, ps);
                float nv[DIM], fs[V];
#pragma unroll
                for (int a = 0; a < DIM; ++a) nv[a] = (a == k) ? fnv : 0.0f;
                ranocha<float, DIM, -1>(PL, PR, nv, inv_gm1, fs);
                if (P.es) {
                    const float lam = max_speed_nn<float, DIM>(PL, PR, nv, fabsf(fnv), gam);
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const float uL = self_plus ? us[v] : un[t][v], uR = self_plus ? un[t][v] : us[v];
                        fs[v] -= 0.5f * lam * (uR - uL);
                    }
                }
                if constexpr (MORT) {
                    // a 2:1 mortar face: the mortar kernel's flux for this element face
                    const int ms = __ldg(P.face_mortar + (size_t)e * NF + f);
                    if (ms >= 0) {
#pragma unroll
                        for (int v = 0; v < V; ++v)
                            fs[v] = __ldg(static_cast<const float *>(P.mtrace) + ((size_t)ms * B::NFP + (sl % B::NFP)) * V + v);
                    }
                }
                const float sc = self_plus ? inv_w : -inv_w;
#pragma unroll
                for (int v = 0; v < V; ++v) fs[v] *= sc;
                vec_store<V>(&S.sf[el][sl], &S.sf5[el][X ? sl : 0], fs);
            }
        }

        // ---- C: symmetric two-point volume fluxes, each pair once
#pragma unroll
        for (int t = 0; t < PPT; ++t) {
            const int pp = q + NP * t;
            if (pp < NPAIR) {
                const int pd = T.pd[t];
                const int sa = pd & 0xff, sb = (pd >> 8) & 0xff;
                const Prim<float, DIM> A = prim_load<DIM>(&S.pa[el][sa], &S.pb[el][sa]);
                const Prim<float, DIM> Bq = prim_load<DIM>(&S.pa[el][sb], &S.pb[el][sb]);
                const int k = pd >> 16;
                float jk = jak[0];
#pragma unroll
                for (int a = 1; a < DIM; ++a) jk = (k == a) ? jak[a] : jk;
                float nv[DIM], F[V];
#pragma unroll
                for (int a = 0; a < DIM; ++a) nv[a] = (a == k) ? jk : 0.0f;
                ranocha<float, DIM, -1>(A, Bq, nv, inv_gm1, F);
                const int pw = T.pw[t];
                vec_store<V>(&S.pf[el][pw], &S.pf5[el][X ? pw : 0], F);
            }
        }
        __syncthreads();

        // ---- D: sum_k sum_m 2 D_qm f#(q, m) + lift at end nodes; K = -acc / J
        float acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.0f;
        // (volume terms of every direction first, then the face terms: the
        // summation order of the generic stage kernel, so that every kernel
        // variant gives bit-identical results)
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int as = T.aslot[k];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int sl = (as >> (10 * c)) & 0x3ff;
                const float cf = T.acoef[k][c];
                float F[V];
                vec_load<V>(&S.pf[el][sl], &S.pf5[el][X ? sl : 0], F);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = fmaf(cf, F[v], acc[v]);
            }
        }
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
            const int fsl = T.fslot[k];
            if (fsl >= 0) {
                float F[V];
                vec_load<V>(&S.sf[el][fsl], &S.sf5[el][X ? fsl : 0], F);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] += F[v];
            }
        }
        float Kr[V], ksum = 0.0f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if constexpr (VISC) {
                // one rounding: fma(-acc, 1/J, div f_v), as in the generic kernel
                Kr[v] = v > 0 ? fmaf(-acc[v], invJ, static_cast<const float *>(P.visc_kv)[(size_t)(v - 1) * NPtot + idx])
                              : -acc[v] * invJ;
            } else {
                Kr[v] = -acc[v] * invJ;
            }
            ksum += Kr[v];
        }
        if (!isfinite(ksum)) bad |= PERRK_FLAG_NONFINITE;
        if (valid && P.k_store) {
#pragma unroll
            for (int v = 0; v < V; ++v) P.Koutf[v * NPtot + idx] = Kr[v];
        }

        // ---- E: stages with b_i != 0 (FP32 pipe only): entropy integrand
        // <w(U_{n,i}), K_i> from the FP32 primitives, element sum by shuffles,
        // d += b_i K_i and the element's running sum as float pairs
        if (P.do_b) {
            const float4 cb = __ldg(reinterpret_cast<const float4 *>(P.coef_f + g));        // a1, asub, b_hi, b_lo
            const int4 fl = __ldg(reinterpret_cast<const int4 *>(&P.coef_f[g].has_b));     // has_b, first_b, d_final
            float wdf = 0.0f;
            if (fl.x) {
                if constexpr (!PIPE) {
                    wj = __ldg(P.wJ_f + idx);
                    if (!fl.y && !P.d_fused) {
#pragma unroll
                        for (int v = 0; v < V; ++v) {
                            dprev[v] = P.dh[v * NPtot + idx];
                            dprev[V + v] = P.dl[v * NPtot + idx];
                        }
                    }
                }
                const float Sl = (1.0f - gam) * pr.lrho - pr.lbeta;   // log p - gamma log rho
                const float ip = rcp(pr.p);
                float v2 = 0.0f, mk = 0.0f;
#pragma unroll
                for (int a = 0; a < DIM; ++a) {
                    v2 = fmaf(pr.v[a], pr.v[a], v2);
                    mk = fmaf(pr.v[a], Kr[1 + a], mk);
                }
                const float w0 = gam - Sl - gm1 * 0.5f * pr.rho * v2 * ip;
                wdf = fmaf(w0, Kr[0], gm1 * pr.rho * ip * (mk - Kr[DIM + 1])) * wj;
                if (valid && (!P.d_fused || fl.z)) {
                    const df bb{cb.z, cb.w};
                    const float4 cbm = __ldg(reinterpret_cast<const float4 *>(&P.coef_f[g].b1_hi));   // b1, bm pairs
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const size_t j = v * NPtot + idx;
                        df dn;
                        if (P.d_fused) {
                            // d = b_1 K_1 + b_m K_{S-1} + b_S K_S (the sums of the stage-by-stage form)
                            dn = df_mul_f(df{cbm.x, cbm.y}, __ldg(P.K1f + j));   // L2-resident: read by the stage row
                            dn = df_fma_f(dn, df{cbm.z, cbm.w}, __ldg(P.Kprevf + j));
                            dn = df_fma_f(dn, bb, Kr[v]);
                        } else {
                            dn = fl.y ? df_mul_f(bb, Kr[v]) : df_fma_f(df{dprev[v], dprev[V + v]}, bb, Kr[v]);
                        }
                        P.dh[j] = dn.hi;
                        P.dl[j] = dn.lo;
                    }
                }
            }
            constexpr int W = NP < 32 ? NP : 32;
#pragma unroll
            for (int off = W / 2; off > 0; off >>= 1) wdf += __shfl_xor_sync(0xffffffffu, wdf, off);
            if constexpr (NP > 32) {
                if ((q & 31) == 0) S.red[el][q >> 5] = wdf;
                __syncthreads();
                if (q == 0)
                    for (int w = 1; w < NP / 32; ++w) wdf += S.red[el][w];
            }
            if (q == 0 && valid && fl.x) {
                const df bs = df_mul_f(df{cb.z, cb.w}, wdf);
                const df en = fl.y ? bs : df_add(df{P.e_dhf[2 * e], P.e_dhf[2 * e + 1]}, bs);
                P.e_dhf[2 * e] = en.hi;
                P.e_dhf[2 * e + 1] = en.lo;
            }
        }
        __syncthreads();
    }
    if (__syncthreads_or(bad != 0)) {
        if (bad) atomicOr(P.flags, bad);
    }
}

}  // namespace perrk
