// Mixed-form P-ERK stage kernel for 2D axis-aligned box elements with its
// element data staged on chip ahead of the flux arithmetic: a persistent CTA
// with one producer warp and NCG consumer groups (one thread per node of EPB
// elements each), around a ring of NBUF staging buffers in shared memory.
//
//  * The producer warp fills buffer j % NBUF with element group j of the CTA:
//    the own elements' rows of U_n, K_1, K_{i-1} (and omega J at stages with
//    b_i != 0) by bulk asynchronous copies (cp.async.bulk, the TMA engine; one
//    64-byte row per element, variable and array), the neighbours' face
//    nodes of the same arrays by cp.async (16 bytes for a face whose nodes
//    are contiguous, 4 bytes per node otherwise), the element's geometry and
//    face normals by cp.async, and element and partition ids by plain stores.
//    Completion is tracked by one mbarrier per buffer ("full"): the bulk
//    copies' byte count (expect_tx / complete_tx), one cp.async-completion
//    arrival and one ordinary (release) arrival per producer lane.
//  * Consumer group j % NCG waits for buffer j's "full" barrier, computes the
//    stage exactly as k_stage_box does (same operations in the same order,
//    so the results are bit-identical), and releases the buffer on its
//    "empty" barrier once it no longer reads it.  Its own barriers are named
//    barriers over its threads.
//  * Every wait is bounded in time: a wait that gives up sets
//    PERRK_FLAG_TIMEOUT, and the thread leaves its loop; the producer waits
//    for its own copies in flight before it returns.
//
// The paper's stage (Sec. 2.2, eq. PartitionedRKSystem) and the DGSEM right
// -hand side with EC volume and EC/ES surface fluxes (Sec. 2.1) are those of
// k_stage_box; only where the operands come from differs.
#pragma once

#include "stage_box.cuh"

namespace perrk {

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make the initialised barriers visible to the async proxy (the bulk copies'
// complete_tx) as well as to the other threads
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

// arrival triggered when all of this thread's earlier cp.async copies are complete
__device__ __forceinline__ void mbar_arrive_cp_async(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Wait for the phase of the given parity to complete; false after limit_ns.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

// bulk asynchronous global -> shared copy (TMA engine), completion counted
// in bytes on the barrier; both addresses 16-byte aligned, size a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *smem, const void *gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(smem)),
                 "l"(gmem), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// 16-byte asynchronous copy (L2 only), both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}

__device__ __forceinline__ void named_barrier(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

// a bounded wait gives up after about one second
constexpr uint64_t kWaitLimitNs = 1000000000ull;

// ------------------------------------------------------------ shared memory

// One staging buffer: element group j's operands (2D: NP = 16, V = 4; slot
// t = el * NP + q is the thread of node q of element el, and also that
// thread's face slot: face f = q / 4, face node kk = q % 4).
template <int EPB>
struct alignas(16) WsStage {
    static constexpr int NP = 16, V = 4, NT = EPB * NP;
    float own[3 * V + 1][NT];   // rows U_n (0..V-1), K_1 (V..2V-1), K_{i-1} (2V..3V-1), omega J (3V)
    float nb[3 * V][NT];        // the neighbour's face node of each face slot, same rows
    float4 geo[EPB];            // Ja_00, Ja_11, -, 1/J (the first four box metric values)
    float4 fn[EPB];             // scaled normals of faces 0..3
    int e[EPB];                 // element ids (clamped past the active prefix)
    int gp[EPB];                // global partition of the element
    int gpn[NT];                // global partition of each face slot's neighbour
};

// A consumer group's scratch: primitives, states, pair and face fluxes (as in k_stage_box).
template <int EPB>
struct alignas(16) WsGroup {
    float4 pa[EPB][16], pb[EPB][16], u[EPB][16];
    float4 pf[EPB][BoxShape<2>::NPAIR];
    float4 sf[EPB][BoxShape<2>::NSF];
    int ok;                     // the group's leader's verdict on the last wait
};

template <int EPB, int NCG, int NBUF>
struct alignas(128) WsSmem {
    WsStage<EPB> st[NBUF];
    WsGroup<EPB> grp[NCG];
    NodeTable<2> tab[16];
    uint64_t full[NBUF], empty[NBUF];
};

template <int EPB, int NCG, int NBUF>
constexpr size_t stage_ws_smem_bytes() {
    return sizeof(WsSmem<EPB, NCG, NBUF>);
}

template <int EPB, int NCG>
constexpr int ws_threads() {
    return NCG * EPB * 16 + 32;
}

// Stage row U_n + a1 K_1 + asub K_{i-1} from staging rows (the operations of
// row_staged in k_stage_box).
template <int NT>
__device__ __forceinline__ void ws_row(const float (*col)[NT], int t, int g, const StageParams &P, bool need_k,
                                       float *u) {
    constexpr int V = 4;
    if (!need_k) {
#pragma unroll
        for (int v = 0; v < V; ++v) u[v] = col[v][t];
        return;
    }
    const float2 c = __ldg(reinterpret_cast<const float2 *>(P.coef_f + g));   // (a1, asub)
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float kp = (c.y != 0.0f) ? col[2 * V + v][t] : 0.0f;
        u[v] = fmaf(c.y, kp, fmaf(c.x, col[V + v][t], col[v][t]));
    }
}

// ---------------------------------------------------------------- producer

// Fill staging buffers with the CTA's element groups blockIdx.x + j gridDim.x,
// j = 0, 1, ...; returns false if a wait for a free buffer gave up.  The ids
// of group j + 1 (element, neighbours and their partitions) are loaded while
// group j's copies are issued and buffer j + 1 is awaited, so the chain of
// dependent index loads overlaps the ring.  OWN_BULK: the own rows by 64-byte
// bulk copies (TMA); otherwise by 16-byte cp.async (four per row).
template <int EPB, int NCG, int NBUF, bool OWN_BULK>
__device__ __forceinline__ bool ws_produce(const StageParams &P, WsSmem<EPB, NCG, NBUF> &S, int lane, int ngroups) {
    constexpr int NP = 16, NF = 4, V = 4, NFP = 4;
    const size_t NPtot = P.NE * NP;
    const bool need_k = !P.stage1;
    const int narr = need_k ? 3 : 1;
    const int nrow = narr * V + (P.do_b ? 1 : 0);          // own rows per element
    const uint32_t tx = OWN_BULK ? (uint32_t)(EPB * nrow * NP * sizeof(float)) : 0u;
    if (P.ws_stall) return true;   // test hook: no fill, so the consumers' waits run out
    // per-lane ids of one group: lane < EPB holds its element; lane t < EPB NF
    // the neighbour across face t % NF of element t / NF and its partition
    const int f_l = lane % NF, el_l = lane / NF;
    auto load_ids = [&](int grp, int &e, int &gpe, int &nb, int &gn) {
        e = 0;
        gpe = 0;
        nb = 0;
        gn = 0;
        if (grp >= ngroups) return;
        if (lane < EPB) {
            const int slot = grp * EPB + lane;
            e = __ldg(P.elist + (slot < P.n_active ? slot : P.n_active - 1));
            gpe = __ldg(P.gp + e);
        }
        const int eo = __shfl_sync(0xffffffffu, e, el_l < EPB ? el_l : 0);
        if (lane < EPB * NF) {
            nb = __ldg(P.nbr + (size_t)eo * NF + f_l);
            gn = __ldg(P.gp + nb);
        }
    };
    int e_c, gp_c, nb_c, gn_c;
    load_ids(blockIdx.x, e_c, gp_c, nb_c, gn_c);
    bool ok = true;
    int filled = 0;
    for (int j = 0;; ++j) {
        const int grp = blockIdx.x + j * gridDim.x;
        if (grp >= ngroups) break;
        const int b = j % NBUF, use = j / NBUF;
        if (use > 0) {
            // lane 0 decides, so that the warp stays converged; the other
            // lanes then find the phase complete at once (acquire)
            int w = lane == 0 ? (int)mbar_wait_bounded(&S.empty[b], (use - 1) & 1, kWaitLimitNs) : 0;
            w = __shfl_sync(0xffffffffu, w, 0);
            if (!w) {
                ok = false;
                break;
            }
            mbar_wait_bounded(&S.empty[b], (use - 1) & 1, kWaitLimitNs);
        }
        WsStage<EPB> &T = S.st[b];
        if (lane < EPB) {
            T.e[lane] = e_c;
            T.gp[lane] = gp_c;
            cp_async16(&T.geo[lane], P.g_elem_f + (size_t)e_c * 8);
            cp_async16(&T.fn[lane], P.fnorm_f + (size_t)e_c * NF);
        }
        if (OWN_BULK && lane == 0) mbar_expect_tx(&S.full[b], tx);
        __syncwarp();
        // own rows: element el's row r (array r / V, variable r % V; omega J last)
        if constexpr (OWN_BULK) {
            for (int t = lane; t < EPB * nrow; t += 32) {
                const int el = t / nrow, r = t % nrow;
                const size_t e = (size_t)T.e[el];
                const float *src = r < narr * V ? (r / V == 0 ? P.Uf : (r / V == 1 ? P.K1f : P.Kprevf)) + (r % V) * NPtot + e * NP
                                                : P.wJ_f + e * NP;
                float *dst = r < narr * V ? &T.own[r][el * NP] : &T.own[3 * V][el * NP];
                bulk_g2s(dst, src, NP * sizeof(float), &S.full[b]);
            }
        } else {
            // four 16-byte pieces per row, consecutive lanes on consecutive pieces
            for (int t = lane; t < EPB * nrow * 4; t += 32) {
                const int piece = t & 3, row = t >> 2;
                const int el = row / nrow, r = row % nrow;
                const size_t e = (size_t)T.e[el];
                const float *src = r < narr * V ? (r / V == 0 ? P.Uf : (r / V == 1 ? P.K1f : P.Kprevf)) + (r % V) * NPtot + e * NP
                                                : P.wJ_f + e * NP;
                float *dst = r < narr * V ? &T.own[r][el * NP] : &T.own[3 * V][el * NP];
                cp_async16(dst + 4 * piece, src + 4 * piece);
            }
        }
        // neighbour face nodes: lane t < EPB NF takes face t % NF of element t / NF
        if (lane < EPB * NF) {
            const int s0 = el_l * NP + f_l * NFP;   // the face's four slots
#pragma unroll
            for (int kk = 0; kk < NFP; ++kk) T.gpn[s0 + kk] = gn_c;
            for (int arr = 0; arr < narr; ++arr) {
                const float *base = arr == 0 ? P.Uf : (arr == 1 ? P.K1f : P.Kprevf);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float *src = base + v * NPtot + (size_t)nb_c * NP;
                    float *dst = &T.nb[arr * V + v][s0];
                    if (f_l >= 2) {
                        // eta faces: the neighbour's four face nodes are contiguous and 16-byte aligned
                        cp_async16(dst, src + face_node_dev<2>(f_l ^ 1, 0));
                    } else {
#pragma unroll
                        for (int kk = 0; kk < NFP; ++kk) cp_async4(dst + kk, src + face_node_dev<2>(f_l ^ 1, kk));
                    }
                }
            }
        }
        mbar_arrive_cp_async(&S.full[b]);   // when this lane's copies have landed
        mbar_arrive(&S.full[b]);            // this lane's plain stores (release)
        ++filled;
        load_ids(grp + gridDim.x, e_c, gp_c, nb_c, gn_c);   // the next group's ids, in flight during the next wait
    }
    cp_async_wait_all();
    // no bulk copy may still be in flight when the CTA's threads are gone:
    // wait (bounded) for the last fill of every buffer
    if (lane == 0) {
        const int j0 = filled > NBUF ? filled - NBUF : 0;
        for (int jj = j0; jj < filled; ++jj) mbar_wait_bounded(&S.full[jj % NBUF], (jj / NBUF) & 1, kWaitLimitNs);
    }
    __syncwarp();
    return ok;
}

// ---------------------------------------------------------------- kernel

template <int EPB, int NCG, int NBUF, bool VISC, bool OWN_BULK>
__global__ void __launch_bounds__(ws_threads<EPB, NCG>()) k_stage_ws(const StageParams P) {
    using B = BoxShape<2>;
    constexpr int NP = 16, NF = 4, V = 4, NPAIR = B::NPAIR, PPT = B::PPT, NSF = B::NSF;
    constexpr int GT = EPB * NP;   // threads of a consumer group
    constexpr int NCONS = NCG * GT;
    extern __shared__ __align__(128) unsigned char ws_raw[];
    WsSmem<EPB, NCG, NBUF> &S = *reinterpret_cast<WsSmem<EPB, NCG, NBUF> *>(ws_raw);
    const size_t NPtot = P.NE * NP;
    const bool need_k = !P.stage1;
    const int ngroups = (P.n_active + EPB - 1) / EPB;

    if (threadIdx.x < NP) S.tab[threadIdx.x] = reinterpret_cast<const NodeTable<2> *>(P.box_tab)[threadIdx.x];
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&S.full[b], 64);          // 32 cp.async-completion + 32 plain arrivals (+ bulk bytes)
            mbar_init(&S.empty[b], GT / 32);    // one arrival per consumer warp
        }
        mbar_fence_init();
    }
    __syncthreads();   // the last CTA-wide barrier: the producer warp leaves early

    if (threadIdx.x >= NCONS) {
        if (!ws_produce<EPB, NCG, NBUF, OWN_BULK>(P, S, threadIdx.x - NCONS, ngroups) && threadIdx.x == NCONS)
            atomicOr(P.flags, PERRK_FLAG_TIMEOUT);
        return;
    }

    const int cg = threadIdx.x / GT, tid = threadIdx.x % GT, el = tid / NP, q = tid % NP;
    const int bar_id = 1 + cg;
    WsGroup<EPB> &G = S.grp[cg];
    const NodeTable<2> &Tb = S.tab[q];
    const float gm1 = P.gm1_f, inv_gm1 = P.inv_gm1_f, gam = P.gam_f, inv_w = P.inv_w_f;
    uint32_t bad = 0;

    for (int j = cg;; j += NCG) {
        const int grp = blockIdx.x + j * gridDim.x;
        if (grp >= ngroups) break;
        const int b = j % NBUF, use = j / NBUF;
        // the group's leader decides (bounded) and tells the group; the
        // others then find the phase complete at once (their own acquire)
        if (tid == 0) G.ok = (int)mbar_wait_bounded(&S.full[b], use & 1, kWaitLimitNs);
        named_barrier(bar_id, GT);
        if (!G.ok) {
            if (tid == 0) bad |= PERRK_FLAG_TIMEOUT;
            break;
        }
        mbar_wait_bounded(&S.full[b], use & 1, kWaitLimitNs);
        const WsStage<EPB> &T = S.st[b];
        const int slot = grp * EPB + el;
        const bool valid = slot < P.n_active;
        const int e = T.e[el];
        const size_t idx = (size_t)e * NP + q;
        const int g = T.gp[el];

        // ---- A: stage rows of the own node and of the neighbour face node
        float un[V], u[V], dprev[2 * V], wj = 0.0f;
#pragma unroll
        for (int v = 0; v < 2 * V; ++v) dprev[v] = 0.0f;
        ws_row<GT>(T.nb, tid, T.gpn[tid], P, need_k, un);
        ws_row<GT>(T.own, tid, g, P, need_k, u);
        if (P.do_b) wj = T.own[3 * V][tid];
        const float4 geo = T.geo[el];
        const float jak[3] = {geo.x, geo.y, geo.z};
        const float invJ = geo.w;
        const float4 fn4 = T.fn[el];
        const Prim<float, 2> pr = make_prim<float, 2>(u, gm1, bad);
        const int qsl = Tb.qsl;
        prim_store<2>(&G.pa[el][qsl], &G.pb[el][qsl], pr);
        vec_store<V>(&G.u[el][qsl], nullptr, u);
        named_barrier(bar_id, GT);

        // ---- B: interface flux at this thread's face node (2D: one per node)
        {
            const int sfd = Tb.sfd[0];
            const int f = sfd & 0xff, k = f >> 1, qs = (sfd >> 8) & 0xff;
            const Prim<float, 2> ps = prim_load<2>(&G.pa[el][qs], &G.pb[el][qs]);
            float us[V];
            vec_load<V>(&G.u[el][qs], nullptr, us);
            const Prim<float, 2> pn = make_prim<float, 2>(un, gm1, bad);
            const float fnv = f == 0 ? fn4.x : (f == 1 ? fn4.y : (f == 2 ? fn4.z : fn4.w));
            const bool self_plus = (f & 1);
            const Prim<float, 2> PL = prim_select<2>(self_plus, ps, pn);
            const Prim<float, 2> PR = prim_select<2>(self_plus, pn, ps);
            float nv[2], fs[V];
#pragma unroll
            for (int a = 0; a < 2; ++a) nv[a] = (a == k) ? fnv : 0.0f;
            ranocha<float, 2, -1>(PL, PR, nv, inv_gm1, fs);
            if (P.es) {
                const float lam = max_speed_nn<float, 2>(PL, PR, nv, fabsf(fnv), gam);
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const float uL = self_plus ? us[v] : un[v], uR = self_plus ? un[v] : us[v];
                    fs[v] -= 0.5f * lam * (uR - uL);
                }
            }
            const float sc = self_plus ? inv_w : -inv_w;
#pragma unroll
            for (int v = 0; v < V; ++v) fs[v] *= sc;
            vec_store<V>(&G.sf[el][q], nullptr, fs);
        }

        // ---- C: symmetric two-point volume fluxes, each pair once
#pragma unroll
        for (int t = 0; t < PPT; ++t) {
            const int pd = Tb.pd[t];
            const int sa = pd & 0xff, sb = (pd >> 8) & 0xff;
            const Prim<float, 2> A = prim_load<2>(&G.pa[el][sa], &G.pb[el][sa]);
            const Prim<float, 2> Bq = prim_load<2>(&G.pa[el][sb], &G.pb[el][sb]);
            const int kd = pd >> 16;
            float jk = jak[0];
            jk = (kd == 1) ? jak[1] : jk;
            float nv[2], F[V];
#pragma unroll
            for (int a = 0; a < 2; ++a) nv[a] = (a == kd) ? jk : 0.0f;
            ranocha<float, 2, -1>(A, Bq, nv, inv_gm1, F);
            vec_store<V>(&G.pf[el][Tb.pw[t]], nullptr, F);
        }
        named_barrier(bar_id, GT);

        // ---- D: sum_k sum_m 2 D_qm f#(q, m), then the lift at end nodes; K = -acc / J
        float acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.0f;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int as = Tb.aslot[k];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int sl = (as >> (10 * c)) & 0x3ff;
                const float cf = Tb.acoef[k][c];
                float F[V];
                vec_load<V>(&G.pf[el][sl], nullptr, F);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = fmaf(cf, F[v], acc[v]);
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int fsl = Tb.fslot[k];
            if (fsl >= 0) {
                float F[V];
                vec_load<V>(&G.sf[el][fsl], nullptr, F);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] += F[v];
            }
        }
        float Kr[V], ksum = 0.0f;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if constexpr (VISC) {
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


        // ---- E: stages with b_i != 0: entropy integrand <w(U_{n,i}), K_i> from
        // the FP32 primitives, element sum by shuffles, d and the element's
        // running sum as float pairs (the operations of k_stage_box)
        if (P.do_b) {
            const float4 cb = __ldg(reinterpret_cast<const float4 *>(P.coef_f + g));        // a1, asub, b_hi, b_lo
            const int4 fl = __ldg(reinterpret_cast<const int4 *>(&P.coef_f[g].has_b));     // has_b, first_b, d_final
            float wdf = 0.0f;
            if (fl.x) {
                if (!fl.y && !P.d_fused) {
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        dprev[v] = P.dh[v * NPtot + idx];
                        dprev[V + v] = P.dl[v * NPtot + idx];
                    }
                }
                const float Sl = (1.0f - gam) * pr.lrho - pr.lbeta;   // log p - gamma log rho
                const float ip = rcp(pr.p);
                float v2 = 0.0f, mk = 0.0f;
#pragma unroll
                for (int a = 0; a < 2; ++a) {
                    v2 = fmaf(pr.v[a], pr.v[a], v2);
                    mk = fmaf(pr.v[a], Kr[1 + a], mk);
                }
                const float w0 = gam - Sl - gm1 * 0.5f * pr.rho * v2 * ip;
                wdf = fmaf(w0, Kr[0], gm1 * pr.rho * ip * (mk - Kr[3])) * wj;
                if (valid && (!P.d_fused || fl.z)) {
                    const df bb{cb.z, cb.w};
                    const float4 cbm = __ldg(reinterpret_cast<const float4 *>(&P.coef_f[g].b1_hi));   // b1, bm pairs
#pragma unroll
                    for (int v = 0; v < V; ++v) {
                        const size_t jv = v * NPtot + idx;
                        df dn;
                        if (P.d_fused) {
                            // d = b_1 K_1 + b_m K_{S-1} + b_S K_S from the staged K_1 and K_{S-1}
                            dn = df_mul_f(df{cbm.x, cbm.y}, T.own[V + v][tid]);
                            dn = df_fma_f(dn, df{cbm.z, cbm.w}, T.own[2 * V + v][tid]);
                            dn = df_fma_f(dn, bb, Kr[v]);
                        } else {
                            dn = fl.y ? df_mul_f(bb, Kr[v]) : df_fma_f(df{dprev[v], dprev[V + v]}, bb, Kr[v]);
                        }
                        P.dh[jv] = dn.hi;
                        P.dl[jv] = dn.lo;
                    }
                }
            }
#pragma unroll
            for (int off = NP / 2; off > 0; off >>= 1) wdf += __shfl_xor_sync(0xffffffffu, wdf, off);
            if (q == 0 && valid && fl.x) {
                const df bs = df_mul_f(df{cb.z, cb.w}, wdf);
                const df en = fl.y ? bs : df_add(df{P.e_dhf[2 * e], P.e_dhf[2 * e + 1]}, bs);
                P.e_dhf[2 * e] = en.hi;
                P.e_dhf[2 * e + 1] = en.lo;
            }
        }
        // the group's scratch is rewritten by its next item, and the staging
        // buffer is free once every warp of the group is past this point
        named_barrier(bar_id, GT);
        if ((tid & 31) == 0) mbar_arrive(&S.empty[b]);
    }
    if (bad) atomicOr(P.flags, bad);
}

}  // namespace perrk
