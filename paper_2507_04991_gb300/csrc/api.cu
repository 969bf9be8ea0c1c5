// C ABI of libperrk: context lifetime, state transfer, the P-ERRK step
// sequence and its CUDA-graph capture.  One step is
//   S stage launches (stage i over its active element prefix)
//   -> relax_init (Delta H, Newton guess) [-> MLP guess]
//   -> newton_max_it Newton passes (each returns at once when the solve is done)
//   -> update (U_{n+1} = U_n + gamma dt d, t += gamma dt, step record).
// Nothing in a step depends on host control flow, so the whole step is one
// capturable launch sequence.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "perrk_internal.h"

struct perrk_ctx {
    perrk::Ctx c;
    cudaStream_t capture_stream = nullptr;
    long long host_steps = 0;  // steps since the last set_state (mirrors the device counter)
};

namespace perrk {

cudaError_t stage_ws_prepare_2d();

// the mixed form on 2D axis-aligned box elements (stage kernel variants 0-3)
static bool box2d(const Ctx &c) {
    return c.opt.precision == PERRK_MIXED && c.equation != PERRK_BURGERS_1D && !c.curved && c.dim == 2;
}

static thread_local std::string g_err;

void set_error(const std::string &e) { g_err = e; }

perrk_status cuda_check(int err, const char *what) {
    if (err == (int)cudaSuccess) return PERRK_OK;
    char buf[256];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString((cudaError_t)err));
    g_err = buf;
    return err == (int)cudaErrorMemoryAllocation ? PERRK_OUT_OF_MEMORY : PERRK_CUDA_ERROR;
}

#define PERRK_TRY(x)                          \
    do {                                      \
        perrk_status _s = (x);                \
        if (_s != PERRK_OK) return _s;        \
    } while (0)
#define PERRK_CUDA(x, what) PERRK_TRY(cuda_check((int)(x), what))

// a device copy of a host vector in its own allocation (caller frees)
template <typename T>
static perrk_status upload(T *&dst, const std::vector<T> &src, const char *what) {
    if (src.empty()) {
        dst = nullptr;
        return PERRK_OK;
    }
    PERRK_CUDA(cudaMalloc((void **)&dst, src.size() * sizeof(T)), what);
    PERRK_CUDA(cudaMemcpy(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice), what);
    return PERRK_OK;
}

// The buffers a context sizes when it is created live in one device
// allocation (one cudaMalloc, one cudaFree): zero-initialised buffers first
// (one memset), then the tables copied from the host (one copy from a host
// staging buffer), then buffers the kernels fill before reading.  Every
// buffer starts on a 256-byte boundary.
class ArenaPlan {
  public:
    void zeroed(void **slot, size_t bytes) { add(slot, bytes, nullptr, 0); }
    void raw(void **slot, size_t bytes) { add(slot, bytes, nullptr, 2); }
    template <typename T>
    void upload(T *&slot, const std::vector<T> &v) {
        add(reinterpret_cast<void **>(&slot), v.size() * sizeof(T), v.data(), 1);
    }
    perrk_status commit(Ctx &c) {
        size_t off = 0, zero_end = 0, up0 = 0, up1 = 0;
        for (int kind = 0; kind < 3; ++kind) {
            if (kind == 1) up0 = off;
            for (Item &it : items_)
                if (it.kind == kind) {
                    it.offset = off;
                    off += (it.bytes + 255) / 256 * 256;
                }
            if (kind == 0) zero_end = off;
            if (kind == 1) up1 = off;
        }
        c.arena_bytes = off;
        if (off == 0) return PERRK_OK;
        PERRK_CUDA(cudaMalloc(&c.arena, off), "context alloc");
        char *base = static_cast<char *>(c.arena);
        for (Item &it : items_) *it.slot = base + it.offset;
        if (zero_end > 0) PERRK_CUDA(cudaMemset(base, 0, zero_end), "context clear");
        if (up1 > up0) {
            std::vector<char> staging(up1 - up0, 0);
            for (const Item &it : items_)
                if (it.kind == 1) memcpy(staging.data() + (it.offset - up0), it.data.data(), it.bytes);
            PERRK_CUDA(cudaMemcpy(base + up0, staging.data(), staging.size(), cudaMemcpyHostToDevice), "context upload");
        }
        return PERRK_OK;
    }

  private:
    struct Item {
        void **slot;
        size_t bytes, offset;
        std::vector<char> data;
        int kind;   // 0 zeroed, 1 uploaded, 2 raw
    };
    void add(void **slot, size_t bytes, const void *src, int kind) {
        *slot = nullptr;
        if (bytes == 0) return;
        Item it{slot, bytes, 0, {}, kind};
        if (src) it.data.assign(static_cast<const char *>(src), static_cast<const char *>(src) + bytes);
        items_.push_back(std::move(it));
    }
    std::vector<Item> items_;
};

static void free_ctx(Ctx &c) {
    void *ptrs[] = {c.g_box_tab, c.U, c.K1, c.Ka, c.Kb, c.d, c.Uf, c.Ul, c.dh, c.dl, c.e_dhf, c.g_wJ_lo, c.K1f, c.Kaf, c.Kbf, c.e_dh, c.g_node, c.g_elem, c.g_fnorm, c.g_wJ, c.g_nbr, c.g_gp,
                    c.g_elist, c.g_chunk_inst, c.g_chunk_e0, c.g_chunk_e1, c.g_inst_chunk0, c.g_inst_nchunks,
                    c.g_coef, c.g_coef_f, c.g_scal, c.g_partials, c.g_counters, c.g_flags, c.g_records, c.g_mlp,
                    c.g_dftab, c.g_node_f, c.g_elem_f, c.g_fnorm_f, c.g_wJ_f, c.g_ring, c.visc_fv,
                    c.visc_kv, c.g_mortars, c.g_face_mortar, c.g_mtrace};
    const char *a0 = static_cast<const char *>(c.arena), *a1 = a0 + c.arena_bytes;
    for (void *p : ptrs)   // buffers allocated on their own later (the MLP weights)
        if (p && !(c.arena && static_cast<const char *>(p) >= a0 && static_cast<const char *>(p) < a1)) cudaFree(p);
    if (c.arena) cudaFree(c.arena);
    c.arena = nullptr;
    c.arena_bytes = 0;
    if (c.graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)c.graph_exec);
    if (c.graph) cudaGraphDestroy((cudaGraph_t)c.graph);
    c.graph_exec = c.graph = nullptr;
}

// Stage coefficients of every (stage, global partition) and, with dt_too,
// each instance's dt in its scalar record (one strided copy).
static perrk_status upload_coefficients(Ctx &c, bool dt_too = true) {
    std::vector<StageCoef> coef;
    std::vector<StageCoefF> coef_f;
    stage_coefficients(c, coef, coef_f);
    PERRK_CUDA(cudaMemcpy(c.g_coef, coef.data(), coef.size() * sizeof(StageCoef), cudaMemcpyHostToDevice), "coef upload");
    PERRK_CUDA(cudaMemcpy(c.g_coef_f, coef_f.data(), coef_f.size() * sizeof(StageCoefF), cudaMemcpyHostToDevice),
               "coef upload");
    if (dt_too && c.n_inst > 0) {
        std::vector<double> dts(c.n_inst);
        for (int k = 0; k < c.n_inst; ++k) dts[k] = c.inst[k].dt;
        PERRK_CUDA(cudaMemcpy2D(&c.g_scal[0].dt, sizeof(InstScalars), dts.data(), sizeof(double), sizeof(double),
                                (size_t)c.n_inst, cudaMemcpyHostToDevice),
                   "dt upload");
    }
    c.graph_dirty = true;
    return PERRK_OK;
}

static perrk_status alloc_ctx(Ctx &c) {
    int dev = 0, sms = 152;
    PERRK_CUDA(cudaGetDevice(&dev), "device query");
    PERRK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device query");
    c.sm_count = sms;
    make_chunks(c, sms);
    const size_t nstate = (size_t)c.V * c.n_elem * c.NP;
    const bool mixed = c.opt.precision == PERRK_MIXED;
    ArenaPlan A;
    // float64 form: U, K_1, two stage registers, d.  Mixed form: U and d as
    // float pairs (hi, lo), FP32 stage registers, U (float64) as the staging
    // buffer of set_state / get_state.
    A.zeroed(reinterpret_cast<void **>(&c.U), nstate * sizeof(double));
    if (!mixed)
        for (double **b : {&c.d, &c.K1, &c.Ka, &c.Kb}) A.zeroed(reinterpret_cast<void **>(b), nstate * sizeof(double));
    if (mixed) {
        for (float **b : {&c.Uf, &c.Ul, &c.dh, &c.dl, &c.K1f, &c.Kaf, &c.Kbf})
            A.zeroed(reinterpret_cast<void **>(b), nstate * sizeof(float));
        A.zeroed(reinterpret_cast<void **>(&c.e_dhf), (size_t)c.n_elem * 2 * sizeof(float));
    } else {
        A.zeroed(reinterpret_cast<void **>(&c.e_dh), (size_t)c.n_elem * sizeof(double));
    }
    A.upload(c.g_node, c.geo_node);
    A.upload(c.g_elem, c.geo_elem);
    A.upload(c.g_fnorm, c.fnorm);
    A.upload(c.g_wJ, c.wJ);
    if (mixed) {
        auto tof = [](const std::vector<double> &v) { return std::vector<float>(v.begin(), v.end()); };
        A.upload(c.g_node_f, tof(c.geo_node));
        A.upload(c.g_elem_f, tof(c.geo_elem));
        A.upload(c.g_fnorm_f, tof(c.fnorm));
        A.upload(c.g_wJ_f, tof(c.wJ));
        std::vector<float> wlo(c.wJ.size());
        for (size_t i = 0; i < wlo.size(); ++i) wlo[i] = (float)(c.wJ[i] - (double)(float)c.wJ[i]);
        A.upload(c.g_wJ_lo, wlo);
    }
    A.upload(c.g_nbr, c.nbr);
    if (c.n_mortars > 0) {
        A.upload(c.g_mortars, c.mortars);
        A.upload(c.g_face_mortar, c.face_mortar);
        const size_t nt = (size_t)3 * c.n_mortars * ipow4(c.dim - 1) * c.V * (mixed ? sizeof(float) : sizeof(double));
        A.zeroed(&c.g_mtrace, nt);
    }
    A.upload(c.g_gp, c.gp_of_elem);
    A.upload(c.g_elist, c.elist);
    if (c.viscous) {
        A.upload(c.g_ring, c.ring);
        const size_t wsz = mixed ? sizeof(float) : sizeof(double);
        const size_t nn = (size_t)c.n_elem * c.NP * (c.V - 1);
        A.zeroed(&c.visc_fv, nn * c.dim * wsz);
        A.zeroed(&c.visc_kv, nn * wsz);
    }
    A.upload(c.g_chunk_inst, c.chunk_inst);
    A.upload(c.g_chunk_e0, c.chunk_e0);
    A.upload(c.g_chunk_e1, c.chunk_e1);
    std::vector<int32_t> ic0(c.n_inst), inc(c.n_inst);
    for (int k = 0; k < c.n_inst; ++k) {
        ic0[k] = c.inst[k].chunk0;
        inc[k] = c.inst[k].n_chunks;
    }
    A.upload(c.g_inst_chunk0, ic0);
    A.upload(c.g_inst_nchunks, inc);
    A.raw(reinterpret_cast<void **>(&c.g_coef), (size_t)c.S * c.n_gp * sizeof(StageCoef));      // upload_coefficients
    A.raw(reinterpret_cast<void **>(&c.g_coef_f), (size_t)c.S * c.n_gp * sizeof(StageCoefF));
    std::vector<InstScalars> scal(c.n_inst);
    for (auto &s : scal) {
        memset(&s, 0, sizeof s);
        s.gamma = 1.0;
        for (int k = 0; k < 3; ++k) s.hist_gamma[k] = 1.0;
    }
    for (int k = 0; k < c.n_inst; ++k) scal[k].dt = c.inst[k].dt;
    A.upload(c.g_scal, scal);
    A.raw(reinterpret_cast<void **>(&c.g_partials), c.chunk_inst.size() * 8 * sizeof(double));
    A.zeroed(reinterpret_cast<void **>(&c.g_counters), (size_t)c.n_inst * sizeof(uint32_t));
    A.zeroed(reinterpret_cast<void **>(&c.g_flags), sizeof(uint32_t));
    {
        std::vector<float> tab, consts;
        df_tables(c.gamma_gas, tab, consts);
        A.upload(c.g_dftab, tab);
        for (int i = 0; i < 8; ++i) c.df_consts[i] = consts[i];
    }
    if (mixed && c.equation != PERRK_BURGERS_1D && !c.curved && c.dim >= 2) {
        float Df[16];
        for (int i = 0; i < 16; ++i) Df[i] = (float)c.lgl_D[i];
        const size_t nb = c.dim == 2 ? box_node_table_2d(Df, nullptr) : box_node_table_3d(Df, nullptr);
        std::vector<uint8_t> tab(nb);
        if (c.dim == 2) box_node_table_2d(Df, tab.data());
        else box_node_table_3d(Df, tab.data());
        A.upload(*reinterpret_cast<uint8_t **>(&c.g_box_tab), tab);
    }
    c.rec_cap = 256;
    A.raw(reinterpret_cast<void **>(&c.g_records), (size_t)c.rec_cap * c.n_inst * sizeof(perrk_step_info));
    PERRK_TRY(A.commit(c));
    return upload_coefficients(c, false);   // (each instance's dt is in its uploaded scalar record)
}

static perrk_status enqueue_step(Ctx &c, cudaStream_t st) {
    for (int i = 0; i < c.S; ++i) PERRK_TRY(launch_stage(c, i, false, nullptr, nullptr, nullptr, nullptr, st));
    PERRK_TRY(launch_relax_init(c, st));
    if (c.opt.relaxation) {
        if (c.opt.guess == PERRK_GUESS_MLP && c.mlp_on && c.opt.solver == PERRK_SOLVER_NEWTON)
            PERRK_TRY(launch_mlp_guess(c, st));
        for (int it = 0; it < c.opt.newton_max_it; ++it) PERRK_TRY(launch_newton_pass(c, st));
    }
    return launch_update(c, 0, st);
}

}  // namespace perrk

using namespace perrk;

extern "C" {

void perrk_default_options(perrk_options *o) {
    if (!o) return;
    o->precision = PERRK_FP64;
    o->relaxation = 1;
    o->newton_max_it = 10;
    o->newton_tol_r = 1e-14;
    o->newton_tol_g = 1e-14;
    o->guess = PERRK_GUESS_PREV;
    o->target = PERRK_TARGET_DELTA_H;
    o->use_graph = 0;
    o->fuse_direction = 1;
    o->solver = PERRK_SOLVER_NEWTON;
    o->bracket_lo = 0.8;
    o->bracket_hi = 1.2;
}

perrk_status perrk_create_batched(int n, const perrk_mesh_desc *mesh, const perrk_scheme_desc *scheme,
                                  const perrk_options *opts, perrk_ctx **out) {
    if (!out) {
        set_error("out is NULL");
        return PERRK_INVALID_ARG;
    }
    *out = nullptr;
    perrk_ctx *h = new (std::nothrow) perrk_ctx();
    if (!h) return PERRK_OUT_OF_MEMORY;
    std::string err;
    perrk_status st = build_ctx(h->c, n, mesh, scheme, opts, err);
    if (st != PERRK_OK) {
        set_error(err);
        delete h;
        return st;
    }
    st = alloc_ctx(h->c);
    if (st == PERRK_OK) st = cuda_check((int)cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking), "stream");
    // the staged 2D box kernel's shared-memory opt-in, outside any capture
    if (st == PERRK_OK && box2d(h->c)) st = cuda_check((int)stage_ws_prepare_2d(), "staged stage kernel set-up");
    if (st != PERRK_OK) {
        free_ctx(h->c);
        delete h;
        return st;
    }
    *out = h;
    return PERRK_OK;
}

perrk_status perrk_create(const perrk_mesh_desc *mesh, const perrk_scheme_desc *scheme, const perrk_options *opts,
                          perrk_ctx **out) {
    return perrk_create_batched(1, mesh, scheme, opts, out);
}

void perrk_destroy(perrk_ctx *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    free_ctx(h->c);
    if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
    delete h;
}

perrk_status perrk_shape(const perrk_ctx *h, int *n_elem, int *nvar, int *np, int *n_inst) {
    if (!h) return PERRK_INVALID_ARG;
    if (n_elem) *n_elem = h->c.n_elem;
    if (nvar) *nvar = h->c.V;
    if (np) *np = h->c.NP;
    if (n_inst) *n_inst = h->c.n_inst;
    return PERRK_OK;
}

perrk_status perrk_set_state(perrk_ctx *h, const double *u, int on_device, void *stream) {
    if (!h || !u || on_device < 0 || on_device > 2) return PERRK_INVALID_ARG;
    Ctx &c = h->c;
    const size_t bytes = (size_t)c.V * c.n_elem * c.NP * sizeof(double);
    cudaStream_t st = (cudaStream_t)stream;
    PERRK_CUDA(cudaMemcpyAsync(c.U, u, bytes, on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st),
               "set_state copy");
    PERRK_CUDA(cudaMemsetAsync(c.g_flags, 0, sizeof(uint32_t), st), "flags clear");
    if (c.Uf) PERRK_TRY(launch_split_entropy_set(c, st));
    else PERRK_TRY(launch_entropy_set(c, st));
    h->host_steps = 0;
    if (on_device == 0) PERRK_CUDA(cudaStreamSynchronize(st), "set_state sync");
    return PERRK_OK;
}

perrk_status perrk_get_state(perrk_ctx *h, double *u, int on_device, void *stream) {
    if (!h || !u || on_device < 0 || on_device > 2) return PERRK_INVALID_ARG;
    Ctx &c = h->c;
    const size_t bytes = (size_t)c.V * c.n_elem * c.NP * sizeof(double);
    cudaStream_t st = (cudaStream_t)stream;
    if (c.Uf) PERRK_TRY(launch_join(c.Uf, c.Ul, c.U, (size_t)c.V * c.n_elem * c.NP, st));
    PERRK_CUDA(cudaMemcpyAsync(u, c.U, bytes, on_device == 1 ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st),
               "get_state copy");
    if (on_device == 0) PERRK_CUDA(cudaStreamSynchronize(st), "get_state sync");
    return PERRK_OK;
}

static size_t state_section_bytes(const Ctx &c) {
    const size_t n = (size_t)c.V * c.n_elem * c.NP;
    return c.Uf ? 2 * n * sizeof(float) : n * sizeof(double);
}

size_t perrk_checkpoint_size(const perrk_ctx *h) {
    if (!h) return 0;
    return sizeof(perrk_checkpoint_header) + (size_t)h->c.n_inst * sizeof(perrk_resume_info) +
           state_section_bytes(h->c);
}

perrk_status perrk_checkpoint_save(perrk_ctx *h, void *buf, size_t size, void *stream) {
    if (!h || !buf || size < perrk_checkpoint_size(h)) {
        set_error("checkpoint_save: null context or buffer, or buffer smaller than perrk_checkpoint_size");
        return PERRK_INVALID_ARG;
    }
    const Ctx &c = h->c;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *out = static_cast<unsigned char *>(buf);
    perrk_checkpoint_header hd{};
    hd.magic = PERRK_CHECKPOINT_MAGIC;
    hd.version = 1;
    hd.precision = c.opt.precision;
    hd.n_inst = c.n_inst;
    hd.n_elem = c.n_elem;
    hd.nvar = c.V;
    hd.np = c.NP;
    hd.state_bytes = state_section_bytes(c);
    std::vector<InstScalars> sc(c.n_inst);
    PERRK_CUDA(cudaMemcpyAsync(sc.data(), c.g_scal, sc.size() * sizeof(InstScalars), cudaMemcpyDeviceToHost, st),
               "checkpoint scalars");
    unsigned char *state = out + sizeof hd + (size_t)c.n_inst * sizeof(perrk_resume_info);
    const size_t n = (size_t)c.V * c.n_elem * c.NP;
    if (c.Uf) {
        PERRK_CUDA(cudaMemcpyAsync(state, c.Uf, n * sizeof(float), cudaMemcpyDeviceToHost, st), "checkpoint state");
        PERRK_CUDA(cudaMemcpyAsync(state + n * sizeof(float), c.Ul, n * sizeof(float), cudaMemcpyDeviceToHost, st),
                   "checkpoint state");
    } else {
        PERRK_CUDA(cudaMemcpyAsync(state, c.U, n * sizeof(double), cudaMemcpyDeviceToHost, st), "checkpoint state");
    }
    PERRK_CUDA(cudaStreamSynchronize(st), "checkpoint sync");
    memcpy(out, &hd, sizeof hd);
    for (int k = 0; k < c.n_inst; ++k) {
        perrk_resume_info r{};
        r.t = sc[k].t;
        r.dt = c.inst[k].dt;
        r.H_n = sc[k].H_n;
        r.A_n = sc[k].A_n;
        r.H0 = sc[k].H0;
        for (int j = 0; j < 3; ++j) {
            r.gamma_hist[j] = sc[k].hist_gamma[j];
            r.dh_hist[j] = sc[k].hist_dh[j];
        }
        r.steps = sc[k].nsteps_done;
        memcpy(out + sizeof hd + (size_t)k * sizeof r, &r, sizeof r);
    }
    return PERRK_OK;
}

perrk_status perrk_checkpoint_load(perrk_ctx *h, const void *buf, size_t size, void *stream) {
    if (!h || !buf || size < sizeof(perrk_checkpoint_header)) {
        set_error("checkpoint_load: null context or buffer, or buffer shorter than the header");
        return PERRK_INVALID_ARG;
    }
    Ctx &c = h->c;
    const unsigned char *in = static_cast<const unsigned char *>(buf);
    perrk_checkpoint_header hd;
    memcpy(&hd, in, sizeof hd);
    if (hd.magic != PERRK_CHECKPOINT_MAGIC || hd.version != 1 || hd.precision != c.opt.precision ||
        hd.n_inst != c.n_inst || hd.n_elem != c.n_elem || hd.nvar != c.V || hd.np != c.NP ||
        hd.state_bytes != state_section_bytes(c) || size < perrk_checkpoint_size(h)) {
        set_error("checkpoint_load: the checkpoint does not match this context (format, precision or shapes)");
        return PERRK_INVALID_ARG;
    }
    std::vector<perrk_resume_info> rs(c.n_inst);
    memcpy(rs.data(), in + sizeof hd, rs.size() * sizeof(perrk_resume_info));
    for (int k = 0; k < c.n_inst; ++k)
        if (!std::isfinite(rs[k].t) || !std::isfinite(rs[k].H_n) || !(rs[k].dt > 0.0) || !std::isfinite(rs[k].dt) ||
            rs[k].steps < 0 || rs[k].steps != rs[0].steps) {
            set_error("checkpoint_load: non-finite history, bad dt, or instances at different step counts");
            return PERRK_INVALID_ARG;
        }
    cudaStream_t st = (cudaStream_t)stream;
    PERRK_CUDA(cudaStreamSynchronize(st), "checkpoint sync");
    bool dt_changed = false;
    for (int k = 0; k < c.n_inst; ++k)
        if (c.inst[k].dt != rs[k].dt) {
            c.inst[k].dt = rs[k].dt;
            dt_changed = true;
        }
    if (dt_changed) PERRK_TRY(upload_coefficients(c));
    const unsigned char *state = in + sizeof hd + rs.size() * sizeof(perrk_resume_info);
    const size_t n = (size_t)c.V * c.n_elem * c.NP;
    if (c.Uf) {
        PERRK_CUDA(cudaMemcpyAsync(c.Uf, state, n * sizeof(float), cudaMemcpyHostToDevice, st), "checkpoint state");
        PERRK_CUDA(cudaMemcpyAsync(c.Ul, state + n * sizeof(float), n * sizeof(float), cudaMemcpyHostToDevice, st),
                   "checkpoint state");
    } else {
        PERRK_CUDA(cudaMemcpyAsync(c.U, state, n * sizeof(double), cudaMemcpyHostToDevice, st), "checkpoint state");
    }
    PERRK_CUDA(cudaMemsetAsync(c.g_flags, 0, sizeof(uint32_t), st), "flags clear");
    // the per-step scalars start from what set_state leaves, then take the history
    PERRK_TRY(launch_entropy_set(c, st));
    std::vector<InstScalars> sc(c.n_inst);
    PERRK_CUDA(cudaMemcpyAsync(sc.data(), c.g_scal, sc.size() * sizeof(InstScalars), cudaMemcpyDeviceToHost, st),
               "checkpoint scalars");
    PERRK_CUDA(cudaStreamSynchronize(st), "checkpoint sync");
    for (int k = 0; k < c.n_inst; ++k) {
        const perrk_resume_info &r = rs[k];
        sc[k].t = r.t;
        sc[k].dt = r.dt;
        sc[k].H_n = r.H_n;
        sc[k].A_n = r.A_n;
        sc[k].H0 = r.H0;
        for (int j = 0; j < 3; ++j) {
            sc[k].hist_gamma[j] = r.gamma_hist[j];
            sc[k].hist_dh[j] = r.dh_hist[j];
        }
        sc[k].gamma = r.gamma_hist[0];
        sc[k].nsteps_done = (int32_t)r.steps;
    }
    PERRK_CUDA(cudaMemcpyAsync(c.g_scal, sc.data(), sc.size() * sizeof(InstScalars), cudaMemcpyHostToDevice, st),
               "checkpoint scalars");
    PERRK_CUDA(cudaStreamSynchronize(st), "checkpoint sync");
    h->host_steps = rs[0].steps;
    return PERRK_OK;
}

perrk_status perrk_set_dt(perrk_ctx *h, int inst, double dt) {
    if (!h || !(dt > 0.0) || !std::isfinite(dt) || inst < -1 || inst >= h->c.n_inst) {
        set_error("bad instance or dt");
        return PERRK_INVALID_ARG;
    }
    Ctx &c = h->c;
    PERRK_CUDA(cudaDeviceSynchronize(), "set_dt sync");
    for (int k = 0; k < c.n_inst; ++k)
        if (inst < 0 || inst == k) c.inst[k].dt = dt;
    return upload_coefficients(c);
}

perrk_status perrk_step(perrk_ctx *h, int nsteps, perrk_step_info *info, void *stream) {
    if (!h || nsteps < 0) return PERRK_INVALID_ARG;
    Ctx &c = h->c;
    for (const Instance &I : c.inst)
        if (!(I.dt > 0.0)) {
            set_error("dt not set (perrk_set_dt)");
            return PERRK_INVALID_ARG;
        }
    cudaStream_t st = (cudaStream_t)stream;
    PERRK_CUDA(cudaMemsetAsync(c.g_flags, 0, sizeof(uint32_t), st), "flags clear");
    if (c.opt.use_graph && c.graph_dirty) {
        if (c.graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)c.graph_exec);
        if (c.graph) cudaGraphDestroy((cudaGraph_t)c.graph);
        c.graph_exec = c.graph = nullptr;
        PERRK_CUDA(cudaStreamSynchronize(st), "pre-capture sync");
        PERRK_CUDA(cudaStreamBeginCapture(h->capture_stream, cudaStreamCaptureModeThreadLocal), "capture begin");
        perrk_status s = enqueue_step(c, h->capture_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->capture_stream, &g);
        if (s != PERRK_OK) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return s;
        }
        PERRK_CUDA(e, "capture end");
        cudaGraphExec_t ex = nullptr;
        PERRK_CUDA(cudaGraphInstantiate(&ex, g, 0), "graph instantiate");
        c.graph = g;
        c.graph_exec = ex;
        c.graph_dirty = false;
    }
    long long done = 0;
    while (done < nsteps) {
        const long long batch = info ? std::min<long long>(nsteps - done, c.rec_cap) : (nsteps - done);
        const long long first_slot = h->host_steps % c.rec_cap;
        for (long long k = 0; k < batch; ++k) {
            if (c.opt.use_graph) PERRK_CUDA(cudaGraphLaunch((cudaGraphExec_t)c.graph_exec, st), "graph launch");
            else PERRK_TRY(enqueue_step(c, st));
            h->host_steps++;
        }
        if (info) {
            std::vector<perrk_step_info> recs((size_t)c.rec_cap * c.n_inst);
            PERRK_CUDA(cudaMemcpyAsync(recs.data(), c.g_records, recs.size() * sizeof(perrk_step_info),
                                       cudaMemcpyDeviceToHost, st),
                       "records copy");
            PERRK_CUDA(cudaStreamSynchronize(st), "step sync");
            for (long long k = 0; k < batch; ++k) {
                long long slot = (first_slot + k) % c.rec_cap;
                memcpy(info + (size_t)(done + k) * c.n_inst, recs.data() + (size_t)slot * c.n_inst,
                       (size_t)c.n_inst * sizeof(perrk_step_info));
            }
        }
        done += batch;
    }
    if (info) {
        uint32_t fl = 0;
        PERRK_CUDA(cudaMemcpy(&fl, c.g_flags, sizeof fl, cudaMemcpyDeviceToHost), "flags read");
        if (fl & PERRK_FLAG_TIMEOUT) {
            set_error("a bounded device wait of the stage kernel gave up");
            return PERRK_TIMEOUT;
        }
        if (fl & (PERRK_FLAG_NONPHYSICAL | PERRK_FLAG_NONFINITE)) {
            set_error("non-physical or non-finite state met during the step");
            return PERRK_NONPHYSICAL_STATE;
        }
    }
    return PERRK_OK;
}

perrk_status perrk_autotune(perrk_ctx *h, void *stream, float *best_ms_out) {
    if (!h) return PERRK_INVALID_ARG;
    Ctx &c = h->c;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 152;
    PERRK_CUDA(cudaGetDevice(&dev), "device query");
    PERRK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device query");
    std::vector<int> epbs = c.dim == 1 ? std::vector<int>{16, 32} : (c.dim == 2 ? std::vector<int>{4, 8, 16}
                                                                              : std::vector<int>{1, 2, 4});
    std::vector<int> grids = {0, 2 * sms, 4 * sms, 8 * sms};
    cudaEvent_t e0, e1;
    PERRK_CUDA(cudaEventCreate(&e0), "event");
    PERRK_CUDA(cudaEventCreate(&e1), "event");
    // kernel variants: the mixed form on box elements has three stage kernels
    const bool box = c.opt.precision == PERRK_MIXED && c.equation != PERRK_BURGERS_1D && !c.curved && c.dim >= 2;
    const std::vector<int> variants = box ? (c.dim == 2 ? std::vector<int>{0, 1, 2, 3, 4} : std::vector<int>{0, 1, 2})
                                          : std::vector<int>{c.stage_variant};
    // box kernels: also the persistent grids of exactly one wave (2D: 1280 /
    // (16 EPB) resident CTAs per SM at 48 registers, i.e. 20, 10, 5 for
    // EPB = 4, 8, 16; 3D: 768 / (64 EPB), i.e. 12, 6, 3 for EPB = 1, 2, 4)
    if (box)
        for (int k : c.dim == 2 ? std::vector<int>{5, 10, 20} : std::vector<int>{3, 6, 12}) grids.push_back(k * sms);
    // timed: every stage of a step in order, as the step graph runs them
    // (the stages with partial active prefixes weigh in), after a warm-up of
    // the first and the last stage
    auto sweep = [&]() {
        bool ok = true;
        for (int si = 0; si < c.S && ok; ++si)
            ok = launch_stage(c, si, false, nullptr, nullptr, nullptr, nullptr, st) == PERRK_OK;
        return ok;
    };
    float best = 1e30f;
    int best_epb = c.stage_epb, best_grid = c.stage_persistent, best_var = c.stage_variant;
    const int save_epb = c.stage_epb, save_grid = c.stage_persistent, save_var = c.stage_variant;
    for (int var : variants)
        for (int epb : epbs)
            for (int g : grids) {
                c.stage_variant = var;
                c.stage_epb = epb;
                c.stage_persistent = g;
                // warm-up; an unsupported configuration reports an error and is skipped
                bool ok = launch_stage(c, 0, false, nullptr, nullptr, nullptr, nullptr, st) == PERRK_OK &&
                          launch_stage(c, c.S - 1, false, nullptr, nullptr, nullptr, nullptr, st) == PERRK_OK;
                if (!ok) {
                    cudaGetLastError();
                    continue;
                }
                cudaEventRecord(e0, st);
                ok = sweep();
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float tot = 0.0f;
                cudaEventElapsedTime(&tot, e0, e1);
                if (ok && tot < best) {
                    best = tot;
                    best_epb = epb;
                    best_grid = g;
                    best_var = var;
                }
            }
    c.stage_epb = best < 1e29f ? best_epb : save_epb;
    c.stage_persistent = best < 1e29f ? best_grid : save_grid;
    c.stage_variant = best < 1e29f ? best_var : save_var;
    // relaxation block size: time the entropy pass (a full-state float64/double-float pass)
    float best_r = 1e30f;
    int best_t = c.relax_threads;
    for (int t : {128, 256}) {
        c.relax_threads = t;
        PERRK_TRY(launch_entropy(c, 1, st));
        cudaEventRecord(e0, st);
        PERRK_TRY(launch_entropy(c, 1, st));
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_r) {
            best_r = ms;
            best_t = t;
        }
    }
    c.relax_threads = best_t;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c.tuned = true;
    c.graph_dirty = true;
    if (best_ms_out) *best_ms_out = best / (float)c.S;
    return cuda_check((int)cudaStreamSynchronize(st), "autotune sync");
}

perrk_status perrk_tuning(const perrk_ctx *h, int *elems_per_cta, int *persistent_grid, int *relax_threads,
                          int *stage_variant) {
    if (!h) return PERRK_INVALID_ARG;
    if (elems_per_cta) *elems_per_cta = h->c.stage_epb;
    if (persistent_grid) *persistent_grid = h->c.stage_persistent;
    if (relax_threads) *relax_threads = h->c.relax_threads;
    if (stage_variant) *stage_variant = h->c.stage_variant;
    return PERRK_OK;
}

perrk_status perrk_set_tuning(perrk_ctx *h, int elems_per_cta, int persistent_grid, int relax_threads,
                              int stage_variant) {
    if (!h) return PERRK_INVALID_ARG;
    Ctx &c = h->c;
    const bool epb_ok = c.dim == 1 ? (elems_per_cta == 16 || elems_per_cta == 32)
                                   : (c.dim == 2 ? (elems_per_cta == 4 || elems_per_cta == 8 || elems_per_cta == 16)
                                                 : (elems_per_cta == 1 || elems_per_cta == 2 || elems_per_cta == 4));
    const bool box = c.opt.precision == PERRK_MIXED && c.equation != PERRK_BURGERS_1D && !c.curved && c.dim >= 2;
    const bool ws_ok = stage_variant < 3 || (box && c.dim == 2 && (elems_per_cta == 4 || elems_per_cta == 8));
    if (!epb_ok || !ws_ok || persistent_grid < 0 || (relax_threads != 128 && relax_threads != 256) ||
        stage_variant < 0 || stage_variant > 4 || (!box && stage_variant != 0 && stage_variant != c.stage_variant)) {
        set_error("set_tuning: unsupported mapping for this context");
        return PERRK_INVALID_ARG;
    }
    c.stage_epb = elems_per_cta;
    c.stage_persistent = persistent_grid;
    c.relax_threads = relax_threads;
    c.stage_variant = box ? stage_variant : c.stage_variant;
    c.graph_dirty = true;
    return PERRK_OK;
}

static bool amr_ok(const Ctx &c) {
    return c.dim == 2 && !c.curved && c.equation == PERRK_EULER_2D && c.n_inst == 1;
}

perrk_status perrk_amr_indicator(perrk_ctx *h, double *alpha, void *stream) {
    if (!h || !alpha) return PERRK_INVALID_ARG;
    Ctx &c = h->c;
    if (!amr_ok(c)) {
        set_error("amr_indicator: single-instance 2D Euler contexts on box elements only");
        return PERRK_NOT_SUPPORTED;
    }
    std::vector<double> x, w, D;
    lgl_tables(x, w, D);
    AmrIndicatorConsts K;
    amr_indicator_consts(x, K);
    cudaStream_t st = (cudaStream_t)stream;
    double *dev = nullptr;
    PERRK_CUDA(cudaMalloc((void **)&dev, (size_t)c.n_elem * sizeof(double)), "amr indicator alloc");
    perrk_status s = launch_amr_indicator(c, K, dev, st);
    if (s == PERRK_OK)
        s = cuda_check((int)cudaMemcpyAsync(alpha, dev, (size_t)c.n_elem * sizeof(double), cudaMemcpyDeviceToHost, st),
                       "amr indicator copy");
    if (s == PERRK_OK) s = cuda_check((int)cudaStreamSynchronize(st), "amr indicator sync");
    cudaFree(dev);
    return s;
}

perrk_status perrk_amr_transfer(const perrk_ctx *hs, perrk_ctx *hd, const int32_t *map, void *stream) {
    if (!hs || !hd || !map || hs == hd) return PERRK_INVALID_ARG;
    const Ctx &a = hs->c;
    Ctx &b = hd->c;
    if (!amr_ok(a) || !amr_ok(b) || a.V != b.V) {
        set_error("amr_transfer: single-instance 2D Euler contexts on box elements only");
        return PERRK_NOT_SUPPORTED;
    }
    for (int e = 0; e < b.n_elem; ++e) {
        const int32_t *r = map + 5 * (size_t)e;
        const int kind = r[0];
        bool ok = kind >= 0 && kind <= 2 && r[1] >= 0 && r[1] < a.n_elem;
        if (kind == 1) ok = ok && r[2] >= 0 && r[2] < 4;
        if (kind == 2)
            for (int k = 2; k <= 4; ++k) ok = ok && r[k] >= 0 && r[k] < a.n_elem;
        if (!ok) {
            set_error("amr_transfer: map row out of range");
            return PERRK_INVALID_ARG;
        }
    }
    std::vector<double> x, w, D;
    lgl_tables(x, w, D);
    AmrOps O;
    mortar_operators(x, O.P, O.R);
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *dmap = nullptr;
    const size_t mb = (size_t)b.n_elem * 5 * sizeof(int32_t);
    PERRK_CUDA(cudaMalloc((void **)&dmap, mb), "amr map alloc");
    perrk_status s = cuda_check((int)cudaMemcpyAsync(dmap, map, mb, cudaMemcpyHostToDevice, st), "amr map copy");
    if (s == PERRK_OK) s = launch_amr_transfer(a, b, dmap, O, st);
    if (s == PERRK_OK) s = cuda_check((int)cudaMemsetAsync(b.g_flags, 0, sizeof(uint32_t), st), "flags clear");
    // the new state's entropy scalars (and, mixed form, its float pair), as set_state would
    if (s == PERRK_OK) s = b.Uf ? launch_split_entropy_set(b, st) : launch_entropy_set(b, st);
    if (s == PERRK_OK) s = launch_amr_history(a, b, st);
    if (s == PERRK_OK) s = cuda_check((int)cudaStreamSynchronize(st), "amr transfer sync");
    cudaFree(dmap);
    if (s == PERRK_OK) hd->host_steps = hs->host_steps;
    return s;
}

perrk_status perrk_test_stall_producer(perrk_ctx *h, int on) {
    if (!h) return PERRK_INVALID_ARG;
    h->c.ws_stall = on ? 1 : 0;
    h->c.graph_dirty = true;
    return PERRK_OK;
}

perrk_status perrk_entropy(perrk_ctx *h, double *H, void *stream) {
    if (!h || !H) return PERRK_INVALID_ARG;
    Ctx &c = h->c;
    cudaStream_t st = (cudaStream_t)stream;
    PERRK_TRY(launch_entropy(c, 1, st));
    std::vector<InstScalars> scal(c.n_inst);
    PERRK_CUDA(cudaMemcpyAsync(scal.data(), c.g_scal, scal.size() * sizeof(InstScalars), cudaMemcpyDeviceToHost, st),
               "scalars copy");
    PERRK_CUDA(cudaStreamSynchronize(st), "entropy sync");
    for (int k = 0; k < c.n_inst; ++k) H[k] = scal[k].H_next;
    return PERRK_OK;
}

perrk_status perrk_launch_stage(perrk_ctx *h, int stage, void *stream) {
    if (!h || stage < 0 || stage >= h->c.S) return PERRK_INVALID_ARG;
    return launch_stage(h->c, stage, false, nullptr, nullptr, nullptr, nullptr, stream);
}

perrk_status perrk_stage_info(const perrk_ctx *h, int stage, int64_t *n_active, int64_t *bytes, int *n_stages,
                              int *kernels_per_step, int64_t *dof_stage_per_step) {
    if (!h || stage < 0 || stage >= h->c.S) return PERRK_INVALID_ARG;
    const Ctx &c = h->c;
    const int NF = 2 * c.dim, NFP = ipow4(c.dim - 1);
    const int64_t vals = (int64_t)c.V * c.NP;
    const int64_t per_arr = vals * (c.opt.precision == PERRK_MIXED ? 4 : 8);  // U / K arrays, one element
    const int64_t per_d = vals * 8;                                          // float64 direction
    std::vector<StageCoef> coef;
    std::vector<StageCoefF> coef_f;
    stage_coefficients(c, coef, coef_f);
    int64_t tot = 0;
    const int na = c.n_active[stage];
    for (int k = 0; k < na; ++k) {
        const int e = c.elist[k];
        const StageCoef &sc = coef[(size_t)stage * c.n_gp + c.gp_of_elem[e]];
        int64_t arrays = 1 /*U*/ + (stage == c.S - 1 ? 0 : 1) /*K out (not stored at the last stage)*/;
        if (stage > 0) arrays += 1;               // K_1
        if (stage > 0 && sc.asub != 0.0) arrays += 1;  // K_{i-1}
        int64_t dbytes = 0;
        if (c.d_fused) dbytes = sc.d_final != 0.0 ? per_d : 0;             // d written once, at the last stage
        else if (sc.b != 0.0) dbytes = ((sc.first_b != 0.0) ? 1 : 2) * per_d;  // d write (and read)
        int64_t geo = c.curved ? (int64_t)c.NP * 5 * 8 + (int64_t)NF * NFP * 2 * 8 : (int64_t)(c.dim + 1 + NF) * 8;
        if (sc.b != 0.0) geo += (int64_t)c.NP * 8 + 8;  // omega J and the element's Delta H slot
        tot += arrays * per_arr + dbytes + geo + 4 * (2 + NF);  // element list, partition id, neighbours
    }
    if (c.viscous && na > 0) {
        // BR1: node fluxes over the gradient set (stage state read again, f_v
        // written), their divergence over the active prefix (f_v read, the
        // result written and read back by the stage kernel)
        const int64_t real = c.opt.precision == PERRK_MIXED ? 4 : 8;
        const int64_t fvb = (int64_t)c.dim * (c.V - 1) * c.NP * real, kvb = (int64_t)(c.V - 1) * c.NP * real;
        const int64_t geo_v = c.curved ? (int64_t)c.NP * 5 * real + (int64_t)NF * NFP * 2 * real : (int64_t)(c.dim + 1 + NF) * real;
        const int32_t *ring = c.ring.data() + c.ring_off[stage];
        const int n_ring = c.ring_off[stage + 1] - c.ring_off[stage];
        for (int k = 0; k < na + n_ring; ++k) {
            const int e = k < na ? c.elist[k] : ring[k - na];
            const StageCoef &sc = coef[(size_t)stage * c.n_gp + c.gp_of_elem[e]];
            int64_t arrays = 1;
            if (stage > 0) arrays += 1;
            if (stage > 0 && sc.asub != 0.0) arrays += 1;
            tot += arrays * per_arr + fvb + geo_v + 4 * (2 + NF);
        }
        tot += (int64_t)na * (fvb + 2 * kvb + geo_v + 4 * (1 + NF));
    }
    if (c.n_mortars > 0 && c.mortar_active[stage] > 0) {
        // mortar kernel: the stage rows at the three elements' face nodes
        // (U_n, K_1, K_{i-1}) and the traces of the three element faces written
        const int64_t real = c.opt.precision == PERRK_MIXED ? 4 : 8;
        const int64_t face = (int64_t)NFP * c.V * real;
        tot += (int64_t)c.mortar_active[stage] * (3 * face * (stage > 0 ? 3 : 1) + 3 * face + 4 * 4);
    }
    if (n_active) *n_active = na;
    if (bytes) *bytes = tot;
    if (n_stages) *n_stages = c.S;
    if (kernels_per_step) {
        int k = 0;
        for (int i = 0; i < c.S; ++i)
            k += (c.n_active[i] > 0 ? (c.viscous ? 3 : 1) : 0) + (c.n_mortars > 0 && c.mortar_active[i] > 0 ? 1 : 0);
        k += 2;  // relax_init + update
        if (c.opt.relaxation)
            k += c.opt.newton_max_it +
                 ((c.opt.guess == PERRK_GUESS_MLP && c.mlp_on && c.opt.solver == PERRK_SOLVER_NEWTON) ? 1 : 0);
        *kernels_per_step = k;
    }
    if (dof_stage_per_step) {
        int64_t s = 0;
        for (int i = 0; i < c.S; ++i) s += (int64_t)c.n_active[i];
        // stage 1 counts once per element for every member (it is one of the E evaluations)
        *dof_stage_per_step = s * c.V * c.NP;
    }
    return PERRK_OK;
}

perrk_status perrk_rhs(perrk_ctx *h, const double *u_in, double *k_out, void *stream) {
    if (!h || !u_in || !k_out) return PERRK_INVALID_ARG;
    Ctx &c = h->c;
    if (c.opt.precision != PERRK_MIXED) return launch_stage(c, 0, true, u_in, nullptr, k_out, nullptr, stream);
    // mixed form: FP32 input copy and FP32 result in the (transient) stage registers
    const size_t n = (size_t)c.V * c.n_elem * c.NP;
    PERRK_TRY(launch_convert(u_in, c.Kbf, nullptr, nullptr, n, stream));
    PERRK_TRY(launch_stage(c, 0, true, nullptr, c.Kbf, nullptr, c.Kaf, stream));
    return launch_convert(nullptr, nullptr, c.Kaf, k_out, n, stream);
}

int perrk_mlp_size(void) {
    const int F = kMlpFeatures, H = kMlpHidden;
    return H * F + H + H * H + H + H + 1 + 2 * F + 1;
}

int perrk_mlp_features(void) { return kMlpFeatures; }

perrk_status perrk_set_mlp(perrk_ctx *h, const float *w, int n) {
    if (!h) return PERRK_INVALID_ARG;
    Ctx &c = h->c;
    if (!w) {
        c.mlp_on = 0;
        c.graph_dirty = true;
        return PERRK_OK;
    }
    if (n != perrk_mlp_size()) {
        set_error("MLP weight count mismatch");
        return PERRK_INVALID_ARG;
    }
    if (!c.g_mlp) PERRK_CUDA(cudaMalloc((void **)&c.g_mlp, n * sizeof(float)), "mlp alloc");
    PERRK_CUDA(cudaMemcpy(c.g_mlp, w, n * sizeof(float), cudaMemcpyHostToDevice), "mlp upload");
    c.mlp_on = 1;
    c.graph_dirty = true;
    return PERRK_OK;
}

perrk_status perrk_mlp_train(const float *feats, const float *target, int n, float *weights, int epochs, float lr,
                             float *loss_out, void *stream) {
    if (!feats || !target || !weights || n <= 0 || epochs < 0) return PERRK_INVALID_ARG;
    return mlp_train_device(feats, target, n, weights, epochs, lr, loss_out, nullptr, stream);
}

perrk_status perrk_mlp_grad(const float *feats, const float *target, int n, const float *weights, float *grad_out,
                            float *loss_out, void *stream) {
    if (!feats || !target || !weights || !grad_out || n <= 0) return PERRK_INVALID_ARG;
    std::vector<float> w(weights, weights + perrk_mlp_size());
    return mlp_train_device(feats, target, n, w.data(), 0, 0.0f, loss_out, grad_out, stream);
}

perrk_status perrk_df_log(const double *x, double *y, int n, void *stream) {
    if (!x || !y || n < 0) return PERRK_INVALID_ARG;
    std::vector<float> tab, consts;
    df_tables(1.4, tab, consts);
    float *dtab = nullptr, *dk = nullptr;
    PERRK_TRY(upload(dtab, tab, "df table"));
    perrk_status s = upload(dk, consts, "df consts");
    if (s == PERRK_OK) s = launch_df_log(dtab, dk, x, y, n, stream);
    if (s == PERRK_OK) s = cuda_check((int)cudaStreamSynchronize((cudaStream_t)stream), "df_log sync");
    cudaFree(dtab);
    if (dk) cudaFree(dk);
    return s;
}

const char *perrk_last_error(void) { return g_err.c_str(); }

const char *perrk_status_string(perrk_status s) {
    switch (s) {
        case PERRK_OK: return "ok";
        case PERRK_INVALID_ARG: return "invalid argument";
        case PERRK_CUDA_ERROR: return "CUDA error";
        case PERRK_NONPHYSICAL_STATE: return "non-physical state";
        case PERRK_TIMEOUT: return "timeout";
        case PERRK_OUT_OF_MEMORY: return "out of memory";
        case PERRK_NOT_SUPPORTED: return "not supported";
    }
    return "unknown status";
}

}  // extern "C"
