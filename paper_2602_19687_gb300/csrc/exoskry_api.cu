// C ABI of the library: context management, validation, device copies of
// tables/grids/data, workspace, and the launch sequence of each call.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "context.cuh"
#include "quadrature.h"

using namespace es;


namespace {

// polls of a bounded mbarrier wait before a kernel gives up (seconds), and the
// short limit of the wait-timeout test hook (milliseconds)
constexpr unsigned WAIT_POLLS = 1u << 24, WAIT_POLLS_TEST = 1u << 12;

es_status fail(es_ctx *c, es_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

es_status cuda_fail(es_ctx *c, cudaError_t e, const char *where) {
    return fail(c, ES_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Every device allocation of a context goes through dev_alloc / dev_free,
// which keep the context's live byte count and enforce its limit
// (es_set_memory_limit): a request past the limit fails with ES_ENOMEM
// before cudaMalloc is called.
es_status dev_alloc(es_ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 1;
    if (c->mem_limit && c->dev_bytes + bytes > c->mem_limit)
        return fail(c, ES_ENOMEM, "device memory limit of " + std::to_string(c->mem_limit) + " bytes: " +
                                      std::to_string(c->dev_bytes) + " held, " + std::to_string(bytes) +
                                      " more requested");
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(c, ES_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    c->dev_sizes[*p] = bytes;
    c->dev_bytes += bytes;
    return ES_OK;
}

void dev_free(es_ctx *c, void *p) {
    if (!p) return;
    auto it = c->dev_sizes.find(p);
    if (it != c->dev_sizes.end()) {
        c->dev_bytes -= it->second;
        c->dev_sizes.erase(it);
    }
    cudaFree(p);
}

template <class T>
es_status dalloc(es_ctx *c, std::vector<void *> &owner, T **p, size_t count) {
    *p = nullptr;
    void *q = nullptr;
    es_status s = dev_alloc(c, &q, (count ? count : 1) * sizeof(T));
    if (s != ES_OK) return s;
    owner.push_back(q);
    *p = static_cast<T *>(q);
    return ES_OK;
}

template <class T>
es_status upload(es_ctx *c, std::vector<void *> &owner, T **p, const T *src, size_t count) {
    es_status s = dalloc(c, owner, p, count);
    if (s != ES_OK) return s;
    cudaError_t e = cudaMemcpy(*p, src, count * sizeof(T), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? ES_OK : cuda_fail(c, e, "cudaMemcpy");
}

void free_all(es_ctx *c, std::vector<void *> &v) {
    for (void *p : v) dev_free(c, p);
    v.clear();
}

bool ascending(const double *g, int n) {
    for (int i = 1; i < n; ++i)
        if (!(g[i] > g[i - 1])) return false;
    return true;
}

// same bracket convention as the device code, in double on the host
void host_bracket(const double *grid, int n, double x, int &i, double &w) {
    if (x <= grid[0]) x = grid[0];
    if (x >= grid[n - 1]) x = grid[n - 1];
    i = 0;
    for (int q = 0; q < n; ++q)
        if (grid[q] <= x) i = q;
    if (i > n - 2) i = n - 2;
    w = (x - grid[i]) / (grid[i + 1] - grid[i]);
}

uint16_t to_bf16_rne(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    return (uint16_t)(u >> 16);
}

double planck_host(double nu, double t) {
    return TWO_HC2 * nu * nu * nu / std::expm1(C2_RAD * nu / t);
}

cudaEvent_t take_event(es_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(void *p, const char *name, cudaStream_t st) {
    es_ctx *c = static_cast<es_ctx *>(p);
    int idx = -1;
    for (size_t k = 0; k < c->prof.size(); ++k)
        if (c->prof[k].name == name) idx = (int)k;
    if (idx < 0) {
        c->prof.push_back(es_ctx::ProfEntry{name, 0.0, 0});
        idx = (int)c->prof.size() - 1;
    }
    c->open_entry = idx;
    c->open_ev = take_event(c);
    cudaEventRecord(c->open_ev, st);
}

void prof_end(void *p, cudaStream_t st) {
    es_ctx *c = static_cast<es_ctx *>(p);
    cudaEvent_t e = take_event(c);
    cudaEventRecord(e, st);
    c->pending.push_back(es_ctx::Pending{c->open_entry, c->open_ev, e});
    c->open_entry = -1;
}

void prof_resolve(es_ctx *c) {
    for (auto &q : c->pending) {
        cudaEventSynchronize(q.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, q.a, q.b);
        c->prof[q.entry].ms += ms;
        c->prof[q.entry].n += 1;
        c->ev_pool.push_back(q.a);
        c->ev_pool.push_back(q.b);
    }
    c->pending.clear();
}

es_status check_launch(es_ctx *c, const char *what) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ES_OK : cuda_fail(c, e, what);
}

void drop_graph(es_ctx::GraphSlot &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.epoch = -1;
    g.calls = 0;
}

// Run `enqueue(stream)` eagerly, or, from the second call with an unchanged
// batch shape and buffers on, capture it once into a CUDA graph and replay it.
// The graph is captured and launched on a private non-blocking stream joined
// to the caller's stream by events, so callers on the legacy default stream
// get replay too. Profiling runs stay eager (their events are per launch).
template <class F>
es_status launch_or_replay(es_ctx *c, es_ctx::GraphSlot &g, cudaStream_t st, F &&enqueue) {
    if (!c->use_graph || c->prof_on) return enqueue(st);
    if (g.epoch != c->graph_epoch) {
        drop_graph(g);
        g.epoch = c->graph_epoch;
    }
    if (!g.exec) {
        if (g.calls++ == 0) return enqueue(st);   // first call eager: sets attributes, warms caches
        cudaError_t e = cudaSuccess;
        if (!c->gstream) {
            e = cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(c, e, "graph stream");
        }
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
        es_status s = enqueue(c->gstream);
        e = cudaStreamEndCapture(c->gstream, &graph);
        if (s != ES_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return s != ES_OK ? s : cuda_fail(c, e, "graph capture");
        }
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g.exec = nullptr;
            return cuda_fail(c, e, "graph instantiate");
        }
    }
    cudaError_t e = cudaEventRecord(c->ev_fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->gstream, c->ev_fork, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(g.exec, c->gstream);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, c->gstream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->ev_join, 0);
    return e == cudaSuccess ? ES_OK : cuda_fail(c, e, "graph launch");
}

es_status alloc_forward(es_ctx *c, int B) {
    if (B <= c->cap_b) return ES_OK;
    ++c->graph_epoch;
    free_all(c, c->work_bufs);
    free_all(c, c->bwd_bufs);
    // until the new buffers are all in place the context holds no batch (a
    // failed allocation leaves it in the "no batch set" state)
    c->cap_b = c->cap_b_bwd = 0;
    c->batch = 0;
    c->n_kind[0] = c->n_kind[1] = 0;
    const Model &m = c->m;
    const size_t L = m.L, S = m.S, N = m.N;
    Work &w = c->w;
    es_status s = ES_OK;
    double *theta_user;
#define ALLOC(p, n) if ((s = dalloc(c, c->work_bufs, &(p), (size_t)(n))) != ES_OK) return s
    ALLOC(theta_user, (size_t)B * m.nfree);
    w.theta_user = theta_user;
    ALLOC(w.theta, (size_t)B * m.nfull);
    ALLOC(w.kind, B);
    ALLOC(w.flags, B);
    ALLOC(w.err, 1);
    ALLOC(w.t_lay, B * L);
    ALLOC(w.t_lev, B * (L + 1));
    ALLOC(w.r_lev, B * (L + 1));
    ALLOC(w.xs, B * (S + 2));
    ALLOC(w.n_lay, B * L);
    ALLOC(w.rc, B);
    ALLOC(w.base, B);
    ALLOC(w.scale, B);
    ALLOC(w.lmat, B * L * L);
    ALLOC(w.area, B * L);
    ALLOC(w.dr, B * L);
    ALLOC(w.it, B * L);
    ALLOC(w.gt, B * L);
    ALLOC(w.wtr, B * L);
    ALLOC(w.itc, B * L);
    ALLOC(w.wtc, B * L);
    ALLOC(w.gtc, B * L);
    ALLOC(w.ccia, B * L * 2);
    ALLOC(w.ray, B * L);
    ALLOC(w.cloud_c, B * L);
    ALLOC(w.cloud_d, B * L);
    ALLOC(w.cloud_g, B * N_CG);
    ALLOC(w.spec, (size_t)B * N);
    ALLOC(w.arows, (size_t)B * 2);
    ALLOC(w.lnl, B);
    ALLOC(w.misc, (size_t)B * 4);
    ALLOC(c->d_lnl, B);
#undef ALLOC
    if (cudaMemset(w.err, 0, sizeof(int)) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "status word");
    c->cap_b = B;
    return ES_OK;
}

es_status alloc_backward(es_ctx *c) {
    const int B = c->cap_b;
    if (B <= c->cap_b_bwd) return ES_OK;
    ++c->graph_epoch;
    free_all(c, c->bwd_bufs);
    c->cap_b_bwd = 0;
    const Model &m = c->m;
    const size_t L = m.L, S = m.S, N = m.N;
    Work &w = c->w;
    es_status s = ES_OK;
#define ALLOC(p, n) if ((s = dalloc(c, c->bwd_bufs, &(p), (size_t)(n))) != ES_OK) return s
    ALLOC(w.dbar, (size_t)B * m.Np);
    ALLOC(w.lbar, (size_t)B * L * L);
    ALLOC(w.red, (size_t)B * L * N_RED);
    ALLOC(w.qtot, (size_t)B * S);
    ALLOC(w.zbar, (size_t)B * L);
    ALLOC(w.areabar, (size_t)B * L);
    ALLOC(w.levbar, (size_t)B * (L + 1));
    ALLOC(w.drbar, (size_t)B * L);
    ALLOC(w.grad, (size_t)B * c->m.nfree);
    ALLOC(w.cloud_dbar, (size_t)B * L);
    ALLOC(w.cloud_pbar, (size_t)B * N_CG);
#undef ALLOC
    c->cap_b_bwd = B;
    return ES_OK;
}

// Large per-kind buffers, allocated on first need and kept until the batch
// capacity grows: alpha/abar for emission samples, estore for the
// transmission adjoint.
es_status ensure_big(es_ctx *c, float **p, size_t &cap, size_t count) {
    if (count <= cap && *p) return ES_OK;
    ++c->graph_epoch;
    dev_free(c, *p);
    *p = nullptr;
    cap = 0;
    void *q = nullptr;
    es_status s = dev_alloc(c, &q, count * sizeof(float));
    if (s != ES_OK) return s;
    *p = static_cast<float *>(q);
    cap = count;
    return ES_OK;
}

es_status ready(es_ctx *c) {
    if (!c->have_tables) return fail(c, ES_ESTATE, "tables not loaded");
    if (!c->have_grid) return fail(c, ES_ESTATE, "instrument grid not set");
    if (c->batch <= 0) return fail(c, ES_ESTATE, "no batch set");
    for (int k = 0; k < 2; ++k)
        if (c->n_kind[k] > 0 && !c->have_data[k])
            return fail(c, ES_ESTATE, std::string("no data for ") + (k ? "emission" : "transmission") + " samples");
    return ES_OK;
}

es_status ensure_ymod(es_ctx *c) {
    size_t need = (size_t)c->cap_b * c->m.nbins;
    if (need <= c->ymod_cap) return ES_OK;
    ++c->graph_epoch;
    dev_free(c, c->w.ymod);
    c->w.ymod = nullptr;
    c->ymod_cap = 0;
    void *q = nullptr;
    es_status s = dev_alloc(c, &q, need * sizeof(double));
    if (s != ES_OK) return s;
    c->w.ymod = static_cast<double *>(q);
    c->ymod_cap = need;
    return ES_OK;
}

// The one-vector (plain per-sample) transmission path: a batch of a single
// transmission vector runs its opacity stage as a table stream of its own
// (k_trans_alpha, the raw bracketing rows read once) and the chord kernel on
// the extinction it wrote, instead of the fused interpolating forward.
bool one_vector_path(const es_ctx *c) { return c->batch == 1 && c->n_kind[0] == 1; }

// Emission samples solved by the delta-EAA (k_eaa.cu) instead of the fused
// emission kernels.
bool eaa_path(const es_ctx *c) { return c->m.emis_solver == ES_RT_DELTA_EAA && c->n_kind[1] > 0; }

// Device buffers a call needs (allocated before any launch or capture).
es_status prepare(es_ctx *c, bool adjoint) {
    es_status s;
    if ((s = ensure_ymod(c)) != ES_OK) return s;
    if ((one_vector_path(c) || eaa_path(c)) &&
        (s = ensure_big(c, &c->w.ext, c->ext_cap, (size_t)c->batch * c->m.L * c->m.Np)) != ES_OK)
        return s;
    if (eaa_path(c) && (s = ensure_big(c, &c->eaa_scr, c->eaa_scr_cap, eaa_scratch_floats(c->m))) != ES_OK)
        return s;

    if (adjoint) {
        if ((s = alloc_backward(c)) != ES_OK) return s;
        if (c->n_kind[0] &&
            (s = ensure_big(c, &c->w.estore, c->estore_cap, (size_t)c->batch * c->m.L * c->m.Np)) != ES_OK)
            return s;
        // emission: I_toa per angle, a second (cloudy) column with the non-grey cloud
        const size_t cols = c->m.cloud_kind == ES_CLOUD_KH18 ? 2 : 1;
        if (c->n_kind[1] &&
            (s = ensure_big(c, &c->w.itop, c->alpha_cap, (size_t)c->batch * c->m.Np * N_MU * cols)) != ES_OK)
            return s;
    }
    return ES_OK;
}

// The status word of the fused kernels' bounded waits: cleared at the start
// of every call, copied to the context's pinned host word at its end (both
// steps inside a captured graph too), read by finish() for host-buffer calls.
void clear_status(es_ctx *c, cudaStream_t st) { cudaMemsetAsync(c->w.err, 0, sizeof(int), st); }
void post_status(es_ctx *c, cudaStream_t st) {
    cudaMemcpyAsync(c->h_err, c->w.err, sizeof(int), cudaMemcpyDeviceToHost, st);
}

es_status run_forward(es_ctx *c, bool adjoint, float *spec_out, double *binned_out, double *lnl_out,
                      cudaStream_t st, bool post = true) {
    Work w = c->w;
    w.B = c->batch;
    int launches = 0;
    const Hook &h = c->hook;
    clear_status(c, st);
    launches += launch_setup(c->m, w, st, h);
    c->last_one_vector = false;
    const es_ctx::Shape *sh = c->shape;
    if (eaa_path(c)) {   // emission by the delta-EAA; transmission samples by their fused kernel
        if (c->n_kind[0]) {
            const es_ctx::Shape &x = sh[es_ctx::FUSED_TRANS_FWD];
            launches += launch_trans_fused_forward(c->m, w, adjoint, x.chunk, x.sample_major, st, h);
        }
        launches += launch_eaa_forward(c->m, w, c->eaa_scr, adjoint, st, h);
    } else if (c->n_kind[0] && c->n_kind[1]) {   // both kinds: one kernel over all items
        const es_ctx::Shape &x = sh[es_ctx::FUSED_MIXED_FWD];
        launches += launch_mixed_fused_forward(c->m, w, adjoint, x.chunk, x.sample_major, st, h);
    } else if (one_vector_path(c)) {
        c->last_one_vector = true;
        launches += launch_trans_alpha(c->m, w, st, h);
        launches += launch_trans_chord_forward(c->m, w, adjoint, st, h);
    } else if (c->n_kind[0]) {
        const es_ctx::Shape &x = sh[es_ctx::FUSED_TRANS_FWD];
        launches += launch_trans_fused_forward(c->m, w, adjoint, x.chunk, x.sample_major, st, h);
    } else if (c->n_kind[1]) {
        const es_ctx::Shape &x = sh[es_ctx::FUSED_EMIS_FWD];
        launches += launch_emis_fused_forward(c->m, w, adjoint, x.chunk, x.sample_major, st, h);
    }
    if (adjoint) {
        cudaMemsetAsync(w.dbar, 0, sizeof(float) * (size_t)w.B * c->m.Np, st);
    }
    launches += launch_bins(c->m, w, adjoint, spec_out, binned_out, lnl_out, st, h);
    if (post) post_status(c, st);
    c->last_launches = launches;
    return check_launch(c, "forward launch");
}

}  // namespace

extern "C" {

es_status es_create(es_ctx **out, int device, const es_model_desc *d) {
    if (!out || !d) return ES_EINVAL;
    *out = nullptr;
    if (d->n_layers < 2 || d->n_layers > ES_MAX_LAYERS) return ES_EINVAL;
    if (d->n_species < 1 || d->n_species > ES_MAX_SPECIES) return ES_EINVAL;
    if (!(d->p_top_bar > 0) || !(d->p_bot_bar > d->p_top_bar) || !(d->p_ref_bar > 0)) return ES_EINVAL;
    if (d->tp_kind < 0 || d->tp_kind > ES_TP_MILNE || d->cloud_kind < 0 || d->cloud_kind > ES_CLOUD_KH18) return ES_EINVAL;
    if (d->emission_flux != ES_FLUX_PLANET_STAR && d->emission_flux != ES_FLUX_BROWN_DWARF) return ES_EINVAL;
    if (d->emission_flux == ES_FLUX_BROWN_DWARF && !(d->distance_cm > 0)) return ES_EINVAL;
    if (d->cloud_profile < ES_QC_POWER_LAW || d->cloud_profile > ES_QC_SLAB_BAND) return ES_EINVAL;
    if (d->cloud_feature != 0 && d->cloud_feature != 1) return ES_EINVAL;
    if (d->emission_quadrature != ES_QUAD_GAUSS_LEGENDRE && d->emission_quadrature != ES_QUAD_GAUSS_JACOBI)
        return ES_EINVAL;
    if (!(d->r_star_cm > 0) || !(d->t_star_k > 0)) return ES_EINVAL;
    if (d->emission_solver != ES_RT_ABSORPTION && d->emission_solver != ES_RT_DELTA_EAA) return ES_EINVAL;
    if (d->emission_solver == ES_RT_DELTA_EAA &&
        (d->cloud_kind == ES_CLOUD_DECK || !(d->cloud_ssa >= 0.0 && d->cloud_ssa <= 1.0) ||
         !(d->cloud_g >= 0.0 && d->cloud_g < 1.0)))
        return ES_EINVAL;
    const int nfull = d->n_species + ES_P_N_EXTRA;
    if (d->n_free < 1 || d->n_free > 32 || d->n_free > nfull) return ES_EINVAL;
    for (int k = 0; k < d->n_free; ++k) {
        if (d->free_idx[k] < 0 || d->free_idx[k] >= nfull) return ES_EINVAL;
        for (int q = 0; q < k; ++q)
            if (d->free_idx[q] == d->free_idx[k]) return ES_EINVAL;
    }
    for (int s = 0; s < d->n_species; ++s)
        if (!(d->species_mass_amu[s] > 0)) return ES_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return ES_ECUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return ES_ECUDA;
    es_ctx *c = new es_ctx();
    c->device = device;
    c->desc = *d;
    Model &m = c->m;
    m.L = d->n_layers;
    m.S = d->n_species;
    m.nfree = d->n_free;
    m.nfull = nfull;
    m.tp_kind = d->tp_kind;
    m.cloud_kind = d->cloud_kind;
    m.emis_flux = d->emission_flux;
    m.distance = d->distance_cm;
    m.cloud_profile = d->cloud_profile;
    m.cloud_feature = d->cloud_feature;
    m.wait_polls = WAIT_POLLS;
    m.wait_test = 0;
    m.p_ref = d->p_ref_bar * BAR;
    m.r_star = d->r_star_cm;
    m.t_star = d->t_star_k;
    m.ray_h2 = d->ray_h2_cm2;
    m.ray_he = d->ray_he_cm2;
    m.ray_nu_ref = d->ray_nu_ref > 0 ? d->ray_nu_ref : 1.0;
    for (int s = 0; s < m.S; ++s) m.mass[s] = d->species_mass_amu[s];
    for (int k = 0; k < nfull; ++k) m.theta_fixed[k] = d->theta_fixed[k];
    for (int k = 0; k < m.nfree; ++k) m.free_idx[k] = d->free_idx[k];
    // flux angles: the kernels form 2 pi w_j mu_j, so a Gauss-Jacobi weight
    // W_j (of the weight mu) is stored as W_j / mu_j
    if (d->emission_quadrature == ES_QUAD_GAUSS_JACOBI) {
        double W[N_MU];
        gauss_jacobi_mu_01(N_MU, m.mu_gl, W);
        for (int j = 0; j < N_MU; ++j) m.w_gl[j] = W[j] / m.mu_gl[j];
    } else {
        gauss_legendre4_01(m.mu_gl, m.w_gl);
    }
    m.emis_solver = d->emission_solver;
    m.cloud_ssa = (float)d->cloud_ssa;
    m.cloud_gasym = (float)d->cloud_g;
    interp_weights_01(N_MU, m.mu_gl, m.c_mu);
    // pressure levels (top to bottom) and layers
    std::vector<double> p_lev(m.L + 1), p_lay(m.L);
    for (int k = 0; k <= m.L; ++k)
        p_lev[k] = d->p_top_bar * std::pow(d->p_bot_bar / d->p_top_bar, (double)k / m.L) * BAR;
    for (int l = 0; l < m.L; ++l) p_lay[l] = std::sqrt(p_lev[l] * p_lev[l + 1]);
    double *dp;
    es_status s;
    if ((s = upload(c, c->model_bufs, &dp, p_lev.data(), p_lev.size())) != ES_OK) { es_destroy(c); return s; }
    m.p_lev = dp;
    if ((s = upload(c, c->model_bufs, &dp, p_lay.data(), p_lay.size())) != ES_OK) { es_destroy(c); return s; }
    m.p_lay = dp;
    std::vector<double> lnp(m.L + 1);
    for (int k = 0; k <= m.L; ++k) lnp[k] = std::log(p_lev[k]);
    if ((s = upload(c, c->model_bufs, &dp, lnp.data(), lnp.size())) != ES_OK) { es_destroy(c); return s; }
    m.lnp_lev = dp;
    m.ln_p_ref = std::log(m.p_ref);
    if (cudaHostAlloc(reinterpret_cast<void **>(&c->h_err), sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        c->h_err = nullptr;
        es_destroy(c);
        return ES_ENOMEM;
    }
    *c->h_err = 0;
    *out = c;
    return ES_OK;
}

es_status es_load_tables(es_ctx *c, const es_tables_desc *t) {
    if (!c) return ES_EINVAL;
    if (!t || !t->nu || !t->t_grid || !t->p_grid_bar || !t->log10_sigma || !t->cia_t_grid || !t->cia_h2h2 ||
        !t->cia_h2he)
        return fail(c, ES_EINVAL, "null table pointer");
    if (t->n_nu < 2 || t->n_t < 2 || t->n_p < 2 || t->n_t_cia < 2 || t->n_t > 64 || t->n_p > 64 || t->n_t_cia > 64)
        return fail(c, ES_EINVAL, "table sizes out of range");
    if (!ascending(t->nu, t->n_nu) || !ascending(t->t_grid, t->n_t) || !ascending(t->p_grid_bar, t->n_p) ||
        !ascending(t->cia_t_grid, t->n_t_cia) || !(t->t_grid[0] > 0) || !(t->p_grid_bar[0] > 0) ||
        !(t->nu[0] > 0))
        return fail(c, ES_EINVAL, "grids must be positive and strictly ascending");
    if (t->storage != ES_TABLE_F32 && t->storage != ES_TABLE_BF16) return fail(c, ES_EINVAL, "bad storage");
    {
        // every table value finite (a NaN or Inf would reach every spectrum silently)
        const size_t per_row = (size_t)t->n_nu, rows = (size_t)c->m.S * t->n_t * t->n_p;
        for (size_t r = 0; r < rows; ++r)
            for (size_t n = 0; n < per_row; ++n)
                if (!std::isfinite(t->log10_sigma[r * per_row + n])) {
                    const size_t ip = r % t->n_p, it = (r / t->n_p) % t->n_t, sp = r / ((size_t)t->n_p * t->n_t);
                    return fail(c, ES_EINVAL, "log10_sigma[" + std::to_string(sp) + "][" + std::to_string(it) + "][" +
                                                  std::to_string(ip) + "][" + std::to_string(n) + "] is not finite");
                }
        for (int pair = 0; pair < 2; ++pair) {
            const float *src = pair ? t->cia_h2he : t->cia_h2h2;
            for (size_t k = 0; k < (size_t)t->n_t_cia * per_row; ++k)
                if (!std::isfinite(src[k]))
                    return fail(c, ES_EINVAL, std::string(pair ? "cia_h2he" : "cia_h2h2") + " value " +
                                                  std::to_string(k) + " is not finite");
        }
    }
    cudaSetDevice(c->device);
    free_all(c, c->table_bufs);
    free_all(c, c->grid_bufs);
    c->have_tables = c->have_grid = false;
    c->have_data[0] = c->have_data[1] = false;
    c->cap_b = c->cap_b_bwd = 0;
    c->batch = 0;   // the workspace is gone: the batch must be set again
    c->n_kind[0] = c->n_kind[1] = 0;
    free_all(c, c->work_bufs);
    free_all(c, c->bwd_bufs);
    Model &m = c->m;
    m.N = t->n_nu;
    m.NT = t->n_t;
    m.NP = t->n_p;
    m.NTc = t->n_t_cia;
    m.bf16 = t->storage == ES_TABLE_BF16;
    c->nu_host.assign(t->nu, t->nu + t->n_nu);
    // device rows are padded to Np (a multiple of 128, the widest tile) by
    // repeating the last value, so the last tile's loads stay inside their row
    m.Np = (m.N + 127) / 128 * 128;
    const size_t N = m.N, Np = m.Np, S = m.S, rows = S * m.NT * m.NP;
    es_status s;
    std::vector<float> off(rows, 0.f);
    if (m.bf16) {
        std::vector<uint16_t> q(rows * Np);
        for (size_t r = 0; r < rows; ++r) {
            const float *src = t->log10_sigma + r * N;
            double mean = 0.0;
            for (size_t n = 0; n < N; ++n) mean += src[n];
            float o = (float)(mean / (double)N);
            off[r] = o;
            for (size_t n = 0; n < Np; ++n) q[r * Np + n] = to_bf16_rne(src[n < N ? n : N - 1] - o);
        }
        uint16_t *d16;
        if ((s = upload(c, c->table_bufs, &d16, q.data(), q.size())) != ES_OK) return s;
        m.tab16 = d16;
        m.tab32 = nullptr;
    } else {
        std::vector<float> q(rows * Np);
        for (size_t r = 0; r < rows; ++r)
            for (size_t n = 0; n < Np; ++n) q[r * Np + n] = t->log10_sigma[r * N + (n < N ? n : N - 1)];
        float *d32;
        if ((s = upload(c, c->table_bufs, &d32, q.data(), q.size())) != ES_OK) return s;
        m.tab32 = d32;
        m.tab16 = nullptr;
    }
    float *df;
    if ((s = upload(c, c->table_bufs, &df, off.data(), rows)) != ES_OK) return s;
    m.row_off = df;
    std::vector<float> cia(2 * (size_t)m.NTc * Np);
    for (int pair = 0; pair < 2; ++pair) {
        const float *src = pair ? t->cia_h2he : t->cia_h2h2;
        for (size_t r = 0; r < (size_t)m.NTc; ++r)
            for (size_t n = 0; n < Np; ++n)
                cia[((size_t)pair * m.NTc + r) * Np + n] = src[r * N + (n < N ? n : N - 1)];
    }
    if ((s = upload(c, c->table_bufs, &df, cia.data(), cia.size())) != ES_OK) return s;
    m.cia = df;
    // CIA interpolation coefficients per temperature bracket and wavenumber pair
    {
        const size_t np2 = Np / 2, nb = (size_t)m.NTc - 1;
        std::vector<float> c4(2 * nb * np2 * 4);
        for (int pair = 0; pair < 2; ++pair)
            for (size_t r = 0; r < nb; ++r)
                for (size_t q = 0; q < np2; ++q)
                    for (int k = 0; k < 2; ++k) {
                        const double k0 = cia[((size_t)pair * m.NTc + r) * Np + 2 * q + k];
                        const double k1 = cia[((size_t)pair * m.NTc + r + 1) * Np + 2 * q + k];
                        float *o = &c4[((r * np2 + q) * 2 + pair) * 4];
                        o[k] = (float)(LOG2_10 * k0);
                        o[2 + k] = (float)(LOG2_10 * (k1 - k0));
                    }
        float4 *d4;
        if ((s = upload(c, c->table_bufs, &d4, reinterpret_cast<const float4 *>(c4.data()), c4.size() / 4)) != ES_OK)
            return s;
        m.cia4 = d4;
    }
    std::vector<float> nuf(Np), ifs(Np);
    for (size_t n = 0; n < Np; ++n) {
        const double nv = t->nu[n < N ? n : N - 1];
        nuf[n] = (float)nv;
        // Fp/F* divides by the stellar flux; a brown dwarf's flux is absolute
        ifs[n] = (m.emis_flux == ES_FLUX_BROWN_DWARF) ? 1.f : (float)(1.0 / (PI * planck_host(nv, m.t_star)));
    }
    if ((s = upload(c, c->table_bufs, &df, nuf.data(), Np)) != ES_OK) return s;
    m.nu = df;
    if ((s = upload(c, c->table_bufs, &df, ifs.data(), Np)) != ES_OK) return s;
    m.inv_fstar = df;
    std::vector<double> logt(m.NT), logp(m.NP);
    for (int i = 0; i < m.NT; ++i) logt[i] = std::log10(t->t_grid[i]);
    for (int i = 0; i < m.NP; ++i) logp[i] = std::log10(t->p_grid_bar[i]);
    double *dd;
    if ((s = upload(c, c->table_bufs, &dd, logt.data(), logt.size())) != ES_OK) return s;
    m.log_t = dd;
    if ((s = upload(c, c->table_bufs, &dd, t->cia_t_grid, (size_t)m.NTc)) != ES_OK) return s;
    m.cia_t = dd;
    // fixed pressure bracket of every layer (log10 p in bar)
    std::vector<int> ip(m.L);
    std::vector<float> wp(m.L);
    for (int l = 0; l < m.L; ++l) {
        double pl = c->desc.p_top_bar * std::pow(c->desc.p_bot_bar / c->desc.p_top_bar, (double)l / m.L) * BAR;
        double pu = c->desc.p_top_bar * std::pow(c->desc.p_bot_bar / c->desc.p_top_bar, (double)(l + 1) / m.L) * BAR;
        double play = std::sqrt(pl * pu);
        int i;
        double wv;
        host_bracket(logp.data(), m.NP, std::log10(play / BAR), i, wv);
        ip[l] = i;
        wp[l] = (float)wv;
    }
    int *di;
    if ((s = upload(c, c->table_bufs, &di, ip.data(), ip.size())) != ES_OK) return s;
    m.ip = di;
    if ((s = upload(c, c->table_bufs, &df, wp.data(), wp.size())) != ES_OK) return s;
    m.wp = df;
    // per-cell bilinear coefficients used by the fused kernels
    float4 *coef;
    m.SP = 2 * spl_for(m.S);
    const size_t ncoef = (size_t)(m.NT - 1) * (m.NP - 1) * m.SP * m.Np;
    if ((s = dalloc(c, c->table_bufs, &coef, ncoef)) != ES_OK) return s;
    m.coef4 = nullptr;
    cudaError_t e = cudaMemset(coef, 0, ncoef * sizeof(float4));
    if (e != cudaSuccess) return cuda_fail(c, e, "coefficient table");
    launch_build_coef(m, coef, nullptr);
    e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "coefficient table");
    m.coef4 = coef;
    c->have_tables = true;
    ++c->graph_epoch;
    return ES_OK;
}

es_status es_set_grid(es_ctx *c, const double *lo, const double *hi, int nbins) {
    if (!c) return ES_EINVAL;
    if (!c->have_tables) return fail(c, ES_ESTATE, "load tables before the grid");
    if (!lo || !hi || nbins < 1) return fail(c, ES_EINVAL, "bad bin arrays");
    cudaSetDevice(c->device);
    const int N = c->m.N;
    // lambda = 1e4/nu decreases with the index, so each bin's members
    // {n : lo <= lambda_n < hi} form one contiguous index range.
    std::vector<double> lam(N);
    for (int n = 0; n < N; ++n) lam[n] = 1.0e4 / c->nu_host[n];
    std::vector<int> blo(nbins), bhi(nbins), owner(N, -1);
    for (int k = 0; k < nbins; ++k) {
        if (!(hi[k] > lo[k])) return fail(c, ES_EINVAL, "bin " + std::to_string(k) + ": hi <= lo");
        int a = 0, b = N;   // first index with lam < hi
        while (a < b) {
            int mid = (a + b) / 2;
            if (lam[mid] < hi[k]) b = mid; else a = mid + 1;
        }
        int first = a;
        a = 0, b = N;       // first index with lam < lo
        while (a < b) {
            int mid = (a + b) / 2;
            if (lam[mid] < lo[k]) b = mid; else a = mid + 1;
        }
        int end = a;
        if (end <= first) return fail(c, ES_EINVAL, "bin " + std::to_string(k) + " holds no native point");
        for (int n = first; n < end; ++n) {
            if (owner[n] >= 0) return fail(c, ES_EINVAL, "bins " + std::to_string(owner[n]) + " and " +
                                                           std::to_string(k) + " overlap");
            owner[n] = k;
        }
        blo[k] = first;
        bhi[k] = end;
    }
    free_all(c, c->grid_bufs);
    free_all(c, c->data_bufs);
    c->have_grid = false;
    c->have_data[0] = c->have_data[1] = false;
    es_status s;
    int *di;
    if ((s = upload(c, c->grid_bufs, &di, blo.data(), (size_t)nbins)) != ES_OK) return s;
    c->m.bin_lo = di;
    if ((s = upload(c, c->grid_bufs, &di, bhi.data(), (size_t)nbins)) != ES_OK) return s;
    c->m.bin_hi = di;
    if ((s = upload(c, c->grid_bufs, &di, owner.data(), (size_t)N)) != ES_OK) return s;
    c->m.bin_of = di;
    if ((s = dalloc(c, c->grid_bufs, &c->d_data, (size_t)4 * nbins)) != ES_OK) return s;
    c->m.nbins = nbins;
    c->m.y_obs = c->d_data;
    c->m.sigma = c->d_data + 2 * (size_t)nbins;
    for (int k = 0; k < 2; ++k) {
        c->y_host[k].assign(nbins, 0.0);
        c->s_host[k].assign(nbins, 1.0);
    }
    c->have_grid = true;
    ++c->graph_epoch;
    return ES_OK;
}

es_status es_set_data(es_ctx *c, int kind, const double *y_obs, const double *sigma, int nbins) {
    if (!c) return ES_EINVAL;
    if (!c->have_grid) return fail(c, ES_ESTATE, "set the instrument grid before the data");
    if (kind != ES_KIND_TRANSMISSION && kind != ES_KIND_EMISSION) return fail(c, ES_EINVAL, "bad kind");
    if (!y_obs || !sigma || nbins != c->m.nbins) return fail(c, ES_EINVAL, "data size differs from the grid");
    for (int k = 0; k < nbins; ++k)
        if (!(sigma[k] > 0) || !std::isfinite(y_obs[k])) return fail(c, ES_EINVAL, "sigma must be > 0, y finite");
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemcpy(c->d_data + (size_t)kind * nbins, y_obs, sizeof(double) * nbins,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_data + (size_t)(2 + kind) * nbins, sigma, sizeof(double) * nbins,
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "es_set_data");
    c->have_data[kind] = true;
    return ES_OK;
}

es_status es_set_batch(es_ctx *c, const double *theta, const int32_t *kind, int batch, int mem,
                       es_stream_t stream) {
    if (!c) return ES_EINVAL;
    if (!c->have_tables) return fail(c, ES_ESTATE, "load tables before the batch");
    if (!theta || batch < 1 || (mem != ES_MEM_HOST && mem != ES_MEM_DEVICE))
        return fail(c, ES_EINVAL, "bad batch arguments");
    cudaSetDevice(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    es_status s = alloc_forward(c, batch);
    if (s != ES_OK) return s;
    const cudaMemcpyKind dir = mem == ES_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaMemcpyAsync(const_cast<double *>(c->w.theta_user), theta,
                                    sizeof(double) * (size_t)batch * c->m.nfree, dir, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "theta copy");
    std::vector<int32_t> kh(batch, ES_KIND_TRANSMISSION);
    if (kind) {
        if (mem == ES_MEM_HOST) {
            std::memcpy(kh.data(), kind, sizeof(int32_t) * batch);
        } else {
            e = cudaMemcpyAsync(kh.data(), kind, sizeof(int32_t) * batch, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return cuda_fail(c, e, "kind copy");
        }
    }
    int nk[2] = {0, 0};
    for (int b = 0; b < batch; ++b) {
        if (kh[b] != ES_KIND_TRANSMISSION && kh[b] != ES_KIND_EMISSION)
            return fail(c, ES_EINVAL, "kind must be 0 (transmission) or 1 (emission)");
        nk[kh[b]]++;
    }
    e = cudaMemcpyAsync(c->w.kind, kh.data(), sizeof(int32_t) * batch, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && mem == ES_MEM_HOST) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && kind && mem == ES_MEM_DEVICE) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "kind upload");
    if (mem == ES_MEM_DEVICE && !kind) {
        e = cudaStreamSynchronize(st);   // the host vector kh goes out of scope
        if (e != cudaSuccess) return cuda_fail(c, e, "kind upload");
    }
    if (batch != c->batch || nk[0] != c->n_kind[0] || nk[1] != c->n_kind[1]) ++c->graph_epoch;
    c->batch = batch;
    c->n_kind[0] = nk[0];
    c->n_kind[1] = nk[1];
    return ES_OK;
}

namespace {

es_status copy_out(es_ctx *c, void *dst, const void *src, size_t bytes, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? ES_OK : cuda_fail(c, e, "result copy");
}

// Host-buffer calls synchronise here and report a kernel that gave up on a
// bounded wait as ES_ETIMEOUT; device-buffer calls return at once (their
// samples carry ES_FLAG_TIMEOUT and ln L = -1e300 instead).
es_status finish(es_ctx *c, int mem, cudaStream_t st) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && mem == ES_MEM_HOST) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel execution");
    if (mem == ES_MEM_HOST && *c->h_err)
        return fail(c, ES_ETIMEOUT, "a tensor-core kernel gave up on a bounded wait; every sample of the call "
                                    "is flagged invalid (ES_FLAG_TIMEOUT)");
    return ES_OK;
}

}  // namespace

es_status es_forward(es_ctx *c, float *spectrum, double *binned, double *lnl, int mem, es_stream_t stream) {
    if (!c) return ES_EINVAL;
    if (mem != ES_MEM_HOST && mem != ES_MEM_DEVICE) return fail(c, ES_EINVAL, "bad mem");
    es_status s = ready(c);
    if (s != ES_OK) return s;
    cudaSetDevice(c->device);
    if ((s = prepare(c, false)) != ES_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int B = c->batch;
    float *d_spec = spectrum;
    double *d_bin = binned, *d_lnl = lnl;
    std::vector<void *> tmp;
    if (mem == ES_MEM_HOST) {
        d_lnl = lnl ? c->d_lnl : nullptr;
        if (spectrum && (s = dalloc(c, tmp, &d_spec, (size_t)B * c->m.N)) != ES_OK) return s;
        if (binned && (s = dalloc(c, tmp, &d_bin, (size_t)B * c->m.nbins)) != ES_OK) { free_all(c, tmp); return s; }
    }
    s = run_forward(c, false, d_spec, d_bin, d_lnl, st);
    if (s == ES_OK && mem == ES_MEM_HOST) {
        if (lnl) s = copy_out(c, lnl, d_lnl, sizeof(double) * B, st);
        if (s == ES_OK && spectrum) s = copy_out(c, spectrum, d_spec, sizeof(float) * (size_t)B * c->m.N, st);
        if (s == ES_OK && binned) s = copy_out(c, binned, d_bin, sizeof(double) * (size_t)B * c->m.nbins, st);
    }
    if (s == ES_OK) s = finish(c, mem, st);
    if (!tmp.empty()) {
        cudaStreamSynchronize(st);
        free_all(c, tmp);
    }
    return s;
}

es_status es_loglike(es_ctx *c, double *lnl, int mem, es_stream_t stream) {
    if (!c) return ES_EINVAL;
    if (!lnl) return fail(c, ES_EINVAL, "lnL pointer is NULL");
    if (mem != ES_MEM_HOST && mem != ES_MEM_DEVICE) return fail(c, ES_EINVAL, "bad mem");
    es_status s = ready(c);
    if (s != ES_OK) return s;
    cudaSetDevice(c->device);
    if ((s = prepare(c, false)) != ES_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = launch_or_replay(c, c->graph_ll, st,
                         [&](cudaStream_t q) { return run_forward(c, false, nullptr, nullptr, c->d_lnl, q); });
    if (s != ES_OK) return s;
    cudaError_t e = cudaMemcpyAsync(lnl, c->d_lnl, sizeof(double) * c->batch,
                                    mem == ES_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "lnL copy");
    return finish(c, mem, st);
}

// Forward + adjoint into the context's buffers (lnL in d_lnl, gradient in w.grad).
es_status enqueue_forward_backward(es_ctx *c, cudaStream_t st) {
    const int B = c->batch;
    const Model &m = c->m;
    Work w = c->w;
    w.B = B;
    const size_t L = m.L, S = m.S;
    cudaMemsetAsync(w.red, 0, sizeof(double) * B * L * N_RED, st);
    cudaMemsetAsync(w.qtot, 0, sizeof(double) * B * S, st);
    cudaMemsetAsync(w.zbar, 0, sizeof(double) * B * L, st);
    cudaMemsetAsync(w.areabar, 0, sizeof(double) * B * L, st);
    cudaMemsetAsync(w.levbar, 0, sizeof(double) * B * (L + 1), st);
    cudaMemsetAsync(w.drbar, 0, sizeof(double) * B * L, st);
    cudaMemsetAsync(w.lbar, 0, sizeof(float) * B * L * L, st);
    cudaMemsetAsync(w.cloud_dbar, 0, sizeof(double) * B * L, st);
    cudaMemsetAsync(w.cloud_pbar, 0, sizeof(double) * B * N_CG, st);
    es_status s = run_forward(c, true, nullptr, nullptr, c->d_lnl, st, false);
    if (s != ES_OK) return s;
    int launches = (int)c->last_launches;
    const Hook &h = c->hook;
    const es_ctx::Shape *sh = c->shape;
    if (eaa_path(c)) {
        if (c->n_kind[0]) {
            const es_ctx::Shape &x = sh[es_ctx::FUSED_TRANS_BWD];
            launches += launch_trans_fused_backward(m, w, x.chunk, x.sample_major, st, h);
        }
        launches += launch_eaa_backward(m, w, c->eaa_scr, st, h);
    } else if (c->n_kind[0] && c->n_kind[1]) {
        const es_ctx::Shape &x = sh[es_ctx::FUSED_MIXED_BWD];
        launches += launch_mixed_fused_backward(m, w, x.chunk, x.sample_major, st, h);
    } else if (c->n_kind[0]) {
        const es_ctx::Shape &x = sh[es_ctx::FUSED_TRANS_BWD];
        launches += launch_trans_fused_backward(m, w, x.chunk, x.sample_major, st, h);
    } else if (c->n_kind[1]) {
        const es_ctx::Shape &x = sh[es_ctx::FUSED_EMIS_BWD];
        launches += launch_emis_fused_backward(m, w, x.chunk, x.sample_major, st, h);
    }
    launches += launch_setup_backward(m, w, c->d_lnl, st, h);
    post_status(c, st);
    c->last_launches = launches;
    return check_launch(c, "backward launch");
}

es_status es_forward_backward(es_ctx *c, double *lnl, double *grad, int mem, es_stream_t stream) {
    if (!c) return ES_EINVAL;
    if (mem != ES_MEM_HOST && mem != ES_MEM_DEVICE) return fail(c, ES_EINVAL, "bad mem");
    es_status s = ready(c);
    if (s != ES_OK) return s;
    cudaSetDevice(c->device);
    if ((s = prepare(c, true)) != ES_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = launch_or_replay(c, c->graph_fb, st, [&](cudaStream_t q) { return enqueue_forward_backward(c, q); });
    if (s != ES_OK) return s;
    const int B = c->batch;
    const cudaMemcpyKind dir = mem == ES_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    cudaError_t e = cudaSuccess;
    if (lnl) e = cudaMemcpyAsync(lnl, c->d_lnl, sizeof(double) * B, dir, st);
    if (e == cudaSuccess && grad)
        e = cudaMemcpyAsync(grad, c->w.grad, sizeof(double) * (size_t)B * c->m.nfree, dir, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "result copy");
    return finish(c, mem, st);
}

es_status es_autotune(es_ctx *c, es_stream_t stream) {
    if (!c) return ES_EINVAL;
    es_status s = ready(c);
    if (s != ES_OK) return s;
    cudaSetDevice(c->device);
    if ((s = prepare(c, true)) != ES_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // one full pass with the built-in shapes, so that the forward's stores the
    // adjoint kernels read (exp(-tau), I_toa, dbar) are valid while they are timed
    for (auto &x : c->shape) x = es_ctx::Shape{};
    if ((s = enqueue_forward_backward(c, st)) != ES_OK) return s;
    Work w = c->w;
    w.B = c->batch;
    const Hook none{};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_it = [&](auto &&launch) {
        float best = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, st);
            launch();
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        return best;
    };
    // the fastest (work-item size, item order) of one kernel
    auto tune = [&](int which, const std::vector<int> &sizes, auto &&launch) {
        float best = 1e30f;
        for (int order = 0; order < 2; ++order)
            for (int ch : sizes) {
                const float ms = time_it([&]() { launch(ch, order); });
                if (ms < best) {
                    best = ms;
                    c->shape[which] = es_ctx::Shape{ch, order};
                }
            }
    };
    const Model &m = c->m;
    if (eaa_path(c)) {   // the delta-EAA kernels have fixed shapes: only a transmission part is tuned
        if (c->n_kind[0]) {
            tune(es_ctx::FUSED_TRANS_FWD, {2, 4, 8, 16, 32, 64, 128},
                 [&](int ch, int o) { launch_trans_fused_forward(m, w, true, ch, o, st, none); });
            tune(es_ctx::FUSED_TRANS_BWD, {2, 4, 8, 16, 32, 64},
                 [&](int ch, int o) { launch_trans_fused_backward(m, w, ch, o, st, none); });
        }
    } else if (c->n_kind[0] && c->n_kind[1]) {
        const std::vector<int> win = {4, 8, 16, 32, 64};
        tune(es_ctx::FUSED_MIXED_FWD, win,
             [&](int ch, int o) { launch_mixed_fused_forward(m, w, true, ch, o, st, none); });
        tune(es_ctx::FUSED_MIXED_BWD, win, [&](int ch, int o) { launch_mixed_fused_backward(m, w, ch, o, st, none); });
    } else if (c->n_kind[0]) {
        tune(es_ctx::FUSED_TRANS_FWD, {2, 4, 8, 16, 32, 64, 128},
             [&](int ch, int o) { launch_trans_fused_forward(m, w, true, ch, o, st, none); });
        tune(es_ctx::FUSED_TRANS_BWD, {2, 4, 8, 16, 32, 64},
             [&](int ch, int o) { launch_trans_fused_backward(m, w, ch, o, st, none); });
    } else if (c->n_kind[1]) {
        tune(es_ctx::FUSED_EMIS_FWD, {1, 2, 4, 8, 16},
             [&](int ch, int o) { launch_emis_fused_forward(m, w, true, ch, o, st, none); });
        tune(es_ctx::FUSED_EMIS_BWD, {1, 2, 4, 8, 16},
             [&](int ch, int o) { launch_emis_fused_backward(m, w, ch, o, st, none); });
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ++c->graph_epoch;
    return check_launch(c, "autotune");
}

es_status es_set_graphs(es_ctx *c, int on) {
    if (!c) return ES_EINVAL;
    c->use_graph = on != 0;
    ++c->graph_epoch;
    return ES_OK;
}

es_status es_set_memory_limit(es_ctx *c, uint64_t bytes) {
    if (!c) return ES_EINVAL;
    c->mem_limit = (size_t)bytes;
    return ES_OK;
}

es_status es_set_test_hooks(es_ctx *c, int hooks) {
    if (!c) return ES_EINVAL;
    if (hooks & ~ES_TEST_WAIT_TIMEOUT) return fail(c, ES_EINVAL, "unknown test hook");
    const bool wt = (hooks & ES_TEST_WAIT_TIMEOUT) != 0;
    c->m.wait_test = wt ? 1 : 0;
    c->m.wait_polls = wt ? WAIT_POLLS_TEST : WAIT_POLLS;
    ++c->graph_epoch;   // the model is baked into captured graphs
    return ES_OK;
}

es_status es_get_flags(es_ctx *c, int32_t *flags, int mem, es_stream_t stream) {
    if (!c) return ES_EINVAL;
    if (!flags || c->batch <= 0) return fail(c, ES_EINVAL, "no batch or NULL flags");
    cudaSetDevice(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(flags, c->w.flags, sizeof(int32_t) * c->batch,
                                    mem == ES_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && mem == ES_MEM_HOST) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? ES_OK : cuda_fail(c, e, "flags copy");
}

int64_t es_query(const es_ctx *c, int key) {
    if (!c) return -1;
    switch (key) {
        case 0: return c->m.N;
        case 1: return c->m.nbins;
        case 2: return c->m.nfree;
        case 3: return c->batch;
        case 4: return c->m.L;
        case 5: return c->m.S;
        case 6: return (int64_t)c->dev_bytes;
        case 7: return c->last_launches;
        case 8: return c->shape[es_ctx::FUSED_TRANS_FWD].chunk;
        case 9: return c->shape[es_ctx::FUSED_TRANS_BWD].chunk;
        case 12: return c->shape[es_ctx::FUSED_EMIS_FWD].chunk;
        case 13: return c->shape[es_ctx::FUSED_EMIS_BWD].chunk;
        case 14: return c->shape[es_ctx::FUSED_MIXED_FWD].chunk;
        case 15: return c->shape[es_ctx::FUSED_MIXED_BWD].chunk;
        case 16: {
            int64_t bits = 0;
            for (int k = 0; k < es_ctx::N_FUSED; ++k) bits |= (int64_t)(c->shape[k].sample_major ? 1 : 0) << k;
            return bits;
        }
        case 10: return c->use_graph ? 1 : 0;
        case 11: {
            int v = -1;
            if (!c->w.err || cudaMemcpy(&v, c->w.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
            return v;
        }
        case 17: {   // bytes of raw table and CIA rows the one-vector opacity stage read
            if (!c->last_one_vector || !c->w.arows) return 0;
            int r[2] = {0, 0};
            if (cudaMemcpy(r, c->w.arows, sizeof(r), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
            const int64_t esz = c->m.bf16 ? 2 : 4;
            return ((int64_t)r[0] * esz + (int64_t)r[1] * 4) * c->m.N;
        }
        default: return -1;
    }
}

es_status es_set_profiling(es_ctx *c, int on) {
    if (!c) return ES_EINVAL;
    cudaSetDevice(c->device);
    prof_resolve(c);
    c->prof.clear();
    c->prof_on = on != 0;
    c->hook = Hook{};
    if (c->prof_on) {
        c->hook.ctx = c;
        c->hook.begin = prof_begin;
        c->hook.end = prof_end;
    }
    return ES_OK;
}

es_status es_get_profile(es_ctx *c, int index, char *name, int name_len, double *total_ms, int64_t *launches) {
    if (!c) return ES_EINVAL;
    cudaSetDevice(c->device);
    prof_resolve(c);
    if (index < 0 || index >= (int)c->prof.size()) return fail(c, ES_EINVAL, "no such profile entry");
    const auto &e = c->prof[index];
    if (name && name_len > 0) {
        std::strncpy(name, e.name.c_str(), (size_t)name_len - 1);
        name[name_len - 1] = 0;
    }
    if (total_ms) *total_ms = e.ms;
    if (launches) *launches = e.n;
    return ES_OK;
}

const char *es_last_error(const es_ctx *c) { return c ? c->err.c_str() : "NULL context"; }

void es_destroy(es_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    free_all(c, c->bwd_bufs);
    free_all(c, c->work_bufs);
    free_all(c, c->data_bufs);
    free_all(c, c->grid_bufs);
    free_all(c, c->table_bufs);
    free_all(c, c->model_bufs);
    drop_graph(c->graph_fb);
    drop_graph(c->graph_ll);
    if (c->gstream) {
        cudaStreamSynchronize(c->gstream);
        cudaStreamDestroy(c->gstream);
        cudaEventDestroy(c->ev_fork);
        cudaEventDestroy(c->ev_join);
    }
    dev_free(c, c->w.ymod);
    dev_free(c, c->w.itop);
    dev_free(c, c->w.estore);
    dev_free(c, c->w.ext);
    dev_free(c, c->eaa_scr);
    if (c->h_err) cudaFreeHost(c->h_err);
    prof_resolve(c);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
}

}  // extern "C"
