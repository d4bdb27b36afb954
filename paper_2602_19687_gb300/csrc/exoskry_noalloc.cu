// es_loglike_noalloc: the log-likelihood of a small batch with every piece of
// per-call device workspace taken from one fixed-size array that is part of
// the library image, so the call itself never allocates device memory.
//
// Who needs this: callers that must not call cudaMalloc on the hot path, for
// example a host framework that owns all device memory through its own pool
// and forbids other allocations (custom operators of array frameworks), or a
// long-running sampler that has to be sure it cannot hit an out-of-memory
// error in the middle of a run.
//
// The array (NOALLOC_SCRATCH_BYTES, 32 MiB) exists on every GPU that loads
// the library, from module load until the process exits. Every call on a GPU
// uses the same array and leaves the last call's contents behind; two calls
// that overlap on the GPU (different streams, or different host threads)
// race on it and must be serialised by the caller.
#include <mutex>

#include "context.cuh"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;

// workspace of es_loglike_noalloc; host code may only use the address
// obtained from cudaGetSymbolAddress, never the name itself
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_scratch_mu;
unsigned char *g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device (looked up once
// per device; the first call on a device must not happen during capture).
cudaError_t scratch_address(int device, unsigned char **out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Carver {
    unsigned char *base;
    size_t used = 0;
    template <class T>
    T *take(size_t count) {
        used = (used + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + used) : nullptr;
        used += (count ? count : 1) * sizeof(T);
        return p;
    }
};

// Lay out the forward workspace of a batch of B vectors; returns bytes needed.
size_t carve(const es::Model &m, int B, unsigned char *base, es::Work &w, int **kind_slot) {
    Carver c{base};
    const size_t L = m.L, S = m.S, N = m.N;
    w.B = B;
    w.theta = c.take<double>((size_t)B * m.nfull);
    *kind_slot = c.take<int>(B);
    w.flags = c.take<int>(B);
    w.err = c.take<int>(1);
    w.t_lay = c.take<double>(B * L);
    w.t_lev = c.take<double>(B * (L + 1));
    w.r_lev = c.take<double>(B * (L + 1));
    w.xs = c.take<double>(B * (S + 2));
    w.n_lay = c.take<double>(B * L);
    w.rc = c.take<double>(B);
    w.base = c.take<double>(B);
    w.scale = c.take<double>(B);
    w.lmat = c.take<float>(B * L * L);
    w.area = c.take<float>(B * L);
    w.dr = c.take<float>(B * L);
    w.it = c.take<int>(B * L);
    w.gt = c.take<float>(B * L);
    w.wtr = c.take<float>(B * L);
    w.itc = c.take<int>(B * L);
    w.wtc = c.take<float>(B * L);
    w.gtc = c.take<float>(B * L);
    w.ccia = c.take<float>(B * L * 2);
    w.ray = c.take<float>(B * L);
    if (m.cloud_kind == ES_CLOUD_KH18) {   // non-grey cloud: C_l, D_i and the g(nu) constants
        w.cloud_c = c.take<float>(B * L);
        w.cloud_d = c.take<float>(B * L);
        w.cloud_g = c.take<float>((size_t)B * es::N_CG);
    }
    w.spec = c.take<float>((size_t)B * N);
    w.ymod = c.take<double>((size_t)B * m.nbins);
    w.lnl = c.take<double>(B);
    w.misc = c.take<double>((size_t)B * 4);
    return c.used;
}

es_status fail(es_ctx *c, es_status s, const std::string &msg) {
    c->err = msg;
    return s;
}

}  // namespace

extern "C" es_status es_loglike_noalloc(es_ctx *c, const double *theta, const int32_t *kind, int batch,
                                        double *lnl, es_stream_t stream) {
    if (!c) return ES_EINVAL;
    if (!theta || !lnl || batch < 1) return fail(c, ES_EINVAL, "es_loglike_noalloc: NULL theta/lnL or batch < 1");
    if (!c->have_tables) return fail(c, ES_ESTATE, "tables not loaded");
    if (!c->have_grid) return fail(c, ES_ESTATE, "instrument grid not set");
    if (!c->have_data[ES_KIND_TRANSMISSION] || (kind && !c->have_data[ES_KIND_EMISSION]))
        return fail(c, ES_ESTATE, "es_loglike_noalloc needs transmission data, and emission data when kind is given");
    if (c->device < 0 || c->device >= MAX_DEVICES) return fail(c, ES_EINVAL, "device ordinal too large");
    if (kind && c->m.emis_solver == ES_RT_DELTA_EAA)
        return fail(c, ES_EINVAL, "es_loglike_noalloc: the delta-EAA emission solver needs es_loglike");
    es::Work w{};
    int *kind_slot = nullptr;
    const size_t need = carve(c->m, batch, nullptr, w, &kind_slot);
    if (need > NOALLOC_SCRATCH_BYTES)
        return fail(c, ES_EINVAL,
                    "es_loglike_noalloc: batch of " + std::to_string(batch) + " needs " + std::to_string(need) +
                        " bytes of workspace, more than the fixed " + std::to_string(NOALLOC_SCRATCH_BYTES) +
                        " bytes; use es_set_batch + es_loglike or a smaller batch");
    cudaError_t e = cudaSetDevice(c->device);
    unsigned char *base = nullptr;
    if (e == cudaSuccess) e = scratch_address(c->device, &base);
    if (e != cudaSuccess) return fail(c, ES_ECUDA, std::string("scratch address: ") + cudaGetErrorString(e));
    carve(c->m, batch, base, w, &kind_slot);
    w.theta_user = theta;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (kind) {
        w.kind = const_cast<int *>(reinterpret_cast<const int *>(kind));
    } else {
        w.kind = kind_slot;   // all transmission (ES_KIND_TRANSMISSION == 0)
        e = cudaMemsetAsync(kind_slot, 0, sizeof(int) * (size_t)batch, st);
        if (e != cudaSuccess) return fail(c, ES_ECUDA, std::string("kind fill: ") + cudaGetErrorString(e));
    }
    e = cudaMemsetAsync(w.err, 0, sizeof(int), st);
    if (e != cudaSuccess) return fail(c, ES_ECUDA, std::string("status word: ") + cudaGetErrorString(e));
    const es::Hook none{};
    int launches = 0;
    launches += es::launch_setup(c->m, w, st, none);
    // (the kinds are device data here: one kernel per kind, each skipping the other kind's items)
    launches += es::launch_trans_fused_forward(c->m, w, false, 0, 0, st, none);
    if (kind) {
        launches += es::launch_emis_fused_forward(c->m, w, false, 0, 0, st, none);
    }
    launches += es::launch_bins(c->m, w, false, nullptr, nullptr, lnl, st, none);
    c->last_launches = launches;
    e = cudaGetLastError();
    return e == cudaSuccess ? ES_OK : fail(c, ES_ECUDA, std::string("es_loglike_noalloc: ") + cudaGetErrorString(e));
}
