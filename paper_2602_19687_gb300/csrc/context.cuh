// The context object behind the opaque es_ctx handle (private to the library).
#pragma once

#include <string>
#include <unordered_map>
#include <vector>

#include "internal.cuh"

struct es_ctx {
    int device = 0;
    es_model_desc desc{};
    es::Model m{};
    es::Work w{};
    std::string err = "no error";
    std::vector<void *> model_bufs;   // freed on destroy
    std::vector<void *> table_bufs;   // replaced by es_load_tables
    std::vector<void *> grid_bufs;    // replaced by es_set_grid
    std::vector<void *> data_bufs;
    std::vector<void *> work_bufs;    // forward workspace
    std::vector<void *> bwd_bufs;     // adjoint workspace
    bool have_tables = false, have_grid = false, have_data[2] = {false, false};
    int cap_b = 0, cap_b_bwd = 0, batch = 0, n_kind[2] = {0, 0};
    // device bytes held by the context (every allocation: tables, grids, data,
    // workspace), the size of each allocation, and the limit (0: none)
    size_t dev_bytes = 0, mem_limit = 0;
    std::unordered_map<void *, size_t> dev_sizes;
    int *h_err = nullptr;             // pinned copy of the device status word, written at the end of every call
    int64_t last_launches = 0;
    bool last_one_vector = false;     // the last forward ran the one-vector path
    std::vector<double> y_host[2], s_host[2];
    std::vector<double> nu_host;      // FP64 wavenumber grid (bin membership)
    size_t ymod_cap = 0, alpha_cap = 0, estore_cap = 0;   // alpha_cap: the emission I_toa store
    size_t ext_cap = 0;               // the extinction buffer (one-vector path; delta-EAA emission)
    float *eaa_scr = nullptr;         // delta-EAA: the RT kernels' per-thread scratch array
    size_t eaa_scr_cap = 0;
    double *d_data = nullptr;         // [2][nbins] y_obs then sigma
    double *d_lnl = nullptr, *d_grad = nullptr;
    // per-kernel CUDA-event profiling
    struct ProfEntry { std::string name; double ms = 0.0; int64_t n = 0; };
    struct Pending { int entry; cudaEvent_t a, b; };
    bool prof_on = false;
    std::vector<ProfEntry> prof;
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> ev_pool;
    int open_entry = -1;
    cudaEvent_t open_ev = nullptr;
    es::Hook hook;
    // launch shapes of the fused kernels (es_autotune): work-item size (0: the
    // built-in heuristic) and item order, per kernel (FUSED_* indices)
    struct Shape { int chunk = 0, sample_major = 0; };
    enum { FUSED_TRANS_FWD, FUSED_TRANS_BWD, FUSED_EMIS_FWD, FUSED_EMIS_BWD, FUSED_MIXED_FWD, FUSED_MIXED_BWD,
           N_FUSED };
    Shape shape[N_FUSED];
    // CUDA-graph replay of es_loglike / es_forward_backward
    bool use_graph = true;
    int graph_epoch = 0;
    cudaStream_t gstream = nullptr;   // private stream the graphs run on
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;              // bumped whenever buffers or the batch shape change
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        int epoch = -1, calls = 0;
    } graph_fb, graph_ll;
};
