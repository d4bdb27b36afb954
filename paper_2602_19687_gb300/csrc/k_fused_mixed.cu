// One persistent kernel per direction for a batch that holds both
// transmission (Sect. 4) and emission (Sect. 5) samples. Work items are
// (sample, wavenumber window) pairs over every sample of the batch, in
// chunk-major order by default, so the blocks running at a time work on one
// window of the coefficient table, whichever kind their samples are: the
// transmission and emission items of a window share its lines in L2. A block
// runs an item of either kind with the same shared memory: the transmission
// engine's buffers (its layer constants, cloud constants, adjoint sums and
// coefficient staging are the emission engine's too) plus the emission
// levels. A window is `wtiles` 128-wavenumber transmission tiles, i.e.
// wtiles / 4 emission tiles of 512 wavenumbers (wtiles a multiple of 4).
#include <algorithm>

#include "fused_emis.cuh"
#include "fused_trans.cuh"

namespace es {

namespace {

struct MixedFwdSmem {
    TransFwdSmem t;
    EmisLevels lv;
};

struct MixedBwdSmem {
    TransBwdSmem t;
    EmisLevels lv;
};

static_assert(F2_THREADS == EM_THREADS && BW_THREADS == EM_THREADS && BW_WARPS == EM_WARPS,
              "the mixed kernels run both engines with one block shape");
static_assert(ET % FT2 == 0, "an emission tile spans whole transmission tiles");
constexpr int E_PER_W = ET / FT2;   // transmission tiles per emission tile (4)

template <int SPL, bool STORE, bool CLOUD>
__global__ void __launch_bounds__(F2_THREADS, 1) k_mixed_fwd(Model m, Work w, int wtiles, int sample_major) {
    extern __shared__ float4 smem4[];
    MixedFwdSmem &sm = *reinterpret_cast<MixedFwdSmem *>(smem4);
    TransFwdEngine<SPL, STORE, CLOUD> te(m, w, sm.t);
    te.setup();
    const EmisView v{&sm.t.sc, &sm.lv, sm.t.cg, nullptr, nullptr, nullptr, nullptr};
    const int ntiles_t = (m.N + FT2 - 1) / FT2, ntiles_e = (m.N + ET - 1) / ET, etiles = wtiles / E_PER_W;
    const ItemOrder order{w.B, (ntiles_t + wtiles - 1) / wtiles, sample_major};
    int cur_b = -1;
    for (long long item = blockIdx.x; item < order.total() && !te.abort; item += gridDim.x) {
        int c, b;
        order.at(item, c, b);
        const bool trans = w.kind[b] == ES_KIND_TRANSMISSION;
        if (b != cur_b) {
            te.drain();   // the transmission tiles in flight, before the shared constants are replaced
            if (sm.t.abort) {
                te.abort = true;
                break;
            }
            tc_fence_before();
            __syncthreads();
            stage_sample(m, w, b, sm.t.sc, RUN_COST_FWD, SBO_NU, F2_WARPS / 4);
            if (trans) te.stage_operands(b);
            else stage_levels<CLOUD>(m, w, b, v);
            cur_b = b;
            fence_async_smem();
            __syncthreads();
        }
        if (trans) te.tiles(b, c * wtiles, min(ntiles_t, (c + 1) * wtiles));
        else {
            // (the emission engine exists only on this branch: its constants do
            // not take registers while transmission tiles run)
            EmisFwdEngine<SPL, STORE, CLOUD> ee(m, w, v);
            ee.tiles(b, c * etiles, min(ntiles_e, (c + 1) * etiles));
        }
    }
    te.teardown();
}

template <int SPL, bool CLOUD>
__global__ void __launch_bounds__(BW_THREADS, 1) k_mixed_bwd(Model m, Work w, int wtiles, int sample_major) {
    extern __shared__ float4 smem4[];
    MixedBwdSmem &sm = *reinterpret_cast<MixedBwdSmem *>(smem4);
    TransBwdEngine<SPL, CLOUD> te(m, w, sm.t);
    te.setup();
    const EmisView v{&sm.t.sc, &sm.lv, sm.t.cg, sm.t.red, sm.t.qtot, sm.t.cpbar, &sm.t.stage[0][0]};
    // the emission engine is built on the branches that use it, so that its
    // constants take no registers while transmission tiles run
    using Emis = EmisBwdEngine<SPL, CLOUD>;
    const int ntiles_t = (m.N + FT2 - 1) / FT2, ntiles_e = (m.N + ET - 1) / ET, etiles = wtiles / E_PER_W;
    const ItemOrder order{w.B, (ntiles_t + wtiles - 1) / wtiles, sample_major};
    const long long total = order.total();
    // the block's next transmission item after `item` (its first tile is
    // prefetched to L2 during the current item's last tile)
    auto next_trans = [&](long long item, int &nb, int &nt) {
        nb = -1;
        for (long long nx = item + gridDim.x; nx < total; nx += gridDim.x) {
            int c, b;
            order.at(nx, c, b);
            if (w.flags[b]) continue;
            if (w.kind[b] == ES_KIND_TRANSMISSION) {
                nb = b;
                nt = c * wtiles;
            }
            return;
        }
    };
    if (blockIdx.x < total) {
        int c, b;
        order.at(blockIdx.x, c, b);
        if (w.kind[b] == ES_KIND_TRANSMISSION) te.prefetch_tile(b, c * wtiles);
    }
    int cur_b = -1;
    bool cur_trans = false;
    for (long long item = blockIdx.x; item < total && !te.abort; item += gridDim.x) {
        int c, b;
        order.at(item, c, b);
        if (w.flags[b]) continue;
        const bool trans = w.kind[b] == ES_KIND_TRANSMISSION;
        if (b != cur_b) {
            if (cur_b >= 0) {
                if (cur_trans) {
                    te.wait_lbar();
                    te.flush(cur_b);
                } else {
                    Emis(m, w, v).flush(cur_b);
                }
            }
            tc_fence_before();
            __syncthreads();
            if (trans) {
                stage_sample(m, w, b, sm.t.sc, RUN_COST_BWD, SBO_NU, BW_WARPS / 4);
                te.stage_operands(b);
            } else {
                stage_sample(m, w, b, sm.t.sc, RUN_COST_FWD, SBO_NU, BW_WARPS / 4);
                stage_levels<CLOUD>(m, w, b, v);
                Emis(m, w, v).reset();
            }
            cur_b = b;
            cur_trans = trans;
            fence_async_smem();
            __syncthreads();
        }
        if (trans) {
            int nb, nt = 0;
            next_trans(item, nb, nt);
            te.tiles(b, c * wtiles, min(ntiles_t, (c + 1) * wtiles), nb, nt);
        } else {
            Emis(m, w, v).tiles(b, c * etiles, min(ntiles_e, (c + 1) * etiles));
        }
    }
    if (cur_b >= 0 && !te.abort) {
        if (cur_trans) {
            te.wait_lbar();
            te.flush(cur_b);
        } else {
            Emis(m, w, v).flush(cur_b);
        }
    }
    te.teardown();
}

int sm_count_m() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace

size_t mixed_fwd_smem() { return sizeof(MixedFwdSmem); }
size_t mixed_bwd_smem() { return sizeof(MixedBwdSmem); }

// Window width in 128-wavenumber tiles: the transmission kernels' heuristic,
// rounded up to whole emission tiles.
int mixed_window(const Model &m, int B) {
    const int c = chunk_tiles(m, B, sm_count_m(), FT2);
    return std::max(E_PER_W, (c + E_PER_W - 1) / E_PER_W * E_PER_W);
}

int launch_mixed_fused_forward(const Model &m, const Work &w, bool store, int wtiles_req, int sample_major,
                               cudaStream_t st, const Hook &h) {
    const int ntiles = (m.N + FT2 - 1) / FT2;
    const int wt = wtiles_req > 0 ? std::max(E_PER_W, wtiles_req / E_PER_W * E_PER_W) : mixed_window(m, w.B);
    const long long items = (long long)w.B * ((ntiles + wt - 1) / wt);
    const int grid = (int)std::min<long long>(items, (long long)sm_count_m());
    const size_t sm = mixed_fwd_smem();
#define ES_MF1(SPL, SE, CL)                                                                     \
    do {                                                                                        \
        cudaFuncSetAttribute(k_mixed_fwd<SPL, SE, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        ES_LAUNCH(h, "k_mixed_fwd", st, k_mixed_fwd<SPL, SE, CL><<<grid, F2_THREADS, sm, st>>>(m, w, wt, sample_major)); \
    } while (0)
#define ES_MF(SPL, SE) \
    do { if (cloud) ES_MF1(SPL, SE, true); else ES_MF1(SPL, SE, false); } while (0)
    const bool cloud = m.cloud_kind == ES_CLOUD_KH18;
    const int spl = spl_for(m.S);
    if (spl == 2) { if (store) ES_MF(2, true); else ES_MF(2, false); }
    else if (spl == 4) { if (store) ES_MF(4, true); else ES_MF(4, false); }
    else { if (store) ES_MF(8, true); else ES_MF(8, false); }
#undef ES_MF
#undef ES_MF1
    return 1;
}

int launch_mixed_fused_backward(const Model &m, const Work &w, int wtiles_req, int sample_major, cudaStream_t st,
                                const Hook &h) {
    const int ntiles = (m.N + FT2 - 1) / FT2;
    const int wt = wtiles_req > 0 ? std::max(E_PER_W, wtiles_req / E_PER_W * E_PER_W) : mixed_window(m, w.B);
    const long long items = (long long)w.B * ((ntiles + wt - 1) / wt);
    const int grid = (int)std::min<long long>(items, (long long)sm_count_m());
    const size_t sm = mixed_bwd_smem();
#define ES_MB1(SPL, CL)                                                                         \
    do {                                                                                        \
        cudaFuncSetAttribute(k_mixed_bwd<SPL, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        ES_LAUNCH(h, "k_mixed_bwd", st, k_mixed_bwd<SPL, CL><<<grid, BW_THREADS, sm, st>>>(m, w, wt, sample_major)); \
    } while (0)
#define ES_MB(SPL) \
    do { if (cloud) ES_MB1(SPL, true); else ES_MB1(SPL, false); } while (0)
    const bool cloud = m.cloud_kind == ES_CLOUD_KH18;
    const int spl = spl_for(m.S);
    if (spl == 2) ES_MB(2);
    else if (spl == 4) ES_MB(4);
    else ES_MB(8);
#undef ES_MB
#undef ES_MB1
    return 1;
}

}  // namespace es
