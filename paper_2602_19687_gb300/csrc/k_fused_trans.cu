// Transmission-only persistent kernels over (sample, wavenumber-chunk) work
// items of transmission samples: the tile engines of fused_trans.cuh (Sect. 3
// opacities -> Sect. 4 chord optical depth and transit depth, and their
// adjoint), items in chunk-major or sample-major order.
#include <algorithm>

#include "fused_trans.cuh"

namespace es {

namespace {

// Block shapes of the transmission-only kernels (measured at B = 1024): the
// forward with 24 warps (6 layer groups x 4 wavenumber quarters, 78-80
// registers) per SM; the adjoint with 16 warps, its coefficients staged
// per warp through shared memory, L split in alpha_bar = L^T tau_bar.
constexpr int FWD_WARPS = 24, BWD_WARPS = 16;
constexpr bool BWD_STAGE = true, BWD_LSPLIT = true;
using FwdSmem = TransFwdSmemT<FWD_WARPS>;
using BwdSmem = TransBwdSmemT<BWD_WARPS, BWD_STAGE, BWD_LSPLIT>;

template <int SPL, bool STORE_E, bool CLOUD>
__global__ void __launch_bounds__(FWD_WARPS * 32, 1) k_trans_fwd(Model m, Work w, int chunk_tiles, int sample_major) {
    extern __shared__ float4 smem4[];
    FwdSmem &sm = *reinterpret_cast<FwdSmem *>(smem4);
    TransFwdEngine<SPL, STORE_E, CLOUD, FWD_WARPS> e(m, w, sm);
    e.setup();
    const int ntiles = (m.N + FT2 - 1) / FT2;
    const ItemOrder order{w.B, (ntiles + chunk_tiles - 1) / chunk_tiles, sample_major};
    int cur_b = -1;
    for (long long item = blockIdx.x; item < order.total() && !e.abort; item += gridDim.x) {
        int c, b;
        order.at(item, c, b);
        if (w.kind[b] != ES_KIND_TRANSMISSION) continue;
        if (b != cur_b) {
            e.drain();   // the previous sample's tiles, before its constants are replaced
            if (sm.abort) {
                e.abort = true;
                break;
            }
            tc_fence_before();
            __syncthreads();
            stage_sample(m, w, b, sm.sc, RUN_COST_FWD, SBO_NU, FWD_WARPS / 4);
            e.stage_operands(b);
            cur_b = b;
            fence_async_smem();
            __syncthreads();
        }
        e.tiles(b, c * chunk_tiles, min(ntiles, (c + 1) * chunk_tiles));
    }
    e.teardown();
}

// The chord product, transit depth and exp(-tau) store of the one-vector
// path: the forward's tiles with the extinction read from the buffer that
// k_trans_alpha wrote (no interpolation, no layer constants).
template <bool STORE_E, bool CLOUD>
__global__ void __launch_bounds__(FWD_WARPS * 32, 1) k_trans_chord(Model m, Work w, int chunk_tiles) {
    extern __shared__ float4 smem4[];
    FwdSmem &sm = *reinterpret_cast<FwdSmem *>(smem4);
    TransFwdEngine<4, STORE_E, CLOUD, FWD_WARPS> e(m, w, sm);
    e.setup();
    const int ntiles = (m.N + FT2 - 1) / FT2;
    const ItemOrder order{w.B, (ntiles + chunk_tiles - 1) / chunk_tiles, 0};
    int cur_b = -1;
    for (long long item = blockIdx.x; item < order.total() && !e.abort; item += gridDim.x) {
        int c, b;
        order.at(item, c, b);
        if (w.kind[b] != ES_KIND_TRANSMISSION) continue;
        if (b != cur_b) {
            e.drain();
            if (sm.abort) {
                e.abort = true;
                break;
            }
            tc_fence_before();
            __syncthreads();
            e.stage_operands(b);
            cur_b = b;
            fence_async_smem();
            __syncthreads();
        }
        e.tiles_from(b, c * chunk_tiles, min(ntiles, (c + 1) * chunk_tiles), w.ext);
    }
    e.teardown();
}

template <int SPL, bool CLOUD>
__global__ void __launch_bounds__(BWD_WARPS * 32, 1) k_trans_bwd(Model m, Work w, int chunk_tiles, int sample_major) {
    extern __shared__ float4 smem4[];
    BwdSmem &sm = *reinterpret_cast<BwdSmem *>(smem4);
    TransBwdEngine<SPL, CLOUD, BWD_WARPS, BWD_STAGE, BWD_LSPLIT> e(m, w, sm);
    e.setup();
    const int ntiles = (m.N + BT - 1) / BT;
    const ItemOrder order{w.B, (ntiles + chunk_tiles - 1) / chunk_tiles, sample_major};
    const long long total = order.total();
    // the block's next transmission item after `item` that the adjoint runs
    auto next_item = [&](long long item, int &nb, int &nt) {
        nb = -1;
        for (long long nx = item + gridDim.x; nx < total; nx += gridDim.x) {
            int c, b;
            order.at(nx, c, b);
            if (w.kind[b] == ES_KIND_TRANSMISSION && !w.flags[b]) {
                nb = b;
                nt = c * chunk_tiles;
                return;
            }
        }
    };
    if (blockIdx.x < total) {
        int c, b;
        order.at(blockIdx.x, c, b);
        e.prefetch_tile(b, c * chunk_tiles);
    }
    int cur_b = -1;
    for (long long item = blockIdx.x; item < total && !e.abort; item += gridDim.x) {
        int c, b;
        order.at(item, c, b);
        if (w.kind[b] != ES_KIND_TRANSMISSION || w.flags[b]) continue;
        if (b != cur_b) {
            if (cur_b >= 0) {
                e.wait_lbar();
                e.flush(cur_b);
            }
            tc_fence_before();
            __syncthreads();
            stage_sample(m, w, b, sm.sc, RUN_COST_BWD, SBO_NU, BWD_WARPS / 4);
            e.stage_operands(b);
            cur_b = b;
            fence_async_smem();
            __syncthreads();
        }
        int nb, nt = 0;
        next_item(item, nb, nt);
        e.tiles(b, c * chunk_tiles, min(ntiles, (c + 1) * chunk_tiles), nb, nt);
    }
    if (cur_b >= 0 && !e.abort) {
        e.wait_lbar();
        e.flush(cur_b);
    }
    e.teardown();
}

size_t fwd_smem() { return sizeof(FwdSmem); }
size_t bwd_smem() { return sizeof(BwdSmem); }

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace

// Tiles of `tile` wavenumbers per work item: up to 16 (amortises staging the
// sample), fewer when the batch is small so that every resident block gets items.
int chunk_tiles(const Model &m, int B, int blocks, int tile) {
    const int ntiles = (m.N + tile - 1) / tile;
    long long c = ((long long)ntiles * B) / (4LL * blocks);
    return (int)std::max<long long>(1, std::min<long long>(16, c));
}

int launch_trans_fused_forward(const Model &m, const Work &w, bool store_e, int chunk_req, int sample_major,
                               cudaStream_t st, const Hook &h) {
    const int ntiles = (m.N + FT2 - 1) / FT2;
    const int chunk = chunk_req > 0 ? chunk_req : chunk_tiles(m, w.B, sm_count(), FT2);
    const long long items = (long long)w.B * ((ntiles + chunk - 1) / chunk);
    const int grid = (int)std::min<long long>(items, (long long)sm_count());
    const size_t sm = fwd_smem();
#define ES_FWD1(SPL, SE, CL)                                                                    \
    do {                                                                                        \
        cudaFuncSetAttribute(k_trans_fwd<SPL, SE, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        ES_LAUNCH(h, "k_trans_fwd", st, k_trans_fwd<SPL, SE, CL><<<grid, FWD_WARPS * 32, sm, st>>>(m, w, chunk, sample_major)); \
    } while (0)
#define ES_FWD(SPL, SE) \
    do { if (cloud) ES_FWD1(SPL, SE, true); else ES_FWD1(SPL, SE, false); } while (0)
    const bool cloud = m.cloud_kind == ES_CLOUD_KH18;
    const int spl = spl_for(m.S);
    if (spl == 2) { if (store_e) ES_FWD(2, true); else ES_FWD(2, false); }
    else if (spl == 4) { if (store_e) ES_FWD(4, true); else ES_FWD(4, false); }
    else { if (store_e) ES_FWD(8, true); else ES_FWD(8, false); }
#undef ES_FWD1
#undef ES_FWD
    return 1;
}

int launch_trans_chord_forward(const Model &m, const Work &w, bool store_e, cudaStream_t st, const Hook &h) {
    const int ntiles = (m.N + FT2 - 1) / FT2;
    const int chunk = chunk_tiles(m, w.B, sm_count(), FT2);
    const long long items = (long long)w.B * ((ntiles + chunk - 1) / chunk);
    const int grid = (int)std::min<long long>(items, (long long)sm_count());
    const size_t sm = fwd_smem();
#define ES_CHORD(SE, CL)                                                                        \
    do {                                                                                        \
        cudaFuncSetAttribute(k_trans_chord<SE, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        ES_LAUNCH(h, "k_trans_chord", st, k_trans_chord<SE, CL><<<grid, FWD_WARPS * 32, sm, st>>>(m, w, chunk)); \
    } while (0)
    const bool cloud = m.cloud_kind == ES_CLOUD_KH18;
    if (store_e) { if (cloud) ES_CHORD(true, true); else ES_CHORD(true, false); }
    else { if (cloud) ES_CHORD(false, true); else ES_CHORD(false, false); }
#undef ES_CHORD
    return 1;
}

int launch_trans_fused_backward(const Model &m, const Work &w, int chunk_req, int sample_major, cudaStream_t st,
                                const Hook &h) {
    const int ntiles = (m.N + BT - 1) / BT;
    const int chunk = chunk_req > 0 ? chunk_req : chunk_tiles(m, w.B, sm_count(), BT);
    const long long items = (long long)w.B * ((ntiles + chunk - 1) / chunk);
    const int grid = (int)std::min<long long>(items, (long long)sm_count());
    const size_t sm = bwd_smem();
#define ES_BWD1(SPL, CL)                                                                        \
    do {                                                                                        \
        cudaFuncSetAttribute(k_trans_bwd<SPL, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        ES_LAUNCH(h, "k_trans_bwd", st, k_trans_bwd<SPL, CL><<<grid, BWD_WARPS * 32, sm, st>>>(m, w, chunk, sample_major)); \
    } while (0)
#define ES_BWD(SPL) \
    do { if (cloud) ES_BWD1(SPL, true); else ES_BWD1(SPL, false); } while (0)
    const bool cloud = m.cloud_kind == ES_CLOUD_KH18;
    const int spl = spl_for(m.S);
    if (spl == 2) ES_BWD(2);
    else if (spl == 4) ES_BWD(4);
    else ES_BWD(8);
#undef ES_BWD
#undef ES_BWD1
    return 1;
}

}  // namespace es
