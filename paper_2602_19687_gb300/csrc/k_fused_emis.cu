// Emission-only persistent kernels over (sample, wavenumber-chunk) work items
// of emission samples: the tile engines of fused_emis.cuh (Sect. 3 opacities
// -> Sect. 5 Schwarzschild integration, and its adjoint), items in
// chunk-major or sample-major order.
#include <algorithm>

#include "fused_emis.cuh"

namespace es {

namespace {

template <int SPL, bool STORE_I, bool CLOUD>
__global__ void __launch_bounds__(EM_THREADS, 1) k_emis_fwd(Model m, Work w, int chunk_tiles, int sample_major) {
    extern __shared__ float4 smem4[];
    EmisSmem &sm = *reinterpret_cast<EmisSmem *>(smem4);
    const EmisView v = emis_view(sm, nullptr);
    EmisFwdEngine<SPL, STORE_I, CLOUD> e(m, w, v);
    const int ntiles = (m.N + ET - 1) / ET;
    const ItemOrder order{w.B, (ntiles + chunk_tiles - 1) / chunk_tiles, sample_major};
    int cur_b = -1;
    for (long long item = blockIdx.x; item < order.total(); item += gridDim.x) {
        int c, b;
        order.at(item, c, b);
        if (w.kind[b] != ES_KIND_EMISSION) continue;
        if (b != cur_b) {
            __syncthreads();
            stage_sample(m, w, b, sm.sc, RUN_COST_FWD);
            stage_levels<CLOUD>(m, w, b, v);
            cur_b = b;
            __syncthreads();
        }
        e.tiles(b, c * chunk_tiles, min(ntiles, (c + 1) * chunk_tiles));
    }
}

template <int SPL, bool CLOUD>
__global__ void __launch_bounds__(EM_THREADS, 1) k_emis_bwd(Model m, Work w, int chunk_tiles, int sample_major) {
    extern __shared__ float4 smem4[];
    EmisSmem &sm = *reinterpret_cast<EmisSmem *>(smem4);
    const EmisView v = emis_view(sm, reinterpret_cast<unsigned char *>(smem4) + EM_STAGE_OFFSET);
    EmisBwdEngine<SPL, CLOUD> e(m, w, v);
    const int ntiles = (m.N + ET - 1) / ET;
    const ItemOrder order{w.B, (ntiles + chunk_tiles - 1) / chunk_tiles, sample_major};
    int cur_b = -1;
    for (long long item = blockIdx.x; item < order.total(); item += gridDim.x) {
        int c, b;
        order.at(item, c, b);
        if (w.kind[b] != ES_KIND_EMISSION || w.flags[b]) continue;
        if (b != cur_b) {
            if (cur_b >= 0) e.flush(cur_b);
            __syncthreads();
            stage_sample(m, w, b, sm.sc, RUN_COST_FWD);
            stage_levels<CLOUD>(m, w, b, v);
            e.reset();
            cur_b = b;
            __syncthreads();
        }
        e.tiles(b, c * chunk_tiles, min(ntiles, (c + 1) * chunk_tiles));
    }
    if (cur_b >= 0) e.flush(cur_b);
}

size_t emis_smem() { return sizeof(EmisSmem); }

int sm_count_e() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace

// 512-wavenumber tiles per work item: up to 8, fewer when the batch is small
// so that every resident block gets items.
int emis_chunk(const Model &m, int B) {
    const int ntiles = (m.N + ET - 1) / ET;
    long long c = ((long long)ntiles * B) / (4LL * sm_count_e());
    return (int)std::max<long long>(1, std::min<long long>(8, c));
}

int launch_emis_fused_forward(const Model &m, const Work &w, bool store_i, int chunk_req, int sample_major,
                              cudaStream_t st, const Hook &h) {
    const int ntiles = (m.N + ET - 1) / ET;
    const int chunk = chunk_req > 0 ? chunk_req : emis_chunk(m, w.B);
    const long long items = (long long)w.B * ((ntiles + chunk - 1) / chunk);
    const int grid = (int)std::min<long long>(items, (long long)sm_count_e());
    const size_t sm = emis_smem();
#define ES_EF1(SPL, SI, CL)                                                                     \
    do {                                                                                        \
        cudaFuncSetAttribute(k_emis_fwd<SPL, SI, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        ES_LAUNCH(h, "k_emis_fwd", st, k_emis_fwd<SPL, SI, CL><<<grid, EM_THREADS, sm, st>>>(m, w, chunk, sample_major)); \
    } while (0)
#define ES_EF(SPL, SI) \
    do { if (cloud) ES_EF1(SPL, SI, true); else ES_EF1(SPL, SI, false); } while (0)
    const bool cloud = m.cloud_kind == ES_CLOUD_KH18;
    const int spl = spl_for(m.S);
    if (spl == 2) { if (store_i) ES_EF(2, true); else ES_EF(2, false); }
    else if (spl == 4) { if (store_i) ES_EF(4, true); else ES_EF(4, false); }
    else { if (store_i) ES_EF(8, true); else ES_EF(8, false); }
#undef ES_EF
#undef ES_EF1
    return 1;
}

int launch_emis_fused_backward(const Model &m, const Work &w, int chunk_req, int sample_major, cudaStream_t st,
                               const Hook &h) {
    const int ntiles = (m.N + ET - 1) / ET;
    const int chunk = chunk_req > 0 ? chunk_req : emis_chunk(m, w.B);
    const long long items = (long long)w.B * ((ntiles + chunk - 1) / chunk);
    const int grid = (int)std::min<long long>(items, (long long)sm_count_e());
    const size_t sm = EM_STAGE_OFFSET + (size_t)EM_WARPS * STAGE_BYTES_PER_WARP;
#define ES_EB1(SPL, CL)                                                                         \
    do {                                                                                        \
        cudaFuncSetAttribute(k_emis_bwd<SPL, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        ES_LAUNCH(h, "k_emis_bwd", st, k_emis_bwd<SPL, CL><<<grid, EM_THREADS, sm, st>>>(m, w, chunk, sample_major)); \
    } while (0)
#define ES_EB(SPL) \
    do { if (cloud) ES_EB1(SPL, true); else ES_EB1(SPL, false); } while (0)
    const bool cloud = m.cloud_kind == ES_CLOUD_KH18;
    const int spl = spl_for(m.S);
    if (spl == 2) ES_EB(2);
    else if (spl == 4) ES_EB(4);
    else ES_EB(8);
#undef ES_EB
#undef ES_EB1
    return 1;
}

}  // namespace es
