// Transmission (Sect. 4): chord optical depth tau_i(nu) = sum_l L_il alpha_l(nu)
// with the path-length matrix L_il = P_il dr_l (Eq. P_1D, tau_trans =
// P . dtau_vert), and the transit depth
//   delta(nu) = base + sum_i A_i (1 - exp(-tau_i(nu))),
// A_i the annulus areas / R_*^2 and base = r_c^2 / R_*^2 (the spectrum
// buffer holds delta - base; the base is added in FP64 at binning).
// The adjoint gives tau_bar, alpha_bar = L^T tau_bar, the geometry adjoint
// L_bar = sum_nu tau_bar alpha^T and the area/base adjoints.
#include "internal.cuh"

namespace es {

namespace {

constexpr int TR_THREADS = 128;   // one wavenumber per thread
constexpr int CH = 16;            // rows per register chunk
constexpr int LB_THREADS = 256;   // L_bar kernel: 16 x 16 threads, 7 x 7 outputs each
constexpr int LB_BLK = 7;
constexpr int LB_NU = 32;         // wavenumbers staged per step
constexpr int LB_RANGE = 2048;    // wavenumbers per L_bar block

__host__ __device__ inline int round_up(int x, int a) { return (x + a - 1) / a * a; }

__device__ __forceinline__ float block_sum128(float v, float *scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncwarp();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int q = 0; q < TR_THREADS / 32; ++q) t += scratch[q];
    __syncthreads();
    return t;
}

// Stage L^T (Lt[l][i], i contiguous, zero-padded to Lp) and a column tile of
// `src` ([B][L][N] layout) for wavenumbers n0 + t.
__device__ void stage_tiles(const Model &m, const float *lmat_b, const float *src_b, int n0, float *Lt,
                            float *tile, bool transpose) {
    const int L = m.L, Lp = round_up(L, CH), N = m.N;
    for (int idx = threadIdx.x; idx < L * Lp; idx += TR_THREADS) {
        int r = idx / Lp, c = idx % Lp;
        float v = 0.f;
        if (c < L) v = transpose ? lmat_b[(size_t)c * L + r] : lmat_b[(size_t)r * L + c];
        Lt[idx] = v;
    }
    const int n = n0 + threadIdx.x;
    for (int l = 0; l < L; ++l) tile[l * TR_THREADS + threadIdx.x] = (n < N) ? src_b[(size_t)l * N + n] : 0.f;
}

// tau for one i-chunk: acc[u] = sum_{l} L_{i0+u, l} a_l (Lt transposed layout)
__device__ __forceinline__ void chunk_tau(const float *Lt, const float *tile, int Lp, int i0, int lmax,
                                          float acc[CH]) {
#pragma unroll
    for (int u = 0; u < CH; ++u) acc[u] = 0.f;
    for (int l = 0; l < lmax; ++l) {
        const float a = tile[l * TR_THREADS + threadIdx.x];
        const float4 *row = reinterpret_cast<const float4 *>(Lt + l * Lp + i0);
#pragma unroll
        for (int q = 0; q < CH / 4; ++q) {
            float4 v = row[q];
            acc[4 * q + 0] = fmaf(v.x, a, acc[4 * q + 0]);
            acc[4 * q + 1] = fmaf(v.y, a, acc[4 * q + 1]);
            acc[4 * q + 2] = fmaf(v.z, a, acc[4 * q + 2]);
            acc[4 * q + 3] = fmaf(v.w, a, acc[4 * q + 3]);
        }
    }
}

__global__ void __launch_bounds__(TR_THREADS) k_transit(Model m, Work w) {
    const int b = blockIdx.y;
    if (w.kind[b] != ES_KIND_TRANSMISSION) return;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const int L = m.L, Lp = round_up(L, CH), N = m.N;
    float *Lt = sm, *tile = sm + L * Lp, *ar = tile + L * TR_THREADS;
    const int n0 = blockIdx.x * TR_THREADS, n = n0 + threadIdx.x;
    stage_tiles(m, w.lmat + (size_t)b * L * L, w.alpha + (size_t)b * L * N, n0, Lt, tile, true);
    for (int i = threadIdx.x; i < Lp; i += TR_THREADS) ar[i] = (i < L) ? w.area[(size_t)b * L + i] : 0.f;
    __syncthreads();
    float atm = 0.f, acc[CH];
    for (int i0 = 0; i0 < L; i0 += CH) {
        chunk_tau(Lt, tile, Lp, i0, min(L, i0 + CH), acc);
#pragma unroll
        for (int u = 0; u < CH; ++u) atm = fmaf(ar[i0 + u], -expm1f(-acc[u]), atm);
    }
    if (n < N) w.spec[(size_t)b * N + n] = atm;
}

// tau_bar_i = dbar A_i exp(-tau_i); area_bar_i += sum dbar (1 - exp(-tau_i)).
__global__ void __launch_bounds__(TR_THREADS) k_transit_taubar(Model m, Work w) {
    const int b = blockIdx.y;
    if (w.kind[b] != ES_KIND_TRANSMISSION || w.flags[b]) return;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    __shared__ float scratch[TR_THREADS / 32];
    const int L = m.L, Lp = round_up(L, CH), N = m.N;
    float *Lt = sm, *tile = sm + L * Lp, *ar = tile + L * TR_THREADS;
    const int n0 = blockIdx.x * TR_THREADS, n = n0 + threadIdx.x;
    stage_tiles(m, w.lmat + (size_t)b * L * L, w.alpha + (size_t)b * L * N, n0, Lt, tile, true);
    for (int i = threadIdx.x; i < Lp; i += TR_THREADS) ar[i] = (i < L) ? w.area[(size_t)b * L + i] : 0.f;
    __syncthreads();
    const float db = (n < N) ? w.dbar[(size_t)b * N + n] : 0.f;
    float *tb = w.taubar + (size_t)b * L * N;
    float acc[CH];
    for (int i0 = 0; i0 < L; i0 += CH) {
        chunk_tau(Lt, tile, Lp, i0, min(L, i0 + CH), acc);
        for (int u = 0; u < CH && i0 + u < L; ++u) {
            const int i = i0 + u;
            float e = expf(-acc[u]);
            if (n < N) tb[(size_t)i * N + n] = db * ar[i] * e;
            float part = block_sum128(db * -expm1f(-acc[u]), scratch);
            if (threadIdx.x == 0 && part != 0.f) atomicAdd(w.areabar + (size_t)b * L + i, (double)part);
        }
    }
}

// alpha_bar_l = sum_{i >= l} L_il tau_bar_i
__global__ void __launch_bounds__(TR_THREADS) k_transit_abar(Model m, Work w) {
    const int b = blockIdx.y;
    if (w.kind[b] != ES_KIND_TRANSMISSION) return;
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const int L = m.L, Lp = round_up(L, CH), N = m.N;
    float *Lm = sm, *tile = sm + L * Lp;
    const int n0 = blockIdx.x * TR_THREADS, n = n0 + threadIdx.x;
    const bool bad = w.flags[b] != 0;
    if (!bad) stage_tiles(m, w.lmat + (size_t)b * L * L, w.taubar + (size_t)b * L * N, n0, Lm, tile, false);
    __syncthreads();
    float *ab = w.abar + (size_t)b * L * N;
    for (int l0 = 0; l0 < L; l0 += CH) {
        float acc[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) acc[u] = 0.f;
        if (!bad) {
            for (int i = l0; i < L; ++i) {
                const float t = tile[i * TR_THREADS + threadIdx.x];
                const float4 *row = reinterpret_cast<const float4 *>(Lm + i * Lp + l0);
#pragma unroll
                for (int q = 0; q < CH / 4; ++q) {
                    float4 v = row[q];
                    acc[4 * q + 0] = fmaf(v.x, t, acc[4 * q + 0]);
                    acc[4 * q + 1] = fmaf(v.y, t, acc[4 * q + 1]);
                    acc[4 * q + 2] = fmaf(v.z, t, acc[4 * q + 2]);
                    acc[4 * q + 3] = fmaf(v.w, t, acc[4 * q + 3]);
                }
            }
        }
        if (n < N)
            for (int u = 0; u < CH && l0 + u < L; ++u) ab[(size_t)(l0 + u) * N + n] = acc[u];
    }
}

// L_bar_il = sum_nu tau_bar_i(nu) alpha_l(nu) over a wavenumber range, then
// atomically added (FP64) into the per-sample matrix.
__global__ void __launch_bounds__(LB_THREADS) k_transit_lbar(Model m, Work w) {
    const int b = blockIdx.y;
    if (w.kind[b] != ES_KIND_TRANSMISSION || w.flags[b]) return;
    const int L = m.L, N = m.N;
    __shared__ float st[LB_NU][16 * LB_BLK + 1], sa[LB_NU][16 * LB_BLK + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i0 = ty * LB_BLK, l0 = tx * LB_BLK;
    float acc[LB_BLK][LB_BLK];
#pragma unroll
    for (int u = 0; u < LB_BLK; ++u)
#pragma unroll
        for (int v = 0; v < LB_BLK; ++v) acc[u][v] = 0.f;
    const float *tb = w.taubar + (size_t)b * L * N, *al = w.alpha + (size_t)b * L * N;
    const int nbeg = blockIdx.x * LB_RANGE, nend = min(N, nbeg + LB_RANGE);
    for (int c0 = nbeg; c0 < nend; c0 += LB_NU) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < LB_NU * 16 * LB_BLK; idx += LB_THREADS) {
            int r = idx / LB_NU, c = idx % LB_NU;   // r: layer/impact index, c: wavenumber
            int n = c0 + c;
            bool ok = (r < L) && (n < nend);
            st[c][r] = ok ? tb[(size_t)r * N + n] : 0.f;
            sa[c][r] = ok ? al[(size_t)r * N + n] : 0.f;
        }
        __syncthreads();
        if (l0 <= i0 + LB_BLK - 1) {
            for (int c = 0; c < LB_NU; ++c) {
                float tv[LB_BLK], av[LB_BLK];
#pragma unroll
                for (int u = 0; u < LB_BLK; ++u) {
                    tv[u] = st[c][i0 + u];
                    av[u] = sa[c][l0 + u];
                }
#pragma unroll
                for (int u = 0; u < LB_BLK; ++u)
#pragma unroll
                    for (int v = 0; v < LB_BLK; ++v) acc[u][v] = fmaf(tv[u], av[v], acc[u][v]);
            }
        }
    }
    double *lb = w.lbar + (size_t)b * L * L;
    for (int u = 0; u < LB_BLK; ++u)
        for (int v = 0; v < LB_BLK; ++v) {
            int i = i0 + u, l = l0 + v;
            if (i < L && l <= i && acc[u][v] != 0.f) atomicAdd(lb + (size_t)i * L + l, (double)acc[u][v]);
        }
}

size_t transit_smem(const Model &m, bool with_area) {
    int Lp = round_up(m.L, CH);
    return sizeof(float) * ((size_t)m.L * Lp + (size_t)m.L * TR_THREADS + (with_area ? Lp : 0));
}

}  // namespace

int launch_transit(const Model &m, const Work &w, cudaStream_t st, const Hook &h) {
    size_t sm = transit_smem(m, true);
    cudaFuncSetAttribute(k_transit, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((m.N + TR_THREADS - 1) / TR_THREADS, w.B);
    ES_LAUNCH(h, "k_transit", st, k_transit<<<grid, TR_THREADS, sm, st>>>(m, w));
    return 1;
}

int launch_transit_backward(const Model &m, const Work &w, cudaStream_t st, const Hook &h) {
    size_t sm = transit_smem(m, true);
    cudaFuncSetAttribute(k_transit_taubar, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncSetAttribute(k_transit_abar, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    dim3 grid((m.N + TR_THREADS - 1) / TR_THREADS, w.B);
    ES_LAUNCH(h, "k_transit_taubar", st, k_transit_taubar<<<grid, TR_THREADS, sm, st>>>(m, w));
    ES_LAUNCH(h, "k_transit_abar", st, k_transit_abar<<<grid, TR_THREADS, sm, st>>>(m, w));
    dim3 grid2((m.N + LB_RANGE - 1) / LB_RANGE, w.B);
    ES_LAUNCH(h, "k_transit_lbar", st, k_transit_lbar<<<grid2, LB_THREADS, 0, st>>>(m, w));
    return 3;
}

}  // namespace es
