// Opacity interpolation and extinction (Sect. 3):
//   alpha_l(nu) = sum_s n_l X_s 10^{bilerp log10 sigma_s(T_l, p_l, nu)}
//               + n_l^2 X_H2 (X_H2 k_H2H2 + X_He k_H2He)(T_l, nu)
//               + n_l (X_H2 s_H2 + X_He s_He) (nu / nu_ref)^4
// evaluated in base 2 with the log2(X n) and table row offsets folded into a
// per-(sample, layer, species) constant, and its adjoint (recomputing the
// terms instead of storing them).
#include "internal.cuh"
#include <cuda_bf16.h>

namespace es {

namespace {

constexpr int EXT_THREADS = 128;
constexpr int BWD_NU_PER_THREAD = 16;

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <bool BF16>
__device__ __forceinline__ float tab_load(const Model &m, size_t idx) {
    if (BF16) return __uint_as_float(((uint32_t)__ldg(m.tab16 + idx)) << 16);
    return __ldg(m.tab32 + idx);
}

template <bool BF16>
__global__ void __launch_bounds__(EXT_THREADS) k_extinction(Model m, Work w, int only_kind) {
    const int b = blockIdx.y;
    if (only_kind >= 0 && w.kind[b] != only_kind) return;
    const int n = blockIdx.x * EXT_THREADS + threadIdx.x;
    const int L = m.L, S = m.S, N = m.N;
    __shared__ float4 s_w4[ES_MAX_LAYERS];
    __shared__ int s_it[ES_MAX_LAYERS], s_ip[ES_MAX_LAYERS], s_itc[ES_MAX_LAYERS];
    __shared__ float s_wtc[ES_MAX_LAYERS], s_ray[ES_MAX_LAYERS], s_cc[2 * ES_MAX_LAYERS];
    __shared__ float s_coef[ES_MAX_LAYERS * ES_MAX_SPECIES];
    for (int l = threadIdx.x; l < L; l += EXT_THREADS) {
        size_t bl = (size_t)b * L + l;
        s_w4[l] = w.w4[bl];
        s_it[l] = w.it[bl];
        s_ip[l] = m.ip[l];
        s_itc[l] = w.itc[bl];
        s_wtc[l] = w.wtc[bl];
        s_ray[l] = w.ray[bl];
        s_cc[2 * l] = w.ccia[2 * bl];
        s_cc[2 * l + 1] = w.ccia[2 * bl + 1];
    }
    for (int i = threadIdx.x; i < L * S; i += EXT_THREADS) s_coef[i] = w.coef[(size_t)b * L * S + i];
    __syncthreads();
    if (n >= N) return;
    const float nf = m.nu[n] / (float)m.ray_nu_ref;
    const float nu4 = (nf * nf) * (nf * nf);
    const size_t strideP = m.Np, strideT = (size_t)m.NP * m.Np, strideS = (size_t)m.NT * strideT;
    const float *cia1 = m.cia + n, *cia2 = m.cia + (size_t)m.NTc * m.Np + n;
    float *out = w.alpha + (size_t)b * L * N + n;
    for (int l = 0; l < L; ++l) {
        const float4 wv = s_w4[l];
        const size_t row = (size_t)s_it[l] * strideT + (size_t)s_ip[l] * strideP + n;
        float acc = 0.f;
        for (int s = 0; s < S; ++s) {
            const size_t r = row + s * strideS;
            float q00 = tab_load<BF16>(m, r), q01 = tab_load<BF16>(m, r + strideP);
            float q10 = tab_load<BF16>(m, r + strideT), q11 = tab_load<BF16>(m, r + strideT + strideP);
            float e = fmaf(wv.x, q00, fmaf(wv.y, q01, fmaf(wv.z, q10, fmaf(wv.w, q11, s_coef[l * S + s]))));
            acc += ex2(e);
        }
        const size_t c = (size_t)s_itc[l] * m.Np;
        float k0 = __ldg(cia1 + c), k1 = __ldg(cia1 + c + m.Np);
        acc += ex2(fmaf((float)LOG2_10, fmaf(s_wtc[l], k1 - k0, k0), s_cc[2 * l]));
        k0 = __ldg(cia2 + c);
        k1 = __ldg(cia2 + c + m.Np);
        acc += ex2(fmaf((float)LOG2_10, fmaf(s_wtc[l], k1 - k0, k0), s_cc[2 * l + 1]));
        acc = fmaf(s_ray[l], nu4, acc);
        out[(size_t)l * N] = acc;
    }
}

// Block-wide sum of `v` across EXT_THREADS threads; result valid in thread 0.
__device__ __forceinline__ float block_sum(float v, float *scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncwarp();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int q = 0; q < EXT_THREADS / 32; ++q) t += scratch[q];
    __syncthreads();
    return t;
}

// Adjoint: with abar = d lnL / d alpha_l(nu), accumulate per (sample, layer)
//   Q_s = sum abar e_s, D = sum abar sum_s e_s dlog10sigma_s/dlog10T,
//   C1 = sum abar c1, C2 = sum abar c2, C1T = sum abar c1 dlog10k1/dT,
//   C2T = sum abar c2 dlog10k2/dT, W4 = sum abar (nu/nu_ref)^4,
// where e_s, c1, c2 are the species and CIA extinction terms.
template <bool BF16>
__global__ void __launch_bounds__(EXT_THREADS) k_extinction_bwd(Model m, Work w, int only_kind) {
    const int b = blockIdx.y;
    if (only_kind >= 0 && w.kind[b] != only_kind) return;
    const int L = m.L, S = m.S, N = m.N, NR = S + 6;   // species, then D, C1, C2, C1T, C2T, W4
    const int n0 = blockIdx.x * EXT_THREADS * BWD_NU_PER_THREAD + threadIdx.x;
    __shared__ float scratch[EXT_THREADS / 32];
    const size_t strideP = m.Np, strideT = (size_t)m.NP * m.Np, strideS = (size_t)m.NT * strideT;
    for (int l = 0; l < L; ++l) {
        const size_t bl = (size_t)b * L + l;
        const float4 wv = w.w4[bl];
        const int it = w.it[bl], ip = m.ip[l], itc = w.itc[bl];
        const float wp = m.wp[l], gt = w.gt[bl], wtc = w.wtc[bl], gtc = w.gtc[bl];
        const float cc1 = w.ccia[2 * bl], cc2 = w.ccia[2 * bl + 1];
        float acc[ES_MAX_SPECIES + 6];
        for (int q = 0; q < NR; ++q) acc[q] = 0.f;
        const float *abar = w.abar + bl * N;
        for (int k = 0; k < BWD_NU_PER_THREAD; ++k) {
            const int n = n0 + k * EXT_THREADS;
            if (n >= N) break;
            const float a = abar[n];
            float dsum = 0.f;
            for (int s = 0; s < S; ++s) {
                const size_t r = (size_t)it * strideT + (size_t)ip * strideP + n + s * strideS;
                float q00 = tab_load<BF16>(m, r), q01 = tab_load<BF16>(m, r + strideP);
                float q10 = tab_load<BF16>(m, r + strideT), q11 = tab_load<BF16>(m, r + strideT + strideP);
                float e = ex2(fmaf(wv.x, q00, fmaf(wv.y, q01, fmaf(wv.z, q10, fmaf(wv.w, q11,
                                                                               w.coef[bl * S + s])))));
                const float *off = m.row_off + ((size_t)s * m.NT + it) * m.NP + ip;
                float slope = gt * ((1.f - wp) * ((q10 - q00) + (off[m.NP] - off[0]))
                                    + wp * ((q11 - q01) + (off[m.NP + 1] - off[1])));
                float ae = a * e;
                acc[s] += ae;
                dsum = fmaf(ae, slope, dsum);
            }
            acc[S] += dsum;
            const size_t c = (size_t)itc * m.Np + n;
            float k0 = __ldg(m.cia + c), k1 = __ldg(m.cia + c + m.Np);
            float c1 = ex2(fmaf((float)LOG2_10, fmaf(wtc, k1 - k0, k0), cc1));
            float sl1 = gtc * (k1 - k0);
            const size_t c2i = c + (size_t)m.NTc * m.Np;
            k0 = __ldg(m.cia + c2i);
            k1 = __ldg(m.cia + c2i + m.Np);
            float c2 = ex2(fmaf((float)LOG2_10, fmaf(wtc, k1 - k0, k0), cc2));
            float sl2 = gtc * (k1 - k0);
            acc[S + 1] += a * c1;
            acc[S + 2] += a * c2;
            acc[S + 3] += a * c1 * sl1;
            acc[S + 4] += a * c2 * sl2;
            const float nf = m.nu[n] / (float)m.ray_nu_ref;
            acc[S + 5] += a * (nf * nf) * (nf * nf);
        }
        // species: per-species totals (qtot) and their sum for this layer (red
        // slot 0); then D, C1, C2, C1T, C2T, W4 into slots 2, 4, 5, 6, 7, 8
        float qs = 0.f;
        for (int q = 0; q < NR; ++q) {
            float t = block_sum(acc[q], scratch);
            if (threadIdx.x == 0) {
                if (q < S) {
                    qs += t;
                    if (t != 0.f) atomicAdd(w.qtot + (size_t)b * S + q, (double)t);
                } else if (t != 0.f) {
                    atomicAdd(w.red + bl * N_RED + (q == S ? 2 : 3 + (q - S)), (double)t);
                }
            }
        }
        if (threadIdx.x == 0 && qs != 0.f) atomicAdd(w.red + bl * N_RED, (double)qs);
    }
}

}  // namespace

int launch_extinction(const Model &m, const Work &w, int only_kind, cudaStream_t st, const Hook &h) {
    dim3 grid((m.N + EXT_THREADS - 1) / EXT_THREADS, w.B);
    if (m.bf16) ES_LAUNCH(h, "k_extinction", st, k_extinction<true><<<grid, EXT_THREADS, 0, st>>>(m, w, only_kind));
    else ES_LAUNCH(h, "k_extinction", st, k_extinction<false><<<grid, EXT_THREADS, 0, st>>>(m, w, only_kind));
    return 1;
}

int launch_extinction_backward(const Model &m, const Work &w, int only_kind, cudaStream_t st, const Hook &h) {
    const int per_block = EXT_THREADS * BWD_NU_PER_THREAD;
    dim3 grid((m.N + per_block - 1) / per_block, w.B);
    if (m.bf16) ES_LAUNCH(h, "k_extinction_bwd", st, k_extinction_bwd<true><<<grid, EXT_THREADS, 0, st>>>(m, w, only_kind));
    else ES_LAUNCH(h, "k_extinction_bwd", st, k_extinction_bwd<false><<<grid, EXT_THREADS, 0, st>>>(m, w, only_kind));
    return 1;
}

}  // namespace es
