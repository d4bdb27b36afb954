// Instrument binning (equal-weight mean over the native points of each bin)
// and the Gaussian log-likelihood of Sect. 2.3,
//   ln L = sum_k [-ln s_k - 1/2 ln 2 pi - 1/2 (r_k/s_k)^2],
//   r_k = y_obs,k - y_k, s_k^2 = sigma_k^2 + 10^(2c) (Eq. c_error),
// in FP64, one block per sample: bin sums with one warp per bin, the
// likelihood terms with one thread per bin. With the adjoint requested it
// also writes d lnL / d spectrum (dbar) and the base / error-inflation
// adjoints.
#include "internal.cuh"

namespace es {

namespace {

constexpr int BIN_THREADS = 256;

__device__ __forceinline__ double block_sum_d(double v, double *scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncwarp();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int q = 0; q < BIN_THREADS / 32; ++q) t += scratch[q];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(BIN_THREADS) k_bins(Model m, Work w, int adjoint, float *spec_out,
                                                      double *binned_out, double *lnl_out) {
    const int b = blockIdx.x;
    // a kind other than transmission / emission (possible only through the
    // no-allocation entry point, whose device-side kinds are not checked on the
    // host) makes the sample invalid; it never indexes the data
    const int kind_in = w.kind[b];
    const bool kind_ok = kind_in == ES_KIND_TRANSMISSION || kind_in == ES_KIND_EMISSION;
    const int N = m.N, S = m.S, kind = kind_ok ? kind_in : ES_KIND_TRANSMISSION;
    __shared__ double scratch[BIN_THREADS / 32];
    __shared__ int s_bad, s_flag;
    if (threadIdx.x == 0) {
        // a fused kernel that gave up on a bounded wait left its spectra
        // unfinished: every sample of the call is invalid
        const int timed_out = *w.err != 0;
        s_flag = w.flags[b] | ((kind_ok && !timed_out) ? 0 : ES_FLAG_INVALID) | (timed_out ? ES_FLAG_TIMEOUT : 0);
        s_bad = s_flag;
    }
    __syncthreads();
    const double base = (kind == ES_KIND_TRANSMISSION) ? w.base[b] : 0.0;
    const double c = w.theta[(size_t)b * m.nfull + S + ES_P_C_INFL];
    const double infl = exp10(2.0 * c);
    const float *sp = w.spec + (size_t)b * N;
    const double *yo = m.y_obs + (size_t)kind * m.nbins, *sg = m.sigma + (size_t)kind * m.nbins;
    // bin means: one warp per bin, coalesced reads of its native points, FP64 sums
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *ym = w.ymod + (size_t)b * m.nbins;
    // (FP32 partial sums of at most 32 points per lane group, FP64 for the
    // last two combining stages: GB300's FP64 rate is a small fraction of FP32)
    for (int k = warp; k < m.nbins; k += BIN_THREADS / 32) {
        const int lo = m.bin_lo[k], hi = m.bin_hi[k];
        float acc = 0.f;
        for (int n = lo + lane; n < hi; n += 32) acc += sp[n];
        for (int o = 16; o > 2; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        double d = (double)acc;
        for (int o = 2; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) ym[k] = d;   // the bin sum; its mean is formed below
    }
    __syncthreads();
    // likelihood terms: one thread per bin
    double lsum = 0.0, cbar = 0.0, bbar = 0.0;
    for (int k = threadIdx.x; k < m.nbins; k += BIN_THREADS) {
        const double y = base + ym[k] / (double)(m.bin_hi[k] - m.bin_lo[k]);
        ym[k] = y;
        if (!isfinite(y)) s_bad = 1;
        if (binned_out) binned_out[(size_t)b * m.nbins + k] = y;
        const double se2 = sg[k] * sg[k] + infl;
        const double r = yo[k] - y;
        lsum += -0.5 * log(se2) - 0.5 * log(2.0 * PI) - 0.5 * r * r / se2;
        cbar += (-0.5 / se2 + 0.5 * r * r / (se2 * se2)) * 2.0 * LN10 * infl;
        bbar += r / se2;
    }
    lsum = block_sum_d(lsum, scratch);
    cbar = block_sum_d(cbar, scratch);
    bbar = block_sum_d(bbar, scratch);
    const bool bad = s_bad != 0;
    if (threadIdx.x == 0) {
        w.flags[b] = bad ? (s_flag | ES_FLAG_INVALID) : 0;
        const double v = bad ? INVALID_LNL : lsum;
        w.lnl[b] = v;
        if (lnl_out) lnl_out[b] = v;
        if (adjoint) {
            w.misc[(size_t)b * 4 + 0] = bad ? 0.0 : bbar;
            w.misc[(size_t)b * 4 + 1] = 0.0;
            w.misc[(size_t)b * 4 + 2] = bad ? 0.0 : cbar;
            w.misc[(size_t)b * 4 + 3] = 0.0;
        }
    }
    if (adjoint && !bad) {
        // d lnL / d spec(n) = (y_obs - y_k) / s_k^2 / n_k for n in bin k
        for (int k = warp; k < m.nbins; k += BIN_THREADS / 32) {
            const int lo = m.bin_lo[k], hi = m.bin_hi[k];
            const float g = (float)(yo[k] - ym[k]) / (float)(sg[k] * sg[k] + infl) / (float)(hi - lo);
            for (int n = lo + lane; n < hi; n += 32) w.dbar[(size_t)b * m.Np + n] = g;
        }
    }
    if (spec_out)
        for (int n = threadIdx.x; n < N; n += BIN_THREADS)
            spec_out[(size_t)b * N + n] = (float)(base + (double)sp[n]);
}

}  // namespace

int launch_bins(const Model &m, const Work &w, bool want_adjoint, float *spectrum_out, double *binned_out,
                double *lnl_out, cudaStream_t st, const Hook &h) {
    ES_LAUNCH(h, "k_bins", st,
              k_bins<<<w.B, BIN_THREADS, 0, st>>>(m, w, want_adjoint ? 1 : 0, spectrum_out, binned_out, lnl_out));
    return 1;
}

}  // namespace es
