// Emission (Sect. 5): absorption-only Schwarzschild integration with a
// source linear in optical depth inside each layer, from I = B(T_bottom)
// upward, at 4 Gauss-Legendre angles on [0, 1]:
//   E = exp(-x), x = dtau/mu,  I <- I E + B_top (1 - E) + (B_bot - B_top) f(x),
//   f(x) = (1 - E)/x - E,   F_toa = 2 pi sum_j w_j mu_j I_j,
//   Fp/F* = s F_toa / (pi B(T_*)) (R_p/R_*)^2,
// B the Planck function per unit wavenumber; and its adjoint.
#include "internal.cuh"

namespace es {

namespace {

constexpr int EM_THREADS = 128;

__device__ __forceinline__ float planck(float nu, double t) {
    // B = 2 h c^2 nu^3 / (exp(c2 nu / T) - 1); zero when the exponent overflows
    float x = (float)C2_RAD * nu * (float)(1.0 / t);
    return (float)TWO_HC2 * nu * nu * nu / expm1f(x);
}

__device__ __forceinline__ float dplanck_dt(float nu, double t, float bval) {
    float x = (float)C2_RAD * nu * (float)(1.0 / t);
    float em = -expm1f(-x);   // 1 - exp(-x)
    return (em > 0.f) ? bval * x / ((float)t * em) : 0.f;
}

// f(x) = (1 - e^-x)/x - e^-x and f'(x); series below x = 0.1 (cancellation).
__device__ __forceinline__ void lin_factor(float x, float e, float &f, float &fp) {
    if (x < 0.1f) {
        f = x * (0.5f + x * (-1.f / 3.f + x * (0.125f + x * (-1.f / 30.f + x * (1.f / 144.f - x * (1.f / 840.f))))));
        fp = 0.5f + x * (-2.f / 3.f + x * (0.375f + x * (-2.f / 15.f + x * (5.f / 144.f - x * (1.f / 140.f)))));
    } else {
        float em = -expm1f(-x);
        float ix = 1.f / x;
        f = em * ix - e;
        fp = (e * x + e * x * x - em) * ix * ix;
    }
}

__global__ void __launch_bounds__(EM_THREADS) k_emission(Model m, Work w) {
    const int b = blockIdx.y;
    if (w.kind[b] != ES_KIND_EMISSION) return;
    const int n = blockIdx.x * EM_THREADS + threadIdx.x;
    const int L = m.L, N = m.N;
    if (n >= N) return;
    const float nu = m.nu[n];
    const double *tlev = w.t_lev + (size_t)b * (L + 1);
    const float *al = w.alpha + (size_t)b * L * N + n;
    const float *dr = w.dr + (size_t)b * L;
    float inten[N_MU];
    float bb = planck(nu, tlev[L]);
#pragma unroll
    for (int j = 0; j < N_MU; ++j) inten[j] = bb;
    for (int l = L - 1; l >= 0; --l) {
        const float bt = planck(nu, tlev[l]);
        const float dtau = al[(size_t)l * N] * dr[l];
#pragma unroll
        for (int j = 0; j < N_MU; ++j) {
            const float x = dtau * (float)(1.0 / m.mu_gl[j]);
            const float e = expf(-x);
            float f, fp;
            lin_factor(x, e, f, fp);
            inten[j] = fmaf(inten[j], e, fmaf(bt, -expm1f(-x), (bb - bt) * f));
        }
        bb = bt;
    }
    float flux = 0.f;
#pragma unroll
    for (int j = 0; j < N_MU; ++j) flux = fmaf((float)(2.0 * PI * m.w_gl[j] * m.mu_gl[j]), inten[j], flux);
    w.spec[(size_t)b * N + n] = (float)w.scale[b] * flux * m.inv_fstar[n];
}

__device__ __forceinline__ float block_sum(float v, float *scratch) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncwarp();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x == 0)
        for (int q = 0; q < EM_THREADS / 32; ++q) t += scratch[q];
    __syncthreads();
    return t;
}

// Adjoint: forward sweep storing the upward intensity at every level, then
// a top-down sweep. Produces alpha_bar (via dtau_bar dr), per-layer dr_bar,
// per-level T_lev_bar and the scale adjoint.
__global__ void __launch_bounds__(EM_THREADS) k_emission_bwd(Model m, Work w) {
    const int b = blockIdx.y;
    if (w.kind[b] != ES_KIND_EMISSION) return;
    __shared__ float scratch[EM_THREADS / 32];
    const int n = blockIdx.x * EM_THREADS + threadIdx.x;
    const int L = m.L, N = m.N;
    if (w.flags[b]) {   // invalid sample: zero alpha_bar so the extinction adjoint adds nothing
        if (n < N)
            for (int l = 0; l < L; ++l) w.abar[((size_t)b * L + l) * N + n] = 0.f;
        return;
    }
    const bool live = n < N;
    const int nn = live ? n : N - 1;
    const float nu = m.nu[nn];
    const double *tlev = w.t_lev + (size_t)b * (L + 1);
    const float *al = w.alpha + (size_t)b * L * N + nn;
    const float *dr = w.dr + (size_t)b * L;
    float ist[ES_MAX_LAYERS + 1][N_MU];
    float blev[ES_MAX_LAYERS + 1];
    blev[L] = planck(nu, tlev[L]);
#pragma unroll
    for (int j = 0; j < N_MU; ++j) ist[L][j] = blev[L];
    for (int l = L - 1; l >= 0; --l) {
        blev[l] = planck(nu, tlev[l]);
        const float dtau = al[(size_t)l * N] * dr[l];
#pragma unroll
        for (int j = 0; j < N_MU; ++j) {
            const float x = dtau * (float)(1.0 / m.mu_gl[j]);
            const float e = expf(-x);
            float f, fp;
            lin_factor(x, e, f, fp);
            ist[l][j] = fmaf(ist[l + 1][j], e, fmaf(blev[l], -expm1f(-x), (blev[l + 1] - blev[l]) * f));
        }
    }
    float flux = 0.f;
#pragma unroll
    for (int j = 0; j < N_MU; ++j) flux = fmaf((float)(2.0 * PI * m.w_gl[j] * m.mu_gl[j]), ist[0][j], flux);
    const float db = live ? w.dbar[(size_t)b * m.Np + n] : 0.f;
    const float sc = (float)w.scale[b];
    const float fbar = db * sc * m.inv_fstar[nn];
    float sbar = db * flux * m.inv_fstar[nn];
    float ib[N_MU];
#pragma unroll
    for (int j = 0; j < N_MU; ++j) ib[j] = fbar * (float)(2.0 * PI * m.w_gl[j] * m.mu_gl[j]);
    float btop_bar = 0.f;   // adjoint of B at level l accumulated from the layer above
    float *abar = w.abar + (size_t)b * L * N;
    for (int l = 0; l < L; ++l) {
        const float alpha = al[(size_t)l * N];
        const float dtau = alpha * dr[l];
        const float bt = blev[l], bbv = blev[l + 1];
        float dtb = 0.f, btb = btop_bar, bbb = 0.f;
#pragma unroll
        for (int j = 0; j < N_MU; ++j) {
            const float imu = (float)(1.0 / m.mu_gl[j]);
            const float x = dtau * imu;
            const float e = expf(-x);
            float f, fp;
            lin_factor(x, e, f, fp);
            const float iin = ist[l + 1][j];
            const float xbar = ib[j] * (-iin * e + bt * e + (bbv - bt) * fp);
            dtb = fmaf(xbar, imu, dtb);
            btb = fmaf(ib[j], -expm1f(-x) - f, btb);
            bbb = fmaf(ib[j], f, bbb);
            ib[j] *= e;
        }
        if (live) abar[(size_t)l * N + n] = dtb * dr[l];
        float part = block_sum(live ? dtb * alpha : 0.f, scratch);
        if (threadIdx.x == 0 && part != 0.f) atomicAdd(w.drbar + (size_t)b * L + l, (double)part);
        // level l is complete: from layer l (top) and layer l-1 (bottom)
        part = block_sum(live ? btb * dplanck_dt(nu, tlev[l], bt) : 0.f, scratch);
        if (threadIdx.x == 0 && part != 0.f) atomicAdd(w.levbar + (size_t)b * (L + 1) + l, (double)part);
        btop_bar = bbb;
    }
    // bottom level: from the last layer and the boundary condition I = B_bottom
    float bl = btop_bar;
#pragma unroll
    for (int j = 0; j < N_MU; ++j) bl += ib[j];
    float part = block_sum(live ? bl * dplanck_dt(nu, tlev[L], blev[L]) : 0.f, scratch);
    if (threadIdx.x == 0 && part != 0.f) atomicAdd(w.levbar + (size_t)b * (L + 1) + L, (double)part);
    part = block_sum(live ? sbar : 0.f, scratch);
    if (threadIdx.x == 0 && part != 0.f) atomicAdd(w.misc + (size_t)b * 4 + 1, (double)part);
}

}  // namespace

int launch_emission(const Model &m, const Work &w, cudaStream_t st, const Hook &h) {
    dim3 grid((m.N + EM_THREADS - 1) / EM_THREADS, w.B);
    ES_LAUNCH(h, "k_emission", st, k_emission<<<grid, EM_THREADS, 0, st>>>(m, w));
    return 1;
}

int launch_emission_backward(const Model &m, const Work &w, cudaStream_t st, const Hook &h) {
    dim3 grid((m.N + EM_THREADS - 1) / EM_THREADS, w.B);
    ES_LAUNCH(h, "k_emission_bwd", st, k_emission_bwd<<<grid, EM_THREADS, 0, st>>>(m, w));
    return 1;
}

}  // namespace es
