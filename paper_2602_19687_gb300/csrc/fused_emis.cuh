// Tile engines of the fused emission kernels (Sect. 3 opacities -> Sect. 5
// Schwarzschild integration), driven by the persistent kernels over
// (sample, wavenumber-chunk) items (emission-only in k_fused_emis.cu, mixed
// transmission/emission in k_fused_mixed.cu). Each warp owns 32 consecutive wavenumbers and walks all layers
// from the top down: a lane pair interpolates the extinction of its
// wavenumber pair (species split between the lanes, as in the transmission
// kernels), combines it by one shuffle, and each lane integrates the
// upward intensity of its own wavenumber at 4 Gauss-Legendre angles. With the
// source linear in optical depth inside a layer and x = dtau / mu,
//   E = exp(-x),  Src = B_top (1 - E) + (B_bot - B_top) f(x),
//   f(x) = (1 - E)/x - E,
// the bottom-up recursion I <- I E + Src telescopes to the top-down sum
//   I_toa = sum_l T_l Src_l + T_L B_surface,  T_l = prod_{k < l} E_k,
// which is what a top-down walk accumulates. Fp/F* = s F / (pi B(T_*)) with
// F = 2 pi sum_j w_j mu_j I_j. No block barrier inside a tile: the block only
// shares the sample's per-layer constants.
//
// The adjoint walks the layers top-down again with the stored I_toa: with
// the prefix P_l = sum_{k <= l} T_k Src_k, the part of I_toa from below
// layer l is I_toa - P_l, so
//   dI/d dtau_l = (1/mu) [T_l (B_top E + (B_bot - B_top) f'(x)) - (I_toa - P_l)],
//   dI/dB_top = T_l (1 - E - f),  dI/dB_bot = T_l f,  dI/dB_surface = T_L,
// and the interpolation is recomputed and reduced against
// alpha_bar = dtau_bar dr.
//
// With the non-grey cloud (Sect. 2.5) each lane also integrates a cloudy
// column, dtau_l + C_l g(nu) dr_l, and the emergent fluxes are mixed by the
// cloud fraction; its adjoint adds the cloudy column's dtau_bar to alpha_bar
// and returns d lnL / d C_l, d lnL / d g(nu) and d lnL / d f_cld.
#pragma once

#include "fused_common.cuh"

namespace es {

namespace {

constexpr int EM_WARPS = 16;
constexpr int EM_THREADS = EM_WARPS * 32;
constexpr int ET = EM_WARPS * 32;       // wavenumbers per block tile (32 per warp)

// The per-sample arrays of the emission engines, wherever a kernel keeps them
// in shared memory (EmisSmem in the emission-only kernels, beside the
// transmission engine's buffers in the mixed kernels).
struct EmisLevels {
    float inv_t[ES_MAX_LAYERS + 1];    // 1 / T at the levels
    float dr[ES_MAX_LAYERS];           // layer thickness
    float ccl[ES_MAX_LAYERS];          // non-grey cloud: C_l (extinction per unit g(nu))
    float levb_bot;                    // adjoint: T_bar of the bottom level
    float sbar;                        // adjoint: d lnL / d (emission scale)
};

struct EmisView {
    SampleConst *sc;
    EmisLevels *lv;
    float *cg;                         // [N_CG] non-grey cloud: g(nu) constants (kh18_g)
    // adjoint accumulators of the current sample: per layer 32 partial sums
    // [value 0..7][lane parity][lane bit 1] (values: QS, D, C, CT, W4, dr_bar,
    // T_bar of the level, C_l bar of the cloud), combined at the flush
    float *red;                        // [ES_MAX_LAYERS * 32]
    float *qtot;                       // [ES_MAX_SPECIES]
    float *cpbar;                      // [N_CG] d lnL / d (ln r_eff via g, a, ln Q0, f_cld, A, lambda_0, omega, xi)
    unsigned char *stage;              // adjoint: per-warp coefficient staging, EM_WARPS x STAGE_BYTES_PER_WARP
};

struct EmisSmem {
    SampleConst sc;
    EmisLevels lv;
    float cg[N_CG];
    float red[ES_MAX_LAYERS * 32];
    float qtot[ES_MAX_SPECIES];
    float cpbar[N_CG];
};

// The adjoint's per-warp coefficient staging follows EmisSmem in dynamic
// shared memory (the forward has none: its loads go through L1).
constexpr size_t EM_STAGE_OFFSET = (sizeof(EmisSmem) + 127) / 128 * 128;

__device__ __forceinline__ EmisView emis_view(EmisSmem &sm, unsigned char *stage) {
    return EmisView{&sm.sc, &sm.lv, sm.cg, sm.red, sm.qtot, sm.cpbar, stage};
}

template <bool CLOUD>
__device__ __forceinline__ void stage_levels(const Model &m, const Work &w, int b, const EmisView &v) {
    const int L = m.L;
    for (int k = threadIdx.x; k <= L; k += blockDim.x) v.lv->inv_t[k] = (float)(1.0 / w.t_lev[(size_t)b * (L + 1) + k]);
    for (int l = threadIdx.x; l < L; l += blockDim.x) v.lv->dr[l] = w.dr[(size_t)b * L + l];
    if (CLOUD) {
        for (int l = threadIdx.x; l < L; l += blockDim.x) v.lv->ccl[l] = w.cloud_c[(size_t)b * L + l];
        if (threadIdx.x < N_CG) v.cg[threadIdx.x] = w.cloud_g[(size_t)b * N_CG + threadIdx.x];
    }
}

// Planck function per unit wavenumber at a level: B = nu3c e / (1 - e) with
// nu3c = 2 h c^2 nu^3, e = 2^-a and a = (h c nu / k T) log2 e (the same as
// nu3c / (2^a - 1), with the same precision where a is small). Where a
// passes 126, e flushes to zero and so does B (its true value is then below
// 2^-126 of nu3c). Optionally dB/dT = B a ln 2 / ((1 - e) T).
struct Planck {
    float nu3c, xc;   // 2 h c^2 nu^3; (h c / k) nu log2 e
    __device__ __forceinline__ void init(float nu) {
        nu3c = (float)TWO_HC2 * nu * nu * nu;
        xc = (float)(C2_RAD * 1.4426950408889634) * nu;
    }
    __device__ __forceinline__ float value(float inv_t) const {
        const float e = ex2f(-xc * inv_t);
        return nu3c * e * __frcp_rn(1.f - e);
    }
    __device__ __forceinline__ float value_dt(float inv_t, float &dbdt) const {
        const float a = xc * inv_t;
        const float e = ex2f(-a), r = __frcp_rn(1.f - e);
        const float bv = nu3c * e * r;
        dbdt = bv * (a * 0.6931471805599453f) * r * inv_t;
        return bv;
    }
};

// Angle-pair constants: mu, 1/mu, log2(e)/mu for angles (0,1) and (2,3).
struct Angles {
    float2 mu[2], imu[2], c[2], wt[2];   // wt = 2 pi w mu
    __device__ __forceinline__ void init(const Model &m) {
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const double a = m.mu_gl[2 * p], bq = m.mu_gl[2 * p + 1];
            mu[p] = make_float2((float)a, (float)bq);
            imu[p] = make_float2((float)(1.0 / a), (float)(1.0 / bq));
            c[p] = make_float2((float)(1.4426950408889634 / a), (float)(1.4426950408889634 / bq));
            wt[p] = make_float2((float)(2.0 * PI * m.w_gl[2 * p] * a), (float)(2.0 * PI * m.w_gl[2 * p + 1] * bq));
        }
    }
};

// Layer factors for an angle pair, x = dtau / mu, E = exp(-x) (MUFU, relative
// error ~2^-22): 1 - E and f(x) = (1 - E)/x - E. Below x = 1/4 both come from
// their Taylor series, since the direct forms magnify the error of E by 1/x
// (f' by 1/x^2); above, from the direct forms, whose error there stays below
// ~1e-5 relative (f) and ~4e-6 (f'). Six terms of the series for 1 - E and f,
// seven for f', leave truncation errors below 1e-7 relative at x = 1/4:
//   1 - E = x sum_{k>=0} (-x)^k / (k+1)!,   f = sum_{k>=1} (-1)^(k+1) k x^k / (k+1)!
template <int NC>
__device__ __forceinline__ float2 poly(float2 x, const float (&c)[NC]) {
    float2 r = fma2(x, f2(c[NC - 1]), f2(c[NC - 2]));
#pragma unroll
    for (int k = NC - 3; k >= 0; --k) r = fma2(x, r, f2(c[k]));
    return r;
}
constexpr float X_SERIES = 0.25f;
__device__ __forceinline__ float2 pick(float2 x, float2 series, float2 direct) {
    return make_float2(x.x < X_SERIES ? series.x : direct.x, x.y < X_SERIES ? series.y : direct.y);
}
__device__ __forceinline__ void lin_factors(float2 x, float2 e, float2 ix, float2 &ome, float2 &f) {
    const float cg[6] = {1.f, -1.f / 2, 1.f / 6, -1.f / 24, 1.f / 120, -1.f / 720};
    const float cf[6] = {1.f / 2, -1.f / 3, 1.f / 8, -1.f / 30, 1.f / 144, -1.f / 840};
    const float2 ome_d = fma2(e, f2(-1.f), f2(1.f));
    ome = pick(x, mul2(x, poly(x, cg)), ome_d);
    f = pick(x, mul2(x, poly(x, cf)), fma2(ome_d, ix, mul2(e, f2(-1.f))));
}
// f'(x) = (E x + E x^2 - (1 - E)) / x^2 = sum_{k>=1} (-1)^(k+1) k^2 x^(k-1) / (k+1)!
__device__ __forceinline__ float2 lin_fp(float2 x, float2 e, float2 ome, float2 ix) {
    const float cp[7] = {1.f / 2, -2.f / 3, 3.f / 8, -2.f / 15, 5.f / 144, -1.f / 140, 7.f / 5760};
    const float2 ex = mul2(e, x);
    const float2 fd = mul2(fma2(ex, x, add2(ex, mul2(ome, f2(-1.f)))), mul2(ix, ix));
    return pick(x, poly(x, cp), fd);
}

// Lane's alpha at its own wavenumber from the pair sum.
__device__ __forceinline__ float own(float2 a, int half) { return half ? a.y : a.x; }

// One layer of the top-down sum for the lane's wavenumber at both angle
// pairs: I += T Src, T *= E (see the header comment).
__device__ __forceinline__ void rt_layer(const Angles &ang, float dtau, float bt, float bb, float2 (&tr)[2],
                                         float2 (&in)[2]) {
    const float rdt = __frcp_rn(dtau);
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float2 x = mul2(f2(dtau), ang.imu[p]);
        const float2 e = ex2x2(mul2(f2(-dtau), ang.c[p]));
        float2 ome, f;
        lin_factors(x, e, mul2(ang.mu[p], f2(rdt)), ome, f);
        const float2 src = fma2(f2(bt), ome, mul2(f2(bb - bt), f));
        in[p] = fma2(tr[p], src, in[p]);
        tr[p] = mul2(tr[p], e);
    }
}

// Adjoint of rt_layer for one column with the stored I_toa: returns
// d lnL / d dtau_l and adds the adjoints of the layer's top and bottom Planck
// values to btb and bbb; ib = d lnL / d I_toa per angle.
__device__ __forceinline__ float rt_layer_bwd(const Angles &ang, float dtau, float bt, float bb,
                                              const float2 (&itoa)[2], const float2 (&ib)[2], float2 (&tr)[2],
                                              float2 (&pre)[2], float &btb, float &bbb) {
    const float rdt = __frcp_rn(dtau);
    float dtb = 0.f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float2 x = mul2(f2(dtau), ang.imu[q]);
        const float2 e = ex2x2(mul2(f2(-dtau), ang.c[q]));
        const float2 ix = mul2(ang.mu[q], f2(rdt));
        float2 ome, f;
        lin_factors(x, e, ix, ome, f);
        const float2 fp = lin_fp(x, e, fma2(e, f2(-1.f), f2(1.f)), ix);
        const float2 src = fma2(f2(bt), ome, mul2(f2(bb - bt), f));
        pre[q] = fma2(tr[q], src, pre[q]);
        const float2 below = add2(itoa[q], mul2(pre[q], f2(-1.f)));
        // dI/d dtau = (1/mu) [T (B_top E + dB f') - below]
        const float2 g = mul2(ang.imu[q], fma2(tr[q], fma2(f2(bt), e, mul2(f2(bb - bt), fp)), mul2(below, f2(-1.f))));
        const float2 it = mul2(ib[q], tr[q]);
        dtb = fmaf(ib[q].x, g.x, fmaf(ib[q].y, g.y, dtb));
        const float2 omf = add2(ome, mul2(f, f2(-1.f)));
        btb = fmaf(it.x, omf.x, fmaf(it.y, omf.y, btb));
        bbb = fmaf(it.x, f.x, fmaf(it.y, f.y, bbb));
        tr[q] = mul2(tr[q], e);
    }
    return dtb;
}

__device__ __forceinline__ float flux_of(const Angles &ang, const float2 (&in)[2]) {
    return fmaf(ang.wt[0].x, in[0].x, fmaf(ang.wt[0].y, in[0].y, fmaf(ang.wt[1].x, in[1].x, ang.wt[1].y * in[1].y)));
}

// ---------------------------------------------------------------- forward engine
// CLOUD: the non-grey cloud and cloud fraction (ES_CLOUD_KH18). A second
// column with dtau_l + C_l g(nu) dr_l is integrated beside the clear one and
// the fluxes are mixed, F = f F_cld + (1 - f) F_cf (Sect. 2.5).
template <int SPL, bool STORE_I, bool CLOUD>
struct EmisFwdEngine {
    const Model &m;
    const Work &w;
    const EmisView v;
    const int warp, lane, half, L, N;
    Angles ang;

    __device__ __forceinline__ EmisFwdEngine(const Model &m_, const Work &w_, const EmisView &v_)
        : m(m_), w(w_), v(v_), warp(threadIdx.x >> 5), lane(threadIdx.x & 31), half(lane & 1), L(m_.L), N(m_.N) {
        ang.init(m_);
    }

    // 512-wavenumber tiles [t0, t1) of the staged emission sample b (each warp
    // its 32 wavenumbers of every tile; no block barrier)
    __device__ __forceinline__ void tiles(int b, int t0, int t1) {
        const float scale = (float)w.scale[b];
        for (int t = t0; t < t1; ++t) {
            const int nw = t * ET + 32 * warp;   // the warp's first wavenumber
            if (nw >= m.Np) continue;
            const int n = nw + 2 * (lane >> 1), nme = n + half;
            PairInterp<SPL> pi;
            pi.init(m, n, half, lane);
            Planck pl;
            pl.init(m.nu[nme]);
            const float gc = CLOUD ? kh18_g(v.cg, m.nu[nme]) : 0.f;
            float bt = pl.value(v.lv->inv_t[0]);
            float2 tr[2] = {f2(1.f), f2(1.f)}, in[2] = {f2(0.f), f2(0.f)};
            float2 trc[2] = {f2(1.f), f2(1.f)}, inc[2] = {f2(0.f), f2(0.f)};   // cloudy column
            for (int l = 0; l < L;) {
                // broadcast from lane 0: provably warp-uniform for the compiler
                const int end = __shfl_sync(0xffffffffu, v.sc->lay[l].run_end, 0);
                pi.load(*v.sc, v.sc->lay[l].cell, v.sc->lay[l].itc);
                if (end < L) pi.prefetch(v.sc->lay[end].cell, v.sc->lay[end].itc);
                for (; l < end; ++l) {
                    const LayerConst &lc = v.sc->lay[l];
                    float2 tt, sum = ex2x2(pi.expo(0, lc.wp, lc.wt, tt));
#pragma unroll
                    for (int j = 1; j < SPL; ++j) sum = add2(sum, ex2x2(pi.expo(j, lc.wp, lc.wt, tt)));
                    const float2 mine = pi.part(lc, sum, pi.cia(lc));
                    const float dtau = own(add2(mine, shfl_xor2(mine, 1)), half) * v.lv->dr[l];
                    const float bb = pl.value(v.lv->inv_t[l + 1]);
                    rt_layer(ang, dtau, bt, bb, tr, in);
                    if (CLOUD) rt_layer(ang, fmaf(v.lv->ccl[l] * gc, v.lv->dr[l], dtau), bt, bb, trc, inc);
                    bt = bb;
                }
            }
            // surface: I = B(bottom level) below the last layer
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                in[p] = fma2(tr[p], f2(bt), in[p]);
                if (CLOUD) inc[p] = fma2(trc[p], f2(bt), inc[p]);
            }
            float flux = flux_of(ang, in);
            if (CLOUD) flux = v.cg[3] * flux_of(ang, inc) + (1.f - v.cg[3]) * flux;
            if (nme < N) w.spec[(size_t)b * N + nme] = scale * flux * m.inv_fstar[nme];
            if (STORE_I) {   // [B][Np][column][4 angles], the cloudy column second
                float4 *it4 = reinterpret_cast<float4 *>(w.itop) + ((size_t)b * m.Np + nme) * (CLOUD ? 2 : 1);
                it4[0] = make_float4(in[0].x, in[0].y, in[1].x, in[1].y);
                if (CLOUD) it4[1] = make_float4(inc[0].x, inc[0].y, inc[1].x, inc[1].y);
            }
        }
    }
};

// Warp reduction of 8 values per lane that keeps the two lane parities apart:
// on return lane holds the sum of v[4 b4 + 2 b3 + b2] over the 8 lanes of its
// parity that share (b4, b3, b2) (bk = bit k of the lane).
__device__ __forceinline__ float reduce8_parity(const float (&v)[8], int lane) {
    float a[4], c[2];
    {
        const bool up = lane & 16;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            a[k] = (up ? v[k + 4] : v[k]) + __shfl_xor_sync(0xffffffffu, up ? v[k] : v[k + 4], 16);
    }
    {
        const bool up = lane & 8;
#pragma unroll
        for (int k = 0; k < 2; ++k)
            c[k] = (up ? a[k + 2] : a[k]) + __shfl_xor_sync(0xffffffffu, up ? a[k] : a[k + 2], 8);
    }
    const bool up = lane & 4;
    float e = (up ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, up ? c[0] : c[1], 4);
    e += __shfl_xor_sync(0xffffffffu, e, 2);
    return e;
}

// The three transpose stages of reduce8_parity: lane holds the sum of
// v[4 b4 + 2 b3 + b2] over the 8 lanes that differ from it in bits 4, 3, 2.
__device__ __forceinline__ float reduce8_partial(const float (&v)[8], int lane) {
    float a[4], c[2];
    {
        const bool up = lane & 16;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            a[k] = (up ? v[k + 4] : v[k]) + __shfl_xor_sync(0xffffffffu, up ? v[k] : v[k + 4], 16);
    }
    {
        const bool up = lane & 8;
#pragma unroll
        for (int k = 0; k < 2; ++k)
            c[k] = (up ? a[k + 2] : a[k]) + __shfl_xor_sync(0xffffffffu, up ? a[k] : a[k + 2], 8);
    }
    const bool up = lane & 4;
    return (up ? c[1] : c[0]) + __shfl_xor_sync(0xffffffffu, up ? c[0] : c[1], 4);
}

// Warp transpose-reduction of 8 values: on return lane holds the warp-wide
// sum of v[4 b4 + 2 b3 + b2].
__device__ __forceinline__ float transpose_reduce8_e(const float (&v)[8], int lane) {
    float e = reduce8_parity(v, lane);
    return e + __shfl_xor_sync(0xffffffffu, e, 1);
}

__device__ __forceinline__ float warp_total(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------- adjoint engine
template <int SPL, bool CLOUD>
struct EmisBwdEngine {
    const Model &m;
    const Work &w;
    const EmisView v;
    const int warp, lane, half, L, N, S;
    // after three transpose stages every lane holds a distinct partial sum:
    // value 4 b4 + 2 b3 + b2, parity b0, partial b1; one atomic per lane, no branch
    const int rslot, ridx;   // ridx: transpose_reduce8 slot
    const bool qwriter;
    const float ray_ref;
    // coefficients of each run are staged through shared memory one run ahead
    // (the last run of a tile stages the first run of the warp's next tile)
    static constexpr bool STAGED = 2 * SPL + 1 <= STAGE_BLOCKS;
    const uint32_t stg;
    Angles ang;

    __device__ __forceinline__ EmisBwdEngine(const Model &m_, const Work &w_, const EmisView &v_)
        : m(m_), w(w_), v(v_), warp(threadIdx.x >> 5), lane(threadIdx.x & 31), half(lane & 1), L(m_.L), N(m_.N),
          S(m_.S),
          rslot(4 * (4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1)) + 2 * (lane & 1) +
                ((lane >> 1) & 1)),
          ridx(4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1)), qwriter((lane & 3) == 0),
          ray_ref((float)(1.0 / ((double)m_.ray_nu_ref * m_.ray_nu_ref * m_.ray_nu_ref * m_.ray_nu_ref))),
          stg(smem_u32(v_.stage + (size_t)warp * STAGE_BYTES_PER_WARP) + 16u * (uint32_t)lane) {
        ang.init(m_);
    }

    // whole block, after staging sample b: its accumulators start at zero
    __device__ __forceinline__ void reset() {
        for (int idx = threadIdx.x; idx < L * 32; idx += EM_THREADS) v.red[idx] = 0.f;
        for (int s2 = threadIdx.x; s2 < ES_MAX_SPECIES; s2 += EM_THREADS) v.qtot[s2] = 0.f;
        if (threadIdx.x < N_CG) v.cpbar[threadIdx.x] = 0.f;
        if (threadIdx.x == 0) {
            v.lv->sbar = 0.f;
            v.lv->levb_bot = 0.f;
        }
    }

    // whole block: the sample's sums into the workspace by FP64 atomics
    __device__ __forceinline__ void flush(int b) {
        __syncthreads();
        for (int l = threadIdx.x; l < L; l += EM_THREADS) {
            const float *q = v.red + l * 32;
            const LayerConst &lc = v.sc->lay[l];
            // value v, parity h: q[4 v + 2 h] + q[4 v + 2 h + 1]
            float r[N_RED];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                r[0 + h] = q[0 + 2 * h] + q[1 + 2 * h];                    // QS
                r[2 + h] = (q[4 + 2 * h] + q[5 + 2 * h]) * lc.gts;         // D
                r[4 + h] = q[8 + 2 * h] + q[9 + 2 * h];                    // C
                r[6 + h] = (q[12 + 2 * h] + q[13 + 2 * h]) * lc.gtcs;      // CT
            }
            r[8] = ((q[16] + q[17]) + (q[18] + q[19])) * ray_ref;          // W4
            const float drb = (q[20] + q[21]) + (q[22] + q[23]);
            const float lvb = (q[24] + q[25]) + (q[26] + q[27]);
#pragma unroll
            for (int k = 0; k < N_RED; ++k)
                if (r[k] != 0.f) atomicAdd(w.red + ((size_t)b * L + l) * N_RED + k, (double)r[k]);
            if (drb != 0.f) atomicAdd(w.drbar + (size_t)b * L + l, (double)drb);
            if (lvb != 0.f) atomicAdd(w.levbar + (size_t)b * (L + 1) + l, (double)lvb);
            if (CLOUD) {   // d lnL / d C_l
                const float ccb = (q[28] + q[29]) + (q[30] + q[31]);
                if (ccb != 0.f) atomicAdd(w.cloud_dbar + (size_t)b * L + l, (double)ccb);
            }
        }
        if (threadIdx.x == 0 && v.lv->levb_bot != 0.f) atomicAdd(w.levbar + (size_t)b * (L + 1) + L, (double)v.lv->levb_bot);
        if (CLOUD && threadIdx.x < N_CG && v.cpbar[threadIdx.x] != 0.f)
            atomicAdd(w.cloud_pbar + (size_t)b * N_CG + threadIdx.x, (double)v.cpbar[threadIdx.x]);
        for (int s2 = threadIdx.x; s2 < S; s2 += EM_THREADS)
            if (v.qtot[s2] != 0.f) atomicAdd(w.qtot + (size_t)b * S + s2, (double)v.qtot[s2]);
        if (threadIdx.x == 0 && v.lv->sbar != 0.f) atomicAdd(w.misc + (size_t)b * 4 + 1, (double)v.lv->sbar);
    }

    // 512-wavenumber tiles [t0, t1) of the staged emission sample b
    __device__ __forceinline__ void tiles(int b, int t0, int t1) {
        const float scale = (float)w.scale[b];
        bool prestaged = false;
        for (int t = t0; t < t1; ++t) {
            const int nw = t * ET + 32 * warp;
            if (nw >= m.Np) continue;
            const int n = nw + 2 * (lane >> 1), nme = n + half;
            const bool next_ok = t + 1 < t1 && nw + ET < m.Np;   // the warp's next tile of this item
            PairInterp<SPL> pi;
            pi.init(m, n, half, lane);
            if (STAGED && !prestaged) pi.stage(stg, v.sc->lay[0].cell, v.sc->lay[0].itc, 0);
            Planck pl;
            pl.init(m.nu[nme]);
            const float4 *it4 = reinterpret_cast<const float4 *>(w.itop) + ((size_t)b * m.Np + nme) * (CLOUD ? 2 : 1);
            const float4 i4 = it4[0];
            const float2 itoa[2] = {make_float2(i4.x, i4.y), make_float2(i4.z, i4.w)};
            const float db = w.dbar[(size_t)b * m.Np + nme];   // zero beyond N
            const float fsc = m.inv_fstar[nme];
            const float fbar = db * scale * fsc;
            // d lnL / d I_toa per angle: the clear column weighted 1 - f_cld, the cloudy one f_cld
            const float wcf = CLOUD ? 1.f - v.cg[3] : 1.f, wcl = CLOUD ? v.cg[3] : 0.f;
            const float2 ib[2] = {mul2(f2(fbar * wcf), ang.wt[0]), mul2(f2(fbar * wcf), ang.wt[1])};
            const float2 ibc[2] = {mul2(f2(fbar * wcl), ang.wt[0]), mul2(f2(fbar * wcl), ang.wt[1])};
            float2 itc[2] = {f2(0.f), f2(0.f)};
            if (CLOUD) {
                const float4 c4 = it4[1];
                itc[0] = make_float2(c4.x, c4.y);
                itc[1] = make_float2(c4.z, c4.w);
            }
            const float gc = CLOUD ? kh18_g(v.cg, m.nu[nme]) : 0.f;
            float gacc = 0.f;                          // d lnL / d g(nu) of the lane's wavenumber
            float dbdt;
            float bt = pl.value_dt(v.lv->inv_t[0], dbdt);
            float bprev = 0.f;                         // B_bar of the current top level from the layer above
            float2 tr[2] = {f2(1.f), f2(1.f)}, pre[2] = {f2(0.f), f2(0.f)};
            float2 trc[2] = {f2(1.f), f2(1.f)}, prec[2] = {f2(0.f), f2(0.f)};   // cloudy column
            float2 qa[SPL];
#pragma unroll
            for (int j = 0; j < SPL; ++j) qa[j] = f2(0.f);
            for (int l = 0; l < L;) {
                // broadcast from lane 0: provably warp-uniform for the compiler
                const int end = __shfl_sync(0xffffffffu, v.sc->lay[l].run_end, 0);
                if constexpr (STAGED) {
                    pi.load_staged(*v.sc, stg);
                    if (end < L) pi.stage(stg, v.sc->lay[end].cell, v.sc->lay[end].itc, 0);
                    else if (next_ok) pi.stage(stg, v.sc->lay[0].cell, v.sc->lay[0].itc, ET);
                } else {
                    pi.load(*v.sc, v.sc->lay[l].cell, v.sc->lay[l].itc);
                    if (end < L) pi.prefetch(v.sc->lay[end].cell, v.sc->lay[end].itc);
                }
                for (; l < end; ++l) {
                    const LayerConst &lc = v.sc->lay[l];
                    // extinction, keeping this lane's species terms
                    float2 p[SPL];
                    float2 sum = f2(0.f), pt = f2(0.f);
#pragma unroll
                    for (int j = 0; j < SPL; ++j) {
                        float2 tj;
                        p[j] = ex2x2(pi.expo(j, lc.wp, lc.wt, tj));
                        sum = add2(sum, p[j]);
                        pt = fma2(p[j], tj, pt);
                    }
                    const float2 cc = pi.cia(lc);
                    const float2 mine = pi.part(lc, sum, cc);
                    const float alpha = own(add2(mine, shfl_xor2(mine, 1)), half);
                    const float dtau = alpha * v.lv->dr[l];
                    float dbdt_b;
                    const float bb = pl.value_dt(v.lv->inv_t[l + 1], dbdt_b);
                    float btb = bprev, bbb = 0.f;
                    const float dtb = rt_layer_bwd(ang, dtau, bt, bb, itoa, ib, tr, pre, btb, bbb);
                    // cloudy column: dtau + C_l g dr (alpha_bar as the clear one's; C_l bar, g bar)
                    const float acl = CLOUD ? v.lv->ccl[l] * gc : 0.f;
                    float dtbc = 0.f;
                    if (CLOUD) {
                        dtbc = rt_layer_bwd(ang, fmaf(acl, v.lv->dr[l], dtau), bt, bb, itc, ibc, trc, prec, btb, bbb);
                        gacc = fmaf(dtbc * v.lv->dr[l], v.lv->ccl[l], gacc);
                    }
                    // alpha_bar of both wavenumbers of the pair
                    const float abar_me = (dtb + dtbc) * v.lv->dr[l];
                    const float2 ab = make_float2(__shfl_sync(0xffffffffu, abar_me, lane & 30),
                                                  __shfl_sync(0xffffffffu, abar_me, lane | 1));
                    const float2 abn = mul2(ab, lc.nsc);
#pragma unroll
                    for (int j = 0; j < SPL; ++j) qa[j] = fma2(abn, p[j], qa[j]);
                    const float2 ac = mul2(ab, cc);
                    const float2 act = mul2(ac, pi.d);
                    float vr[8];
                    vr[0] = fmaf(abn.x, sum.x, abn.y * sum.y);
                    vr[1] = fmaf(abn.x, pt.x, abn.y * pt.y);                   // x gts at the flush
                    vr[2] = ac.x + ac.y;
                    vr[3] = act.x + act.y;                                     // x gtcs at the flush
                    vr[4] = fmaf(ab.x, pi.nu4.x, ab.y * pi.nu4.y);             // zero on the odd lane; x ray_ref
                    vr[5] = fmaf(dtbc, acl, (dtb + dtbc) * alpha);              // dr_bar
                    vr[6] = btb * dbdt;                                         // T_bar of level l
                    vr[7] = CLOUD ? dtbc * v.lv->dr[l] * gc : 0.f;                 // C_l bar
                    atomicAdd(v.red + l * 32 + rslot, reduce8_partial(vr, lane));
                    bprev = bbb;
                    bt = bb;
                    dbdt = dbdt_b;
                }
            }
            // bottom level: from the last layer and the surface term I = B_bottom below it
            float bl = bprev;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                bl = fmaf(ib[q].x, tr[q].x, fmaf(ib[q].y, tr[q].y, bl));
                if (CLOUD) bl = fmaf(ibc[q].x, trc[q].x, fmaf(ibc[q].y, trc[q].y, bl));
            }
            const float lev_last = warp_total(bl * dbdt);
            float flux = flux_of(ang, itoa);
            if (CLOUD) {
                // f_cld and g(nu) -> the g(nu) parameters at the lane's wavenumber
                const float fcl = flux_of(ang, itc);
                const float fb = warp_total(db * scale * fsc * (fcl - flux));
                float o[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (gacc != 0.f) kh18_g_adjoint(v.cg, m.nu[nme], gacc, o);
                cloud_pbar_add(v.cg, o, v.cpbar, lane);
                if (lane == 0) atomicAdd(v.cpbar + 3, fb);
                flux = wcl * fcl + wcf * flux;
            }
            const float sb = warp_total(db * flux * fsc);
            if (lane == 0) {
                atomicAdd(&v.lv->levb_bot, lev_last);
                atomicAdd(&v.lv->sbar, sb);
            }
            // per-species totals: slot j of lane half h is species SPL h + j
#pragma unroll
            for (int c0 = 0; c0 < 2 * SPL; c0 += 8) {
                float vq[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int sl = c0 + k;
                    vq[k] = (sl < 2 * SPL && sl / SPL == half) ? qa[sl % SPL].x + qa[sl % SPL].y : 0.f;
                }
                const float tq = transpose_reduce8_e(vq, lane);
                if (qwriter && c0 + ridx < S && tq != 0.f) atomicAdd(v.qtot + c0 + ridx, tq);
            }
            prestaged = STAGED && next_ok;
        }
    }
};

}  // namespace
}  // namespace es
