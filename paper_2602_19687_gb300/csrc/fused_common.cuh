// Building blocks of the fused per-tile kernels: packed FP32x2 arithmetic,
// the split of FP32 values into BF16 hi + lo pairs for the tensor-core
// operands, per-sample layer constants, and the register-cached opacity
// interpolation of a wavenumber pair.
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace es {

constexpr int LP = 112;           // layers padded to 7 x 16 (tensor-core K/M blocks)
constexpr float KSHIFT = 64.f;    // log2 scale folded into the species exponents

// ------------------------------------------------------------ packed FP32x2
// Two FP32 lanes per instruction (sm_100+ FFMA2/FADD2/FMUL2 builtins).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// float2 <-> 64-bit register pair (no data movement: keeps the two lanes of
// a packed operand in one aligned pair across inline asm and shuffles)
__device__ __forceinline__ unsigned long long f2_bits(float2 v) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
    return r;
}
__device__ __forceinline__ float2 bits_f2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 ex2x2(float2 x) {
    unsigned long long r;
    asm("{\n\t.reg .f32 a, b;\n\tex2.approx.ftz.f32 a, %1;\n\tex2.approx.ftz.f32 b, %2;\n\tmov.b64 %0, {a, b};\n\t}"
        : "=l"(r) : "f"(x.x), "f"(x.y));
    return bits_f2(r);
}
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// ------------------------------------------------------------ BF16 split
// x = hi + lo with hi, lo BF16 (hi round-to-nearest, lo the rounded residual)
__device__ __forceinline__ void split2(float2 x, uint32_t &hi, uint32_t &lo) {
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x.y), "f"(x.x));
    const float2 h = make_float2(__uint_as_float(hi << 16), __uint_as_float(hi & 0xffff0000u));
    const float2 r = fma2(h, f2(-1.f), x);   // x - hi, exact
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(r.y), "f"(r.x));
}
// round-to-nearest BF16 pair (x.x in the low half)
__device__ __forceinline__ uint32_t bf16x2(float2 x) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(x.y), "f"(x.x));
    return r;
}
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// 16-byte asynchronous global -> shared copies (bypassing L1), their group
// commit and the wait for all of this thread's groups
__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ float4 lds128(uint32_t saddr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(saddr)
                 : "memory");
    return v;
}
// Per-warp staging of a run's coefficients: [2 SPL + 1 blocks][32 lanes] float4
// (species blocks (j, c), then the CIA pair), for SPL <= 4.
constexpr int STAGE_BLOCKS = 9;
constexpr int STAGE_BYTES_PER_WARP = STAGE_BLOCKS * 32 * 16;

// ------------------------------------------------------------ per-sample constants
// Per-layer constants, with the operands of packed FP32x2 instructions stored
// as duplicated pairs so that the layer loop needs no register moves.
struct __align__(16) LayerConst {
    float2 wp, wt;       // pressure / temperature interpolation weights
    float2 nsc, wtc;     // n_l 2^-KSHIFT; CIA temperature weight
    float2 cc[2];        // log2(n^2 X_H2^2), log2(n^2 X_H2 X_He): CIA pair 0 / 1
    float2 ray;          // n (X_H2 s_H2 + X_He s_He) / nu_ref^4
    float gts, gtcs;     // d/dlog10 T of the log2 exponents: gt / log2(10), gtc / log2(10)
    int cell, itc;       // (T, p) table cell = it * (NP - 1) + ip; CIA temperature bracket
    int run_end;         // first layer after l whose (cell, itc) differs (or L)
    int aoff;            // byte offset of row l in a core-matrix operand with 8-row stride asbo
};

struct SampleConst {
    LayerConst lay[ES_MAX_LAYERS];
    float lx[ES_MAX_SPECIES];   // log2 X_s + KSHIFT
    int gb[12];                 // layer-group boundaries gb[0] = 0 <= ... <= gb[groups] = L
};

// Relative cost of starting a run of layers (a coefficient reload from L2)
// against interpolating one layer, for balancing the layer groups: measured
// best at 3 for the forward interpolation and 1 for the adjoint's (whose
// layers cost more: reductions and the pair exchange of alpha_bar).
constexpr float RUN_COST_FWD = 3.f, RUN_COST_BWD = 1.f;

// All threads of the block: per-layer constants of sample b into shared memory,
// and the boundaries of `groups` (<= 11) layer groups of equal cost.
__device__ inline void stage_sample(const Model &m, const Work &w, int b, SampleConst &sc, float run_cost,
                                    int asbo = 0, int groups = 4) {
    const float ry = (float)(1.0 / ((double)m.ray_nu_ref * m.ray_nu_ref * m.ray_nu_ref * m.ray_nu_ref));
    const float il2 = (float)(1.0 / LOG2_10);
    const int L = m.L;
    const size_t b0 = (size_t)b * L;
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        const size_t bl = b0 + l;
        LayerConst c;
        const int it = w.it[bl], itc = w.itc[bl];
        c.cell = it * (m.NP - 1) + m.ip[l];
        c.itc = itc;
        c.run_end = l + 1;   // set below, once every layer's (cell, itc) is staged
        c.aoff = (l >> 3) * asbo + (l & 7) * 16;
        c.wp = f2(m.wp[l]);
        c.wt = f2(w.wtr[bl]);
        c.wtc = f2(w.wtc[bl]);
        c.nsc = f2((float)(w.n_lay[bl] * 5.421010862427522e-20));   // 2^-64
        c.cc[0] = f2(w.ccia[2 * bl]);
        c.cc[1] = f2(w.ccia[2 * bl + 1]);
        c.ray = f2(w.ray[bl] * ry);
        c.gts = w.gt[bl] * il2;
        c.gtcs = w.gtc[bl] * il2;
        sc.lay[l] = c;
    }
    // absent species (s >= S, padding of the per-lane species slots) get a
    // log2 weight so low that their terms are exactly zero
    for (int s = threadIdx.x; s < ES_MAX_SPECIES; s += blockDim.x) {
        const double x = (s < m.S) ? w.xs[(size_t)b * (m.S + 2) + s] : 0.0;
        sc.lx[s] = (x > 0.0) ? (float)(log2(x) + KSHIFT) : -1.0e4f;
    }
    __syncthreads();
    // end of each layer's run of equal (cell, CIA bracket): a short scan in shared memory
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        const int cell = sc.lay[l].cell, itc = sc.lay[l].itc;
        int r = l + 1;
        while (r < L && sc.lay[r].cell == cell && sc.lay[r].itc == itc) ++r;
        sc.lay[l].run_end = r;
    }
    __syncthreads();
    // layer groups of equal cost: one per layer plus run_cost per run start
    if (threadIdx.x == 0) {
        float total = 0.f;
        for (int l = 0; l < L; ++l) total += 1.f + ((l == 0 || sc.lay[l - 1].run_end == l) ? run_cost : 0.f);
        const float share = 1.f / (float)groups;
        int g = 1;
        float acc = 0.f;
        sc.gb[0] = 0;
        for (int l = 0; l < L && g < groups; ++l) {
            acc += 1.f + ((l == 0 || sc.lay[l - 1].run_end == l) ? run_cost : 0.f);
            if (acc >= total * (float)g * share) sc.gb[g++] = l + 1;
        }
        while (g < groups) sc.gb[g++] = L;
        sc.gb[groups] = L;
    }
}


// ------------------------------------------------------------ interpolation
// Coefficient table layout (k_tables.cu): per (cell, wavenumber pair) the SP
// species slots, each as two float4 (a0, a0', a1, a1'), (a2, a2', a3, a3'),
// so a lane's SPL slots are one contiguous 32 SPL-byte block and each
// coefficient loads straight into an aligned register pair.

// Per-lane interpolation state for SPL species per lane. A wavenumber pair is
// shared by two lanes (h = lane & 1): lane h interpolates species SPL h ..
// SPL h + SPL - 1 (slots beyond S read species S-1 with a zero weight) and
// CIA pair h, keeping the current (T, p) cell's coefficients in registers.
// The layer loops run over runs of layers with one (cell, CIA bracket), so
// coefficients are loaded once per run and the per-layer body has no tests.
template <int SPL>
struct PairInterp {
    float2 a0[SPL], a1[SPL], a2[SPL], a3[SPL];
    float2 b, d;
    float2 nu4;          // nu^4 on lane h = 0, zero on h = 1 (Rayleigh counted once per pair)
    int h = 0;
    const float4 *cp;    // this lane's slot j = 0, c = 0 of its wavenumber pair in cell 0
    const float4 *pfp;   // the line this lane prefetches for the warp, in cell 0
    const float4 *ciap;  // this lane's CIA pair at bracket 0
    size_t cstride;      // float4 per cell
    int jstride;         // float4 between (j, c) blocks: Np (= 2 x pairs x halves / 2)
    int cia_stride;      // float4 per CIA temperature bracket

    // n: the pair's first wavenumber; the warp's lanes 2q, 2q + 1 cover 16
    // consecutive pairs, the first at n - 2 q
    __device__ __forceinline__ void init(const Model &m, int n, int half, int lane) {
        const int n_warp = n - (lane & 30);
        const float2 nu = __ldg(reinterpret_cast<const float2 *>(m.nu + n));
        const float2 nu2 = mul2(nu, nu);
        nu4 = half ? f2(0.f) : mul2(nu2, nu2);
        h = half;
        jstride = m.Np;
        cstride = (size_t)m.Np * m.SP;
        cp = m.coef4 + (size_t)n + half;            // ((pair) * 2 + h) with pair = n / 2
        // the warp's 2 SPL (j, c) blocks of 512 B = 4 lines each: lane -> one line
        const int blk = (lane >> 2) & ((2 * SPL < 8 ? 2 * SPL : 8) - 1);
        pfp = m.coef4 + (size_t)blk * m.Np + n_warp + 8 * (lane & 3);
        cia_stride = m.Np;
        ciap = m.cia4 + (size_t)n + half;
    }
    // coefficients of a run: this lane's species slots in `cell`, CIA pair h in bracket itc
    __device__ __forceinline__ void load(const SampleConst &sc, int cell, int itc) {
        const float4 *p = cp + (size_t)cell * cstride;
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
            const float4 c0 = __ldg(p + (2 * j) * jstride), c1 = __ldg(p + (2 * j + 1) * jstride);
            a0[j] = add2(make_float2(c0.x, c0.y), f2(sc.lx[SPL * h + j]));
            a1[j] = make_float2(c0.z, c0.w);
            a2[j] = make_float2(c1.x, c1.y);
            a3[j] = make_float2(c1.z, c1.w);
        }
        const float4 k = __ldg(ciap + (size_t)itc * cia_stride);
        b = make_float2(k.x, k.y);
        d = make_float2(k.z, k.w);
    }
    // asynchronous copy of a run's coefficients (shift: float4 offset of the
    // tile, 0 or the next tile's 128) into this lane's staging slots `stg`
    __device__ __forceinline__ void stage(uint32_t stg, int cell, int itc, int shift) const {
        const float4 *p = cp + (size_t)cell * cstride + shift;
#pragma unroll
        for (int k = 0; k < 2 * SPL; ++k) cp_async16(stg + k * 512, p + (size_t)k * jstride);
        cp_async16(stg + 2 * SPL * 512, ciap + (size_t)itc * cia_stride + shift);
        cp_async_commit();
    }
    // the staged run: wait for this lane's copies, then read its own slots
    __device__ __forceinline__ void load_staged(const SampleConst &sc, uint32_t stg) {
        cp_async_wait_all();
#pragma unroll
        for (int j = 0; j < SPL; ++j) {
            const float4 c0 = lds128(stg + (2 * j) * 512), c1 = lds128(stg + (2 * j + 1) * 512);
            a0[j] = add2(make_float2(c0.x, c0.y), f2(sc.lx[SPL * h + j]));
            a1[j] = make_float2(c0.z, c0.w);
            a2[j] = make_float2(c1.x, c1.y);
            a3[j] = make_float2(c1.z, c1.w);
        }
        const float4 k = lds128(stg + 2 * SPL * 512);
        b = make_float2(k.x, k.y);
        d = make_float2(k.z, k.w);
    }
    // L1 prefetch of the next run's coefficients: the warp's 2 SPL x 512 B,
    // one 128-B line per lane (two for SPL = 8), and the lane's CIA entry
    __device__ __forceinline__ void prefetch(int cell, int itc) const {
        const float4 *p = pfp + (size_t)cell * cstride;
#pragma unroll
        for (int k = 0; k < (2 * SPL * 4 + 31) / 32; ++k)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(p + (size_t)k * 8 * jstride));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(ciap + (size_t)itc * cia_stride));
    }
    // exponent of species slot j: e = a0 + wp a1 + wt (a2 + wp a3); t = de/dwt
    __device__ __forceinline__ float2 expo(int j, float2 wp, float2 wt, float2 &t) const {
        t = fma2(wp, a3[j], a2[j]);
        return fma2(wt, t, fma2(wp, a1[j], a0[j]));
    }
    // CIA term of this lane's pair
    __device__ __forceinline__ float2 cia(const LayerConst &lc) const {
        return ex2x2(fma2(lc.wtc, d, add2(b, lc.cc[h])));
    }
    // this lane's part of alpha: n 2^-K (its species sum) + its CIA pair (+ Rayleigh on h = 0)
    __device__ __forceinline__ float2 part(const LayerConst &lc, float2 sum, float2 c) const {
        return fma2(lc.ray, nu4, fma2(sum, lc.nsc, c));
    }
};

__device__ __forceinline__ float2 shfl_xor2(float2 v, int o) {
    return bits_f2(__shfl_xor_sync(0xffffffffu, f2_bits(v), o));
}

// Extinction alpha_l(nu) at wavenumber pair n, n+1 for layers [lb, le), the
// lane pair (lane, lane ^ 1) splitting species and CIA pairs:
//   alpha = n 2^-K sum_s 2^e_s + CIA_H2H2 + CIA_H2He + Rayleigh.
// Calls out(layer constants, alpha) on both lanes of the pair. Coefficients
// are loaded directly at each run's start, with an L1 prefetch of the next
// run (staging them through shared memory costs the forward more in queue
// throttling and L1 than it saves).
template <int SPL, class Out>
__device__ __forceinline__ void extinction_pair(const Model &m, const SampleConst &sc, int lb, int le, int n,
                                                int half, Out &&out) {
    PairInterp<SPL> pi;
    pi.init(m, n, half, threadIdx.x & 31);
    // loop bounds broadcast from lane 0: provably warp-uniform for the compiler
    lb = __shfl_sync(0xffffffffu, lb, 0);
    le = __shfl_sync(0xffffffffu, le, 0);
    for (int l = lb; l < le;) {
        const int end = __shfl_sync(0xffffffffu, min(sc.lay[l].run_end, le), 0);
        pi.load(sc, sc.lay[l].cell, sc.lay[l].itc);
        if (end < le) pi.prefetch(sc.lay[end].cell, sc.lay[end].itc);
        const LayerConst *lp = &sc.lay[l], *const lend = &sc.lay[end];
        // two layers per iteration: independent chains for the schedulers
        for (; lp + 1 < lend; lp += 2) {
            const LayerConst &c0 = lp[0], &c1 = lp[1];
            float2 t, s0 = ex2x2(pi.expo(0, c0.wp, c0.wt, t)), s1 = ex2x2(pi.expo(0, c1.wp, c1.wt, t));
#pragma unroll
            for (int j = 1; j < SPL; ++j) {
                s0 = add2(s0, ex2x2(pi.expo(j, c0.wp, c0.wt, t)));
                s1 = add2(s1, ex2x2(pi.expo(j, c1.wp, c1.wt, t)));
            }
            const float2 m0 = fma2(c0.ray, pi.nu4, fma2(s0, c0.nsc, pi.cia(c0)));
            const float2 m1 = fma2(c1.ray, pi.nu4, fma2(s1, c1.nsc, pi.cia(c1)));
            const float2 o0 = shfl_xor2(m0, 1), o1 = shfl_xor2(m1, 1);
            out(c0, add2(m0, o0));
            out(c1, add2(m1, o1));
        }
        if (lp != lend) {
            const LayerConst &lc = *lp;
            float2 t, sum = ex2x2(pi.expo(0, lc.wp, lc.wt, t));
#pragma unroll
            for (int j = 1; j < SPL; ++j) sum = add2(sum, ex2x2(pi.expo(j, lc.wp, lc.wt, t)));
            const float2 mine = fma2(lc.ray, pi.nu4, fma2(sum, lc.nsc, pi.cia(lc)));
            out(lc, add2(mine, shfl_xor2(mine, 1)));
        }
        l = end;
    }
}

// Work items (sample b, wavenumber chunk c) of the persistent kernels, in one
// of two orders: chunk-major (all samples of chunk 0, then chunk 1, ...: the
// blocks running together share a wavenumber window of the coefficient table
// in L2) or sample-major (all chunks of sample 0, then sample 1, ...: each
// block stages fewer samples). The autotuner picks the order.
struct ItemOrder {
    int B, nchunks, sample_major;
    __device__ __forceinline__ long long total() const { return (long long)B * nchunks; }
    __device__ __forceinline__ void at(long long item, int &c, int &b) const {
        if (sample_major) {
            b = (int)(item / nchunks);
            c = (int)(item % nchunks);
        } else {
            c = (int)(item / B);
            b = (int)(item % B);
        }
    }
};

// Sum over the warp, on every lane.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------ non-grey cloud
// Sect. 2.5 extinction efficiency with Q_1 folded into q_c^eff, g(nu) = Q_ext/Q_1:
// the continuum 1/u, u = Q0 x^-a + x^0.2, x = 2 pi r_eff nu, and with the
// mid-infrared feature (Sect. 2.5.3; on when A = cg[4] != 0)
//   g = min(1/u + W(x) Q_feat, Q_max),  W = exp(-x / x0),
//   Q_feat = 2 A exp(-z^2/2) Phi(xi z),  z = (lambda - lambda_0) / omega,
// lambda in micron. cg = (2 pi r_eff, a, Q0, f_cld, A, lambda_0, omega, xi).
constexpr float FEAT_INV_X0 = 2.f;   // 1 / x0, x0 = 0.5
constexpr float Q_EXT_MAX = 2.f;

struct CloudFeature {
    float z, e, cdf, win, qf;   // z, exp(-z^2/2), Phi(xi z), W(x), Q_feat
    __device__ __forceinline__ CloudFeature(const float *cg, float nu, float x) {
        z = (1.0e4f / nu - cg[5]) / cg[6];
        e = expf(-0.5f * z * z);
        cdf = normcdff(cg[7] * z);
        win = expf(-x * FEAT_INV_X0);
        qf = 2.f * cg[4] * e * cdf;
    }
};

__device__ __forceinline__ float kh18_g(const float *cg, float nu) {
    const float x = cg[0] * nu, lx = log2f(x);
    float g = 1.f / (cg[2] * exp2f(-cg[1] * lx) + exp2f(0.2f * lx));
    if (cg[4] != 0.f) {
        const CloudFeature f(cg, nu, x);
        g = fminf(fmaf(f.win, f.qf, g), Q_EXT_MAX);
    }
    return g;
}

// Given gb = d lnL / d g(nu), the derivatives o = d lnL / d (ln r_eff, a,
// ln Q0, A, lambda_0, omega, xi) at this wavenumber. Continuum (u as above,
// g_c = 1/u): dg/dln x = -g_c^2 (0.2 x^0.2 - a Q0 x^-a), dg/da = g_c^2 Q0
// x^-a ln x, dg/dln Q0 = -g_c^2 Q0 x^-a. Feature: dW/dln x = -(x/x0) W,
// dQ_feat/dA = Q_feat/A, dQ_feat/dz = 2A exp(-z^2/2) (xi phi(xi z) - z Phi(xi z)),
// dz/dlambda_0 = -1/omega, dz/domega = -z/omega, dQ_feat/dxi = 2A exp(-z^2/2)
// phi(xi z) z, phi the normal density. At the cap g is flat: all zero.
__device__ __forceinline__ void kh18_g_adjoint(const float *cg, float nu, float gb, float (&o)[7]) {
    const float x = cg[0] * nu, lx = log2f(x), xa = cg[2] * exp2f(-cg[1] * lx), x2 = exp2f(0.2f * lx);
    const float gc = 1.f / (xa + x2), gg = gb * gc * gc;
    o[0] = -gg * (0.2f * x2 - cg[1] * xa);
    o[1] = gg * xa * lx * 0.6931471805599453f;
    o[2] = -gg * xa;
    o[3] = o[4] = o[5] = o[6] = 0.f;
    if (cg[4] != 0.f) {
        const CloudFeature f(cg, nu, x);
        if (fmaf(f.win, f.qf, gc) < Q_EXT_MAX) {
            const float gw = gb * f.win;
            const float pdf = 0.3989422804014327f * expf(-0.5f * cg[7] * cg[7] * f.z * f.z);
            const float dqdz = 2.f * cg[4] * f.e * (cg[7] * pdf - f.z * f.cdf);
            o[0] -= gw * f.qf * x * FEAT_INV_X0;
            o[3] = gw * 2.f * f.e * f.cdf;
            o[4] = -gw * dqdz / cg[6];
            o[5] = -gw * dqdz * f.z / cg[6];
            o[6] = gw * 2.f * cg[4] * f.e * pdf * f.z;
        } else {
            o[0] = o[1] = o[2] = 0.f;
        }
    }
}

// Sums a warp's g-parameter adjoints (kh18_g_adjoint) and adds them to the
// sample's accumulators: cpbar = (ln r_eff, a, ln Q0, f_cld, A, lambda_0,
// omega, xi); the feature's four only when it is on (cg[4] != 0).
__device__ __forceinline__ void cloud_pbar_add(const float *cg, float (&o)[7], float *cpbar, int lane) {
#pragma unroll
    for (int k = 0; k < 3; ++k) o[k] = warp_sum(o[k]);
    if (lane == 0)
        for (int k = 0; k < 3; ++k) atomicAdd(cpbar + k, o[k]);
    if (cg[4] != 0.f) {
#pragma unroll
        for (int k = 3; k < 7; ++k) o[k] = warp_sum(o[k]);
        if (lane == 0)
            for (int k = 3; k < 7; ++k) atomicAdd(cpbar + k + 1, o[k]);
    }
}

}  // namespace es
