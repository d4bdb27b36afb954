// Building blocks of the fused per-tile kernels: warp-level BF16 tensor-core
// MMA (split-precision), packed FP32x2 arithmetic, and the register-cached
// opacity interpolation of one 64-wavenumber tile.
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace es {

constexpr int FT = 64;            // wavenumbers per tile
constexpr int FWARPS = 8;         // warps per fused block
constexpr int FTHREADS = FWARPS * 32;
constexpr int LP = 112;           // layers padded to 7 x 16 (tensor-core K/M blocks)
constexpr float KSHIFT = 64.f;    // log2 scale folded into the species exponents
constexpr int L_PITCH = 120;      // bf16 pitch of [112][112] path-matrix rows (240 B: 15 x 16 B)
constexpr int R_PITCH = 72;       // bf16 pitch of [row][64 nu] operand rows (144 B: 9 x 16 B)

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
__device__ __forceinline__ float2 ex2x2(float2 x) { return make_float2(ex2f(x.x), ex2f(x.y)); }
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }

// ------------------------------------------------------------ BF16 split and tensor cores
// x = hi + lo with hi, lo BF16 (hi round-to-nearest, lo the rounded residual)
__device__ __forceinline__ void split2(float2 x, uint32_t &hi, uint32_t &lo) {
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x.y), "f"(x.x));
    float hx = __uint_as_float(hi << 16), hy = __uint_as_float(hi & 0xffff0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x.y - hy), "f"(x.x - hx));
}
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void ldsm_x4(uint32_t a, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t a, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2(uint32_t a, uint32_t (&r)[2]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t a, uint32_t (&r)[2]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r[0]), "=r"(r[1]) : "r"(a));
}
// D += A B, m16n8k16, BF16 inputs, FP32 accumulation
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// split-precision product: (Ah + Al)(Bh + Bl) ~ Ah Bh + Ah Bl + Al Bh
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                     const uint32_t (&bh)[2], const uint32_t (&bl)[2]) {
    mma16816(d, al, bh);
    mma16816(d, ah, bl);
    mma16816(d, ah, bh);
}

// Address of lane's ldmatrix row for an A fragment (m16 x k16) of a row-major
// [m][k] BF16 array with `pitch` elements per row.
__device__ __forceinline__ uint32_t a_addr(uint32_t base, int pitch, int m0, int k0, int lane) {
    return base + 2u * (uint32_t)((m0 + (lane & 15)) * pitch + k0 + ((lane >> 4) << 3));
}
// A fragment (m16 x k16) of A = S^T where S is stored row-major [k][m] (ldmatrix .trans)
__device__ __forceinline__ uint32_t at_addr(uint32_t base, int pitch, int m0, int k0, int lane) {
    const int q = lane >> 3, r = lane & 7;   // matrix q: (k half, m half) = (q>>1, q&1)
    return base + 2u * (uint32_t)((k0 + ((q >> 1) << 3) + r) * pitch + m0 + ((q & 1) << 3));
}
// B fragment (k16 x n8) from a row-major [n][k] array (ldmatrix, non-trans)
__device__ __forceinline__ uint32_t b_addr(uint32_t base, int pitch, int n0, int k0, int lane) {
    const int l = lane & 15;
    return base + 2u * (uint32_t)((n0 + (l & 7)) * pitch + k0 + ((l >> 3) << 3));
}
// B fragment (k16 x n8) from a row-major [k][n] array (ldmatrix .trans)
__device__ __forceinline__ uint32_t bt_addr(uint32_t base, int pitch, int n0, int k0, int lane) {
    const int l = lane & 15;
    return base + 2u * (uint32_t)((k0 + l) * pitch + n0);
}

// ------------------------------------------------------------ per-sample constants
struct __align__(16) LayerConst {
    int it, ip, itc, cell;   // temperature / pressure / CIA brackets; cell = it * (NP - 1) + ip
    float wt, wp, wtc;       // raw interpolation weights
    float nsc;               // n_l 2^-KSHIFT
    float cc1, cc2;          // log2(n^2 X_H2^2), log2(n^2 X_H2 X_He)
    float ray;               // n (X_H2 s_H2 + X_He s_He) / nu_ref^4
    float gt, gtc;           // 1/dlog10T and 1/dT of the brackets (0 where clamped)
    float pad[3];
};

struct SampleConst {
    LayerConst lay[ES_MAX_LAYERS];
    float lx[ES_MAX_SPECIES];   // log2 X_s + KSHIFT
};

// All threads of the block: per-layer constants of sample b into shared memory.
__device__ inline void stage_sample(const Model &m, const Work &w, int b, SampleConst &sc) {
    const float ry = (float)(1.0 / ((double)m.ray_nu_ref * m.ray_nu_ref * m.ray_nu_ref * m.ray_nu_ref));
    for (int l = threadIdx.x; l < m.L; l += blockDim.x) {
        const size_t bl = (size_t)b * m.L + l;
        LayerConst c;
        c.it = w.it[bl];
        c.ip = m.ip[l];
        c.itc = w.itc[bl];
        c.cell = c.it * (m.NP - 1) + c.ip;
        c.wt = w.wtr[bl];
        c.wp = m.wp[l];
        c.wtc = w.wtc[bl];
        c.nsc = (float)(w.n_lay[bl] * 5.421010862427522e-20);   // 2^-64
        c.cc1 = w.ccia[2 * bl];
        c.cc2 = w.ccia[2 * bl + 1];
        c.ray = w.ray[bl] * ry;
        c.gt = w.gt[bl];
        c.gtc = w.gtc[bl];
        c.pad[0] = c.pad[1] = c.pad[2] = 0.f;
        sc.lay[l] = c;
    }
    // absent species (s >= S, padding of the per-lane species slots) get a
    // log2 weight so low that their terms are exactly zero
    for (int s = threadIdx.x; s < ES_MAX_SPECIES; s += blockDim.x) {
        const double x = (s < m.S) ? w.xs[(size_t)b * (m.S + 2) + s] : 0.0;
        sc.lx[s] = (x > 0.0) ? (float)(log2(x) + KSHIFT) : -1.0e4f;
    }
}

// Layers of layer group `g` out of `ng` (contiguous ranges).
__device__ __forceinline__ void group_layers(int L, int g, int ng, int &lb, int &le) {
    const int per = (L + ng - 1) / ng;
    lb = g * per;
    le = min(L, lb + per);
}

// ------------------------------------------------------------ interpolation
// Coefficient table layout (see k_tables.cu): per (cell, species) and
// wavenumber pair, two float4: (a0, a0', a1, a1') and (a2, a2', a3, a3') for
// the pair's two wavenumbers, so each coefficient loads straight into an
// aligned register pair.
__device__ __forceinline__ void load_cell(const Model &m, int s, int cell, int n, float lx, float2 &a0, float2 &a1,
                                          float2 &a2, float2 &a3) {
    const float4 *p = m.coef4 + (((size_t)cell * m.S + s) * (m.Np >> 1) + (n >> 1)) * 2;
    const float4 c0 = __ldg(p), c1 = __ldg(p + 1);
    a0 = add2(make_float2(c0.x, c0.y), f2(lx));
    a1 = make_float2(c0.z, c0.w);
    a2 = make_float2(c1.x, c1.y);
    a3 = make_float2(c1.z, c1.w);
}

// CIA coefficients of one temperature bracket: e = b + wtc d + cc
__device__ __forceinline__ void load_cia(const Model &m, int pair, int itc, int n, float2 &b, float2 &d) {
    const size_t st = (size_t)m.Np;
    const float *base = m.cia + ((size_t)pair * m.NTc + itc) * st + n;
    const float2 k0 = __ldg(reinterpret_cast<const float2 *>(base));
    const float2 k1 = __ldg(reinterpret_cast<const float2 *>(base + st));
    const float2 c = f2((float)LOG2_10);
    b = mul2(c, k0);
    d = mul2(c, add2(k1, make_float2(-k0.x, -k0.y)));
}

// Per-lane interpolation state for SPL species per lane. A wavenumber pair is
// shared by two lanes (h = lane & 1): lane h interpolates species SPL h ..
// SPL h + SPL - 1 (slots beyond S read species S-1 with a zero weight) and
// CIA pair h, keeping the current (T, p) cell's coefficients in registers;
// cells change only every few layers.
template <int SPL>
struct PairInterp {
    float2 a0[SPL], a1[SPL], a2[SPL], a3[SPL];
    float2 b, d, nu4;
    int cell = -1, itc = -1, h = 0;

    __device__ __forceinline__ void init(const Model &m, int n, int half) {
        const float2 nu = __ldg(reinterpret_cast<const float2 *>(m.nu + n));
        const float2 nu2 = mul2(nu, nu);
        nu4 = mul2(nu2, nu2);
        cell = itc = -1;
        h = half;
    }
    __device__ __forceinline__ int slot(int j) const { return SPL * h + j; }
    __device__ __forceinline__ int table_species(const Model &m, int j) const { return min(slot(j), m.S - 1); }
    // L1 prefetch of the next layer's cell coefficients when the cell changes
    __device__ __forceinline__ void prefetch(const Model &m, const LayerConst &cur, const LayerConst &next, int n) const {
        if (next.cell == cur.cell) return;
#pragma unroll
        for (int j = 0; j < SPL; ++j)
            asm volatile("prefetch.global.L1 [%0];" ::"l"(
                m.coef4 + (((size_t)next.cell * m.S + table_species(m, j)) * (m.Np >> 1) + (n >> 1)) * 2));
    }
    __device__ __forceinline__ void update(const Model &m, const SampleConst &sc, const LayerConst &lc, int n) {
        if (lc.cell != cell) {
            cell = lc.cell;
#pragma unroll
            for (int j = 0; j < SPL; ++j)
                load_cell(m, table_species(m, j), lc.cell, n, sc.lx[slot(j)], a0[j], a1[j], a2[j], a3[j]);
        }
        if (lc.itc != itc) {
            itc = lc.itc;
            load_cia(m, h, lc.itc, n, b, d);
        }
    }
    // exponent of species slot j: e = a0 + wp a1 + wt (a2 + wp a3); t = de/dwt
    __device__ __forceinline__ float2 expo(int j, float2 wp, float2 wt, float2 &t) const {
        t = fma2(wp, a3[j], a2[j]);
        return fma2(wt, t, fma2(wp, a1[j], a0[j]));
    }
    // CIA term of this lane's pair
    __device__ __forceinline__ float2 cia(const LayerConst &lc) const {
        return ex2x2(fma2(f2(lc.wtc), d, add2(b, f2(h ? lc.cc2 : lc.cc1))));
    }
};

// Species slots per lane for S species (two lanes per wavenumber pair).
__host__ __device__ constexpr int spl_for(int S) { return S <= 4 ? 2 : (S <= 8 ? 4 : 8); }

__device__ __forceinline__ float2 shfl_xor2(float2 v, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// Extinction alpha_l(nu) at wavenumber pair n, n+1 for layers [lb, le), the
// lane pair (lane, lane ^ 1) splitting species and CIA pairs:
//   alpha = n 2^-K sum_s 2^e_s + CIA_H2H2 + CIA_H2He + Rayleigh.
// Calls out(l, alpha) on both lanes of the pair.
template <int SPL, class Out>
__device__ __forceinline__ void extinction_pair(const Model &m, const SampleConst &sc, int lb, int le, int n,
                                                int half, Out &&out) {
    PairInterp<SPL> pi;
    pi.init(m, n, half);
    for (int l = lb; l < le; ++l) {
        const LayerConst &lc = sc.lay[l];
        pi.update(m, sc, lc, n);
        if (l + 1 < le) pi.prefetch(m, lc, sc.lay[l + 1], n);
        const float2 wp = f2(lc.wp), wt = f2(lc.wt);
        float2 sum = f2(0.f), t;
#pragma unroll
        for (int j = 0; j < SPL; ++j) sum = add2(sum, ex2x2(pi.expo(j, wp, wt, t)));
        float2 mine = fma2(sum, f2(lc.nsc), pi.cia(lc));
        if (half == 0) mine = fma2(f2(lc.ray), pi.nu4, mine);
        out(l, add2(mine, shfl_xor2(mine, 1)));
    }
}

// Adjoint reductions of one layer for the lane's pair, with abar = d lnL / d alpha:
// Q_s = sum abar e_s (species), D = sum abar sum_s e_s dlog10(sigma_s)/dlog10 T,
// C1, C2, C1T, C2T (CIA and their temperature slopes), W4 = sum abar (nu/nu_ref)^4.
// Values are reduced over the warp and added to red[l][*] (shared, one warp per layer).
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace es
