// Fused transmission kernels (Sect. 3 opacities -> Sect. 4 chord optical
// depth and transit depth), persistent over (sample, wavenumber-chunk) items.
//
// Forward, per 64-wavenumber tile: the extinction alpha[l][nu] of every
// layer is interpolated into shared memory as a split BF16 pair, the chord
// optical depth tau[i][nu] = sum_l L_il alpha_l(nu) runs on the tensor cores
// (mma.sync m16n8k16, hi*hi + hi*lo + lo*hi, FP32 accumulation; only the
// lower-triangular blocks of L), and the epilogue forms
// delta(nu) - base = sum_i A_i (1 - exp(-tau_i)); exp(-tau) is optionally
// stored for the adjoint.
//
// Backward, per tile: tau_bar = dbar A_i exp(-tau) (split BF16 in shared
// memory), alpha_bar = L^T tau_bar on the tensor cores, the interpolation is
// recomputed and reduced against alpha_bar (per-layer sums over wavenumber),
// and L_bar += tau_bar alpha^T on the tensor cores, accumulated in registers
// across the item's tiles.
#include <algorithm>

#include "fused_common.cuh"

namespace es {

namespace {

constexpr int RB_PITCH = 152;                 // bf16 pitch of the backward row buffer (304 B)
constexpr int RB_LO = 72;                     // bf16 offset of the lo half in a row (144 B)
constexpr float LOG2E_F = 1.4426950408889634f;

struct TransFwdSmem {
    SampleConst sc;
    __nv_bfloat16 lh[LP * L_PITCH], ll[LP * L_PITCH];   // path lengths [i][l]
    __nv_bfloat16 ah[LP * R_PITCH], al[LP * R_PITCH];   // extinction [l][nu]
    float area[LP];
};

// Backward block: 16 warps, 128-wavenumber tiles.
constexpr int BW_WARPS = 16;
constexpr int BW_THREADS = BW_WARPS * 32;
constexpr int BT = 128;              // wavenumbers per backward tile
constexpr int T2_PITCH = 136;        // bf16 pitch of tau_bar rows [i][128 nu] (272 B: 17 x 16 B)
constexpr int RB2_BYTES = 528;       // bytes per row buffer row (33 x 16 B): four 128-B quarters
constexpr int LPR = 120;             // row buffer rows: LP layers, plus row L (the Rayleigh weight), to 8
// Row buffer, per layer and per 32-wavenumber quarter k (bytes [128 k, 128 k + 128)):
// first alpha_bar as 32 FP32, then overwritten by the extinction as BF16 hi
// (bytes 0..63 of the quarter) and lo (bytes 64..127). Each quarter of a row
// belongs to one warp, so the overwrite only needs a warp barrier. Row L holds
// w(nu) = (nu/nu_ref)^4 as split BF16, so that the L_bar product also yields
// z_i = sum_nu tau_bar_i(nu) w(nu), from which the Rayleigh reduction
// W4_l = sum_nu alpha_bar_l(nu) w(nu) = sum_i L_il z_i follows.

struct TransBwdSmem {
    SampleConst sc;
    __nv_bfloat16 lh[LP * L_PITCH], ll[LP * L_PITCH];   // path lengths [i][l]
    __nv_bfloat16 th[LP * T2_PITCH], tl[LP * T2_PITCH]; // tau_bar [i][nu]
    unsigned char rb[LPR * RB2_BYTES];                  // alpha_bar / alpha rows, Rayleigh weight row
    float area[LP];
    float area_acc[LP];                                 // area_bar of the current sample
    float red[ES_MAX_LAYERS * N_RED];                   // per-layer reductions of the current sample
    float qtot[ES_MAX_SPECIES];                         // per-species totals of the current sample
};

// Path-length matrix of sample b as split BF16 [i][l] (zero-padded to LP x LP).
__device__ void stage_lmat(const Model &m, const Work &w, int b, __nv_bfloat16 *lh, __nv_bfloat16 *ll, float *area) {
    const int L = m.L;
    const float *src = w.lmat + (size_t)b * L * L;
    for (int idx = threadIdx.x; idx < LP * (LP / 2); idx += FTHREADS) {
        const int i = idx / (LP / 2), l = 2 * (idx % (LP / 2));
        float2 v = make_float2(0.f, 0.f);
        if (i < L) {
            if (l < L) v.x = src[(size_t)i * L + l];
            if (l + 1 < L) v.y = src[(size_t)i * L + l + 1];
        }
        uint32_t hi, lo;
        split2(v, hi, lo);
        *reinterpret_cast<uint32_t *>(lh + i * L_PITCH + l) = hi;
        *reinterpret_cast<uint32_t *>(ll + i * L_PITCH + l) = lo;
    }
    for (int i = threadIdx.x; i < LP; i += FTHREADS) area[i] = (i < L) ? w.area[(size_t)b * L + i] : 0.f;
}

template <int SPL, bool STORE_E>
__global__ void __launch_bounds__(FTHREADS, 2) k_trans_fwd(Model m, Work w, int chunk_tiles) {
    extern __shared__ float4 smem4[];
    TransFwdSmem &sm = *reinterpret_cast<TransFwdSmem *>(smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = m.L, N = m.N;
    const int ntiles = (N + FT - 1) / FT;
    const int nchunks = (ntiles + chunk_tiles - 1) / chunk_tiles;
    const long long total = (long long)w.B * nchunks;
    // extinction rows of the padding layers stay zero
    for (int idx = threadIdx.x; idx < (LP - L) * R_PITCH; idx += FTHREADS) {
        sm.ah[L * R_PITCH + idx] = __float2bfloat16_rn(0.f);
        sm.al[L * R_PITCH + idx] = __float2bfloat16_rn(0.f);
    }
    // interpolation: 4 layer groups x 2 halves (32 wavenumbers) of the tile; a
    // wavenumber pair is shared by a lane pair splitting the species
    const int half = lane & 1, pair = 16 * (warp & 1) + (lane >> 1);
    int lb, le;
    group_layers(L, warp >> 1, FWARPS / 2, lb, le);
    const uint32_t blh = smem_u32(sm.lh), bll = smem_u32(sm.ll), bah = smem_u32(sm.ah), bal = smem_u32(sm.al);
    const int ksmax = (L + 15) / 16;
    // lane half 0 stores the hi parts of its pair's extinction, half 1 the lo parts
    uint32_t *const a_dst = reinterpret_cast<uint32_t *>((half ? sm.al : sm.ah) + 2 * pair);
    int cur_b = -1;
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        // chunk-major order: blocks running together share a wavenumber window,
        // so its slice of the opacity tables stays resident in L2
        const int c = (int)(item / w.B), b = (int)(item % w.B);
        if (w.kind[b] != ES_KIND_TRANSMISSION) continue;
        if (b != cur_b) {
            __syncthreads();
            stage_sample(m, w, b, sm.sc);
            stage_lmat(m, w, b, sm.lh, sm.ll, sm.area);
            cur_b = b;
            __syncthreads();
        }
        const int t1 = min(ntiles, (c + 1) * chunk_tiles);
        for (int t = c * chunk_tiles; t < t1; ++t) {
            const int nt0 = t * FT;
            extinction_pair<SPL>(m, sm.sc, lb, le, nt0 + 2 * pair, half, [&](int l, float2 a) {
                uint32_t hi, lo;
                split2(a, hi, lo);
                a_dst[l * (R_PITCH / 2)] = half ? lo : hi;
            });
            __syncthreads();
            // tau[i][nu] for this warp's 8 wavenumbers, lower-triangular blocks only
            float acc[7][4];
#pragma unroll
            for (int mi = 0; mi < 7; ++mi) acc[mi][0] = acc[mi][1] = acc[mi][2] = acc[mi][3] = 0.f;
#pragma unroll
            for (int ks = 0; ks < 7; ++ks) {
                if (ks < ksmax) {
                    uint32_t bh[2], bl[2];
                    ldsm_x2_t(bt_addr(bah, R_PITCH, 8 * warp, 16 * ks, lane), bh);
                    ldsm_x2_t(bt_addr(bal, R_PITCH, 8 * warp, 16 * ks, lane), bl);
#pragma unroll
                    for (int mi = ks; mi < 7; ++mi) {
                        uint32_t ah[4], al[4];
                        ldsm_x4(a_addr(blh, L_PITCH, 16 * mi, 16 * ks, lane), ah);
                        ldsm_x4(a_addr(bll, L_PITCH, 16 * mi, 16 * ks, lane), al);
                        mma3(acc[mi], ah, al, bh, bl);
                    }
                }
            }
            // epilogue: sum_i A_i (1 - exp(-tau_i)); lane holds rows r, r+8 and columns c, c+1
            const int col = 8 * warp + 2 * (lane & 3), r = lane >> 2;
            const int n0 = nt0 + col;
            float s0 = 0.f, s1 = 0.f;
#pragma unroll
            for (int mi = 0; mi < 7; ++mi) {
                const int i0 = 16 * mi + r, i1 = i0 + 8;
                const float e00 = ex2f(-acc[mi][0] * LOG2E_F), e01 = ex2f(-acc[mi][1] * LOG2E_F);
                const float e10 = ex2f(-acc[mi][2] * LOG2E_F), e11 = ex2f(-acc[mi][3] * LOG2E_F);
                const float a0 = sm.area[i0], a1 = sm.area[i1];
                s0 += a0 * (1.f - e00) + a1 * (1.f - e10);
                s1 += a0 * (1.f - e01) + a1 * (1.f - e11);
                if (STORE_E) {   // padding wavenumbers too: the adjoint multiplies them by dbar = 0
                    float *eb = w.estore + (size_t)b * L * m.Np + n0;
                    // streaming stores: keep the opacity coefficients, not these, in L2
                    if (i0 < L) __stcs(reinterpret_cast<float2 *>(eb + (size_t)i0 * m.Np), make_float2(e00, e01));
                    if (i1 < L) __stcs(reinterpret_cast<float2 *>(eb + (size_t)i1 * m.Np), make_float2(e10, e11));
                }
            }
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            }
            if (r == 0) {
                float *sp = w.spec + (size_t)b * N;
                if (n0 < N) sp[n0] = s0;
                if (n0 + 1 < N) sp[n0 + 1] = s1;
            }
            __syncthreads();
        }
    }
}

// Warp transpose-reduction of 16 values: on return lane holds the warp-wide
// sum of v[idx] with idx = 8 b4 + 4 b3 + 2 b2 + b1 (bk = bit k of the lane).
__device__ __forceinline__ float transpose_reduce16(float (&v)[16], int lane) {
    float a[8], c[4], d[2];
    {
        const bool up = lane & 16;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float send = up ? v[k] : v[k + 8], keep = up ? v[k + 8] : v[k];
            a[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
    }
    {
        const bool up = lane & 8;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float send = up ? a[k] : a[k + 4], keep = up ? a[k + 4] : a[k];
            c[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
    }
    {
        const bool up = lane & 4;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const float send = up ? c[k] : c[k + 2], keep = up ? c[k + 2] : c[k];
            d[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
    }
    const bool up = lane & 2;
    float e = (up ? d[1] : d[0]) + __shfl_xor_sync(0xffffffffu, up ? d[0] : d[1], 2);
    e += __shfl_xor_sync(0xffffffffu, e, 1);
    return e;
}

// Lower-triangular block pair p (0..55) of L_bar: i-block mi (0..6), l-block nj <= 2 mi + 1.
__device__ __forceinline__ void decode_pair(int p, int &mi, int &nj) {
    mi = 0;
    while (p >= 2 * mi + 2) {
        p -= 2 * mi + 2;
        ++mi;
    }
    nj = p;
}

// Block pair p (0..63) of the L_bar product: the 56 lower-triangular pairs,
// then (mi, L/8) for the i-blocks whose lower triangle stops short of column
// L (the Rayleigh weight row). False for unused slots.
__device__ __forceinline__ bool lbar_pair(int p, int L, int &mi, int &nj) {
    if (p < 56) {
        decode_pair(p, mi, nj);
        return true;
    }
    mi = p - 56;
    nj = L >> 3;
    return mi < 7 && nj > 2 * mi + 1;
}

__device__ __forceinline__ int reduce_index(int lane) {
    return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

// Warp transpose-reduction of 8 values: on return lane holds the warp-wide
// sum of v[idx] with idx = 4 b4 + 2 b3 + b2 (bk = bit k of the lane).
__device__ __forceinline__ float transpose_reduce8(const float (&v)[8], int lane) {
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
    e += __shfl_xor_sync(0xffffffffu, e, 1);
    return e;
}

__device__ __forceinline__ int reduce_index8(int lane) {
    return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// Warp reduction of 4 values per lane that keeps the two lane parities
// apart: on return lane holds the sum of v[2 b4 + b3] over the 16 lanes of its
// parity (bk = bit k of the lane).
__device__ __forceinline__ float reduce4_parity(const float (&v)[4], int lane) {
    float a[2];
    {
        const bool up = lane & 16;
#pragma unroll
        for (int k = 0; k < 2; ++k)
            a[k] = (up ? v[k + 2] : v[k]) + __shfl_xor_sync(0xffffffffu, up ? v[k] : v[k + 2], 16);
    }
    const bool up = lane & 8;
    float e = (up ? a[1] : a[0]) + __shfl_xor_sync(0xffffffffu, up ? a[0] : a[1], 8);
    e += __shfl_xor_sync(0xffffffffu, e, 4);
    e += __shfl_xor_sync(0xffffffffu, e, 2);
    return e;
}

// Backward interpolation for one warp: layers [lb, le), wavenumber pair n, n+1
// shared by the lane pair (lane, lane ^ 1) that splits the species; `quarter`
// points at the warp's 32-wavenumber quarter of row 0 of the row buffer.
// Reads alpha_bar, adds per-layer reductions to red[l][*] and per-species
// totals to qtot[s], then overwrites the quarter-rows with the extinction as
// split BF16. Per layer, summed over wavenumber, with lane half h's species
// and CIA pair h: QS_h = sum abar n sum_s e_s, D_h = sum abar n sum_s e_s
// dlog2(sigma_s)/dlog10 T, C_h = sum abar c_h, CT_h = sum abar c_h dlog2 k_h/dT
// (red slots 0/1, 2/3, 4/5, 6/7 for h = 0/1); per species Q_s = sum_l sum
// abar n e_s. The Rayleigh sum over wavenumber comes from the L_bar product.
template <int SPL>
__device__ void interp_backward(const Model &m, const SampleConst &sc, int lb, int le, int n, int half, int lane,
                                unsigned char *quarter, float *red, float *qtot) {
    const int S = m.S, q = lane >> 1;
    const int ridx = reduce_index8(lane);
    const bool writer = (lane & 3) == 0;
    // after reduce4_parity: lanes with bits 2, 1 clear write slot 2 (2 b4 + b3) + b0
    const bool rwriter = (lane & 6) == 0;
    const int rslot = 2 * (2 * ((lane >> 4) & 1) + ((lane >> 3) & 1)) + (lane & 1);
    PairInterp<SPL> pi;
    pi.init(m, n, half, lane);
    float2 qa[SPL];
#pragma unroll
    for (int j = 0; j < SPL; ++j) qa[j] = f2(0.f);
    const int st_off = (half ? 64 : 0) + 4 * q;
    for (int l = lb; l < le;) {
        const int end = min(sc.lay[l].run_end, le);
        pi.load(sc, sc.lay[l].cell, sc.lay[l].itc);
        if (end < le) pi.prefetch(sc.lay[end].cell, sc.lay[end].itc);
        for (; l < end; ++l) {
            const LayerConst &lc = sc.lay[l];
            unsigned char *row = quarter + (size_t)l * RB2_BYTES;
            const float2 ab = *reinterpret_cast<const float2 *>(row + 8 * q);
            const float2 abn = mul2(ab, lc.nsc);
            float2 t, p = ex2x2(pi.expo(0, lc.wp, lc.wt, t));
            float2 sum = p, pt = mul2(p, t);
            qa[0] = fma2(abn, p, qa[0]);
#pragma unroll
            for (int j = 1; j < SPL; ++j) {
                p = ex2x2(pi.expo(j, lc.wp, lc.wt, t));
                sum = add2(sum, p);
                qa[j] = fma2(abn, p, qa[j]);
                pt = fma2(p, t, pt);
            }
            const float2 c = pi.cia(lc);
            const float2 ac = mul2(ab, c);
            const float2 act = mul2(ac, pi.d);
            float v[4];
            v[0] = fmaf(abn.x, sum.x, abn.y * sum.y);
            v[1] = fmaf(abn.x, pt.x, abn.y * pt.y) * lc.gts;
            v[2] = ac.x + ac.y;
            v[3] = (act.x + act.y) * lc.gtcs;
            const float tot = reduce4_parity(v, lane);
            if (rwriter) atomicAdd(red + l * N_RED + rslot, tot);
            const float2 mine = fma2(lc.ray, pi.nu4, fma2(sum, lc.nsc, c));
            const float2 alpha = add2(mine, shfl_xor2(mine, 1));
            uint32_t hi, lo;
            split2(alpha, hi, lo);
            __syncwarp();
            *reinterpret_cast<uint32_t *>(row + st_off) = half ? lo : hi;
        }
    }
    // per-species totals: slot j of lane half h is species SPL h + j
#pragma unroll
    for (int c0 = 0; c0 < 2 * SPL; c0 += 8) {
        float v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int sl = c0 + k;
            v[k] = (sl < 2 * SPL && sl / SPL == half) ? qa[sl % SPL].x + qa[sl % SPL].y : 0.f;
        }
        const float tq = transpose_reduce8(v, lane);
        if (writer && c0 + ridx < S && tq != 0.f) atomicAdd(qtot + c0 + ridx, tq);
    }
}

// B fragment (k16 x n8) of alpha^T for L_bar = tau_bar alpha^T: rows l of the
// row buffer, wavenumbers [16 ks, 16 ks + 16) of the tile; lo = false/true.
__device__ __forceinline__ uint32_t rb_addr(uint32_t base, int n0, int ks, bool lo, int lane) {
    const int l = lane & 15;
    const int qt = ks >> 1, kin = (ks & 1) * 16 + ((l >> 3) << 3);
    return base + (uint32_t)((n0 + (l & 7)) * RB2_BYTES + 128 * qt + (lo ? 64 : 0) + 2 * kin);
}

template <int SPL>
__global__ void __launch_bounds__(BW_THREADS, 1) k_trans_bwd(Model m, Work w, int chunk_tiles) {
    extern __shared__ float4 smem4[];
    TransBwdSmem &sm = *reinterpret_cast<TransBwdSmem *>(smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = m.L, N = m.N, S = m.S;
    const int ntiles = (N + BT - 1) / BT;
    const int nchunks = (ntiles + chunk_tiles - 1) / chunk_tiles;
    const long long total = (long long)w.B * nchunks;
    const int group = warp >> 1;                        // tau_bar phase: rows i = group + 8 k
    // interpolation: 4 layer groups x 4 quarters (32 wavenumbers); lane pairs split species
    const int half = lane & 1, vq = warp & 3, pair = 16 * vq + (lane >> 1);
    int lb, le;
    group_layers(L, warp >> 2, 4, lb, le);
    // padding rows (impact parameters / layers >= L) of tau_bar and the row buffer stay zero
    for (int idx = threadIdx.x; idx < (LP - L) * T2_PITCH; idx += BW_THREADS) {
        sm.th[L * T2_PITCH + idx] = __float2bfloat16_rn(0.f);
        sm.tl[L * T2_PITCH + idx] = __float2bfloat16_rn(0.f);
    }
    for (int idx = threadIdx.x; idx < (LPR - L) * RB2_BYTES; idx += BW_THREADS) sm.rb[L * RB2_BYTES + idx] = 0;
    const float ray_ref = (float)(1.0 / ((double)m.ray_nu_ref * m.ray_nu_ref * m.ray_nu_ref * m.ray_nu_ref));
    const uint32_t blh = smem_u32(sm.lh), bll = smem_u32(sm.ll), bth = smem_u32(sm.th), btl = smem_u32(sm.tl);
    const uint32_t brb = smem_u32(sm.rb);
    const int ksmax = (L + 15) / 16;
    float lacc[4][4];
    int cur_b = -1;
    auto flush = [&](int b) {
        // L_bar, reductions, per-species totals and area_bar of sample b (FP64 atomics)
        double *lbar = w.lbar + (size_t)b * L * L, *zbar = w.zbar + (size_t)b * L;
        const int r = lane >> 2, col = 2 * (lane & 3);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int mi, nj;
            if (lbar_pair(warp + BW_WARPS * k, L, mi, nj)) {
                const int i0 = 16 * mi + r, l0 = 8 * nj + col;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int ii = i0 + ((e >> 1) << 3), ll = l0 + (e & 1);
                    const float v = lacc[k][e];
                    if (ii >= L || v == 0.f) continue;
                    if (ll == L) atomicAdd(zbar + ii, (double)v);
                    else if (ll <= ii) atomicAdd(lbar + (size_t)ii * L + ll, (double)v);
                }
            }
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < L * N_RED; idx += BW_THREADS) {
            const float v = sm.red[idx];
            if (v != 0.f) atomicAdd(w.red + (size_t)b * L * N_RED + idx, (double)v);
        }
        for (int i = threadIdx.x; i < L; i += BW_THREADS)
            if (sm.area_acc[i] != 0.f) atomicAdd(w.areabar + (size_t)b * L + i, (double)sm.area_acc[i]);
        for (int s2 = threadIdx.x; s2 < S; s2 += BW_THREADS)
            if (sm.qtot[s2] != 0.f) atomicAdd(w.qtot + (size_t)b * S + s2, (double)sm.qtot[s2]);
    };
    // L2 prefetch of the exp(-tau) rows and dbar of tile t of sample b (the
    // tau_bar phase reads them straight from HBM otherwise, with every warp
    // of the block waiting on the same loads)
    uint64_t evict_first;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(evict_first));
    auto prefetch_tile = [&](int pb, int pt) {
        if (threadIdx.x < L) {   // read once: evict-first, the coefficient table stays resident
            const float *src = w.estore + ((size_t)pb * L + threadIdx.x) * m.Np + (size_t)pt * BT;
            asm volatile("cp.async.bulk.prefetch.L2.global.L2::cache_hint [%0], %1, %2;" ::"l"(src), "r"(BT * 4),
                         "l"(evict_first)
                         : "memory");
        } else if (threadIdx.x == L) {
            const float *src = w.dbar + (size_t)pb * m.Np + (size_t)pt * BT;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(BT * 4) : "memory");
        }
    };
    if (blockIdx.x < total) {
        const long long it0 = blockIdx.x;
        prefetch_tile((int)(it0 % w.B), (int)(it0 / w.B) * chunk_tiles);
    }
    for (long long item = blockIdx.x; item < total; item += gridDim.x) {
        // chunk-major order: blocks running together share a wavenumber window
        const int c = (int)(item / w.B), b = (int)(item % w.B);
        if (w.kind[b] != ES_KIND_TRANSMISSION || w.flags[b]) continue;
        if (b != cur_b) {
            if (cur_b >= 0) flush(cur_b);
            __syncthreads();
            stage_sample(m, w, b, sm.sc);
            stage_lmat(m, w, b, sm.lh, sm.ll, sm.area);
            for (int idx = threadIdx.x; idx < L * N_RED; idx += BW_THREADS) sm.red[idx] = 0.f;
            for (int i = threadIdx.x; i < LP; i += BW_THREADS) sm.area_acc[i] = 0.f;
            for (int s2 = threadIdx.x; s2 < ES_MAX_SPECIES; s2 += BW_THREADS) sm.qtot[s2] = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) lacc[k][0] = lacc[k][1] = lacc[k][2] = lacc[k][3] = 0.f;
            cur_b = b;
            __syncthreads();
        }
        const int t1 = min(ntiles, (c + 1) * chunk_tiles);
        for (int t = c * chunk_tiles; t < t1; ++t) {
            const int nt0 = t * BT;
            if (t + 1 < t1) {
                prefetch_tile(b, t + 1);
            } else if (item + gridDim.x < total) {   // first tile of this block's next item
                const long long nx = item + gridDim.x;
                prefetch_tile((int)(nx % w.B), (int)(nx / w.B) * chunk_tiles);
            }
            // Rayleigh weight row w(nu) for the L_bar product
            if (threadIdx.x < BT / 2) {
                const int t2 = threadIdx.x;
                const float2 nu = __ldg(reinterpret_cast<const float2 *>(m.nu + nt0 + 2 * t2));
                const float2 nu2 = mul2(nu, nu);
                uint32_t hi, lo;
                split2(mul2(mul2(nu2, nu2), f2(ray_ref)), hi, lo);
                unsigned char *rw = sm.rb + (size_t)L * RB2_BYTES + 128 * (t2 >> 4) + 4 * (t2 & 15);
                *reinterpret_cast<uint32_t *>(rw) = hi;
                *reinterpret_cast<uint32_t *>(rw + 64) = lo;
            }
            // tau_bar = dbar A_i exp(-tau); area_bar += dbar (1 - exp(-tau))
            {
                const int nl = nt0 + 2 * (lane + 32 * (warp & 1));
                const float2 db = *reinterpret_cast<const float2 *>(w.dbar + (size_t)b * m.Np + nl);
                const float *eb = w.estore + (size_t)b * L * m.Np + nl;
                float av[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    av[k] = 0.f;
                    const int i = group + 8 * k;
                    if (k < 14 && i < L) {
                        const float2 e = *reinterpret_cast<const float2 *>(eb + (size_t)i * m.Np);
                        const float a = sm.area[i];
                        uint32_t hi, lo;
                        split2(make_float2(db.x * a * e.x, db.y * a * e.y), hi, lo);
                        const int col = 2 * (lane + 32 * (warp & 1));
                        *reinterpret_cast<uint32_t *>(sm.th + i * T2_PITCH + col) = hi;
                        *reinterpret_cast<uint32_t *>(sm.tl + i * T2_PITCH + col) = lo;
                        av[k] = db.x * (1.f - e.x) + db.y * (1.f - e.y);
                    }
                }
                const float tot = transpose_reduce16(av, lane);
                const int k = reduce_index(lane), i = group + 8 * k;
                if ((lane & 1) == 0 && k < 14 && i < L && tot != 0.f) atomicAdd(sm.area_acc + i, tot);
            }
            __syncthreads();
            // alpha_bar[l][nu] = sum_{i >= l} L_il tau_bar_i(nu), this warp's 8 wavenumbers
            {
                float acc[7][4];
#pragma unroll
                for (int ml = 0; ml < 7; ++ml) acc[ml][0] = acc[ml][1] = acc[ml][2] = acc[ml][3] = 0.f;
#pragma unroll
                for (int ks = 0; ks < 7; ++ks) {
                    if (ks < ksmax) {
                        uint32_t bh[2], bl[2];
                        ldsm_x2_t(bt_addr(bth, T2_PITCH, 8 * warp, 16 * ks, lane), bh);
                        ldsm_x2_t(bt_addr(btl, T2_PITCH, 8 * warp, 16 * ks, lane), bl);
#pragma unroll
                        for (int ml = 0; ml <= ks; ++ml) {
                            uint32_t ah[4], al[4];
                            ldsm_x4_t(at_addr(blh, L_PITCH, 16 * ml, 16 * ks, lane), ah);
                            ldsm_x4_t(at_addr(bll, L_PITCH, 16 * ml, 16 * ks, lane), al);
                            mma3(acc[ml], ah, al, bh, bl);
                        }
                    }
                }
                const int colt = 8 * warp + 2 * (lane & 3), r = lane >> 2;
                const int qt = colt >> 5, cin = colt & 31;
#pragma unroll
                for (int ml = 0; ml < 7; ++ml) {
                    const int l0 = 16 * ml + r, l1 = l0 + 8;
                    if (l0 < L)
                        *reinterpret_cast<float2 *>(sm.rb + (size_t)l0 * RB2_BYTES + 128 * qt + 4 * cin) =
                            make_float2(acc[ml][0], acc[ml][1]);
                    if (l1 < L)
                        *reinterpret_cast<float2 *>(sm.rb + (size_t)l1 * RB2_BYTES + 128 * qt + 4 * cin) =
                            make_float2(acc[ml][2], acc[ml][3]);
                }
            }
            __syncthreads();
            interp_backward<SPL>(m, sm.sc, lb, le, nt0 + 2 * pair, half, lane, sm.rb + 128 * vq, sm.red, sm.qtot);
            __syncthreads();
            // L_bar[i][l] += sum_nu tau_bar[i][nu] alpha[l][nu] over this tile (8 k-steps)
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int mi, nj;
                if (lbar_pair(warp + BW_WARPS * k, L, mi, nj)) {
#pragma unroll
                    for (int ks = 0; ks < BT / 16; ++ks) {
                        uint32_t ah[4], al[4], bh[2], bl[2];
                        ldsm_x4(a_addr(bth, T2_PITCH, 16 * mi, 16 * ks, lane), ah);
                        ldsm_x4(a_addr(btl, T2_PITCH, 16 * mi, 16 * ks, lane), al);
                        ldsm_x2(rb_addr(brb, 8 * nj, ks, false, lane), bh);
                        ldsm_x2(rb_addr(brb, 8 * nj, ks, true, lane), bl);
                        mma3(lacc[k], ah, al, bh, bl);
                    }
                }
            }
            __syncthreads();
        }
    }
    if (cur_b >= 0) flush(cur_b);
}

size_t fwd_smem() { return sizeof(TransFwdSmem); }
size_t bwd_smem() { return sizeof(TransBwdSmem); }

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace

// Tiles per work item: up to 16 (amortises staging the sample), fewer when the
// batch is small so that every resident block gets items.
int chunk_tiles(const Model &m, int B, int blocks) {
    const int ntiles = (m.N + FT - 1) / FT;
    long long c = ((long long)ntiles * B) / (4LL * blocks);
    return (int)std::max<long long>(1, std::min<long long>(16, c));
}

int launch_trans_fused_forward(const Model &m, const Work &w, bool store_e, int chunk_req, cudaStream_t st,
                               const Hook &h) {
    const int ntiles = (m.N + FT - 1) / FT;
    const int chunk = chunk_req > 0 ? chunk_req : chunk_tiles(m, w.B, 2 * sm_count());
    const long long items = (long long)w.B * ((ntiles + chunk - 1) / chunk);
    const int grid = (int)std::min<long long>(items, 2LL * sm_count());
    const size_t sm = fwd_smem();
#define ES_FWD(SPL, SE)                                                                         \
    do {                                                                                        \
        cudaFuncSetAttribute(k_trans_fwd<SPL, SE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        ES_LAUNCH(h, "k_trans_fwd", st, k_trans_fwd<SPL, SE><<<grid, FTHREADS, sm, st>>>(m, w, chunk)); \
    } while (0)
    const int spl = spl_for(m.S);
    if (spl == 2) { if (store_e) ES_FWD(2, true); else ES_FWD(2, false); }
    else if (spl == 4) { if (store_e) ES_FWD(4, true); else ES_FWD(4, false); }
    else { if (store_e) ES_FWD(8, true); else ES_FWD(8, false); }
#undef ES_FWD
    return 1;
}

int launch_trans_fused_backward(const Model &m, const Work &w, int chunk_req, cudaStream_t st, const Hook &h) {
    const int ntiles = (m.N + BT - 1) / BT;
    const int chunk = chunk_req > 0 ? chunk_req : std::max(1, chunk_tiles(m, w.B, sm_count()) / 2);
    const long long items = (long long)w.B * ((ntiles + chunk - 1) / chunk);
    const int grid = (int)std::min<long long>(items, (long long)sm_count());
    const size_t sm = bwd_smem();
#define ES_BWD(SPL)                                                                             \
    do {                                                                                        \
        cudaFuncSetAttribute(k_trans_bwd<SPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        ES_LAUNCH(h, "k_trans_bwd", st, k_trans_bwd<SPL><<<grid, BW_THREADS, sm, st>>>(m, w, chunk)); \
    } while (0)
    const int spl = spl_for(m.S);
    if (spl == 2) ES_BWD(2);
    else if (spl == 4) ES_BWD(4);
    else ES_BWD(8);
#undef ES_BWD
    return 1;
}

}  // namespace es
