// Tile engines of the fused transmission kernels (Sect. 3 opacities ->
// Sect. 4 chord optical depth and transit depth). The persistent kernels
// (transmission-only in k_fused_trans.cu, mixed transmission/emission in
// k_fused_mixed.cu) walk their (sample, wavenumber-chunk) work items and
// drive these engines.
//
// Forward, per 128-wavenumber tile: the extinction alpha[l][nu] of every
// layer is interpolated into shared memory as a split BF16 pair, the chord
// optical depth tau[i][nu] = sum_l L_il alpha_l(nu) runs on the tcgen05
// tensor cores (hi*hi + hi*lo + lo*hi, FP32 accumulation in TMEM), and the
// epilogue forms delta(nu) - base = sum_i A_i (1 - exp(-tau_i)); exp(-tau) is
// optionally stored for the adjoint.
//
// Backward, per tile: tau_bar = dbar A_i exp(-tau) (BF16 in shared memory),
// alpha_bar = L^T tau_bar on the tensor cores (L split, FP32 accumulation in
// TMEM), the interpolation is recomputed and reduced against alpha_bar
// (per-layer sums over wavenumber), and L_bar += tau_bar alpha^T on the
// tensor cores (BF16 alpha), accumulated in TMEM across the sample's tiles.
// The adjoint products need the gradient's accuracy (1e-3), not the transit
// depth's, so tau_bar and alpha enter them as single BF16; the measured
// gradient error of that choice is ~1e-6 relative.
#pragma once

#include "fused_common.cuh"
#include "tc_common.cuh"

namespace es {

namespace {

constexpr float LOG2E_F = 1.4426950408889634f;

// Forward block: NW (16 or 24) warps, 128-wavenumber tiles; the chord product runs on
// the tcgen05 tensor cores with the accumulator in TMEM, double-buffered: the
// epilogue of tile t - 1 overlaps the product of tile t, whose completion
// then frees the (single) extinction operand for tile t + 1 (one block
// barrier per tile). A second extinction buffer measured slower: the shared
// memory it takes comes out of L1.
constexpr int FT2 = 128;                          // wavenumbers per forward tile (the MMA's M)
constexpr int F2_WARPS = 16;
constexpr int F2_THREADS = F2_WARPS * 32;
constexpr int SBO_NU = (FT2 / 8) * CORE_STRIDE;   // 8-row group stride of [row][128 nu] operands (2304 B)
constexpr int SBO_LP = (LP / 8) * CORE_STRIDE;    // 8-row group stride of [row][112 layers] operands (2016 B)
constexpr int F2_TMEM_COLS = 256;                 // two 112-column accumulators

// NW warps: NW / 4 layer groups x 4 wavenumber quarters (the TMEM lane
// quadrants) in the interpolation, NW / 4 impact-parameter chunks in the epilogue
template <int NW>
struct TransFwdSmemT {
    SampleConst sc;
    alignas(128) unsigned char lh[(LP / 8) * SBO_LP], ll[(LP / 8) * SBO_LP];    // L[i][l], split BF16
    alignas(128) unsigned char ah[1][(LP / 8) * SBO_NU], al[1][(LP / 8) * SBO_NU];   // alpha[l][nu], split BF16
    float area[LP];
    float cd[LP];                                  // non-grey cloud: D_i (0 beyond L)
    float cg[N_CG];                                // non-grey cloud: g(nu) constants (kh18_g)
    float part[2][NW / 4][FT2];                    // per-column-chunk partial transit sums, per buffer
    alignas(8) uint64_t mbar[2];
    uint32_t tmem_base;
    int abort;
};
using TransFwdSmem = TransFwdSmemT<16>;

// Backward block: NW (16 or 24) warps, 128-wavenumber tiles; both products on the
// tcgen05 tensor cores: alpha_bar^T = tau_bar^T L into TMEM columns [0, 112)
// (read there by the interpolation warps) and L_bar = tau_bar alpha^T
// accumulated over the sample's tiles in TMEM columns [128, 256).
constexpr int BW_WARPS = 16;
constexpr int BW_THREADS = BW_WARPS * 32;
constexpr int BT = 128;              // wavenumbers per backward tile
constexpr int LB_ROWS = 128;         // rows of the alpha operand: layers, the Rayleigh weight row (L), zeros
// The alpha operand's row L holds w(nu) = (nu/nu_ref)^4 (BF16), so
// the L_bar product also yields z_i = sum_nu tau_bar_i(nu) w(nu), from which
// the Rayleigh reduction W4_l = sum_nu alpha_bar_l(nu) w(nu) = sum_i L_il z_i
// follows.

// STAGE: per-warp shared-memory staging of the coefficients (see
// interp_backward); LSPLIT: L as split BF16 (hi + lo) in alpha_bar = L^T tau_bar,
// else single BF16 (tau_bar is single BF16 there in any case)
template <int NW, bool STAGE, bool LSPLIT = true>
struct TransBwdSmemT {
    SampleConst sc;
    alignas(128) unsigned char lh[(LP / 8) * SBO_LP], ll[LSPLIT ? (LP / 8) * SBO_LP : 16];      // L[i][l]
    // adjoint operands as single BF16 (the gradient tolerance is 1e-3; the
    // measured error of these products is ~1e-6 relative): tau_bar[i][nu], alpha[l][nu]
    alignas(128) unsigned char th[(LP / 8) * SBO_NU];
    alignas(128) unsigned char ah[(LB_ROWS / 8) * SBO_NU];
    float area[LP];
    float area_acc[LP];                                 // area_bar of the current sample
    // per-layer reductions of the current sample: 8 slots (value, lane parity)
    // x 4 partial sums (one per lane-bit pair b2 b1), summed at the flush
    float red[ES_MAX_LAYERS * 32];
    float qtot[ES_MAX_SPECIES];                         // per-species totals of the current sample
    // non-grey cloud: D_i, its adjoint, d lnL / d g(nu) of the tile, the
    // g(nu) constants and the parameter adjoints of the sample
    float cd[LP], cdbar[LP], gbar[BT], cg[N_CG], cpbar[N_CG];
    alignas(16) unsigned char stage[STAGE ? NW : 1][STAGE_BYTES_PER_WARP];   // per-warp coefficient staging
    alignas(8) uint64_t mbar_a, mbar_l;
    uint32_t tmem_base;
    int abort;
};
using TransBwdSmem = TransBwdSmemT<16, true>;

// Path-length matrix of sample b as the split BF16 tensor-core operand
// L[i][l] (112 x 112, zero-padded, core-matrix layout) and the annulus areas.
__device__ void stage_lmat_tc(const Model &m, const Work &w, int b, unsigned char *lh, unsigned char *ll,
                              float *area) {
    const int L = m.L;
    const float *src = w.lmat + (size_t)b * L * L;
    for (int idx = threadIdx.x; idx < LP * (LP / 2); idx += blockDim.x) {
        const int i = idx / (LP / 2), l = 2 * (idx % (LP / 2));
        float2 v = make_float2(0.f, 0.f);
        if (i < L) {
            if (l < L) v.x = src[(size_t)i * L + l];
            if (l + 1 < L) v.y = src[(size_t)i * L + l + 1];
        }
        uint32_t hi, lo;
        split2(v, hi, lo);
        const uint32_t o = op_off(i, l, SBO_LP);
        *reinterpret_cast<uint32_t *>(lh + o) = hi;
        if (ll) *reinterpret_cast<uint32_t *>(ll + o) = lo;   // (ll NULL: single BF16 L)
    }
    for (int i = threadIdx.x; i < LP; i += blockDim.x) area[i] = (i < L) ? w.area[(size_t)b * L + i] : 0.f;
}

// ---------------------------------------------------------------- forward engine
// The forward's per-tile machinery for one block, as methods on the block's
// state: set-up (padding rows, mbarriers, TMEM), staging of a sample, the
// tiles of one work item, draining the tile still in flight, and teardown.
// The transmission-only kernel and the mixed transmission/emission kernel
// drive it with their own work-item loops.
// CLOUD: the non-grey cloud and cloud fraction (ES_CLOUD_KH18) as a separate
// instantiation, so that the cloud-free kernels carry none of its code.
template <int SPL, bool STORE_E, bool CLOUD, int NW = 16>
struct TransFwdEngine {
    static constexpr int NT = NW * 32, NCK = NW / 4;
    // the warp that issues the chord product: one of the lightest epilogue shares
    static constexpr int ISSUER = NW == 16 ? 12 : (NW == 24 ? 20 : NW - 4);
    static_assert(NW == 16 || NW == 24 || NW == 32, "4, 6 or 8 layer groups");
    const Model &m;
    const Work &w;
    TransFwdSmemT<NW> &sm;
    const int warp, lane, half, vq, pair, grp, ck, L, N, ntiles;
    // interpolation: 4 layer groups x 4 quarters (32 wavenumbers) of the tile;
    // a wavenumber pair is shared by a lane pair splitting the species. Lane
    // half 0 stores the hi parts of its pair's extinction, half 1 the lo parts.
    // Epilogue: TMEM lane quadrant vq (wavenumber 32 vq + lane), impact
    // parameters [28 ck, 28 ck + 28).
    const uint32_t a_off, mbar0, lh_s, ll_s;
    // tau^T[nu][i] = sum_l alpha^T[nu][l] L^T[l][i]: M = 128 wavenumbers, N = 112, K = 112;
    // A = alpha (stored [l][nu]: MN-major), B = L (stored [i][l]: K-major)
    const uint32_t idesc;
    uint32_t tmem = 0;
    uint32_t phases = 0u;   // bit k: parity of the next completion of mbar[k]
    int issued = 0;
    // pend: the last tile issued to the tensor cores (epilogue not yet run);
    // spec: the tile whose epilogue ran (its spectrum written after the next barrier)
    int pend_b = -1, pend_t = 0, pend_buf = 0;
    int spec_b = -1, spec_t = 0, spec_buf = 0;
    bool abort = false;

    __device__ __forceinline__ TransFwdEngine(const Model &m_, const Work &w_, TransFwdSmemT<NW> &sm_)
        : m(m_), w(w_), sm(sm_), warp(threadIdx.x >> 5), lane(threadIdx.x & 31), half(lane & 1), vq(warp & 3),
          pair(16 * vq + (lane >> 1)), grp(warp >> 2), ck(warp >> 2), L(m_.L), N(m_.N), ntiles((m_.N + FT2 - 1) / FT2),
          a_off(op_off(0, 2 * pair, SBO_NU)), mbar0(smem_u32(&sm_.mbar[0])), lh_s(smem_u32(sm_.lh)),
          ll_s(smem_u32(sm_.ll)), idesc(idesc_bf16(FT2, LP, true, false)) {}

    // whole block, once: zero padding rows, mbarriers (mbar[1] 8 bytes above mbar[0]), TMEM
    __device__ __forceinline__ void setup() {
        // extinction rows of the padding layers stay zero
        for (int idx = threadIdx.x; idx < (LP - L) * (FT2 / 2); idx += NT) {
            const uint32_t o = op_off(L + idx / (FT2 / 2), 2 * (idx % (FT2 / 2)), SBO_NU);
            *reinterpret_cast<uint32_t *>(sm.ah[0] + o) = 0u;
            *reinterpret_cast<uint32_t *>(sm.al[0] + o) = 0u;
        }
        if (threadIdx.x == 0) {
            mbar_init(mbar0, 1);
            mbar_init(mbar0 + 8, 1);
            sm.abort = 0;
        }
        if (warp == 0) tmem_alloc(smem_u32(&sm.tmem_base), F2_TMEM_COLS);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        tmem = sm.tmem_base;
    }

    __device__ __forceinline__ void wait_mma(int buf) {
        if (!mbar_wait(mbar0 + 8u * (uint32_t)buf, (phases >> buf) & 1u, m.wait_polls)) sm.abort = 1;
        phases ^= 1u << buf;
        tc_fence_after();
    }

    // impact parameters of epilogue chunk ck from cstart(): 4 chunks of 28 (16
    // warps), 4 of 20 and 2 of 16 (24 warps), or 8 of 14 (32 warps)
    __device__ __forceinline__ int cstart() const {
        return NCK == 4 ? 28 * ck : (NCK == 8 ? 14 * ck : (ck < 4 ? 20 * ck : 80 + 16 * (ck - 4)));
    }

    __device__ __forceinline__ void epilogue(int pb, int pt, int buf) {
        const int nl = 32 * vq + lane;
        const int c0 = cstart();
        // (24 warps: the x8 load and the last columns of the x4 load lie past a
        // 20- or 16-column chunk; they stay inside the allocation and are unused)
        const bool wide = NCK == 4 || ck < 4;   // chunk of 28 / 20 (vs 16) columns
        const uint32_t taddr = tmem + (uint32_t)(buf * 128 + c0) + ((uint32_t)(32 * vq) << 16);
        float v16[16], v8[8], v4[4], v2[2];
        if (NCK == 8) {   // 14 = 8 + 4 + 2 columns
            tmem_ld8(taddr, v8);
            tmem_ld4(taddr + 8, v4);
            tmem_ld2(taddr + 12, v2);
        } else {
            tmem_ld16(taddr, v16);
            if (NCK == 4) tmem_ld8(taddr + 16, v8);
            tmem_ld4(taddr + (NCK == 4 ? 24 : 16), v4);
        }
        tmem_wait_ld();
        // exp(-tau) store, tile-contiguous: [vector][tile][impact parameter][128 nu]
        float *eb = w.estore + (((size_t)pb * ntiles + pt) * L + c0) * FT2 + nl;
        float2 s2 = f2(0.f);
        // terms i0 = c0 + k and i0 + 1 in packed pairs; area[i] = 0 beyond L
        auto term2 = [&](int k, float t0, float t1) {
            const int i0 = c0 + k;
            const float2 e = ex2x2(mul2(make_float2(t0, t1), f2(-LOG2E_F)));
            const float2 a = *reinterpret_cast<const float2 *>(&sm.area[i0]);
            s2 = fma2(a, fma2(e, f2(-1.f), f2(1.f)), s2);
            // streaming stores: keep the opacity coefficients, not these, in L2
            if (STORE_E) {
                if (i0 < L) __stcs(eb + k * FT2, e.x);
                if (i0 + 1 < L) __stcs(eb + (k + 1) * FT2, e.y);
            }
        };
        float s;
        if (!CLOUD && NCK == 8) {
#pragma unroll
            for (int k = 0; k < 8; k += 2) term2(k, v8[k], v8[k + 1]);
#pragma unroll
            for (int k = 0; k < 4; k += 2) term2(8 + k, v4[k], v4[k + 1]);
            term2(12, v2[0], v2[1]);
            s = s2.x + s2.y;
        } else if (!CLOUD) {
#pragma unroll
            for (int k = 0; k < 16; k += 2) term2(k, v16[k], v16[k + 1]);
            if (NCK == 4) {
#pragma unroll
                for (int k = 0; k < 8; k += 2) term2(16 + k, v8[k], v8[k + 1]);
#pragma unroll
                for (int k = 0; k < 4; k += 2) term2(24 + k, v4[k], v4[k + 1]);
            } else if (NCK == 6 && wide) {
#pragma unroll
                for (int k = 0; k < 4; k += 2) term2(16 + k, v4[k], v4[k + 1]);
            }
            s = s2.x + s2.y;
        } else {
            // non-grey cloud (Sect. 2.5): the cloudy chord depth is tau_i + g(nu) D_i,
            // g = 1/(Q0 x^-a + x^0.2), x = 2 pi r_eff nu; the two transit depths
            // mix by the cloud fraction, f delta_cld + (1 - f) delta_cf
            const float g = kh18_g(sm.cg, m.nu[(size_t)pt * FT2 + nl]);
            const float2 gl = f2(-g * LOG2E_F);
            float2 s2c = f2(0.f);
            auto term2c = [&](int k, float t0, float t1) {
                const int i0 = c0 + k;
                const float2 e = ex2x2(mul2(make_float2(t0, t1), f2(-LOG2E_F)));
                const float2 a = *reinterpret_cast<const float2 *>(&sm.area[i0]);
                const float2 d = *reinterpret_cast<const float2 *>(&sm.cd[i0]);
                const float2 ec = mul2(e, ex2x2(mul2(gl, d)));
                s2 = fma2(a, fma2(e, f2(-1.f), f2(1.f)), s2);
                s2c = fma2(a, fma2(ec, f2(-1.f), f2(1.f)), s2c);
                if (STORE_E) {   // the cloud-free exp(-tau); the adjoint rebuilds the cloudy one
                    if (i0 < L) __stcs(eb + k * FT2, e.x);
                    if (i0 + 1 < L) __stcs(eb + (k + 1) * FT2, e.y);
                }
            };
            if (NCK == 8) {
#pragma unroll
                for (int k = 0; k < 8; k += 2) term2c(k, v8[k], v8[k + 1]);
#pragma unroll
                for (int k = 0; k < 4; k += 2) term2c(8 + k, v4[k], v4[k + 1]);
                term2c(12, v2[0], v2[1]);
            } else {
#pragma unroll
            for (int k = 0; k < 16; k += 2) term2c(k, v16[k], v16[k + 1]);
            }
            if (NCK == 4) {
#pragma unroll
                for (int k = 0; k < 8; k += 2) term2c(16 + k, v8[k], v8[k + 1]);
#pragma unroll
                for (int k = 0; k < 4; k += 2) term2c(24 + k, v4[k], v4[k + 1]);
            } else if (NCK == 6 && wide) {
#pragma unroll
                for (int k = 0; k < 4; k += 2) term2c(16 + k, v4[k], v4[k + 1]);
            }
            s = sm.cg[3] * (s2c.x + s2c.y) + (1.f - sm.cg[3]) * (s2.x + s2.y);
        }
        sm.part[buf][ck][nl] = s;
    }

    __device__ __forceinline__ void write_spec(int pb, int pt, int buf) {
        if (threadIdx.x < FT2) {
            const int n = pt * FT2 + threadIdx.x;
            const float(*pp)[FT2] = sm.part[buf];
            float v = (pp[0][threadIdx.x] + pp[1][threadIdx.x]) + (pp[2][threadIdx.x] + pp[3][threadIdx.x]);
            if (NCK >= 6) v += pp[4][threadIdx.x] + pp[5][threadIdx.x];
            if (NCK == 8) v += pp[6][threadIdx.x] + pp[7][threadIdx.x];
            if (n < N) w.spec[(size_t)pb * N + n] = v;
        }
    }

    // finish every tile in flight: its product, epilogue and spectrum
    __device__ __forceinline__ void drain() {
        if (pend_b >= 0) epilogue(pend_b, pend_t, pend_buf);
        tc_fence_before();
        __syncthreads();
        if (spec_b >= 0) write_spec(spec_b, spec_t, spec_buf);
        if (pend_b >= 0) write_spec(pend_b, pend_t, pend_buf);
        pend_b = spec_b = -1;
    }

    // whole block, after drain() and a block barrier: sample b's L operand,
    // areas and cloud constants (its layer constants are staged by the caller)
    __device__ __forceinline__ void stage_operands(int b) {
        stage_lmat_tc(m, w, b, sm.lh, sm.ll, sm.area);
        if (CLOUD) {
            for (int i = threadIdx.x; i < LP; i += NT) sm.cd[i] = (i < L) ? w.cloud_d[(size_t)b * L + i] : 0.f;
            if (threadIdx.x < N_CG) sm.cg[threadIdx.x] = w.cloud_g[(size_t)b * N_CG + threadIdx.x];
        }
    }

    // tiles [t0, t1) of the staged sample b, the extinction operand of each
    // written by fill(first wavenumber of the tile); sets `abort` if a wait gave up
    template <class Fill>
    __device__ __forceinline__ void tiles_with(int b, int t0, int t1, Fill &&fill) {
        for (int t = t0; t < t1; ++t) {
            const int nt0 = t * FT2;
            const int buf = issued & 1;
            fill(nt0);
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            if (sm.abort) {
                abort = true;
                return;
            }
            if (spec_b >= 0) {   // its epilogue ran in every warp before this barrier
                write_spec(spec_b, spec_t, spec_buf);
                spec_b = -1;
            }
            // (wait_test: no product is issued, so the wait below runs out and the block aborts)
            if (threadIdx.x == ISSUER * 32 && !m.wait_test) {   // 7 k-steps x 3 split terms
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * 128);
                // descriptors of k-step 0; a k-step advances the start address field
                // (bits 0-13, 16-byte units) by 2 row groups of alpha / 2 cores of L
                const uint64_t a_h = desc_mn_major(smem_u32(sm.ah[0]), SBO_NU);
                const uint64_t a_l = desc_mn_major(smem_u32(sm.al[0]), SBO_NU);
                const uint64_t b_h = desc_k_major(lh_s, SBO_LP), b_l = desc_k_major(ll_s, SBO_LP);
#pragma unroll
                for (int k = 0; k < LP / 16; ++k) {
                    const uint64_t da = (uint64_t)(k * 2 * SBO_NU / 16), db = (uint64_t)(k * 2 * CORE_STRIDE / 16);
                    tc_mma(d, a_h + da, b_h + db, idesc, k > 0);
                    tc_mma(d, a_h + da, b_l + db, idesc, true);
                    tc_mma(d, a_l + da, b_h + db, idesc, true);
                }
                tc_commit(mbar0 + 8u * (uint32_t)buf);
            }
            // the previous tile's epilogue (its product completed in the
            // previous iteration) overlaps the product just issued
            if (pend_b >= 0) {
                epilogue(pend_b, pend_t, pend_buf);
                spec_b = pend_b;
                spec_t = pend_t;
                spec_buf = pend_buf;
            }
            wait_mma(buf);   // this tile's product: frees the single alpha buffer
            pend_b = b;
            pend_t = t;
            pend_buf = buf;
            ++issued;
        }
    }

    // the extinction interpolated here (the sample's layer constants staged)
    __device__ __forceinline__ void tiles(int b, int t0, int t1) {
        unsigned char *const a_dst = (half ? sm.al[0] : sm.ah[0]) + a_off;
        tiles_with(b, t0, t1, [&](int nt0) {
            extinction_pair<SPL>(m, sm.sc, sm.sc.gb[grp], sm.sc.gb[grp + 1], nt0 + 2 * pair, half,
                                 [&](const LayerConst &lc, float2 a) {
                uint32_t hi, lo;
                split2(a, hi, lo);
                *reinterpret_cast<uint32_t *>(a_dst + lc.aoff) = half ? lo : hi;
            });
        });
    }

    // the extinction read from ext[b][l][Np] (written by the opacity-stage
    // kernel): every thread converts wavenumber pairs of the tile's rows to
    // the split operand, all its loads in flight together
    __device__ __forceinline__ void tiles_from(int b, int t0, int t1, const float *ext) {
        tiles_with(b, t0, t1, [&](int nt0) {
            const float *src = ext + (size_t)b * L * m.Np + nt0;
            constexpr int PER_ROW = FT2 / 2, ITER = (LP * PER_ROW + NT - 1) / NT;
            float2 v[ITER];
#pragma unroll
            for (int k = 0; k < ITER; ++k) {
                const int idx = threadIdx.x + k * NT, l = idx / PER_ROW, c = 2 * (idx % PER_ROW);
                if (l < L) v[k] = *reinterpret_cast<const float2 *>(src + (size_t)l * m.Np + c);
            }
#pragma unroll
            for (int k = 0; k < ITER; ++k) {
                const int idx = threadIdx.x + k * NT, l = idx / PER_ROW, c = 2 * (idx % PER_ROW);
                if (l < L) {
                    uint32_t hi, lo;
                    split2(v[k], hi, lo);
                    const uint32_t o = op_off(l, c, SBO_NU);
                    *reinterpret_cast<uint32_t *>(sm.ah[0] + o) = hi;
                    *reinterpret_cast<uint32_t *>(sm.al[0] + o) = lo;
                }
            }
        });
    }

    // whole block, once at the end: the tiles in flight, the status word, TMEM
    __device__ __forceinline__ void teardown() {
        if (!abort) drain();
        if (sm.abort) abort = true;
        if (abort && threadIdx.x == 0) atomicOr(w.err, 1);
        tc_fence_before();
        __syncthreads();
        if (warp == 0) tmem_free(tmem, F2_TMEM_COLS);
    }
};

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

// Two transpose stages of a warp reduction of 4 values per lane: lane holds
// the sum of v[2 b4 + b3] over the 4 lanes that differ from it in bits 4 and 3
// (bk = bit k of the lane); the remaining sums over bits 2 and 1 (the lane
// parity, bit 0, stays apart) are left to the shared-memory accumulation.
__device__ __forceinline__ float reduce4_partial(const float (&v)[4], int lane) {
    float a[2];
    {
        const bool up = lane & 16;
#pragma unroll
        for (int k = 0; k < 2; ++k)
            a[k] = (up ? v[k + 2] : v[k]) + __shfl_xor_sync(0xffffffffu, up ? v[k] : v[k + 2], 16);
    }
    const bool up = lane & 8;
    return (up ? a[1] : a[0]) + __shfl_xor_sync(0xffffffffu, up ? a[0] : a[1], 8);
}

// Split TMEM load of one column of this warp's lane quadrant: the issue, and
// the wait that binds the value (no use may be scheduled before it).
__device__ __forceinline__ void tmem_issue1(uint32_t taddr, uint32_t &r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr) : "memory");
}
__device__ __forceinline__ void tmem_wait1(uint32_t &r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r)::"memory");
}

// Backward interpolation for one warp: layers [lb, le), wavenumber pair n, n+1
// shared by the lane pair (lane, lane ^ 1) that splits the species. Reads
// alpha_bar from TMEM (`abar_t`: column 0 of the warp's lane quadrant, lane =
// wavenumber), adds per-layer partial reductions to red[l][32] and
// per-species totals to qtot[s], and writes the extinction as split BF16 into
// the alpha operand (`a_dst`: row 0 at this lane's column, hi for half 0, lo
// for half 1). Per layer, summed over wavenumber, with lane half h's species
// and CIA pair h: QS_h = sum abar n sum_s e_s, D_h = sum abar n sum_s e_s
// dlog2(sigma_s)/dw_T, C_h = sum abar c_h, CT_h = sum abar c_h dlog2 k_h/dw_Tc
// (slots 0/1, 2/3, 4/5, 6/7 for h = 0/1, each as 4 partial sums; the flush
// adds them and applies the per-layer weight slopes gts, gtcs); per species
// Q_s = sum_l sum abar n e_s. The Rayleigh sum over wavenumber comes from the
// L_bar product.
template <int SPL, bool STAGE, class Wait>
__device__ void interp_backward(const Model &m, const SampleConst &sc, int lb, int le, int n, int half, int lane,
                                uint32_t abar_t, unsigned char *a_dst, float *red, float *qtot, uint32_t stg,
                                bool prestaged, int next_shift, Wait &&wait_abar) {
    const int S = m.S;
    const int ridx = reduce_index8(lane);
    const bool writer = (lane & 3) == 0;
    // after the two transpose stages every lane holds a distinct partial sum:
    // slot 2 (2 b4 + b3) + b0, partial (b2 b1); one atomic per lane, no branch
    const int rslot = 4 * (2 * (2 * ((lane >> 4) & 1) + ((lane >> 3) & 1)) + (lane & 1)) + ((lane >> 1) & 3);
    PairInterp<SPL> pi;
    pi.init(m, n, half, lane);
    float2 qa[SPL];
#pragma unroll
    for (int j = 0; j < SPL; ++j) qa[j] = f2(0.f);
    bool waited = false;
    uint32_t nxt = 0u;   // alpha_bar of the next layer: its TMEM load runs during the current layer
    // loop bounds broadcast from lane 0: provably warp-uniform for the compiler
    lb = __shfl_sync(0xffffffffu, lb, 0);
    le = __shfl_sync(0xffffffffu, le, 0);
    constexpr bool STAGED = STAGE && 2 * SPL + 1 <= STAGE_BLOCKS;   // else direct loads with an L1 prefetch
    if (STAGED && lb < le && !prestaged) pi.stage(stg, sc.lay[lb].cell, sc.lay[lb].itc, 0);
    for (int l = lb; l < le;) {
        const int end = __shfl_sync(0xffffffffu, min(sc.lay[l].run_end, le), 0);
        if constexpr (STAGED) {
            pi.load_staged(sc, stg);
            if (end < le) pi.stage(stg, sc.lay[end].cell, sc.lay[end].itc, 0);
            else if (next_shift) pi.stage(stg, sc.lay[lb].cell, sc.lay[lb].itc, next_shift);
        } else {
            pi.load(sc, sc.lay[l].cell, sc.lay[l].itc);
            if (end < le) pi.prefetch(sc.lay[end].cell, sc.lay[end].itc);
        }
        if (!waited) {   // the first coefficient loads are in flight while the alpha_bar product completes
            wait_abar();
            waited = true;
            tmem_issue1(abar_t + (uint32_t)l, nxt);
        }
        const LayerConst *lp = &sc.lay[l], *const lend = &sc.lay[end];
        float *rp = red + l * 32 + rslot;
        uint32_t ta = abar_t + (uint32_t)l;
        for (; lp != lend; ++lp, rp += 32, ++ta) {
            const LayerConst &lc = *lp;
            tmem_wait1(nxt);
            const float own = __uint_as_float(nxt);
            // the next column, unconditionally (column le is inside the
            // allocation; its value is never used)
            tmem_issue1(ta + 1u, nxt);
            // both wavenumbers of the pair from the pair's two lanes (two shuffles,
            // no lane-parity selects)
            const float2 ab = make_float2(__shfl_sync(0xffffffffu, own, lane & 30), __shfl_sync(0xffffffffu, own, lane | 1));
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
            v[1] = fmaf(abn.x, pt.x, abn.y * pt.y);   // x gts at the flush
            v[2] = ac.x + ac.y;
            v[3] = act.x + act.y;                     // x gtcs at the flush
            atomicAdd(rp, reduce4_partial(v, lane));
            const float2 mine = fma2(lc.ray, pi.nu4, fma2(sum, lc.nsc, c));
            const float2 alpha = add2(mine, shfl_xor2(mine, 1));
            *reinterpret_cast<uint32_t *>(a_dst + lc.aoff) = bf16x2(alpha);   // both lanes: same word
        }
        l = end;
    }
    if (!waited) wait_abar();   // empty layer group
    else tmem_wait1(nxt);       // the load issued past the last layer
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

// ---------------------------------------------------------------- adjoint engine
// The adjoint's per-tile machinery for one block (set-up, staging, the tiles
// of one work item with the L2 prefetch of the next item's first tile, the
// flush of a sample's sums, teardown), driven by the transmission-only and
// the mixed kernels.
// NW warps (16, 20 or 24); STAGE: coefficients through the per-warp staging
// slots; LSPLIT: split BF16 L in alpha_bar = L^T tau_bar.
template <int SPL, bool CLOUD, int NW = 16, bool STAGE = true, bool LSPLIT = true>
struct TransBwdEngine {
    static constexpr int NT = NW * 32;
    // tau_bar phase: NW / 2 row groups of two warps (128 wavenumbers), rows
    // i = group + ROWG k for k < KR
    static constexpr int ROWG = NW / 2, KR = (LP + ROWG - 1) / ROWG;
    const Model &m;
    const Work &w;
    TransBwdSmemT<NW, STAGE, LSPLIT> &sm;
    const int warp, lane, L, N, S, ntiles;
    const int group;
    // interpolation: 4 layer groups x 4 quarters (32 wavenumbers); lane pairs split species
    const int half, vq, pair, grp;
    const int NL;                                        // L_bar product N: layers and the weight row
    const float ray_ref;
    const uint32_t mbar_a, mbar_l;
    // alpha_bar^T[nu][l] = sum_i tau_bar^T[nu][i] L[i][l]: M = 128 wavenumbers, N = 112, K = 112;
    // A = tau_bar (stored [i][nu]: MN-major), B = L (stored [i][l]: MN-major)
    const uint32_t idesc_a;
    // L_bar[i][l] += sum_nu tau_bar[i][nu] alpha[l][nu]: M = 128, N = NL, K = 128; both K-major
    const uint32_t idesc_l;
    const uint32_t lh_s, ll_s, th_s, ah_s;
    unsigned char *const a_dst;
    const uint32_t stg;
    uint32_t tmem = 0, abar_t = 0;
    uint32_t pa = 0, pl = 0;
    bool l_pending = false, l_started = false, abort = false;

    __device__ __forceinline__ TransBwdEngine(const Model &m_, const Work &w_, TransBwdSmemT<NW, STAGE, LSPLIT> &sm_)
        : m(m_), w(w_), sm(sm_), warp(threadIdx.x >> 5), lane(threadIdx.x & 31), L(m_.L), N(m_.N), S(m_.S),
          ntiles((m_.N + BT - 1) / BT), group(warp >> 1), half(lane & 1), vq(warp & 3), pair(16 * vq + (lane >> 1)),
          grp(warp >> 2), NL((m_.L + 1 + 15) & ~15),
          ray_ref((float)(1.0 / ((double)m_.ray_nu_ref * m_.ray_nu_ref * m_.ray_nu_ref * m_.ray_nu_ref))),
          mbar_a(smem_u32(&sm_.mbar_a)), mbar_l(smem_u32(&sm_.mbar_l)), idesc_a(idesc_bf16(BT, LP, true, true)),
          idesc_l(idesc_bf16(LB_ROWS, NL, false, false)), lh_s(smem_u32(sm_.lh)), ll_s(smem_u32(sm_.ll)),
          th_s(smem_u32(sm_.th)), ah_s(smem_u32(sm_.ah)), a_dst(sm_.ah + op_off(0, 2 * pair, SBO_NU)),
          stg(smem_u32(sm_.stage[STAGE ? warp : 0]) + 16u * (uint32_t)lane) {}

    // whole block, once: zero padding rows, mbarriers, TMEM
    __device__ __forceinline__ void setup() {
        if (CLOUD)
            for (int i = threadIdx.x; i < BT; i += NT) sm.gbar[i] = 0.f;
        // padding rows stay zero: tau_bar rows [L, 112), alpha rows [L + 1, 128)
        for (int idx = threadIdx.x; idx < (LP - L) * (BT / 2); idx += NT) {
            const uint32_t o = op_off(L + idx / (BT / 2), 2 * (idx % (BT / 2)), SBO_NU);
            *reinterpret_cast<uint32_t *>(sm.th + o) = 0u;
        }
        for (int idx = threadIdx.x; idx < (LB_ROWS - L - 1) * (BT / 2); idx += NT) {
            const uint32_t o = op_off(L + 1 + idx / (BT / 2), 2 * (idx % (BT / 2)), SBO_NU);
            *reinterpret_cast<uint32_t *>(sm.ah + o) = 0u;
        }
        if (threadIdx.x == 0) {
            mbar_init(mbar_a, 1);
            mbar_init(mbar_l, 1);
            sm.abort = 0;
        }
        if (warp == 0) tmem_alloc(smem_u32(&sm.tmem_base), 256);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        tmem = sm.tmem_base;
        abar_t = tmem + ((uint32_t)(32 * vq) << 16);
    }

    __device__ __forceinline__ void wait_lbar() {
        if (l_pending) {
            if (!mbar_wait(mbar_l, pl, m.wait_polls)) sm.abort = 1;
            pl ^= 1;
            l_pending = false;
            tc_fence_after();
        }
    }

    // L_bar (TMEM: lane i, column 128 + l; FP32 atomics) and z, the reductions, per-species
    // totals and area_bar of sample b, by FP64 atomics (after wait_lbar)
    __device__ __forceinline__ void flush(int b) {
        float *lbar = w.lbar + (size_t)b * L * L;
        double *zbar = w.zbar + (size_t)b * L;
        const int ck = warp >> 2, ii = 32 * vq + lane;
        // the L_bar columns [128, 256): 4 chunks of 32 over the first 16 warps
        if (ck < 4) {
        float v0[16], v1[16];
        const uint32_t ta = tmem + (uint32_t)(128 + 32 * ck) + ((uint32_t)(32 * vq) << 16);
        tmem_ld16(ta, v0);
        tmem_ld16(ta + 16, v1);
        tmem_wait_ld();
        if (ii < L) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int ll = 32 * ck + j;
                const float v = j < 16 ? v0[j] : v1[j - 16];
                if (v == 0.f) continue;
                if (ll == L) atomicAdd(zbar + ii, (double)v);
                else if (ll <= ii) atomicAdd(lbar + (size_t)ii * L + ll, v);
            }
        }
        }
        tc_fence_before();
        __syncthreads();
        for (int idx = threadIdx.x; idx < L * 8; idx += NT) {
            const int l = idx >> 3, s = idx & 7;
            const float *q = sm.red + l * 32 + 4 * s;
            float v = (q[0] + q[1]) + (q[2] + q[3]);
            if (s == 2 || s == 3) v *= sm.sc.lay[l].gts;   // D: d/dlog10 T of the species exponents
            if (s >= 6) v *= sm.sc.lay[l].gtcs;            // CT: of the CIA exponents
            if (v != 0.f) atomicAdd(w.red + ((size_t)b * L + l) * N_RED + s, (double)v);
        }
        for (int i = threadIdx.x; i < L; i += NT)
            if (sm.area_acc[i] != 0.f) atomicAdd(w.areabar + (size_t)b * L + i, (double)sm.area_acc[i]);
        for (int s2 = threadIdx.x; s2 < S; s2 += NT)
            if (sm.qtot[s2] != 0.f) atomicAdd(w.qtot + (size_t)b * S + s2, (double)sm.qtot[s2]);
        if (CLOUD) {
            for (int i = threadIdx.x; i < L; i += NT)
                if (sm.cdbar[i] != 0.f) atomicAdd(w.cloud_dbar + (size_t)b * L + i, (double)sm.cdbar[i]);
            if (threadIdx.x < N_CG && sm.cpbar[threadIdx.x] != 0.f)
                atomicAdd(w.cloud_pbar + (size_t)b * N_CG + threadIdx.x, (double)sm.cpbar[threadIdx.x]);
        }
    }

    // L2 prefetch of the exp(-tau) rows and dbar of tile t of sample b (the
    // tau_bar phase reads them straight from HBM otherwise, with every warp
    // of the block waiting on the same loads): one 128-byte line per thread
    // (4 lines per row of 128 wavenumbers), issued through the load/store
    // units rather than as bulk copies, which the TMA unit serialises
    __device__ __forceinline__ void prefetch_tile(int pb, int pt) {
        const int row = threadIdx.x >> 2, line = threadIdx.x & 3;
        const float *src = nullptr;
        if (row < L) src = w.estore + (((size_t)pb * ntiles + pt) * L + row) * BT + 32 * line;
        else if (row == L) src = w.dbar + (size_t)pb * m.Np + (size_t)pt * BT + 32 * line;
        if (src) asm volatile("prefetch.global.L2 [%0];" ::"l"(src));
    }

    // whole block, after a block barrier: sample b's L operand, areas, zeroed
    // per-sample sums and cloud constants (its layer constants are staged by
    // the caller); the L_bar accumulator restarts
    __device__ __forceinline__ void stage_operands(int b) {
        stage_lmat_tc(m, w, b, sm.lh, LSPLIT ? sm.ll : nullptr, sm.area);
        for (int idx = threadIdx.x; idx < L * 32; idx += NT) sm.red[idx] = 0.f;
        for (int i = threadIdx.x; i < LP; i += NT) sm.area_acc[i] = 0.f;
        for (int s2 = threadIdx.x; s2 < ES_MAX_SPECIES; s2 += NT) sm.qtot[s2] = 0.f;
        if (CLOUD) {
            for (int i = threadIdx.x; i < LP; i += NT) {
                sm.cd[i] = (i < L) ? w.cloud_d[(size_t)b * L + i] : 0.f;
                sm.cdbar[i] = 0.f;
            }
            if (threadIdx.x < N_CG) {
                sm.cg[threadIdx.x] = w.cloud_g[(size_t)b * N_CG + threadIdx.x];
                sm.cpbar[threadIdx.x] = 0.f;
            }
        }
        l_started = false;
    }

    // tiles [t0, t1) of the staged sample b; (nx_b, nx_t): the first tile of
    // the block's next transmission work item, prefetched during the last
    // tile (nx_b < 0: none). Sets `abort` if a wait gave up.
    __device__ __forceinline__ void tiles(int b, int t0, int t1, int nx_b, int nx_t) {
        for (int t = t0; t < t1; ++t) {
            const int nt0 = t * BT;
            if (t + 1 < t1) prefetch_tile(b, t + 1);
            else if (nx_b >= 0) prefetch_tile(nx_b, nx_t);
            // tau_bar = dbar A_i exp(-tau); area_bar += dbar (1 - exp(-tau)). The
            // loads are issued before waiting for the previous tile's L_bar
            // product, which still reads tau_bar and alpha.
            const int col = 2 * (lane + 32 * (warp & 1));
            const int nl = nt0 + col;
            const float2 db = *reinterpret_cast<const float2 *>(w.dbar + (size_t)b * m.Np + nl);
            const float *eb = w.estore + ((size_t)b * ntiles + t) * L * BT + col;
            float2 ev[KR];
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                const int i = group + ROWG * k;
                ev[k] = (i < L) ? *reinterpret_cast<const float2 *>(eb + i * BT) : make_float2(1.f, 1.f);
            }
            wait_lbar();
            // Rayleigh weight row w(nu) of the alpha operand
            if (threadIdx.x < BT / 2) {
                const int t2 = threadIdx.x;
                const float2 nu = __ldg(reinterpret_cast<const float2 *>(m.nu + nt0 + 2 * t2));
                const float2 nu2 = mul2(nu, nu);
                const uint32_t o = op_off(L, 2 * t2, SBO_NU);
                *reinterpret_cast<uint32_t *>(sm.ah + o) = bf16x2(mul2(mul2(nu2, nu2), f2(ray_ref)));
            }
            if (!CLOUD) {
                float av[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    av[k] = 0.f;
                    const int i = group + ROWG * k;
                    if (k < KR && i < L) {
                        const float2 e = ev[k];
                        const float a = sm.area[i];
                        const uint32_t o = op_off(i, col, SBO_NU);
                        *reinterpret_cast<uint32_t *>(sm.th + o) = bf16x2(make_float2(db.x * a * e.x, db.y * a * e.y));
                        av[k] = db.x * (1.f - e.x) + db.y * (1.f - e.y);
                    }
                }
                const float tot = transpose_reduce16(av, lane);
                const int k = reduce_index(lane), i = group + ROWG * k;
                if ((lane & 1) == 0 && k < KR && i < L && tot != 0.f) atomicAdd(sm.area_acc + i, tot);
            } else {
                // non-grey cloud: E_i = f e_cld + (1 - f) e with e_cld = e 2^(-g D_i log2 e);
                // tau_bar = dbar A_i E_i, area_bar += dbar (1 - E_i), and the
                // adjoints of D_i, of g(nu) and of f
                const float2 nu = *reinterpret_cast<const float2 *>(m.nu + nl);
                const float2 g = make_float2(kh18_g(sm.cg, nu.x), kh18_g(sm.cg, nu.y));
                const float2 gl = mul2(g, f2(-LOG2E_F));
                const float fc = sm.cg[3];
                float av[16], dv[16], fs = 0.f;
                float2 gs = f2(0.f);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    av[k] = dv[k] = 0.f;
                    const int i = group + ROWG * k;
                    if (k < KR && i < L) {
                        const float2 e = ev[k];
                        const float a = sm.area[i], d = sm.cd[i];
                        const float2 ec = mul2(e, ex2x2(mul2(gl, f2(d))));
                        const float2 E = fma2(f2(fc), add2(ec, mul2(e, f2(-1.f))), e);
                        const uint32_t o = op_off(i, col, SBO_NU);
                        *reinterpret_cast<uint32_t *>(sm.th + o) = bf16x2(make_float2(db.x * a * E.x, db.y * a * E.y));
                        av[k] = db.x * (1.f - E.x) + db.y * (1.f - E.y);
                        const float2 wc = mul2(db, ec);
                        dv[k] = fc * a * (wc.x * g.x + wc.y * g.y);
                        gs = fma2(f2(fc * a * d), wc, gs);
                        fs = fmaf(a, db.x * (e.x - ec.x) + db.y * (e.y - ec.y), fs);
                    }
                }
                const float tot = transpose_reduce16(av, lane);
                const float totd = transpose_reduce16(dv, lane);
                const int k = reduce_index(lane), i = group + ROWG * k;
                if ((lane & 1) == 0 && k < KR && i < L) {
                    if (tot != 0.f) atomicAdd(sm.area_acc + i, tot);
                    if (totd != 0.f) atomicAdd(sm.cdbar + i, totd);
                }
                atomicAdd(sm.gbar + col, gs.x);
                atomicAdd(sm.gbar + col + 1, gs.y);
                fs = warp_sum(fs);
                if (lane == 0 && fs != 0.f) atomicAdd(sm.cpbar + 3, fs);
            }
            fence_async_smem();
            __syncthreads();
            if (sm.abort) {
                abort = true;
                return;
            }
            if (threadIdx.x == 0 && !m.wait_test) {   // alpha_bar: 7 k-steps over impact parameters x (L hi, L lo)
                tc_fence_after();
                const uint64_t a_h = desc_mn_major(th_s, SBO_NU);
                const uint64_t b_h = desc_mn_major(lh_s, SBO_LP), b_l = desc_mn_major(ll_s, SBO_LP);
#pragma unroll
                for (int k = 0; k < LP / 16; ++k) {   // start address field advances by 2 row groups
                    const uint64_t da = (uint64_t)(k * 2 * SBO_NU / 16), db2 = (uint64_t)(k * 2 * SBO_LP / 16);
                    tc_mma(tmem, a_h + da, b_h + db2, idesc_a, k > 0);
                    if (LSPLIT) tc_mma(tmem, a_h + da, b_l + db2, idesc_a, true);
                }
                tc_commit(mbar_a);
            }
            if (CLOUD && threadIdx.x < BT) {
                // d lnL / d g(nu) -> the g(nu) parameters at this tile's wavenumbers
                const float gb = sm.gbar[threadIdx.x];
                sm.gbar[threadIdx.x] = 0.f;
                float o[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (gb != 0.f) kh18_g_adjoint(sm.cg, m.nu[nt0 + threadIdx.x], gb, o);
                cloud_pbar_add(sm.cg, o, sm.cpbar, lane);
            }
            interp_backward<SPL, STAGE>(m, sm.sc, sm.sc.gb[grp], sm.sc.gb[grp + 1], nt0 + 2 * pair, half, lane, abar_t, a_dst,
                                 sm.red, sm.qtot, stg, t > t0, t + 1 < t1 ? BT : 0, [&]() {
                                     if (!mbar_wait(mbar_a, pa, m.wait_polls)) sm.abort = 1;
                                     tc_fence_after();
                                 });
            pa ^= 1;
            tc_fence_before();
            fence_async_smem();
            __syncthreads();
            if (sm.abort) {
                abort = true;
                return;
            }
            if (threadIdx.x == 32 && !m.wait_test) {   // L_bar (from another warp than alpha_bar's issuer): 8 k-steps
                tc_fence_after();
                const uint32_t d = tmem + 128u;
                const uint64_t a_h = desc_k_major(th_s, SBO_NU), b_h = desc_k_major(ah_s, SBO_NU);
#pragma unroll
                for (int k = 0; k < BT / 16; ++k) {   // start address field advances by 2 cores
                    const uint64_t dk = (uint64_t)(k * 2 * CORE_STRIDE / 16);
                    tc_mma(d, a_h + dk, b_h + dk, idesc_l, l_started || k > 0);
                }
                tc_commit(mbar_l);
            }
            l_pending = true;
            l_started = true;
        }
    }

    // whole block, once at the end: the status word, TMEM
    __device__ __forceinline__ void teardown() {
        if (sm.abort) abort = true;
        if (abort && threadIdx.x == 0) atomicOr(w.err, 1);
        tc_fence_before();
        __syncthreads();
        if (warp == 0) tmem_free(tmem, 256);
    }
};

}  // namespace
}  // namespace es
