// Opacity stage of the one-vector transmission path (Sect. 3): the layer
// extinction alpha_l(nu) = n_l sum_s X_s sigma_s(T_l, p_l, nu) + CIA + Rayleigh
// of every layer and wavenumber of a sample, written to a [L][Np] buffer that
// the chord kernel reads. The batched kernels interpolate from the per-cell
// coefficient table and keep the extinction on chip; for a single vector the
// stage is a table stream, so this kernel reads the raw table rows instead,
// each row that brackets one of the sample's layers once.
//
// A block takes a window of AW = 64 wavenumbers of one sample:
//  1. it marks the (T, p) table nodes at the corners of any layer's cell, and
//     the CIA temperature nodes, and numbers them (warp ballot scans);
//  2. it copies the window of each marked row into shared memory with
//     cp.async: the species in parts of at most 6 (one part for S <= 6; more
//     parts are separate commit groups, each interpolated as it lands), or
//     in rounds when their rows do not all fit, or not at all (rows read
//     from global memory) when not even one species' rows fit;
//  3. warp w takes layer group w, lane q the wavenumber pair 2q, 2q + 1 of
//     the window; it walks its layers by runs of one cell and CIA bracket,
//     with the cell's bilinear coefficients of the part's species in
//     registers, and sums 2^(e_s + log2 X_s + K);
//  4. the last part adds CIA (both pairs, linear in T between their nodes)
//     and Rayleigh, scales the species sum by n 2^-K and writes alpha (zero
//     beyond N; the windows cover the padded row, so the chord kernel reads
//     no stale value). Earlier parts keep their sums in the output buffer.
// The exponent is the same polynomial as the coefficient table's,
// e = c0 + wp c1 + wt (c2 + wp c3) with c0 = L v00, c1 = L (v01 - v00),
// c2 = L (v10 - v00), c3 = L ((v11 - v10) - (v01 - v00)), L = log2(10).
#include <algorithm>

#include "fused_common.cuh"

namespace es {

namespace {

constexpr int AG = 8;                                   // layer groups per block: one per warp
constexpr int A_THREADS = AG * 32;
constexpr int AW = 64;                                  // wavenumbers per block (a pair per lane)
constexpr int A_SMEM = 72 * 1024;                       // dynamic shared memory per block (3 per SM)
static_assert(ES_MAX_LAYERS <= A_THREADS, "one layer per thread in the set-up");

// Per-layer constants. Corner rows: nodes are numbered in (it, ip) order, so
// the (it, ip + 1) row follows the (it, ip) row (and the CIA itc + 1 row the
// itc row) at the next slot (staged) or node (direct); one index each.
struct __align__(16) ALayer {
    float4 wpt;       // wp, wp, wt, wt (pressure and temperature weights as operand pairs)
    int4 ko;          // cell key it NP + ip; (it, ip) and (it + 1, ip) rows; CIA itc row (staged slots, or nodes)
    float4 wn;        // CIA weight wtc, wtc; n 2^-K, n 2^-K
    float4 rc;        // n (X s) / nu_ref^4 twice; log2(n^2 X_H2 X_H2) twice
    float4 c1;        // log2(n^2 X_H2 X_He) twice; unused
};

struct AlphaSmem {
    ALayer lay[ES_MAX_LAYERS];
    int rend[ES_MAX_LAYERS];    // first layer after l whose cell or CIA bracket differs (or L)
    float lx[ES_MAX_SPECIES];   // log2 X_s + K (absent species: a weight that makes their terms zero)
    int nnodes, ncia;
};

// table element: FP32, or the BF16 residual whose row offset is added separately
template <bool BF16>
struct TabElem;
template <>
struct TabElem<false> {
    using T = float;
    static __device__ __forceinline__ float2 pair(const float *p) { return *reinterpret_cast<const float2 *>(p); }
    static __device__ __forceinline__ float2 lds(uint32_t a) {
        float2 v;
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
        return v;
    }
};
template <>
struct TabElem<true> {
    using T = uint16_t;
    static __device__ __forceinline__ float2 unpack(uint32_t v) {
        return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
    }
    static __device__ __forceinline__ float2 pair(const uint16_t *p) {
        return unpack(*reinterpret_cast<const uint32_t *>(p));
    }
    static __device__ __forceinline__ float2 lds(uint32_t a) {
        uint32_t v;
        asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(a));
        return unpack(v);
    }
};
__device__ __forceinline__ float lds_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

// Where a part's species rows and the CIA rows are. STAGED: shared-memory
// byte addresses (species row (j, slot) at sp + (j nn + slot) row bytes, its
// BF16 offset at ro + 4 (j nn + slot); CIA row (h, slot) at cia + (h ncia +
// slot) 4 AW); else global element pointers at the thread's column.
template <bool BF16, bool STAGED>
struct Rows;
template <bool BF16>
struct Rows<BF16, true> {
    uint32_t sp, ro, cia;
    int nn, ncia;
};
template <bool BF16>
struct Rows<BF16, false> {
    const typename TabElem<BF16>::T *sp;   // species s0, node 0
    const float *ro;                       // BF16 row offsets of species s0
    const float *cia;                      // CIA pair 0, node 0
    size_t sstride, cpair;
    int nodes, Np;
};

// corners (v00, v01, v10, v11) of species j of the part at the layer's cell
template <bool BF16>
__device__ __forceinline__ void corners(const Rows<BF16, true> &r, int j, int4 ko, float2 (&v)[4]) {
    using E = TabElem<BF16>;
    constexpr uint32_t RB = AW * sizeof(typename E::T);
    const uint32_t a0 = r.sp + (uint32_t)(j * r.nn + ko.y) * RB, a1 = r.sp + (uint32_t)(j * r.nn + ko.z) * RB;
    v[0] = E::lds(a0);
    v[1] = E::lds(a0 + RB);
    v[2] = E::lds(a1);
    v[3] = E::lds(a1 + RB);
    if (BF16) {
        const uint32_t q0 = r.ro + 4u * (uint32_t)(j * r.nn + ko.y), q1 = r.ro + 4u * (uint32_t)(j * r.nn + ko.z);
        v[0] = add2(v[0], f2(lds_f32(q0)));
        v[1] = add2(v[1], f2(lds_f32(q0 + 4)));
        v[2] = add2(v[2], f2(lds_f32(q1)));
        v[3] = add2(v[3], f2(lds_f32(q1 + 4)));
    }
}
template <bool BF16>
__device__ __forceinline__ void corners(const Rows<BF16, false> &r, int j, int4 ko, float2 (&v)[4]) {
    using E = TabElem<BF16>;
    const typename E::T *p = r.sp + j * r.sstride;
    const size_t n0 = (size_t)ko.y * r.Np, n1 = (size_t)ko.z * r.Np;
    v[0] = E::pair(p + n0);
    v[1] = E::pair(p + n0 + r.Np);
    v[2] = E::pair(p + n1);
    v[3] = E::pair(p + n1 + r.Np);
    if (BF16) {
        const float *ro = r.ro + (size_t)j * r.nodes;
        v[0] = add2(v[0], f2(ro[ko.y]));
        v[1] = add2(v[1], f2(ro[ko.y + 1]));
        v[2] = add2(v[2], f2(ro[ko.z]));
        v[3] = add2(v[3], f2(ro[ko.z + 1]));
    }
}
// the CIA rows (lo, hi) of pair h at the layer's bracket
template <bool BF16>
__device__ __forceinline__ void cia_rows(const Rows<BF16, true> &r, int h, int co, float2 &lo, float2 &hi) {
    const uint32_t a = r.cia + (uint32_t)(h * r.ncia + co) * (AW * 4);
    lo = TabElem<false>::lds(a);
    hi = TabElem<false>::lds(a + AW * 4);
}
template <bool BF16>
__device__ __forceinline__ void cia_rows(const Rows<BF16, false> &r, int h, int co, float2 &lo, float2 &hi) {
    const float *p = r.cia + h * r.cpair + (size_t)co * r.Np;
    lo = *reinterpret_cast<const float2 *>(p);
    hi = *reinterpret_cast<const float2 *>(p + r.Np);
}

// Extinction of layers [l0, l1) at the thread's wavenumber pair for species
// [s0, s0 + ns), ns <= CH, by runs of layers with one cell and CIA bracket:
// at a run's start the cell's coefficients of the species go to registers,
// then each layer of the run sums the species' 2^e (slots j >= ns, in a last
// part shorter than CH, are exact zeros). A part after the FIRST adds the
// running sum read back from dst; the LAST adds CIA, Rayleigh and n 2^-K and
// writes alpha; other parts store the running sum. Run and loop bounds are
// broadcast from lane 0: warp-uniform for the compiler.
template <bool BF16, bool STAGED, int CH, bool FIRST, bool LAST>
__device__ __forceinline__ void layer_sums(const AlphaSmem &sa, const Rows<BF16, STAGED> &r, int s0, int ns, int l0,
                                           int l1, float2 nu4, float *dst, int Np) {
    const float2 l2t = f2((float)LOG2_10);
    float2 c0[CH], c1[CH], c2[CH], c3[CH];
    l0 = __shfl_sync(0xffffffffu, l0, 0);
    l1 = __shfl_sync(0xffffffffu, l1, 0);
    float2 *out = reinterpret_cast<float2 *>(dst + (size_t)l0 * Np);
    const int step = Np >> 1;
    for (int l = l0; l < l1;) {
        const int e = __shfl_sync(0xffffffffu, min(sa.rend[l], l1), 0);
        const int4 ko = sa.lay[l].ko;
#pragma unroll
        for (int j = 0; j < CH; ++j) {
            if (j < ns) {
                float2 v[4];
                corners(r, j, ko, v);
                const float2 d0 = add2(v[1], mul2(v[0], f2(-1.f)));
                c0[j] = fma2(v[0], l2t, f2(sa.lx[s0 + j]));
                c1[j] = mul2(d0, l2t);
                c2[j] = mul2(add2(v[2], mul2(v[0], f2(-1.f))), l2t);
                c3[j] = mul2(add2(add2(v[3], mul2(v[2], f2(-1.f))), mul2(d0, f2(-1.f))), l2t);
            } else {   // no species in this slot: an exactly zero term
                c0[j] = f2(-1.0e4f);
                c1[j] = c2[j] = c3[j] = f2(0.f);
            }
        }
        if (!FIRST)   // the run's running sums, into L1 ahead of their use
            for (int k = 0; k < e - l; ++k) asm volatile("prefetch.global.L1 [%0];" ::"l"(out + (size_t)k * step));
        for (const ALayer *lp = sa.lay + l; l < e; ++l, ++lp, out += step) {
            const float4 wpt = lp->wpt;
            const float2 wp = make_float2(wpt.x, wpt.y), wt = make_float2(wpt.z, wpt.w);
            float2 sum = ex2x2(fma2(wt, fma2(wp, c3[0], c2[0]), fma2(wp, c1[0], c0[0])));
#pragma unroll
            for (int j = 1; j < CH; ++j) sum = add2(sum, ex2x2(fma2(wt, fma2(wp, c3[j], c2[j]), fma2(wp, c1[j], c0[j]))));
            if (!FIRST) sum = add2(sum, *out);
            if (!LAST) {
                *out = sum;
                continue;
            }
            // CIA: log2 k = L (k_lo + wtc (k_hi - k_lo)) + log2(n^2 X X'), both pairs (the
            // bracket's rows read per layer: registers are kept for the species)
            const float4 wn = lp->wn, rc = lp->rc, cx = lp->c1;
            const float2 wtc = make_float2(wn.x, wn.y), nsc = make_float2(wn.z, wn.w);
            const float2 ray = make_float2(rc.x, rc.y), cc0 = make_float2(rc.z, rc.w), cc1 = make_float2(cx.x, cx.y);
            float2 a0, b0, a1, b1;
            cia_rows(r, 0, ko.w, a0, b0);
            cia_rows(r, 1, ko.w, a1, b1);
            const float2 e0 = fma2(mul2(wtc, l2t), add2(b0, mul2(a0, f2(-1.f))), fma2(a0, l2t, cc0));
            const float2 e1 = fma2(mul2(wtc, l2t), add2(b1, mul2(a1, f2(-1.f))), fma2(a1, l2t, cc1));
            const float2 c = add2(ex2x2(e0), ex2x2(e1));
            *out = fma2(ray, nu4, fma2(sum, nsc, c));
        }
    }
}

// One part of species with its role (first / last) as template arguments.
template <bool BF16, bool STAGED, int CH>
__device__ __forceinline__ void part_sums(const AlphaSmem &sa, const Rows<BF16, STAGED> &r, int s0, int ns, int l0,
                                          int l1, bool first, bool last, float2 nu4, float *dst, int Np) {
    if (first && last) layer_sums<BF16, STAGED, CH, true, true>(sa, r, s0, ns, l0, l1, nu4, dst, Np);
    else if (first) layer_sums<BF16, STAGED, CH, true, false>(sa, r, s0, ns, l0, l1, nu4, dst, Np);
    else if (last) layer_sums<BF16, STAGED, CH, false, true>(sa, r, s0, ns, l0, l1, nu4, dst, Np);
    else layer_sums<BF16, STAGED, CH, false, false>(sa, r, s0, ns, l0, l1, nu4, dst, Np);
}

// cp.async of the window [n0, n0 + AW) of rows q in [0, nrows) to shared
// memory row q (row bytes AW * sizeof(T)); row q's source row is src_of(q).
// Thread t copies 16-byte piece t % P of rows t / P, t / P + R, ... with
// P pieces per row and R = threads / P rows per sweep.
template <class T, class Src>
__device__ __forceinline__ void stage_rows(uint32_t dst, int nrows, int n0, int Np, Src &&src_of) {
    constexpr int EPP = 16 / sizeof(T), P = AW / EPP, R = A_THREADS / P;
    const int j = threadIdx.x % P;
    if (n0 + j * EPP >= Np) return;
    for (int q = threadIdx.x / P; q < nrows; q += R)
        cp_async16(dst + (uint32_t)(q * AW + j * EPP) * (uint32_t)sizeof(T), src_of(q) + n0 + j * EPP);
}

// Species rows of [s0, s0 + ns) to shared memory rows (s - s0) nn + slot,
// without a division per row: the thread's rows advance by R slots.
template <class T>
__device__ __forceinline__ void stage_species(uint32_t dst, const T *tab, const unsigned short *node_of, int s0,
                                              int ns, int nn, int nodes, int n0, int Np) {
    constexpr int EPP = 16 / sizeof(T), P = AW / EPP, R = A_THREADS / P;
    const int j = threadIdx.x % P, q0 = threadIdx.x / P;
    if (n0 + j * EPP >= Np || q0 >= ns * nn) return;
    int s = s0 + q0 / nn, slot = q0 % nn;
    for (int q = q0; q < ns * nn; q += R) {
        cp_async16(dst + (uint32_t)(q * AW + j * EPP) * (uint32_t)sizeof(T),
                   tab + ((size_t)s * nodes + node_of[slot]) * Np + n0 + j * EPP);
        slot += R;
        while (slot >= nn) {
            slot -= nn;
            ++s;
        }
    }
}

template <bool BF16, int CH>
__global__ void __launch_bounds__(A_THREADS, 3) k_trans_alpha(Model m, Work w) {
    using E = TabElem<BF16>;
    using T = typename E::T;
    extern __shared__ float4 smem4[];
    unsigned char *const smem = reinterpret_cast<unsigned char *>(smem4);
    AlphaSmem &sa = *reinterpret_cast<AlphaSmem *>(smem);
    const int b = blockIdx.y, n0 = blockIdx.x * AW;
    const int kind = w.kind[b];   // checked after the first barrier (its latency overlaps the set-up)
    const int L = m.L, S = m.S, NT = m.NT, NP = m.NP, NTc = m.NTc, Np = m.Np;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *const dst0 = w.ext + (size_t)b * L * Np;
    if (n0 >= m.N) {   // a window of padding columns only (the grid covers Np): zero extinction
        if (kind != ES_KIND_TRANSMISSION) return;
        const int wn = min(AW, Np - n0);
        for (int i = tid; i < L * wn; i += A_THREADS) dst0[(size_t)(i / wn) * Np + n0 + i % wn] = 0.f;
        return;
    }
    const int nodes = NT * NP;
    // node marks / slots, CIA marks / slots, slot -> node, CIA slot -> node, staging
    unsigned short *slot_of = reinterpret_cast<unsigned short *>(smem + sizeof(AlphaSmem));
    unsigned short *cslot = slot_of + nodes;
    unsigned short *node_of = cslot + NTc;
    unsigned short *cnode_of = node_of + nodes;
    const uint32_t fixed = (uint32_t)((sizeof(AlphaSmem) + 2 * (size_t)(2 * nodes + 2 * NTc) + 15) & ~(size_t)15);
    const uint32_t stage = smem_u32(smem) + fixed;
    const uint32_t stage_bytes = (A_SMEM - fixed) & ~15u;

    // 1. the sample's inputs, every load issued before any store (read-only
    // path: written by the set-up kernel before this launch); FP32 log of
    // X_s, off the FP64 unit
    const float ry = (float)(1.0 / ((double)m.ray_nu_ref * m.ray_nu_ref * m.ray_nu_ref * m.ray_nu_ref));
    const int l = tid;   // one layer per thread (L <= 112 < A_THREADS)
    const size_t bl = (size_t)b * L + l;
    int it = 0, ip = 0, itc = 0;
    float wp = 0.f, wt = 0.f, wtc = 0.f, nsc = 0.f, ray = 0.f, cc0 = 0.f, cc1 = 0.f;
    if (l < L) {
        it = __ldg(w.it + bl);
        ip = __ldg(m.ip + l);
        itc = __ldg(w.itc + bl);
        wp = __ldg(m.wp + l);
        wt = __ldg(w.wtr + bl);
        wtc = __ldg(w.wtc + bl);
        nsc = (float)__ldg(w.n_lay + bl) * 5.421010862427522e-20f;   // n 2^-64
        ray = __ldg(w.ray + bl) * ry;
        cc0 = __ldg(w.ccia + 2 * bl);
        cc1 = __ldg(w.ccia + 2 * bl + 1);
    }
    float lxs = -1.0e4f;   // absent species: a weight that makes their terms zero
    if (tid < S) {
        const float x = (float)__ldg(w.xs + (size_t)b * (S + 2) + tid);
        if (x > 0.f) lxs = log2f(x) + KSHIFT;
    }
    for (int i = tid; i < nodes; i += A_THREADS) slot_of[i] = 0;
    for (int i = tid; i < NTc; i += A_THREADS) cslot[i] = 0;
    if (tid < ES_MAX_SPECIES) sa.lx[tid] = lxs;
    __syncthreads();
    if (kind != ES_KIND_TRANSMISSION) return;
    // the layer constants (corners as nodes for now), and the marks of the
    // nodes they bracket
    if (l < L) {
        it = min(max(it, 0), NT - 2);
        ip = min(max(ip, 0), NP - 2);
        itc = min(max(itc, 0), NTc - 2);
        const int n00 = it * NP + ip, n10 = (it + 1) * NP + ip;
        ALayer &la = sa.lay[l];
        la.wpt = make_float4(wp, wp, wt, wt);
        la.ko = make_int4(n00, n00, n10, itc);
        la.wn = make_float4(wtc, wtc, nsc, nsc);
        la.rc = make_float4(ray, ray, cc0, cc0);
        la.c1 = make_float4(cc1, cc1, 0.f, 0.f);
        slot_of[n00] = slot_of[n00 + 1] = slot_of[n10] = slot_of[n10 + 1] = 1;
        cslot[itc] = cslot[itc + 1] = 1;
    }
    __syncthreads();
    // run ends (the other warps), while warp 0 numbers the marked nodes and
    // CIA nodes (ballot scans in node order)
    if (warp != 0) {
        for (int q = tid - 32; q < L; q += A_THREADS - 32) {
            const int4 k = sa.lay[q].ko;
            int e = q + 1;
            while (e < L && sa.lay[e].ko.x == k.x && sa.lay[e].ko.w == k.w) ++e;
            sa.rend[q] = e;
        }
    } else {
        int run = 0;
        for (int base = 0; base < nodes; base += 32) {
            const int i = base + lane;
            const bool mk = i < nodes && slot_of[i];
            const unsigned bal = __ballot_sync(0xffffffffu, mk);
            if (mk) {
                const int q = run + __popc(bal & ((1u << lane) - 1u));
                slot_of[i] = (unsigned short)q;
                node_of[q] = (unsigned short)i;
            }
            run += __popc(bal);
        }
        int nc = 0;
        for (int base = 0; base < NTc; base += 32) {
            const int i = base + lane;
            const bool mk = i < NTc && cslot[i];
            const unsigned bal = __ballot_sync(0xffffffffu, mk);
            if (mk) {
                const int q = nc + __popc(bal & ((1u << lane) - 1u));
                cslot[i] = (unsigned short)q;
                cnode_of[q] = (unsigned short)i;
            }
            nc += __popc(bal);
        }
        if (lane == 0) {
            sa.nnodes = run;
            sa.ncia = nc;
        }
    }
    __syncthreads();
    const int nn = sa.nnodes, ncia = sa.ncia;
    if (blockIdx.x == 0 && tid == 0 && w.arows) {
        w.arows[2 * b] = nn * S;
        w.arows[2 * b + 1] = 2 * ncia;
    }
    // staging plan: the CIA rows, then the species rows (and their BF16 row
    // offsets) in parts of `per` species: all parts in flight at once (each
    // its own commit group, interpolated as it lands), or in rounds when they
    // do not all fit; direct global reads when not one species fits
    constexpr uint32_t RB = AW * sizeof(T);
    const uint32_t cia_bytes = 2u * (uint32_t)ncia * AW * 4u;
    const uint32_t avail = cia_bytes < stage_bytes ? stage_bytes - cia_bytes : 0u;
    // bytes of a part of ns species: rows, then the BF16 row offsets rounded up
    // to 16 bytes (the next part's copies start 16-byte aligned)
    auto part_bytes = [&](int ns) {
        return (uint32_t)ns * nn * RB + (BF16 ? ((uint32_t)ns * nn * 4u + 15u) & ~15u : 0u);
    };
    const int parts = (S + 5) / 6;                        // <= 3
    const int per = (S + parts - 1) / parts;              // <= CH
    uint32_t need = 0;
    for (int s0 = 0; s0 < S; s0 += per) need += part_bytes(min(per, S - s0));
    const bool all = need <= avail;
    int rper = min(per, S);   // species per round when not all fit
    if (!all)
        while (rper > 0 && part_bytes(rper) > avail) --rper;
    const bool staged = all || rper > 0;
    if (staged)
        for (int q = tid; q < L; q += A_THREADS) {
            int4 &ko = sa.lay[q].ko;
            ko.y = slot_of[ko.y];
            ko.z = slot_of[ko.z];
            ko.w = cslot[ko.w];
        }

    // the warp's layer group and the lane's wavenumber pair
    const int n = n0 + 2 * lane;
    const int LG = (L + AG - 1) / AG, l0 = min(L, warp * LG), l1 = min(L, l0 + LG);
    const float2 nu = *reinterpret_cast<const float2 *>(m.nu + n);
    const float2 nu2 = mul2(nu, nu), nu4 = mul2(nu2, nu2);
    float *const dst = dst0 + n;
    const T *tab = BF16 ? reinterpret_cast<const T *>(m.tab16) : reinterpret_cast<const T *>(m.tab32);
    if (!staged) {
        __syncthreads();
        // (the rare fallback: two species per round keeps its registers low)
        for (int s0 = 0; s0 < S; s0 += 2) {
            const int ns = min(2, S - s0);
            Rows<BF16, false> r{tab + (size_t)s0 * nodes * Np + n, m.row_off + (size_t)s0 * nodes, m.cia + n,
                                (size_t)nodes * Np, (size_t)NTc * Np, nodes, Np};
            part_sums<BF16, false, 2>(sa, r, s0, ns, l0, l1, s0 == 0, s0 + 2 >= S, nu4, dst, Np);
        }
    } else {
        // 2. the rows into shared memory; 3.-4. the interpolation as each part lands
        const uint32_t sp = stage + cia_bytes;
        stage_rows<float>(stage, 2 * ncia, n0, Np,
                          [&](int q) { return m.cia + ((size_t)(q / ncia) * NTc + cnode_of[q % ncia]) * Np; });
        // rows and BF16 offsets of species [s0, s0 + ns) at shared address `at`
        auto stage_part = [&](int s0, int ns, uint32_t at) {
            stage_species<T>(at, tab, node_of, s0, ns, nn, nodes, n0, Np);
            cp_async_commit();
            if (BF16) {
                float *ro = reinterpret_cast<float *>(smem + (at - smem_u32(smem)) + (size_t)ns * nn * RB);
                for (int q = tid; q < ns * nn; q += A_THREADS)
                    ro[q] = m.row_off[(size_t)(s0 + q / nn) * nodes + node_of[q % nn]];
            }
        };
        // the part's rows at this lane's column
        auto rows_at = [&](uint32_t at, int ns) {
            return Rows<BF16, true>{at + 2u * lane * (uint32_t)sizeof(T), at + (uint32_t)ns * nn * RB,
                                    stage + 8u * lane, nn, ncia};
        };
        if (all) {
            // every part in flight; part k is interpolated once its group has landed
            // (parts before part k: k full parts of `per` species)
            for (int k = 0, s0 = 0; k < parts; ++k, s0 += per)
                stage_part(s0, min(per, S - s0), sp + (uint32_t)k * part_bytes(per));
            for (int k = 0, s0 = 0; k < parts; ++k, s0 += per) {
                const int left = parts - 1 - k;   // groups that may still be in flight
                if (left >= 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
                else if (left == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
                else cp_async_wait_all();
                __syncthreads();
                const int ns = min(per, S - s0);
                part_sums<BF16, true, CH>(sa, rows_at(sp + (uint32_t)k * part_bytes(per), ns), s0, ns, l0, l1, k == 0,
                                          k + 1 == parts, nu4, dst, Np);
            }
        } else {
            for (int s0 = 0; s0 < S; s0 += rper) {   // rounds: stage, interpolate, release
                const int ns = min(rper, S - s0);
                stage_part(s0, ns, sp);
                cp_async_wait_all();
                __syncthreads();
                part_sums<BF16, true, CH>(sa, rows_at(sp, ns), s0, ns, l0, l1, s0 == 0, s0 + rper >= S, nu4, dst,
                                          Np);
                __syncthreads();
            }
        }
    }
    // the tail window: zero extinction at wavenumbers beyond N
    if (n + 1 >= m.N)
        for (int l = l0; l < l1; ++l) {
            float2 *o = reinterpret_cast<float2 *>(dst + (size_t)l * Np);
            float2 a = *o;
            if (n >= m.N) a.x = 0.f;
            a.y = 0.f;
            *o = a;
        }
}

template <bool BF, int CH>
int launch_alpha(const Model &m, const Work &w, cudaStream_t st, const Hook &h) {
    cudaFuncSetAttribute(k_trans_alpha<BF, CH>, cudaFuncAttributeMaxDynamicSharedMemorySize, A_SMEM);
    cudaFuncSetAttribute(k_trans_alpha<BF, CH>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    dim3 grid((m.Np + AW - 1) / AW, w.B);   // every column of the [L][Np] buffer is written
    ES_LAUNCH(h, "k_trans_alpha", st, k_trans_alpha<BF, CH><<<grid, A_THREADS, A_SMEM, st>>>(m, w));
    return 1;
}

}  // namespace

int launch_trans_alpha(const Model &m, const Work &w, cudaStream_t st, const Hook &h) {
    // species per part held in registers: S in 1, 2 or 3 parts of at most 6
    // (only a last, shorter part carries zero slots)
    const int parts = (m.S + 5) / 6;
    const int ch = (m.S + parts - 1) / parts;
#define ES_ALPHA_CH(BF)                                          \
    switch (ch) {                                                \
        case 1: return launch_alpha<BF, 1>(m, w, st, h);         \
        case 2: return launch_alpha<BF, 2>(m, w, st, h);         \
        case 3: return launch_alpha<BF, 3>(m, w, st, h);         \
        case 4: return launch_alpha<BF, 4>(m, w, st, h);         \
        case 5: return launch_alpha<BF, 5>(m, w, st, h);         \
        default: return launch_alpha<BF, 6>(m, w, st, h);        \
    }
    if (m.bf16) ES_ALPHA_CH(true)
    ES_ALPHA_CH(false)
#undef ES_ALPHA_CH
}

}  // namespace es
