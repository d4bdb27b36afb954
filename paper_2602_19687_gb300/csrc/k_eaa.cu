// Emission with scattering: the delta-M scaled extended absorption
// approximation, linear in optical depth (Sect. 5; ES_RT_DELTA_EAA). The paper
// names the scheme without its formulas; the library's reading, per layer l
// with absorption depth A = alpha_gas dr (gas and CIA), Rayleigh depth R and
// cloud depth C, and per flux angle mu_j:
//   scattering  s = R + w_c C,  asymmetry g = w_c g_c C / s,  f = g^2,
//   delta-M     dtau' = A + (1 - w_c) C + (1 - f) s,  w' = (1 - f) s / dtau',
//               g' = g / (1 + g),
//   zeroth order (absorption approximation): linear-in-tau RT without
//               scattering on the depth A + (1 - w_c) C = (1 - w') dtau', down
//               from the top (nothing incident: D = 0) and up from the bottom
//               (U = B of the bottom level), per angle at every level,
//   moments     J = 1/2 sum_j c_j (U_j + D_j),  H = 1/2 sum_j a_j (U_j - D_j)
//               (a_j the flux weights, c_j the angles' interpolatory weights
//               of int_0^1 dmu),
//   first order one upward pass on dtau' with the level sources
//               S_j = (1 - w') B + w' (J + 3 g' mu_j H) of the layer, linear in
//               tau between its two levels: V_j; F = 2 pi sum_j a_j V_j(top).
// A layer of optical path x = dtau / mu entered with I_in, with a source
// linear from S_entry to S_exit, is left with
//   I_in E + S_exit (1 - E) + (S_entry - S_exit) f(x),  E = e^-x,  f = (1 - E)/x - E.
//
// Kernels (the extinction of the batch's emission samples stays in w.ext,
// [B][L][Np]):
//   k_eaa_ext     alpha_gas of every (sample, layer, wavenumber), interpolated
//                 by the fused kernels' lane pairs (no Rayleigh: it scatters);
//   k_eaa_rt      one thread per (sample, wavenumber) column: the zeroth-order
//                 upward pass (its moments to a scratch array), then the
//                 zeroth-order downward pass with the first order summed
//                 top-down;
//   k_eaa_rt_bwd  the adjoint of k_eaa_rt (three passes per column), which
//                 overwrites w.ext with d lnL / d alpha_gas and sums the other
//                 adjoints per layer (dr, the levels' T, the Rayleigh weight,
//                 the cloud's C_l and g(nu) constants);
//   k_eaa_abar    the interpolation adjoint of alpha_gas (the fused emission
//                 adjoint's per-layer and per-species reductions, fed by the
//                 stored alpha_bar).
// The scratch array holds, per resident thread and level, the values one pass
// leaves for the next (3 floats in the forward, 9 in the adjoint), laid out
// [level][value][thread] so that a warp's accesses are contiguous.
#include <algorithm>

#include "fused_emis.cuh"

namespace es {

namespace {

constexpr int EA_THREADS = 128;     // one column per thread
constexpr int EA_BLOCKS_PER_SM = 4; // resident RT blocks per SM (the scratch array's size follows)
constexpr int EA_BWD_BLOCKS_PER_SM = 3;   // the adjoint's (164 registers, no spills): at 4 it spills, at 2 it is slower
constexpr int EA_SUB = 8;           // 128-wavenumber sub-chunks per RT work item
constexpr int EA_FIELDS = 9;        // scratch values per level and thread (adjoint)

int sm_count_a() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// ---------------------------------------------------------------- k_eaa_ext
// alpha_gas [cm^-1] = n 2^-K sum_s 2^e_s + CIA_H2H2 + CIA_H2He of the staged
// emission sample, for 512-wavenumber tiles [t0, t1): each warp its 32
// wavenumbers of every tile, a lane pair per wavenumber pair (species split
// between the two lanes, combined by one shuffle).
template <int SPL>
__device__ __forceinline__ void ext_tiles(const Model &m, const Work &w, const SampleConst &sc, int b, int t0,
                                          int t1) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane & 1, L = m.L;
    for (int t = t0; t < t1; ++t) {
        const int nw = t * ET + 32 * warp;
        if (nw >= m.Np) continue;
        const int n = nw + 2 * (lane >> 1);
        PairInterp<SPL> pi;
        pi.init(m, n, half, lane);
        float *out = w.ext + (size_t)b * L * m.Np + n + half;
        for (int l = 0; l < L;) {
            // broadcast from lane 0: provably warp-uniform for the compiler
            const int end = __shfl_sync(0xffffffffu, sc.lay[l].run_end, 0);
            pi.load(sc, sc.lay[l].cell, sc.lay[l].itc);
            if (end < L) pi.prefetch(sc.lay[end].cell, sc.lay[end].itc);
            for (; l < end; ++l) {
                const LayerConst &lc = sc.lay[l];
                float2 tt, sum = ex2x2(pi.expo(0, lc.wp, lc.wt, tt));
#pragma unroll
                for (int j = 1; j < SPL; ++j) sum = add2(sum, ex2x2(pi.expo(j, lc.wp, lc.wt, tt)));
                const float2 mine = fma2(sum, lc.nsc, pi.cia(lc));
                out[(size_t)l * m.Np] = own(add2(mine, shfl_xor2(mine, 1)), half);
            }
        }
    }
}

struct ExtSmem {
    SampleConst sc;
};

template <int SPL>
__global__ void __launch_bounds__(EM_THREADS, 1) k_eaa_ext(Model m, Work w, int chunk_tiles) {
    extern __shared__ float4 smem4[];
    ExtSmem &sm = *reinterpret_cast<ExtSmem *>(smem4);
    const int ntiles = (m.Np + ET - 1) / ET;
    const ItemOrder order{w.B, (ntiles + chunk_tiles - 1) / chunk_tiles, 1};
    int cur_b = -1;
    for (long long item = blockIdx.x; item < order.total(); item += gridDim.x) {
        int c, b;
        order.at(item, c, b);
        if (w.kind[b] != ES_KIND_EMISSION) continue;
        if (b != cur_b) {
            __syncthreads();
            stage_sample(m, w, b, sm.sc, RUN_COST_FWD);
            cur_b = b;
            __syncthreads();
        }
        ext_tiles<SPL>(m, w, sm.sc, b, c * chunk_tiles, min(ntiles, (c + 1) * chunk_tiles));
    }
}

// ---------------------------------------------------------------- RT helpers
// Per-sample constants of the RT kernels.
struct EaaSample {
    float inv_t[ES_MAX_LAYERS + 1];   // 1 / T at the levels
    float dr[ES_MAX_LAYERS];          // layer thickness
    float ray[ES_MAX_LAYERS];         // n (X_H2 s_H2 + X_He s_He): alpha_ray = ray (nu / nu_ref)^4
    float ccl[ES_MAX_LAYERS];         // non-grey cloud: alpha_cloud = C_l g(nu)
    float cg[N_CG];                   // g(nu) constants (kh18_g), cg[3] = f_cld
};

template <bool CLOUD>
__device__ __forceinline__ void stage_eaa(const Model &m, const Work &w, int b, EaaSample &s) {
    const int L = m.L;
    for (int k = threadIdx.x; k <= L; k += blockDim.x) s.inv_t[k] = (float)(1.0 / w.t_lev[(size_t)b * (L + 1) + k]);
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        s.dr[l] = w.dr[(size_t)b * L + l];
        s.ray[l] = w.ray[(size_t)b * L + l];
        if (CLOUD) s.ccl[l] = w.cloud_c[(size_t)b * L + l];
    }
    if (CLOUD && threadIdx.x < N_CG) s.cg[threadIdx.x] = w.cloud_g[(size_t)b * N_CG + threadIdx.x];
}

// Angle constants in pairs (0, 1), (2, 3): mu, 1/mu, log2(e)/mu, 2 pi a_j
// (flux), a_j / 2 and c_j / 2 (moments), 3 mu.
struct EaaAngles {
    float2 mu[2], imu[2], c[2], wt[2], ha[2], hc[2], mu3[2];
    __device__ __forceinline__ explicit EaaAngles(const Model &m) {
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            float v[6][2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int j = 2 * p + q;
                const double mj = m.mu_gl[j], aj = m.w_gl[j] * mj;
                v[0][q] = (float)mj;
                v[1][q] = (float)(1.0 / mj);
                v[2][q] = (float)(1.4426950408889634 / mj);
                v[3][q] = (float)(2.0 * PI * aj);
                v[4][q] = (float)(0.5 * aj);
                v[5][q] = (float)(0.5 * m.c_mu[j]);
            }
            mu[p] = make_float2(v[0][0], v[0][1]);
            imu[p] = make_float2(v[1][0], v[1][1]);
            c[p] = make_float2(v[2][0], v[2][1]);
            wt[p] = make_float2(v[3][0], v[3][1]);
            ha[p] = make_float2(v[4][0], v[4][1]);
            hc[p] = make_float2(v[5][0], v[5][1]);
            mu3[p] = make_float2(3.f * v[0][0], 3.f * v[0][1]);
        }
    }
};

__device__ __forceinline__ float dot2(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }
__device__ __forceinline__ float dot4(const float2 (&a)[2], const float2 (&b)[2]) {
    return dot2(a[0], b[0]) + dot2(a[1], b[1]);
}

// E, 1 - E and f(x) of angle pair p for a layer of depth d (rd = 1/d).
__device__ __forceinline__ void layer_factors(const EaaAngles &ang, int p, float d, float rd, float2 &e,
                                              float2 &ome, float2 &f) {
    const float2 x = mul2(f2(d), ang.imu[p]);
    e = ex2x2(mul2(f2(-d), ang.c[p]));
    lin_factors(x, e, mul2(ang.mu[p], f2(rd)), ome, f);
}
// The same and f'(x).
__device__ __forceinline__ void layer_factors_fp(const EaaAngles &ang, int p, float d, float rd, float2 &e,
                                                 float2 &ome, float2 &f, float2 &fp) {
    const float2 x = mul2(f2(d), ang.imu[p]);
    e = ex2x2(mul2(f2(-d), ang.c[p]));
    const float2 ix = mul2(ang.mu[p], f2(rd));
    lin_factors(x, e, ix, ome, f);
    fp = lin_fp(x, e, fma2(e, f2(-1.f), f2(1.f)), ix);
}

// Reciprocal (MUFU, relative error ~2^-23); zero for a zero argument (where
// the callers' products are zero or discarded).
__device__ __forceinline__ float rcpa(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return x != 0.f ? y : 0.f;
}

// Layer optical properties of the reading above from its absorption,
// Rayleigh and cloud depths: the zeroth-order depth da = A + (1 - w_c) C, the
// scaled depth dp = dtau', w' and g'; sca, g, f and the reciprocals of da,
// dp, sca and 1 + g kept for the layer factors and the adjoint.
struct LayerOpt {
    float da, dp, om, gp, sca, g, f, rda, rdp, rsca, r1g;
};
__device__ __forceinline__ LayerOpt layer_opt(float A, float R, float C, float wc, float gcl) {
    LayerOpt o;
    o.sca = fmaf(wc, C, R);
    o.rsca = rcpa(o.sca);
    o.g = wc * gcl * C * o.rsca;
    o.f = o.g * o.g;
    o.da = fmaf(1.f - wc, C, A);
    o.rda = rcpa(o.da);
    const float ssc = (1.f - o.f) * o.sca;
    o.dp = o.da + ssc;
    o.rdp = rcpa(o.dp);
    o.om = ssc * o.rdp;
    o.r1g = rcpa(1.f + o.g);
    o.gp = o.g * o.r1g;
    return o;
}
// Adjoint of layer_opt: from the adjoints of (da, dp, w', g') those of A, R, C.
__device__ __forceinline__ void layer_opt_bwd(const LayerOpt &o, float wc, float gcl, float dab, float dpb,
                                              float omb, float gpb, float &Ab, float &Rb, float &Cb) {
    float sscb = omb * o.rdp;
    dpb -= sscb * o.om;
    dab += dpb;
    sscb += dpb;
    float gb = gpb * o.r1g * o.r1g;
    const float fb = -sscb * o.sca;
    float scab = sscb * (1.f - o.f);
    gb = fmaf(2.f * o.g, fb, gb);
    Cb = fmaf(gb, wc * gcl * o.rsca, (1.f - wc) * dab);
    scab -= gb * o.g * o.rsca;
    Ab = dab;
    Rb = scab;
    Cb = fmaf(wc, scab, Cb);
}

// Level sources of angle pair p: S = (1 - w') B + w' (J + 3 g' mu H).
__device__ __forceinline__ float2 level_source(const EaaAngles &ang, int p, const LayerOpt &o, float bv, float jv,
                                               float hv) {
    return fma2(f2(o.om * o.gp * hv), ang.mu3[p], f2(fmaf(1.f - o.om, bv, o.om * jv)));
}

// ---------------------------------------------------------------- k_eaa_rt
// Scratch address of value q at level k for this thread (nth resident threads).
struct Scratch {
    float *base;
    size_t nth;
    int nf;
    __device__ __forceinline__ float &at(int k, int q) const { return base[((size_t)k * nf + q) * nth]; }
};

__device__ __forceinline__ Scratch my_scratch(float *scr, int nf) {
    const size_t nth = (size_t)gridDim.x * EA_THREADS;
    return Scratch{scr + (size_t)blockIdx.x * EA_THREADS + threadIdx.x, nth, nf};
}

// Work items (sample b, chunk of EA_SUB x 128 wavenumbers), sample-major.
__device__ __forceinline__ int eaa_chunks(const Model &m) { return (m.Np + 128 * EA_SUB - 1) / (128 * EA_SUB); }

// Forward of one column (sample b, wavenumber n): writes the spectrum and,
// with STORE_I, the first-order top intensities per angle (the adjoint's
// input). Pass 1 runs the zeroth order upward and leaves per level its
// moments (1/2 sum c_j U_j, 1/2 sum a_j U_j) and B; pass 2 runs the zeroth
// order downward and sums the first order top-down, V(top) = sum_l T_l Src_l
// + T_L B_L, T_l = prod_{k<l} E'_k: the same operations in the same order as
// the prefix sums of the adjoint's pass 2, so that their difference (the part
// of V(top) from below a layer) carries no rounding of its own where it
// vanishes, deep in an optically thick column.
template <bool CLOUD, bool STORE_I>
__global__ void __launch_bounds__(EA_THREADS, EA_BLOCKS_PER_SM) k_eaa_rt(Model m, Work w, float *scr) {
    __shared__ EaaSample ss;
    const EaaAngles ang(m);
    const int L = m.L, Np = m.Np;
    const Scratch sc = my_scratch(scr, 3);
    const float wc = m.cloud_ssa, gcl = m.cloud_gasym;
    const float ry = (float)(1.0 / m.ray_nu_ref);
    const int nch = eaa_chunks(m);
    int cur_b = -1;
    for (long long item = blockIdx.x; item < (long long)w.B * nch; item += gridDim.x) {
        const int b = (int)(item / nch), ch = (int)(item % nch);
        if (w.kind[b] != ES_KIND_EMISSION) continue;
        if (b != cur_b) {
            __syncthreads();
            stage_eaa<CLOUD>(m, w, b, ss);
            cur_b = b;
            __syncthreads();
        }
        const float scale = (float)w.scale[b], fcl = CLOUD ? ss.cg[3] : 0.f;
        for (int sub = 0; sub < EA_SUB; ++sub) {
            const int n = (ch * EA_SUB + sub) * 128 + threadIdx.x;
            if (n >= Np) break;   // Np is a multiple of 128: the whole block leaves together
            const float nu = m.nu[n];
            Planck pl;
            pl.init(nu);
            const float nr = nu * ry, nr4 = (nr * nr) * (nr * nr);   // (nu / nu_ref)^4
            const float gnu = CLOUD ? kh18_g(ss.cg, nu) : 0.f;
            const float *ex = w.ext + (size_t)b * L * Np + n;
            float flux = 0.f;
            float4 vtop[2];
#pragma unroll 1
            for (int col = 0; col < (CLOUD ? 2 : 1); ++col) {
                const float cg = col ? gnu : 0.f;   // cloud depth C = C_l g(nu) dr in the cloudy column
                // pass 1: zeroth order upward, its moments and B to the scratch array
                // (the extinction of the layers two ahead already in flight)
                {
                    float bb = pl.value(ss.inv_t[L]);
                    float2 up[2] = {f2(bb), f2(bb)};
                    sc.at(L, 0) = dot4(ang.hc, up);
                    sc.at(L, 1) = dot4(ang.ha, up);
                    sc.at(L, 2) = bb;
                    float xa = ex[(size_t)(L - 1) * Np], xb = ex[(size_t)(L - 2) * Np];
                    for (int l = L - 1; l >= 0; --l) {
                        const float alpha = xa;
                        xa = xb;
                        if (l >= 2) xb = ex[(size_t)(l - 2) * Np];
                        const float dr = ss.dr[l];
                        const float C = CLOUD ? ss.ccl[l] * cg * dr : 0.f;
                        const float da = fmaf(1.f - wc, C, alpha * dr), rda = rcpa(da);
                        const float bt = pl.value(ss.inv_t[l]);
#pragma unroll
                        for (int p = 0; p < 2; ++p) {
                            float2 e, ome, f;
                            layer_factors(ang, p, da, rda, e, ome, f);
                            up[p] = fma2(up[p], e, fma2(f2(bt), ome, mul2(f2(bb - bt), f)));
                        }
                        sc.at(l, 0) = dot4(ang.hc, up);
                        sc.at(l, 1) = dot4(ang.ha, up);
                        sc.at(l, 2) = bt;
                        bb = bt;
                    }
                }
                // pass 2: zeroth order downward, first order summed top-down (the
                // next layer's extinction and level values loaded one layer ahead)
                float2 dn[2] = {f2(0.f), f2(0.f)}, tr[2] = {f2(1.f), f2(1.f)}, v[2] = {f2(0.f), f2(0.f)};
                float bt = sc.at(0, 2), jt = sc.at(0, 0), ht = sc.at(0, 1);
                float nx = ex[0], nj = sc.at(1, 0), nh = sc.at(1, 1), nb = sc.at(1, 2);
                for (int l = 0; l < L; ++l) {
                    const float alpha = nx, ju = nj, hu = nh, bb = nb;
                    if (l + 1 < L) {
                        nx = ex[(size_t)(l + 1) * Np];
                        nj = sc.at(l + 2, 0);
                        nh = sc.at(l + 2, 1);
                        nb = sc.at(l + 2, 2);
                    }
                    const float dr = ss.dr[l];
                    const float A = alpha * dr, R = ss.ray[l] * nr4 * dr;
                    const float C = CLOUD ? ss.ccl[l] * cg * dr : 0.f;
                    const LayerOpt o = layer_opt(A, R, C, wc, gcl);
                    const float rda = o.rda, rdp = o.rdp;
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        float2 e, ome, f;
                        layer_factors(ang, p, o.da, rda, e, ome, f);
                        dn[p] = fma2(dn[p], e, fma2(f2(bb), ome, mul2(f2(bt - bb), f)));
                    }
                    const float jb = ju + dot4(ang.hc, dn), hb = hu - dot4(ang.ha, dn);
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        float2 e, ome, f;
                        layer_factors(ang, p, o.dp, rdp, e, ome, f);
                        const float2 st = level_source(ang, p, o, bt, jt, ht), sb = level_source(ang, p, o, bb, jb, hb);
                        const float2 ds = add2(sb, mul2(st, f2(-1.f)));
                        v[p] = fma2(tr[p], fma2(st, ome, mul2(ds, f)), v[p]);
                        tr[p] = mul2(tr[p], e);
                    }
                    bt = bb;
                    jt = jb;
                    ht = hb;
                }
#pragma unroll
                for (int p = 0; p < 2; ++p) v[p] = fma2(tr[p], f2(bt), v[p]);   // the bottom boundary, V = B_L
                const float fl = dot4(ang.wt, v);
                flux = col ? fcl * fl + (1.f - fcl) * flux : fl;
                vtop[col] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
            }
            if (n < m.N) w.spec[(size_t)b * m.N + n] = scale * flux * m.inv_fstar[n];
            if (STORE_I) {   // [B][Np][column][4 angles], the cloudy column second
                float4 *it4 = reinterpret_cast<float4 *>(w.itop) + ((size_t)b * Np + n) * (CLOUD ? 2 : 1);
                it4[0] = vtop[0];
                if (CLOUD) it4[1] = vtop[1];
            }
        }
    }
}

// ---------------------------------------------------------------- k_eaa_rt_bwd
// The adjoint's per-block sums of its current work item.
struct EaaRed {
    float lay[3][ES_MAX_LAYERS];      // per layer: d lnL / d dr; sum_nu alpha_ray_bar (nu / nu_ref)^4; d lnL / d C_l
    float tlev[ES_MAX_LAYERS + 1];    // d lnL / d T of the levels
    float cpbar[N_CG];                // d lnL / d (ln r_eff via g, a, ln Q0, f_cld, A, lambda_0, omega, xi)
    float sbar;                       // d lnL / d (emission scale)
};

// Sums of four values over the warp: lane 8 q + r (r < 8) ends with the sum
// of v_q (two transpose stages, then a butterfly over the low three bits).
__device__ __forceinline__ float reduce4(float v0, float v1, float v2, float v3, int lane) {
    const bool u4 = lane & 16;
    const float a0 = (u4 ? v2 : v0) + __shfl_xor_sync(0xffffffffu, u4 ? v0 : v2, 16);
    const float a1 = (u4 ? v3 : v1) + __shfl_xor_sync(0xffffffffu, u4 ? v1 : v3, 16);
    const bool u3 = lane & 8;
    float c = (u3 ? a1 : a0) + __shfl_xor_sync(0xffffffffu, u3 ? a0 : a1, 8);
    c += __shfl_xor_sync(0xffffffffu, c, 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    return c;
}

__device__ __forceinline__ void store4(const Scratch &sc, int k, const float2 (&v)[2]) {
    sc.at(k, 0) = v[0].x;
    sc.at(k, 1) = v[0].y;
    sc.at(k, 2) = v[1].x;
    sc.at(k, 3) = v[1].y;
}
__device__ __forceinline__ void load4(const Scratch &sc, int k, float2 (&v)[2]) {
    v[0] = make_float2(sc.at(k, 0), sc.at(k, 1));
    v[1] = make_float2(sc.at(k, 2), sc.at(k, 3));
}

// Adjoint of one sample's columns. Per column (the cloudy one first, then the
// clear one), with the seed d lnL / d V_j(top) = 2 pi a_j d lnL / d F:
//   pass 1 (up)   the zeroth-order U_j and B at every level, to the scratch array;
//   pass 2 (down) the zeroth-order D_j again, the first order's adjoint in its
//                 telescoped form (V(top) = sum_l T_l Src_l + T_L B_L with
//                 T_l = prod_{k<l} E'_k, so the part of V(top) from below layer
//                 l is V(top) - sum_{k<=l} T_k Src_k and no intensity of the
//                 first order is stored), the adjoints of the level sources
//                 S_j into B, J, H, w', g', and the adjoint of the upward zeroth
//                 order (its recursion runs bottom-up, so its adjoint top-down
//                 with the stored U_j); leaves D_j, J_bar, H_bar and this pass's
//                 B_bar per level, and A_bar per layer;
//   pass 3 (up)   the adjoint of the downward zeroth order with the stored D_j,
//                 completing A_bar (alpha_gas_bar = A_bar dr into w.ext, summed
//                 over both columns), the levels' B_bar (-> T_bar) and the
//                 cloud's adjoints.
// Scratch values per level: 0-3 U_j then D_j, 4 J_bar, 5 H_bar, 6 B, 7 B_bar
// of pass 2, 8 A_bar of the layer below the level (pass 2's part; then the
// cloudy column's total, which the clear column's pass 2 adds to its own).
template <bool CLOUD>
__global__ void __launch_bounds__(EA_THREADS, EA_BWD_BLOCKS_PER_SM) k_eaa_rt_bwd(Model m, Work w, float *scr) {
    __shared__ EaaSample ss;
    __shared__ EaaRed rd;
    const EaaAngles ang(m);
    const int L = m.L, Np = m.Np, lane = threadIdx.x & 31;
    const Scratch sc = my_scratch(scr, EA_FIELDS);
    const float wc = m.cloud_ssa, gcl = m.cloud_gasym;
    const float ry = (float)(1.0 / m.ray_nu_ref);
    const int nch = eaa_chunks(m);
    int cur_b = -1;
    for (long long item = blockIdx.x; item < (long long)w.B * nch; item += gridDim.x) {
        const int b = (int)(item / nch), ch = (int)(item % nch);
        if (w.kind[b] != ES_KIND_EMISSION || w.flags[b]) continue;
        __syncthreads();
        if (b != cur_b) {
            stage_eaa<CLOUD>(m, w, b, ss);
            cur_b = b;
        }
        for (int l = threadIdx.x; l < L; l += EA_THREADS) rd.lay[0][l] = rd.lay[1][l] = rd.lay[2][l] = 0.f;
        for (int k = threadIdx.x; k <= L; k += EA_THREADS) rd.tlev[k] = 0.f;
        if (threadIdx.x < N_CG) rd.cpbar[threadIdx.x] = 0.f;
        if (threadIdx.x == 0) rd.sbar = 0.f;
        __syncthreads();
        const float scale = (float)w.scale[b], fcl = CLOUD ? ss.cg[3] : 0.f;
        for (int sub = 0; sub < EA_SUB; ++sub) {
            const int n = (ch * EA_SUB + sub) * 128 + threadIdx.x;
            if (n >= Np) break;   // Np is a multiple of 128: the whole block leaves together
            const float nu = m.nu[n];
            Planck pl;
            pl.init(nu);
            const float nr = nu * ry, nr4 = (nr * nr) * (nr * nr);
            const float gnu = CLOUD ? kh18_g(ss.cg, nu) : 0.f;
            const float db = w.dbar[(size_t)b * Np + n];   // zero beyond N
            const float fsc = m.inv_fstar[n], fbar = db * scale * fsc;
            float *ex = w.ext + (size_t)b * L * Np + n;
            const float4 *it4 = reinterpret_cast<const float4 *>(w.itop) + ((size_t)b * Np + n) * (CLOUD ? 2 : 1);
            float gacc = 0.f;   // d lnL / d g(nu)
#pragma unroll 1
            for (int col = CLOUD ? 1 : 0; col >= 0; --col) {
                const float cg = col ? gnu : 0.f;
                const float wcol = CLOUD ? (col ? fcl : 1.f - fcl) : 1.f;
                const float4 vt = it4[col];
                const float2 v0[2] = {make_float2(vt.x, vt.y), make_float2(vt.z, vt.w)};
                const float2 vb[2] = {mul2(f2(fbar * wcol), ang.wt[0]), mul2(f2(fbar * wcol), ang.wt[1])};
                // pass 1: upward zeroth order (the extinction two layers ahead in flight)
                {
                    float bb = pl.value(ss.inv_t[L]);
                    float2 up[2] = {f2(bb), f2(bb)};
                    store4(sc, L, up);
                    sc.at(L, 6) = bb;
                    float xa = ex[(size_t)(L - 1) * Np], xb = ex[(size_t)(L - 2) * Np];
                    for (int l = L - 1; l >= 0; --l) {
                        const float alpha = xa;
                        xa = xb;
                        if (l >= 2) xb = ex[(size_t)(l - 2) * Np];
                        const float dr = ss.dr[l];
                        const float C = CLOUD ? ss.ccl[l] * cg * dr : 0.f;
                        const float da = fmaf(1.f - wc, C, alpha * dr), rda = rcpa(da);
                        const float bt = pl.value(ss.inv_t[l]);
#pragma unroll
                        for (int p = 0; p < 2; ++p) {
                            float2 e, ome, f;
                            layer_factors(ang, p, da, rda, e, ome, f);
                            up[p] = fma2(up[p], e, fma2(f2(bt), ome, mul2(f2(bb - bt), f)));
                        }
                        store4(sc, l, up);
                        sc.at(l, 6) = bt;
                        bb = bt;
                    }
                }
                // pass 2: downward
                float2 dn[2] = {f2(0.f), f2(0.f)}, tr[2] = {f2(1.f), f2(1.f)}, pre[2] = {f2(0.f), f2(0.f)};
                float2 lu[2] = {f2(0.f), f2(0.f)};
                float bt = sc.at(0, 6);
                float jt, ht;
                {
                    float2 u0[2];
                    load4(sc, 0, u0);
                    jt = dot4(ang.hc, u0);
                    ht = dot4(ang.ha, u0);
                }
                float jbt = 0.f, hbt = 0.f, bbt = 0.f;   // adjoints of the top level's J, H, B from the layer above
                // the next layer's extinction and the level below it (U, B) loaded one layer ahead
                float nx = ex[0], nbv = sc.at(1, 6);
                float2 nu2[2];
                load4(sc, 1, nu2);
                for (int l = 0; l < L; ++l) {
                    const float alpha = nx, bb = nbv;
                    const float2 ub[2] = {nu2[0], nu2[1]};
                    if (l + 1 < L) {
                        nx = ex[(size_t)(l + 1) * Np];
                        nbv = sc.at(l + 2, 6);
                        load4(sc, l + 2, nu2);
                    }
                    const float dr = ss.dr[l];
                    const float A = alpha * dr, R = ss.ray[l] * nr4 * dr;
                    const float C = CLOUD ? ss.ccl[l] * cg * dr : 0.f;
                    const LayerOpt o = layer_opt(A, R, C, wc, gcl);
                    const float rda = o.rda, rdp = o.rdp;
                    float2 ea[2], omea[2], fa[2], fpa[2], dnb[2];
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        layer_factors_fp(ang, p, o.da, rda, ea[p], omea[p], fa[p], fpa[p]);
                        dnb[p] = fma2(dn[p], ea[p], fma2(f2(bb), omea[p], mul2(f2(bt - bb), fa[p])));
                    }
                    const float jb = dot4(ang.hc, ub) + dot4(ang.hc, dnb), hb = dot4(ang.ha, ub) - dot4(ang.ha, dnb);
                    // first order through layer l
                    float dpb = 0.f, s0t = 0.f, s1t = 0.f, s0b = 0.f, s1b = 0.f;
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        float2 e, ome, f, fp;
                        layer_factors_fp(ang, p, o.dp, rdp, e, ome, f, fp);
                        const float2 st = level_source(ang, p, o, bt, jt, ht), sb = level_source(ang, p, o, bb, jb, hb);
                        const float2 ds = add2(sb, mul2(st, f2(-1.f)));
                        pre[p] = fma2(tr[p], fma2(st, ome, mul2(ds, f)), pre[p]);
                        const float2 below = add2(v0[p], mul2(pre[p], f2(-1.f)));
                        const float2 g = mul2(ang.imu[p], fma2(tr[p], fma2(st, e, mul2(ds, fp)), mul2(below, f2(-1.f))));
                        dpb += dot2(vb[p], g);
                        const float2 it = mul2(vb[p], tr[p]);
                        const float2 sbt = mul2(it, add2(ome, mul2(f, f2(-1.f)))), sbb = mul2(it, f);
                        s0t += sbt.x + sbt.y;
                        s1t += dot2(sbt, ang.mu[p]);
                        s0b += sbb.x + sbb.y;
                        s1b += dot2(sbb, ang.mu[p]);
                        tr[p] = mul2(tr[p], e);
                    }
                    // the level sources' adjoints
                    bbt = fmaf(1.f - o.om, s0t, bbt);
                    float bbb = (1.f - o.om) * s0b;
                    const float omb = (jt - bt) * s0t + 3.f * o.gp * ht * s1t + (jb - bb) * s0b + 3.f * o.gp * hb * s1b;
                    const float gpb = 3.f * o.om * (ht * s1t + hb * s1b);
                    jbt = fmaf(o.om, s0t, jbt);
                    hbt = fmaf(3.f * o.om * o.gp, s1t, hbt);
                    const float jbb = o.om * s0b, hbb = 3.f * o.om * o.gp * s1b;
                    // level l is complete: the upward zeroth order's adjoint through layer l
                    float dab = 0.f;
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        lu[p] = fma2(ang.hc[p], f2(jbt), fma2(ang.ha[p], f2(hbt), lu[p]));
                        const float2 dx = fma2(add2(f2(bt), mul2(ub[p], f2(-1.f))), ea[p], mul2(f2(bb - bt), fpa[p]));
                        dab += dot2(lu[p], mul2(ang.imu[p], dx));
                        bbt += dot2(lu[p], add2(omea[p], mul2(fa[p], f2(-1.f))));
                        bbb += dot2(lu[p], fa[p]);
                        lu[p] = mul2(lu[p], ea[p]);
                    }
                    store4(sc, l, dn);
                    sc.at(l, 4) = jbt;
                    sc.at(l, 5) = hbt;
                    sc.at(l, 7) = bbt;
                    float Ab, Rb, Cb;
                    layer_opt_bwd(o, wc, gcl, dab, dpb, omb, gpb, Ab, Rb, Cb);
                    sc.at(l, 8) = (CLOUD && col == 0) ? Ab + sc.at(l, 8) : Ab;
                    // Rayleigh (R = ray (nu/nu_ref)^4 dr) and cloud (C = C_l g(nu) dr) depths
                    const float ar = ss.ray[l] * nr4;
                    float drb = Rb * ar, ccb = 0.f;
                    if (CLOUD && col) {
                        drb = fmaf(Cb, ss.ccl[l] * cg, drb);
                        ccb = Cb * cg * dr;
                        gacc = fmaf(Cb, ss.ccl[l] * dr, gacc);
                    }
                    const float r = reduce4(drb, Rb * dr * nr4, ccb, 0.f, lane);
                    if ((lane & 7) == 0 && lane < 24) atomicAdd(&rd.lay[lane >> 3][l], r);
#pragma unroll
                    for (int p = 0; p < 2; ++p) dn[p] = dnb[p];
                    bt = bb;
                    jt = jb;
                    ht = hb;
                    jbt = jbb;
                    hbt = hbb;
                    bbt = bbb;
                }
                // bottom level: the first order's and the zeroth order's boundary I = B_L
                bbt += dot4(vb, tr);
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    lu[p] = fma2(ang.hc[p], f2(jbt), fma2(ang.ha[p], f2(hbt), lu[p]));
                    bbt += lu[p].x + lu[p].y;
                }
                store4(sc, L, dn);
                sc.at(L, 4) = jbt;
                sc.at(L, 5) = hbt;
                sc.at(L, 7) = bbt;
                // pass 3: upward, the downward zeroth order's adjoint
                float2 ld[2];
                {
                    const float jl = sc.at(L, 4), hl = sc.at(L, 5);
#pragma unroll
                    for (int p = 0; p < 2; ++p) ld[p] = fma2(ang.hc[p], f2(jl), mul2(ang.ha[p], f2(-hl)));
                }
                float bb = sc.at(L, 6), bbs = 0.f;   // bbs: this pass's B_bar of level l+1 from layer l+1
                // the layer's extinction and its top level's D and B loaded one layer ahead
                float px = ex[(size_t)(L - 1) * Np], nbt = sc.at(L - 1, 6);
                float2 nd[2];
                load4(sc, L - 1, nd);
                for (int l = L - 1; l >= 0; --l) {
                    const float alpha = px, btl = nbt;
                    const float2 dl[2] = {nd[0], nd[1]};
                    if (l >= 1) {
                        px = ex[(size_t)(l - 1) * Np];
                        nbt = sc.at(l - 1, 6);
                        load4(sc, l - 1, nd);
                    }
                    const float dr = ss.dr[l];
                    const float C = CLOUD ? ss.ccl[l] * cg * dr : 0.f;
                    const float da = fmaf(1.f - wc, C, alpha * dr), rda = rcpa(da);
                    float2 ea[2];
                    float da3 = 0.f, bte = 0.f;
#pragma unroll
                    for (int p = 0; p < 2; ++p) {
                        float2 ome, f, fp;
                        layer_factors_fp(ang, p, da, rda, ea[p], ome, f, fp);
                        const float2 dx = fma2(add2(f2(bb), mul2(dl[p], f2(-1.f))), ea[p], mul2(f2(btl - bb), fp));
                        da3 += dot2(ld[p], mul2(ang.imu[p], dx));
                        bbs += dot2(ld[p], add2(ome, mul2(f, f2(-1.f))));
                        bte += dot2(ld[p], f);
                    }
                    // level l+1 is complete
                    float dbdt;
                    pl.value_dt(ss.inv_t[l + 1], dbdt);
                    const float tl = (sc.at(l + 1, 7) + bbs) * dbdt;
                    // layer l: A_bar complete
                    const float Ab = sc.at(l, 8) + da3;
                    float drb = 0.f, ccb = 0.f;
                    if (col == 0) {   // the last column: alpha_gas_bar of both columns
                        ex[(size_t)l * Np] = Ab * dr;
                        drb = Ab * alpha;
                    } else {
                        sc.at(l, 8) = Ab;
                    }
                    if (CLOUD && col) {
                        const float cb3 = (1.f - wc) * da3;
                        drb = fmaf(cb3, ss.ccl[l] * cg, drb);
                        ccb = cb3 * cg * dr;
                        gacc = fmaf(cb3, ss.ccl[l] * dr, gacc);
                    }
                    const float r = reduce4(drb, 0.f, ccb, tl, lane);
                    if ((lane & 7) == 0 && lane != 8) {
                        if (lane == 24) atomicAdd(&rd.tlev[l + 1], r);
                        else atomicAdd(&rd.lay[lane >> 3][l], r);
                    }
                    // lambda_D at level l
                    const float jl = sc.at(l, 4), hl = sc.at(l, 5);
#pragma unroll
                    for (int p = 0; p < 2; ++p)
                        ld[p] = fma2(ld[p], ea[p], fma2(ang.hc[p], f2(jl), mul2(ang.ha[p], f2(-hl))));
                    bb = btl;
                    bbs = bte;
                }
                {   // level 0
                    float dbdt;
                    pl.value_dt(ss.inv_t[0], dbdt);
                    const float t0 = warp_total((sc.at(0, 7) + bbs) * dbdt);
                    if (lane == 0) atomicAdd(&rd.tlev[0], t0);
                }
            }
            // the emission scale, the cloud fraction and the cloud's g(nu) constants
            const float4 c0 = it4[0];
            const float2 vc[2] = {make_float2(c0.x, c0.y), make_float2(c0.z, c0.w)};
            float flux = dot4(ang.wt, vc);
            if (CLOUD) {
                const float4 c1 = it4[1];
                const float2 vd[2] = {make_float2(c1.x, c1.y), make_float2(c1.z, c1.w)};
                const float fcd = dot4(ang.wt, vd);
                const float fb = warp_total(fbar * (fcd - flux));
                float o[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (gacc != 0.f) kh18_g_adjoint(ss.cg, nu, gacc, o);
                cloud_pbar_add(ss.cg, o, rd.cpbar, lane);
                if (lane == 0) atomicAdd(rd.cpbar + 3, fb);
                flux = fcl * fcd + (1.f - fcl) * flux;
            }
            const float sb = warp_total(db * flux * fsc);
            if (lane == 0) atomicAdd(&rd.sbar, sb);
        }
        // the item's sums into the workspace by FP64 atomics
        __syncthreads();
        for (int l = threadIdx.x; l < L; l += EA_THREADS) {
            const size_t bl = (size_t)b * L + l;
            if (rd.lay[0][l] != 0.f) atomicAdd(w.drbar + bl, (double)rd.lay[0][l]);
            if (rd.lay[1][l] != 0.f) atomicAdd(w.red + bl * N_RED + 8, (double)rd.lay[1][l]);
            if (CLOUD && rd.lay[2][l] != 0.f) atomicAdd(w.cloud_dbar + bl, (double)rd.lay[2][l]);
        }
        for (int k = threadIdx.x; k <= L; k += EA_THREADS)
            if (rd.tlev[k] != 0.f) atomicAdd(w.levbar + (size_t)b * (L + 1) + k, (double)rd.tlev[k]);
        if (CLOUD && threadIdx.x < N_CG && rd.cpbar[threadIdx.x] != 0.f)
            atomicAdd(w.cloud_pbar + (size_t)b * N_CG + threadIdx.x, (double)rd.cpbar[threadIdx.x]);
        if (threadIdx.x == 0 && rd.sbar != 0.f) atomicAdd(w.misc + (size_t)b * 4 + 1, (double)rd.sbar);
    }
}

// ---------------------------------------------------------------- k_eaa_abar
// The interpolation adjoint of alpha_gas: for 512-wavenumber tiles of an
// emission sample, the same per-layer sums as the fused emission adjoint (QS,
// D, C, CT with the lane-parity partials; summed over wavenumber by three
// transpose stages and a shared-memory atomic per lane) and per-species
// totals, with alpha_bar read from w.ext (both wavenumbers of a lane pair in
// one 8-byte load) instead of computed by the RT adjoint. The Rayleigh weight
// and dr come from k_eaa_rt_bwd.
struct AbarSmem {
    SampleConst sc;
    float red[ES_MAX_LAYERS * 32];
    float qtot[ES_MAX_SPECIES];
};

template <int SPL>
__global__ void __launch_bounds__(EM_THREADS, 1) k_eaa_abar(Model m, Work w, int chunk_tiles) {
    extern __shared__ float4 smem4[];
    AbarSmem &sm = *reinterpret_cast<AbarSmem *>(smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane & 1, L = m.L, S = m.S;
    // after three transpose stages every lane holds a distinct partial sum:
    // value 4 b4 + 2 b3 + b2, parity b0, partial b1
    const int rslot = 4 * (4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1)) + 2 * (lane & 1) +
                      ((lane >> 1) & 1);
    const int ridx = 4 * ((lane >> 4) & 1) + 2 * ((lane >> 3) & 1) + ((lane >> 2) & 1);
    const bool qwriter = (lane & 3) == 0;
    const int ntiles = (m.Np + ET - 1) / ET;
    const ItemOrder order{w.B, (ntiles + chunk_tiles - 1) / chunk_tiles, 1};
    auto flush = [&](int b) {
        __syncthreads();
        for (int l = threadIdx.x; l < L; l += EM_THREADS) {
            const float *q = sm.red + l * 32;
            const LayerConst &lc = sm.sc.lay[l];
            float r[8];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                r[0 + h] = q[0 + 2 * h] + q[1 + 2 * h];                 // QS
                r[2 + h] = (q[4 + 2 * h] + q[5 + 2 * h]) * lc.gts;      // D
                r[4 + h] = q[8 + 2 * h] + q[9 + 2 * h];                 // C
                r[6 + h] = (q[12 + 2 * h] + q[13 + 2 * h]) * lc.gtcs;   // CT
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (r[k] != 0.f) atomicAdd(w.red + ((size_t)b * L + l) * N_RED + k, (double)r[k]);
        }
        for (int s2 = threadIdx.x; s2 < S; s2 += EM_THREADS)
            if (sm.qtot[s2] != 0.f) atomicAdd(w.qtot + (size_t)b * S + s2, (double)sm.qtot[s2]);
    };
    int cur_b = -1;
    for (long long item = blockIdx.x; item < order.total(); item += gridDim.x) {
        int c, b;
        order.at(item, c, b);
        if (w.kind[b] != ES_KIND_EMISSION || w.flags[b]) continue;
        if (b != cur_b) {
            if (cur_b >= 0) flush(cur_b);
            __syncthreads();
            stage_sample(m, w, b, sm.sc, RUN_COST_BWD);
            for (int idx = threadIdx.x; idx < L * 32; idx += EM_THREADS) sm.red[idx] = 0.f;
            for (int s2 = threadIdx.x; s2 < ES_MAX_SPECIES; s2 += EM_THREADS) sm.qtot[s2] = 0.f;
            cur_b = b;
            __syncthreads();
        }
        const int t1 = min(ntiles, (c + 1) * chunk_tiles);
        for (int t = c * chunk_tiles; t < t1; ++t) {
            const int nw = t * ET + 32 * warp;
            if (nw >= m.Np) continue;
            const int n = nw + 2 * (lane >> 1);
            PairInterp<SPL> pi;
            pi.init(m, n, half, lane);
            const float2 *abp = reinterpret_cast<const float2 *>(w.ext + (size_t)b * L * m.Np + n);
            float2 qa[SPL];
#pragma unroll
            for (int j = 0; j < SPL; ++j) qa[j] = f2(0.f);
            float2 ab_next = abp[0];   // alpha_bar of the pair's two wavenumbers, one layer ahead
            for (int l = 0; l < L;) {
                const int end = __shfl_sync(0xffffffffu, sm.sc.lay[l].run_end, 0);
                pi.load(sm.sc, sm.sc.lay[l].cell, sm.sc.lay[l].itc);
                if (end < L) pi.prefetch(sm.sc.lay[end].cell, sm.sc.lay[end].itc);
                for (; l < end; ++l) {
                    const LayerConst &lc = sm.sc.lay[l];
                    const float2 ab = ab_next;
                    if (l + 1 < L) ab_next = abp[(size_t)(l + 1) * (m.Np / 2)];
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
                    const float2 abn = mul2(ab, lc.nsc);
#pragma unroll
                    for (int j = 0; j < SPL; ++j) qa[j] = fma2(abn, p[j], qa[j]);
                    const float2 ac = mul2(ab, cc);
                    const float2 act = mul2(ac, pi.d);
                    float vr[8];
                    vr[0] = dot2(abn, sum);
                    vr[1] = dot2(abn, pt);   // x gts at the flush
                    vr[2] = ac.x + ac.y;
                    vr[3] = act.x + act.y;   // x gtcs at the flush
                    vr[4] = vr[5] = vr[6] = vr[7] = 0.f;
                    const float part = reduce8_partial(vr, lane);
                    if (rslot < 16) atomicAdd(sm.red + l * 32 + rslot, part);
                }
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
                if (qwriter && c0 + ridx < S && tq != 0.f) atomicAdd(sm.qtot + c0 + ridx, tq);
            }
        }
    }
    if (cur_b >= 0) flush(cur_b);
}

// 512-wavenumber tiles per work item of k_eaa_ext / k_eaa_abar: up to 8,
// fewer when the batch is small so that every SM gets items.
int eaa_chunk(const Model &m, int B) {
    const int ntiles = (m.Np + ET - 1) / ET;
    long long c = ((long long)ntiles * B) / (4LL * sm_count_a());
    return (int)std::max<long long>(1, std::min<long long>(8, c));
}

int eaa_rt_grid(const Model &m, int B, int per_sm) {
    const long long items = (long long)B * ((m.Np + 128 * EA_SUB - 1) / (128 * EA_SUB));
    return (int)std::max<long long>(1, std::min<long long>(items, (long long)sm_count_a() * per_sm));
}

}  // namespace

size_t eaa_scratch_floats(const Model &m) {
    return (size_t)sm_count_a() * EA_BLOCKS_PER_SM * EA_THREADS * (size_t)(m.L + 1) * EA_FIELDS;
}

int launch_eaa_forward(const Model &m, const Work &w, float *scr, bool store_i, cudaStream_t st, const Hook &h) {
    const int ntiles = (m.Np + ET - 1) / ET;
    const int chunk = eaa_chunk(m, w.B);
    const long long items = (long long)w.B * ((ntiles + chunk - 1) / chunk);
    const int grid = (int)std::min<long long>(items, (long long)sm_count_a());
    const size_t sm = sizeof(ExtSmem);
    const int spl = spl_for(m.S);
    if (spl == 2) ES_LAUNCH(h, "k_eaa_ext", st, k_eaa_ext<2><<<grid, EM_THREADS, sm, st>>>(m, w, chunk));
    else if (spl == 4) ES_LAUNCH(h, "k_eaa_ext", st, k_eaa_ext<4><<<grid, EM_THREADS, sm, st>>>(m, w, chunk));
    else ES_LAUNCH(h, "k_eaa_ext", st, k_eaa_ext<8><<<grid, EM_THREADS, sm, st>>>(m, w, chunk));
    const int g2 = eaa_rt_grid(m, w.B, EA_BLOCKS_PER_SM);
#define ES_ER(CL, SI) ES_LAUNCH(h, "k_eaa_rt", st, k_eaa_rt<CL, SI><<<g2, EA_THREADS, 0, st>>>(m, w, scr))
    if (m.cloud_kind == ES_CLOUD_KH18) {
        if (store_i) ES_ER(true, true); else ES_ER(true, false);
    } else {
        if (store_i) ES_ER(false, true); else ES_ER(false, false);
    }
#undef ES_ER
    return 2;
}

int launch_eaa_backward(const Model &m, const Work &w, float *scr, cudaStream_t st, const Hook &h) {
    const int g2 = eaa_rt_grid(m, w.B, EA_BWD_BLOCKS_PER_SM);
    if (m.cloud_kind == ES_CLOUD_KH18)
        ES_LAUNCH(h, "k_eaa_rt_bwd", st, k_eaa_rt_bwd<true><<<g2, EA_THREADS, 0, st>>>(m, w, scr));
    else
        ES_LAUNCH(h, "k_eaa_rt_bwd", st, k_eaa_rt_bwd<false><<<g2, EA_THREADS, 0, st>>>(m, w, scr));
    const int ntiles = (m.Np + ET - 1) / ET;
    const int chunk = eaa_chunk(m, w.B);
    const long long items = (long long)w.B * ((ntiles + chunk - 1) / chunk);
    const int grid = (int)std::min<long long>(items, (long long)sm_count_a());
    const size_t sm = sizeof(AbarSmem);
    const int spl = spl_for(m.S);
    if (spl == 2) ES_LAUNCH(h, "k_eaa_abar", st, k_eaa_abar<2><<<grid, EM_THREADS, sm, st>>>(m, w, chunk));
    else if (spl == 4) ES_LAUNCH(h, "k_eaa_abar", st, k_eaa_abar<4><<<grid, EM_THREADS, sm, st>>>(m, w, chunk));
    else ES_LAUNCH(h, "k_eaa_abar", st, k_eaa_abar<8><<<grid, EM_THREADS, sm, st>>>(m, w, chunk));
    return 2;
}

}  // namespace es
