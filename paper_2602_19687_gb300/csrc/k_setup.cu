// Per-sample setup: parameter unpack, T-p profile (Sect. 2.4), VMR fill
// (Sect. 3.1), hydrostatic altitude grid (FP64), path-length matrix
// (Sect. 4, Eq. P_1D times dr), annulus areas with the grey deck, and the
// per-layer interpolation coefficients used by the extinction kernels.
// Also the adjoint of all of that (reverse sweep over the geometry, then
// forward-mode tangents of the profile/hydrostatics, one lane per parameter).
//
// GB300 runs FP64 at a small fraction of its FP32 rate, so FP64 is kept for
// the profile, the hydrostatic integration and the sums, and the O(L^2)
// path-length work runs in FP32 on differences that are formed exactly:
// every radius r (and impact parameter b) is split as hi + lo with hi =
// fl32(r), so r_l - b_i = (hi_l - hi_b) + (lo_l - lo_b), the first difference
// exact (Sterbenz) and the second tiny. A chord segment is written without
// cancellation, sqrt(r_l^2 - b^2) - sqrt(r_{l+1}^2 - b^2) =
// (r_l - r_{l+1})(r_l + r_{l+1}) / (s_u + s_d).
#include "physics.cuh"

namespace es {

namespace {

constexpr int SETUP_THREADS = 128;

// Level radii and impact parameters as FP32 hi/lo pairs plus the per-layer
// thickness dr_l = r_l - r_{l+1} and sum r_l + r_{l+1} (all from FP64).
struct SplitRadii {
    float rh[ES_MAX_LAYERS + 1], rlo[ES_MAX_LAYERS + 1];
    float bh[ES_MAX_LAYERS], blo[ES_MAX_LAYERS];
    float dl[ES_MAX_LAYERS], sl[ES_MAX_LAYERS];
};

__device__ inline void split_radii(const double *rl, int L, SplitRadii &q) {
    for (int k = threadIdx.x; k <= L; k += blockDim.x) {
        const float h = (float)rl[k];
        q.rh[k] = h;
        q.rlo[k] = (float)(rl[k] - (double)h);
        if (k < L) {
            const double b = 0.5 * (rl[k] + rl[k + 1]);
            const float bh = (float)b;
            q.bh[k] = bh;
            q.blo[k] = (float)(b - (double)bh);
            q.dl[k] = (float)(rl[k] - rl[k + 1]);
            q.sl[k] = (float)(rl[k] + rl[k + 1]);
        }
    }
}

// r_k^2 - b_i^2 in FP32 from the exact difference r_k - b_i
__device__ __forceinline__ float chord_sq(const SplitRadii &q, int k, int i) {
    const float d = (q.rh[k] - q.bh[i]) + (q.rlo[k] - q.blo[i]);
    return d * (q.rh[k] + q.bh[i]);
}

__global__ void __launch_bounds__(SETUP_THREADS) k_setup(Model m, Work w) {
    const int b = blockIdx.x, tid = threadIdx.x;
    const int L = m.L, S = m.S;
    __shared__ double th[ES_MAX_PARAMS];
    __shared__ double xs[ES_MAX_SPECIES + 2];
    __shared__ double tl[ES_MAX_LAYERS], tv[ES_MAX_LAYERS + 1], rl[ES_MAX_LAYERS + 1];
    __shared__ double s_mu, s_g, s_rref, s_rc;
    __shared__ int s_bad;
    __shared__ SplitRadii q;

    if (tid < m.nfull) th[tid] = m.theta_fixed[tid];
    if (tid == 0) s_bad = 0;
    __syncthreads();
    if (tid < m.nfree) th[m.free_idx[tid]] = w.theta_user[(size_t)b * m.nfree + tid];
    __syncthreads();
    if (tid < m.nfull) w.theta[(size_t)b * m.nfull + tid] = th[tid];

    if (tid == 0) {
        double xh2, xhe, mu, sum = 0.0;
        vmr_fill<double>(m, th, xs, xh2, xhe, mu);
        for (int s = 0; s < S; ++s) sum += xs[s];
        xs[S] = xh2;
        xs[S + 1] = xhe;
        s_mu = mu;
        s_g = exp10(th[S + ES_P_LOG_G]);
        s_rref = reference_radius<double>(m, th, s_g);
        if (!(sum < 1.0) || !(s_rref > 0.0)) s_bad = 1;
    }
    for (int l = tid; l < L; l += blockDim.x) tl[l] = temperature<double>(m, th, m.p_lay[l]);
    for (int k = tid; k <= L; k += blockDim.x) tv[k] = temperature<double>(m, th, m.p_lev[k]);
    __syncthreads();
    for (int l = tid; l < L; l += blockDim.x)
        if (!(tl[l] > 0.0) || !isfinite(tl[l])) atomicOr(&s_bad, 1);
    for (int k = tid; k <= L; k += blockDim.x)
        if (!(tv[k] > 0.0) || !isfinite(tv[k])) atomicOr(&s_bad, 1);
    __syncthreads();
    if (tid == 0) {
        if (!s_bad) {
            double inv_r[ES_MAX_LAYERS + 1];
            hydrostatic<double>(m, tl, s_mu, s_g, s_rref, inv_r);
            for (int k = 0; k <= L; ++k) {
                if (!(inv_r[k] > 0.0)) s_bad = 1;
                rl[k] = 1.0 / inv_r[k];
            }
        }
        if (s_bad) {
            for (int k = 0; k <= L; ++k) rl[k] = s_rref;
        } else {
            s_rc = (m.cloud_kind == ES_CLOUD_DECK) ? deck_radius<double>(m, rl, th[S + ES_P_LOG_P_CLOUD])
                                                   : rl[L];
        }
    }
    __syncthreads();
    const bool bad = s_bad != 0;
    const double rs2 = m.r_star * m.r_star;
    if (tid == 0) {
        w.flags[b] = bad ? ES_FLAG_INVALID : 0;
        w.rc[b] = bad ? 0.0 : s_rc;
        w.base[b] = bad ? 0.0 : s_rc * s_rc / rs2;
        w.scale[b] = bad ? 0.0 : emission_scale<double>(m, th, s_rref);
    }
    if (tid < S + 2) w.xs[(size_t)b * (S + 2) + tid] = xs[tid];
    for (int k = tid; k <= L; k += blockDim.x) {
        w.t_lev[(size_t)b * (L + 1) + k] = bad ? 1000.0 : tv[k];
        w.r_lev[(size_t)b * (L + 1) + k] = rl[k];
    }
    // path-length matrix L_il (row: impact parameter of layer i, column: layer l);
    // b_i lies inside layer i, so only the diagonal chord starts at b_i
    split_radii(rl, L, q);
    __syncthreads();
    for (int idx = tid; idx < L * L; idx += blockDim.x) {
        const int i = idx / L, l = idx % L;
        float v = 0.f;
        if (!bad && l <= i) {
            const float su = sqrtf(chord_sq(q, l, i));
            if (l == i) {
                v = 2.f * su;
            } else {
                const float sd = sqrtf(chord_sq(q, l + 1, i));
                v = 2.f * q.dl[l] * q.sl[l] / (su + sd);
            }
        }
        w.lmat[(size_t)b * L * L + idx] = v;
    }
    if (m.cloud_kind == ES_CLOUD_KH18) {
        // Sect. 2.5: C_l = 3 rho_a q_c^eff(p_l) / (4 r_eff) with the model's
        // q_c profile, and D_i = sum_l L_il C_l (the cloud's chord depth per
        // unit g(nu)); the block's lmat rows are read back after the barrier
        const double r_eff = exp10(th[S + ES_P_LOG_R_EFF]) * 1.0e-4;
        for (int l = tid; l < L; l += blockDim.x) {
            const double p = m.p_lay[l];
            double q = 0.0;   // stays 0 outside the cloud
            cloud_mmr<double>(m, th, th, p, q);
            const double rho = s_mu * AMU * p / (K_B * tl[l]);
            w.cloud_c[(size_t)b * L + l] = bad ? 0.f : (float)(3.0 * rho * q / (4.0 * r_eff));
        }
        __syncthreads();
        const float *cl = w.cloud_c + (size_t)b * L;
        for (int i = tid; i < L; i += blockDim.x) {
            const float *li = w.lmat + (size_t)b * L * L + (size_t)i * L;
            double d = 0.0;
            for (int l = 0; l <= i; ++l) d += (double)li[l] * (double)cl[l];
            w.cloud_d[(size_t)b * L + i] = (float)d;
        }
        if (tid == 0) {
            float *cg = w.cloud_g + (size_t)b * N_CG;
            cg[0] = (float)(2.0 * PI * r_eff);
            cg[1] = (float)th[S + ES_P_A_KH];
            cg[2] = (float)exp10(th[S + ES_P_LOG_Q0]);
            cg[3] = (float)th[S + ES_P_F_CLD];
            // mid-infrared feature (A = 0 switches it off in the kernels)
            cg[4] = m.cloud_feature ? (float)th[S + ES_P_FEAT_A] : 0.f;
            cg[5] = (float)th[S + ES_P_FEAT_LAM0];
            cg[6] = (float)th[S + ES_P_FEAT_W];
            cg[7] = (float)th[S + ES_P_FEAT_XI];
        }
    }
    for (int l = tid; l < L; l += blockDim.x) {
        const size_t bl = (size_t)b * L + l;
        double ru = rl[l], rd = rl[l + 1];
        double area = 0.0;
        if (!bad && ru > s_rc) {
            double inner = (rd >= s_rc) ? rd : s_rc;
            area = (ru - inner) * (ru + inner) / rs2;
        }
        w.area[bl] = (float)area;
        w.dr[bl] = bad ? 0.f : (float)(ru - rd);
        double t = tl[l];
        w.t_lay[bl] = t;
        // opacity-table bracket in log10 T (the pressure bracket is fixed per layer)
        int it;
        double wt;
        bool clamped;
        bracket(m.log_t, m.NT, log10(t), it, wt, clamped);
        w.it[bl] = it;
        w.wtr[bl] = (float)wt;
        w.gt[bl] = clamped ? 0.f : (float)(1.0 / (m.log_t[it + 1] - m.log_t[it]));
        double n = m.p_lay[l] / (K_B * t);
        w.n_lay[bl] = bad ? 0.0 : n;
        int itc;
        double wtc;
        bool cl2;
        bracket(m.cia_t, m.NTc, t, itc, wtc, cl2);
        w.itc[bl] = itc;
        w.wtc[bl] = (float)wtc;
        w.gtc[bl] = cl2 ? 0.f : (float)(1.0 / (m.cia_t[itc + 1] - m.cia_t[itc]));
        w.ccia[bl * 2 + 0] = bad ? -1000.f : (float)log2(n * n * xs[S] * xs[S]);
        w.ccia[bl * 2 + 1] = bad ? -1000.f : (float)log2(n * n * xs[S] * xs[S + 1]);
        w.ray[bl] = bad ? 0.f : (float)(n * (xs[S] * m.ray_h2 + xs[S + 1] * m.ray_he));
    }
}

// ---------------------------------------------------------------------------
// adjoint of the setup
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(SETUP_THREADS) k_setup_bwd(Model m, Work w, double *lnl_out) {
    const int b = blockIdx.x, tid = threadIdx.x;
    // an adjoint kernel that gave up on a bounded wait left its sums
    // unfinished: zero gradient, ln L = -1e300 and the timeout flag for every sample
    if (*w.err != 0) {
        if (tid < m.nfree) w.grad[(size_t)b * m.nfree + tid] = 0.0;
        if (tid == 0) {
            w.flags[b] |= ES_FLAG_INVALID | ES_FLAG_TIMEOUT;
            if (lnl_out) lnl_out[b] = INVALID_LNL;
        }
        return;
    }
    const int L = m.L, S = m.S;
    __shared__ double rl[ES_MAX_LAYERS + 1], rbar[ES_MAX_LAYERS + 1], tvbar[ES_MAX_LAYERS + 1];
    __shared__ double tlbar[ES_MAX_LAYERS];
    __shared__ double xbar[ES_MAX_SPECIES + 2], xs[ES_MAX_SPECIES + 2];
    __shared__ double thv[ES_MAX_PARAMS];
    __shared__ double rcbar;
    __shared__ float tlf[ES_MAX_LAYERS], zf[ES_MAX_LAYERS];
    // non-grey cloud: d lnL / d D_i, C_l and d lnL / d C_l (transmission:
    // sum_i L_il Dbar_i; emission: written directly by the emission adjoint)
    __shared__ float cdb[ES_MAX_LAYERS], ccl[ES_MAX_LAYERS];
    __shared__ double cbar[ES_MAX_LAYERS];
    // temperature tangents dT/dtheta_p at layers and (emission) levels
    __shared__ float dtl[ES_MAX_PARAMS][ES_MAX_LAYERS], dtv[ES_MAX_PARAMS][ES_MAX_LAYERS + 1];
    __shared__ SplitRadii q;
    const bool bad = w.flags[b] != 0;
    const bool emis = w.kind[b] == ES_KIND_EMISSION;
    const double rs2 = m.r_star * m.r_star;
    for (int k = tid; k <= L; k += blockDim.x) {
        rl[k] = w.r_lev[(size_t)b * (L + 1) + k];
        rbar[k] = 0.0;
        tvbar[k] = emis ? w.levbar[(size_t)b * (L + 1) + k] : 0.0;
    }
    if (tid < S + 2) {
        xbar[tid] = 0.0;
        xs[tid] = w.xs[(size_t)b * (S + 2) + tid];
    }
    if (tid < m.nfull) thv[tid] = w.theta[(size_t)b * m.nfull + tid];
    for (int l = tid; l < L; l += blockDim.x) tlf[l] = (float)w.t_lay[(size_t)b * L + l];
    if (tid == 0) rcbar = 0.0;
    const bool cloud_any = m.cloud_kind == ES_CLOUD_KH18;
    const bool cloudy = cloud_any && !emis;   // the chord depths D_i of transmission
    for (int l = tid; l < L; l += blockDim.x) {
        cdb[l] = cloudy ? (float)w.cloud_dbar[(size_t)b * L + l] : 0.f;
        ccl[l] = cloudy ? w.cloud_c[(size_t)b * L + l] : 0.f;
        if (cloud_any && emis) cbar[l] = bad ? 0.0 : w.cloud_dbar[(size_t)b * L + l];
    }
    __syncthreads();
    split_radii(rl, L, q);
    if (cloudy && !bad) {   // D_i = sum_l L_il C_l: Cbar_l = sum_i L_il Dbar_i
        for (int l = tid; l < L; l += blockDim.x) {
            double a = 0.0;
            for (int i = l; i < L; ++i) a += (double)w.lmat[((size_t)b * L + i) * L + l] * (double)cdb[i];
            cbar[l] = a;
        }
    }
    __syncthreads();
    const double rc = w.rc[b];
    if (!bad && !emis) {
        // path lengths: L_ii = 2 s(i, i); L_il (l < i) = 2 [s(l, i) - s(l+1, i)],
        // s(k, i) = sqrt(r_k^2 - b_i^2), b_i = (r_i + r_{i+1})/2.
        // Two contention-free passes over the lower triangle: per row i the
        // impact-parameter terms (to r_i, r_{i+1}), per column l the terms of
        // the layer's own radii (to r_l, r_{l+1}); one shared atomic per sum.
        // Terms in FP32 (1/s_d - 1/s_u without cancellation), sums in FP64.
        const float *lbar = w.lbar + (size_t)b * L * L;
        for (int i = tid; i < L; i += blockDim.x) {
            const float bi = q.bh[i];
            double dsum = 0.0;
            for (int l = 0; l <= i; ++l) {
                const float lb = lbar[(size_t)i * L + l] + cdb[i] * ccl[l];   // + the cloud's D_i = sum L_il C_l
                if (lb == 0.f) continue;
                const float u = chord_sq(q, l, i), ru = rsqrtf(u);
                float t;
                if (l < i) {
                    const float d = chord_sq(q, l + 1, i), rd = rsqrtf(d);
                    // 1/s_d - 1/s_u = (r_l^2 - r_{l+1}^2) / (s_u s_d (s_u + s_d))
                    t = 2.f * bi * (q.dl[l] * q.sl[l]) * ru * rd / (u * ru + d * rd);
                } else {
                    t = -2.f * bi * ru;
                }
                dsum += (double)(lb * t);
            }
            atomicAdd(&rbar[i], 0.5 * dsum);
            atomicAdd(&rbar[i + 1], 0.5 * dsum);
        }
        for (int l = tid; l < L; l += blockDim.x) {
            double up = 0.0, dn = 0.0;
            const float r0 = 2.f * q.rh[l], r1 = 2.f * q.rh[l + 1];
            for (int i = l; i < L; ++i) {
                const float lb = lbar[(size_t)i * L + l] + cdb[i] * ccl[l];
                if (lb == 0.f) continue;
                up += (double)(lb * r0 * rsqrtf(chord_sq(q, l, i)));
                if (l < i) dn += (double)(lb * r1 * rsqrtf(chord_sq(q, l + 1, i)));
            }
            atomicAdd(&rbar[l], up);
            atomicAdd(&rbar[l + 1], -dn);
        }
        // annulus areas A_i = (r_i^2 - max(r_{i+1}, r_c)^2)/R_*^2 and base r_c^2/R_*^2
        for (int i = tid; i < L; i += blockDim.x) {
            double ab = w.areabar[(size_t)b * L + i];
            if (rl[i] > rc) {
                atomicAdd(&rbar[i], ab * 2.0 * rl[i] / rs2);
                if (rl[i + 1] >= rc) atomicAdd(&rbar[i + 1], -ab * 2.0 * rl[i + 1] / rs2);
                else atomicAdd(&rcbar, -ab * 2.0 * rc / rs2);
            }
        }
        if (tid == 0) atomicAdd(&rcbar, w.misc[(size_t)b * 4 + 0] * 2.0 * rc / rs2);
    }
    if (!bad && emis) {
        for (int l = tid; l < L; l += blockDim.x) {
            double d = w.drbar[(size_t)b * L + l];
            atomicAdd(&rbar[l], d);
            atomicAdd(&rbar[l + 1], -d);
        }
    }
    // extinction reductions -> layer temperature and VMR adjoints
    if (!bad && tid < S) atomicAdd(&xbar[tid], w.qtot[(size_t)b * S + tid] / xs[tid]);
    if (!emis && !bad)
        for (int i = tid; i < L; i += blockDim.x) zf[i] = (float)w.zbar[(size_t)b * L + i];
    __syncthreads();
    double xh = 0.0, xe = 0.0;   // this thread's part of xbar[S], xbar[S + 1]
    for (int l = tid; l < L; l += blockDim.x) {
        const double *rd = w.red + ((size_t)b * L + l) * N_RED;
        double n = w.n_lay[(size_t)b * L + l], t = w.t_lay[(size_t)b * L + l];
        const double qsum = rd[0] + rd[1];
        double dd = rd[2] + rd[3], c1 = rd[4], c2 = rd[5], c1t = rd[6], c2t = rd[7], w4 = rd[8];
        if (!emis && !bad) {   // W4_l = sum_nu alpha_bar_l w = sum_i L_il z_i (FP32 products)
            const float *lm = w.lmat + (size_t)b * L * L + l;
            float a = 0.f;
            for (int i = l; i < L; ++i) a = fmaf(lm[(size_t)i * L], zf[i], a);
            w4 += (double)a;
        }
        double nbar = 0.0, tb = 0.0;
        if (!bad) {
            nbar = (qsum + 2.0 * (c1 + c2)) / n + (xs[S] * m.ray_h2 + xs[S + 1] * m.ray_he) * w4;
            tb = dd / t + LN10 * (c1t + c2t) - nbar * n / t;
            xh += (2.0 * c1 + c2) / xs[S] + n * m.ray_h2 * w4;
            xe += c2 / xs[S + 1] + n * m.ray_he * w4;
        }
        tlbar[l] = tb;
    }
    for (int o = 16; o > 0; o >>= 1) {
        xh += __shfl_xor_sync(0xffffffffu, xh, o);
        xe += __shfl_xor_sync(0xffffffffu, xe, o);
    }
    if ((tid & 31) == 0) {
        atomicAdd(&xbar[S], xh);
        atomicAdd(&xbar[S + 1], xe);
    }
    // forward-mode tangents in FP32 (values from the forward's FP64 results).
    // Temperature tangents, parallel over (parameter, layer or level): only
    // the profile parameters (slots up to log g, and T_ratio) reach T.
    const int npts = emis ? 2 * L + 1 : L;
    if (!bad) {
        for (int idx = tid; idx < m.nfree * npts; idx += blockDim.x) {
            const int p = idx / npts, k = idx % npts;
            const int seed = m.free_idx[p];
            float dt = 0.f;
            if (seed >= S && (seed - S <= ES_P_LOG_G || seed - S == ES_P_T_RATIO)) {
                DualF th[ES_MAX_PARAMS];
                for (int j = 0; j < m.nfull; ++j) th[j] = DualF((float)thv[j], j == seed ? 1.f : 0.f);
                dt = temperature<DualF>(m, th, k < L ? m.p_lay[k] : m.p_lev[k - L]).d;
            }
            if (k < L) dtl[p][k] = dt;
            else dtv[p][k - L] = dt;
        }
    }
    __syncthreads();
    // then one lane per free parameter: VMRs, hydrostatics, deck, star scale
    if (tid >= 32) return;
    const int p = tid;
    if (p >= m.nfree) return;
    double *gout = w.grad + (size_t)b * m.nfree;
    if (bad) { gout[p] = 0.0; return; }
    const int seed = m.free_idx[p];
    DualF th[ES_MAX_PARAMS];
    for (int k = 0; k < m.nfull; ++k) th[k] = DualF((float)thv[k], k == seed ? 1.f : 0.f);
    DualF x[ES_MAX_SPECIES], xh2, xhe, mu;
    vmr_fill<DualF>(m, th, x, xh2, xhe, mu);
    double acc = 0.0;
    for (int s = 0; s < S; ++s) acc += xbar[s] * (double)x[s].d;
    acc += xbar[S] * (double)xh2.d + xbar[S + 1] * (double)xhe.d;
    DualF tl[ES_MAX_LAYERS];
    for (int l = 0; l < L; ++l) {
        tl[l] = DualF(tlf[l], dtl[p][l]);
        acc += tlbar[l] * (double)dtl[p][l];
    }
    if (emis)
        for (int k = 0; k <= L; ++k) acc += tvbar[k] * (double)dtv[p][k];
    DualF g = dexp10(th[S + ES_P_LOG_G]);
    DualF rref = reference_radius<DualF>(m, th, g);
    DualF inv_r[ES_MAX_LAYERS + 1];
    hydrostatic<DualF>(m, tl, mu, g, rref, inv_r);
    for (int k = 0; k <= L; ++k) {
        const DualF r = 1.0 / inv_r[k];
        inv_r[k].d = r.d;   // keep dr_k for the deck
        acc += rbar[k] * (double)r.d;
    }
    if (!emis) {
        // deck radius r_c = r_k + f (r_{k+1} - r_k), f linear in ln p_c; the
        // radius difference from the FP64 levels
        float drc;
        const double p_c = exp10(thv[S + ES_P_LOG_P_CLOUD]) * BAR;
        const int k = deck_bracket(m, p_c);
        if (k == -1) {
            drc = inv_r[L].d;
        } else if (k == -2) {
            drc = inv_r[0].d;
        } else {
            const double l0 = m.lnp_lev[k], l1 = m.lnp_lev[k + 1];
            const double f = (thv[S + ES_P_LOG_P_CLOUD] * LN10 + log(BAR) - l0) / (l1 - l0);
            const double df = LN10 * (double)th[S + ES_P_LOG_P_CLOUD].d / (l1 - l0);
            drc = (float)((double)inv_r[k].d + f * (double)(inv_r[k + 1].d - inv_r[k].d) + df * (rl[k + 1] - rl[k]));
        }
        acc += rcbar * (double)drc;
    } else {
        DualF sc = emission_scale<DualF>(m, th, rref);
        acc += w.misc[(size_t)b * 4 + 1] * (double)sc.d;
    }
    if (cloud_any) {
        // C_l = 3 rho_a q_c^eff(p_l) / (4 r_eff), rho_a = mu m_u p / (k_B T_l); the
        // profile's branches are taken on the FP64 values, as in the forward
        const DualF r_eff = dexp10(th[S + ES_P_LOG_R_EFF]) * 1.0e-4;
        for (int l = 0; l < L; ++l) {
            const double pl = m.p_lay[l];
            DualF qc;
            if (cbar[l] == 0.0 || !cloud_mmr<DualF>(m, th, thv, pl, qc)) continue;
            const DualF rho = mu * (AMU * pl / K_B) / tl[l];
            const DualF c = 3.0 * rho * qc / (4.0 * r_eff);
            acc += cbar[l] * (double)c.d;
        }
        // g(nu): the kernel's sums over wavenumber of dbar-weighted dg/d(ln r_eff, a, ln Q0); f_cld;
        // the mid-infrared feature's A, lambda_0, omega, xi
        const double *cp = w.cloud_pbar + (size_t)b * N_CG;
        acc += cp[0] * LN10 * (double)th[S + ES_P_LOG_R_EFF].d + cp[1] * (double)th[S + ES_P_A_KH].d +
               cp[2] * LN10 * (double)th[S + ES_P_LOG_Q0].d + cp[3] * (double)th[S + ES_P_F_CLD].d;
        if (m.cloud_feature)
            acc += cp[4] * (double)th[S + ES_P_FEAT_A].d + cp[5] * (double)th[S + ES_P_FEAT_LAM0].d +
                   cp[6] * (double)th[S + ES_P_FEAT_W].d + cp[7] * (double)th[S + ES_P_FEAT_XI].d;
    }
    acc += w.misc[(size_t)b * 4 + 2] * (double)th[S + ES_P_C_INFL].d;
    gout[p] = acc;
}

}  // namespace

int launch_setup(const Model &m, const Work &w, cudaStream_t st, const Hook &h) {
    ES_LAUNCH(h, "k_setup", st, k_setup<<<w.B, SETUP_THREADS, 0, st>>>(m, w));
    return 1;
}

int launch_setup_backward(const Model &m, const Work &w, double *lnl_out, cudaStream_t st, const Hook &h) {
    ES_LAUNCH(h, "k_setup_bwd", st, k_setup_bwd<<<w.B, SETUP_THREADS, 0, st>>>(m, w, lnl_out));
    return 1;
}

}  // namespace es
