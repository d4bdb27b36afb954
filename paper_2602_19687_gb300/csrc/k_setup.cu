// Per-sample setup (FP64): parameter unpack, T-p profile (Sect. 2.4), VMR
// fill (Sect. 3.1), hydrostatic altitude grid, path-length matrix
// (Sect. 4, Eq. P_1D times dr), annulus areas with the grey deck, and the
// per-layer interpolation coefficients used by the extinction kernels.
// Also the adjoint of all of that (reverse sweep over the geometry, then
// forward-mode tangents of the profile/hydrostatics, one lane per parameter).
#include "physics.cuh"

namespace es {

namespace {

constexpr int SETUP_THREADS = 128;

__global__ void __launch_bounds__(SETUP_THREADS) k_setup(Model m, Work w) {
    const int b = blockIdx.x, tid = threadIdx.x;
    const int L = m.L, S = m.S;
    __shared__ double th[ES_MAX_PARAMS];
    __shared__ double xs[ES_MAX_SPECIES + 2];
    __shared__ double tl[ES_MAX_LAYERS], tv[ES_MAX_LAYERS + 1], rl[ES_MAX_LAYERS + 1];
    __shared__ double s_mu, s_g, s_rref, s_rc;
    __shared__ int s_bad;

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
        s_rref = th[S + ES_P_R_P] * R_JUP;
        if (!(sum < 1.0)) s_bad = 1;
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
        double rp = th[S + ES_P_R_P] * R_JUP;
        w.scale[b] = bad ? 0.0 : th[S + ES_P_DILUTION] * rp * rp / rs2;
    }
    if (tid < S + 2) w.xs[(size_t)b * (S + 2) + tid] = xs[tid];
    for (int k = tid; k <= L; k += blockDim.x) {
        w.t_lev[(size_t)b * (L + 1) + k] = bad ? 1000.0 : tv[k];
        w.r_lev[(size_t)b * (L + 1) + k] = rl[k];
    }
    // path-length matrix L_il (row: impact parameter of layer i, column: layer l)
    for (int idx = tid; idx < L * L; idx += blockDim.x) {
        int i = idx / L, l = idx % L;
        double v = 0.0;
        if (!bad && l <= i) {
            double bi = 0.5 * (rl[i] + rl[i + 1]);
            double ru = rl[l], rd = rl[l + 1];
            if (ru > bi) {
                double su = sqrt((ru - bi) * (ru + bi));
                v = (rd < bi) ? 2.0 * su : 2.0 * (su - sqrt((rd - bi) * (rd + bi)));
            }
        }
        w.lmat[(size_t)b * L * L + idx] = (float)v;
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
__global__ void __launch_bounds__(SETUP_THREADS) k_setup_bwd(Model m, Work w) {
    const int b = blockIdx.x, tid = threadIdx.x;
    const int L = m.L, S = m.S;
    __shared__ double rl[ES_MAX_LAYERS + 1], rbar[ES_MAX_LAYERS + 1], tvbar[ES_MAX_LAYERS + 1];
    __shared__ double tlbar[ES_MAX_LAYERS];
    __shared__ double xbar[ES_MAX_SPECIES + 2], xs[ES_MAX_SPECIES + 2];
    __shared__ double rcbar;
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
    if (tid == 0) rcbar = 0.0;
    __syncthreads();
    const double rc = w.rc[b];
    if (!bad && !emis) {
        // path lengths: L_ii = 2 sqrt(r_i^2 - b_i^2); L_il (l < i) =
        // 2 [sqrt(r_l^2 - b_i^2) - sqrt(r_{l+1}^2 - b_i^2)], b_i = (r_i + r_{i+1})/2.
        // Two contention-free passes over the lower triangle: per row i the
        // impact-parameter terms (to r_i, r_{i+1}), per column l the terms of
        // the layer's own radii (to r_l, r_{l+1}); one shared atomic per sum.
        const double *lbar = w.lbar + (size_t)b * L * L;
        for (int i = tid; i < L; i += blockDim.x) {
            const double bi = 0.5 * (rl[i] + rl[i + 1]);
            double dsum = 0.0;
            for (int l = 0; l <= i; ++l) {
                const double lb = lbar[(size_t)i * L + l];
                if (lb == 0.0) continue;
                const double su = sqrt((rl[l] - bi) * (rl[l] + bi));
                if (l < i) {
                    const double sd = sqrt((rl[l + 1] - bi) * (rl[l + 1] + bi));
                    dsum += lb * 2.0 * bi * (1.0 / sd - 1.0 / su);
                } else {
                    dsum -= lb * 2.0 * bi / su;
                }
            }
            atomicAdd(&rbar[i], 0.5 * dsum);
            atomicAdd(&rbar[i + 1], 0.5 * dsum);
        }
        for (int l = tid; l < L; l += blockDim.x) {
            double up = 0.0, dn = 0.0;
            for (int i = l; i < L; ++i) {
                const double lb = lbar[(size_t)i * L + l];
                if (lb == 0.0) continue;
                const double bi = 0.5 * (rl[i] + rl[i + 1]);
                up += lb * 2.0 * rl[l] / sqrt((rl[l] - bi) * (rl[l] + bi));
                if (l < i) dn += lb * 2.0 * rl[l + 1] / sqrt((rl[l + 1] - bi) * (rl[l + 1] + bi));
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
    for (int l = tid; l < L; l += blockDim.x) {
        const double *rd = w.red + ((size_t)b * L + l) * N_RED;
        double n = w.n_lay[(size_t)b * L + l], t = w.t_lay[(size_t)b * L + l];
        const double qsum = rd[0] + rd[1];
        double dd = rd[2] + rd[3], c1 = rd[4], c2 = rd[5], c1t = rd[6], c2t = rd[7], w4 = rd[8];
        if (!emis && !bad) {   // W4_l = sum_nu alpha_bar_l w = sum_i L_il z_i
            const float *lm = w.lmat + (size_t)b * L * L + l;
            const double *z = w.zbar + (size_t)b * L;
            for (int i = 0; i < L; ++i) w4 += (double)lm[(size_t)i * L] * z[i];
        }
        double nbar = 0.0, tb = 0.0;
        if (!bad) {
            nbar = (qsum + 2.0 * (c1 + c2)) / n + (xs[S] * m.ray_h2 + xs[S + 1] * m.ray_he) * w4;
            tb = dd / t + LN10 * (c1t + c2t) - nbar * n / t;
            atomicAdd(&xbar[S], (2.0 * c1 + c2) / xs[S] + n * m.ray_h2 * w4);
            atomicAdd(&xbar[S + 1], c2 / xs[S + 1] + n * m.ray_he * w4);
        }
        tlbar[l] = tb;
    }
    __syncthreads();
    // forward-mode tangents: lane p differentiates with respect to free slot p
    if (tid >= 32) return;
    const int p = tid;
    if (p >= m.nfree) return;
    double *gout = w.grad + (size_t)b * m.nfree;
    if (bad) { gout[p] = 0.0; return; }
    const int seed = m.free_idx[p];
    Dual th[ES_MAX_PARAMS];
    for (int k = 0; k < m.nfull; ++k) th[k] = Dual(w.theta[(size_t)b * m.nfull + k], k == seed ? 1.0 : 0.0);
    Dual x[ES_MAX_SPECIES], xh2, xhe, mu;
    vmr_fill<Dual>(m, th, x, xh2, xhe, mu);
    double acc = 0.0;
    for (int s = 0; s < S; ++s) acc += xbar[s] * x[s].d;
    acc += xbar[S] * xh2.d + xbar[S + 1] * xhe.d;
    Dual tl[ES_MAX_LAYERS];
    for (int l = 0; l < L; ++l) {
        tl[l] = temperature<Dual>(m, th, m.p_lay[l]);
        acc += tlbar[l] * tl[l].d;
    }
    if (emis)
        for (int k = 0; k <= L; ++k) acc += tvbar[k] * temperature<Dual>(m, th, m.p_lev[k]).d;
    Dual g = dexp10(th[S + ES_P_LOG_G]);
    Dual rref = th[S + ES_P_R_P] * R_JUP;
    Dual inv_r[ES_MAX_LAYERS + 1];
    hydrostatic<Dual>(m, tl, mu, g, rref, inv_r);
    Dual r[ES_MAX_LAYERS + 1];
    for (int k = 0; k <= L; ++k) {
        r[k] = 1.0 / inv_r[k];
        acc += rbar[k] * r[k].d;
    }
    if (!emis) {
        Dual rcd = (m.cloud_kind == ES_CLOUD_DECK) ? deck_radius<Dual>(m, r, th[S + ES_P_LOG_P_CLOUD]) : r[L];
        acc += rcbar * rcd.d;
    } else {
        Dual rp = th[S + ES_P_R_P] * R_JUP;
        Dual sc = th[S + ES_P_DILUTION] * rp * rp / rs2;
        acc += w.misc[(size_t)b * 4 + 1] * sc.d;
    }
    acc += w.misc[(size_t)b * 4 + 2] * th[S + ES_P_C_INFL].d;
    gout[p] = acc;
}

}  // namespace

int launch_setup(const Model &m, const Work &w, cudaStream_t st, const Hook &h) {
    ES_LAUNCH(h, "k_setup", st, k_setup<<<w.B, SETUP_THREADS, 0, st>>>(m, w));
    return 1;
}

int launch_setup_backward(const Model &m, const Work &w, cudaStream_t st, const Hook &h) {
    ES_LAUNCH(h, "k_setup_bwd", st, k_setup_bwd<<<w.B, SETUP_THREADS, 0, st>>>(m, w));
    return 1;
}

}  // namespace es
