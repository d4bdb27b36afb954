// Per-sample atmosphere physics, templated on the scalar type so the same
// code gives values (double) and forward-mode tangents (Dual, DualF) for the
// adjoint.
#pragma once

#include "internal.cuh"

namespace es {

// Forward-mode dual number: value and one directional derivative.
struct Dual {
    double v, d;
    __host__ __device__ Dual() : v(0.0), d(0.0) {}
    __host__ __device__ Dual(double x) : v(x), d(0.0) {}
    __host__ __device__ Dual(double x, double dx) : v(x), d(dx) {}
};
__device__ inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__device__ inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__device__ inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
__device__ inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ inline Dual operator/(Dual a, Dual b) {
    double q = a.v / b.v;
    return Dual(q, (a.d - q * b.d) / b.v);
}
__device__ inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
__device__ inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
__device__ inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
__device__ inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
__device__ inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
__device__ inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
__device__ inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
__device__ inline Dual operator/(double a, Dual b) {
    double q = a / b.v;
    return Dual(q, -q * b.d / b.v);
}
__device__ inline Dual dexp(Dual a) { double e = exp(a.v); return Dual(e, e * a.d); }
__device__ inline Dual dlog(Dual a) { return Dual(log(a.v), a.d / a.v); }
__device__ inline Dual dsqrt(Dual a) { double s = sqrt(a.v); return Dual(s, 0.5 * a.d / s); }
__device__ inline Dual dpow(Dual a, double p) {
    double s = pow(a.v, p);
    return Dual(s, p * s / a.v * a.d);
}
__device__ inline Dual dexp10(Dual a) { double e = exp10(a.v); return Dual(e, e * LN10 * a.d); }
// Forward-mode dual number in FP32 for the adjoint's tangent sweeps: the
// tangents only need ~1e-6 relative accuracy (the gradient is checked to
// 1e-3), and GB300 runs FP32 at many times its FP64 rate.
struct DualF {
    float v, d;
    __host__ __device__ DualF() : v(0.f), d(0.f) {}
    __host__ __device__ DualF(double x) : v((float)x), d(0.f) {}
    __host__ __device__ DualF(float x, float dx) : v(x), d(dx) {}
};
__device__ inline DualF operator+(DualF a, DualF b) { return DualF(a.v + b.v, a.d + b.d); }
__device__ inline DualF operator-(DualF a, DualF b) { return DualF(a.v - b.v, a.d - b.d); }
__device__ inline DualF operator-(DualF a) { return DualF(-a.v, -a.d); }
__device__ inline DualF operator*(DualF a, DualF b) { return DualF(a.v * b.v, a.d * b.v + a.v * b.d); }
__device__ inline DualF operator/(DualF a, DualF b) {
    float q = a.v / b.v;
    return DualF(q, (a.d - q * b.d) / b.v);
}
__device__ inline DualF operator+(DualF a, double b) { return DualF(a.v + (float)b, a.d); }
__device__ inline DualF operator+(double a, DualF b) { return DualF((float)a + b.v, b.d); }
__device__ inline DualF operator-(DualF a, double b) { return DualF(a.v - (float)b, a.d); }
__device__ inline DualF operator-(double a, DualF b) { return DualF((float)a - b.v, -b.d); }
__device__ inline DualF operator*(DualF a, double b) { return DualF(a.v * (float)b, a.d * (float)b); }
__device__ inline DualF operator*(double a, DualF b) { return DualF((float)a * b.v, (float)a * b.d); }
__device__ inline DualF operator/(DualF a, double b) { return DualF(a.v / (float)b, a.d / (float)b); }
__device__ inline DualF operator/(double a, DualF b) {
    float q = (float)a / b.v;
    return DualF(q, -q * b.d / b.v);
}
__device__ inline DualF dexp(DualF a) { float e = expf(a.v); return DualF(e, e * a.d); }
__device__ inline DualF dlog(DualF a) { return DualF(logf(a.v), a.d / a.v); }
__device__ inline DualF dsqrt(DualF a) { float s = sqrtf(a.v); return DualF(s, 0.5f * a.d / s); }
__device__ inline DualF dpow(DualF a, double p) {
    float s = powf(a.v, (float)p);
    return DualF(s, (float)p * s / a.v * a.d);
}
__device__ inline DualF dexp10(DualF a) { float e = exp10f(a.v); return DualF(e, e * (float)LN10 * a.d); }
__device__ inline double val(DualF a) { return (double)a.v; }
__device__ inline double dexp(double a) { return exp(a); }
__device__ inline double dlog(double a) { return log(a); }
__device__ inline double dsqrt(double a) { return sqrt(a); }
__device__ inline double dpow(double a, double p) { return pow(a, p); }
__device__ inline double dexp10(double a) { return exp10(a); }
__device__ inline double val(double a) { return a; }
__device__ inline double val(Dual a) { return a.v; }

// Parameter access in the canonical layout (log-VMR slots first).
template <class R>
struct Params {
    const R *th;
    int S;
    __device__ R slot(int k) const { return th[S + k]; }
};

// Volume mixing ratios: X_s = 10^theta_s; Sect. 3.1 background fill.
template <class R>
__device__ void vmr_fill(const Model &m, const R *th, R *x, R &x_h2, R &x_he, R &mu) {
    R sum = R(0.0), mx = R(0.0);
    for (int s = 0; s < m.S; ++s) {
        x[s] = dexp10(th[s]);
        sum = sum + x[s];
        mx = mx + x[s] * m.mass[s];
    }
    x_h2 = (1.0 - sum) / (1.0 + HE_TO_H2);
    x_he = HE_TO_H2 * x_h2;
    mu = mx + x_h2 * M_H2 + x_he * M_HE;
}

// Temperature at pressure p [dyn cm^-2] for the model's profile
// (Sect. 2.4.1 isothermal; Sect. 2.4.4 modified Guillot, 4- or 7-parameter).
template <class R>
__device__ R temperature(const Model &m, const R *th, double p) {
    Params<R> P{th, m.S};
    if (m.tp_kind == ES_TP_ISOTHERMAL) return P.slot(ES_P_T_ISO);
    if (m.tp_kind == ES_TP_MILNE) {
        // Sect. 2.4.3: T^4 = 3/4 T_int^4 [tau + q(p)], tau = kappa_ir p / g,
        // q(p) = q_inf + (q0 - q_inf) exp[-(p/p_t)^beta], q0 = 4/3 T_ratio^4
        R g = dexp10(P.slot(ES_P_LOG_G));
        R kappa = dexp10(P.slot(ES_P_LOG_KAPPA_IR));
        R tint = P.slot(ES_P_T_INT), tr = P.slot(ES_P_T_RATIO);
        R tau = kappa * p / g;
        R tr2 = tr * tr;
        R q0 = (4.0 / 3.0) * (tr2 * tr2);
        R p_t = dexp10(P.slot(ES_P_LOG_P_T)) * BAR;
        R z = dexp(P.slot(ES_P_BETA) * dlog(p / p_t));   // (p/p_t)^beta
        R q = Q_MILNE_INF + (q0 - Q_MILNE_INF) * dexp(-z);
        R tint2 = tint * tint;
        return dsqrt(dsqrt(0.75 * (tint2 * tint2) * (tau + q)));
    }
    R g = dexp10(P.slot(ES_P_LOG_G));
    R kappa = dexp10(P.slot(ES_P_LOG_KAPPA_IR));
    R gamma = dexp10(P.slot(ES_P_LOG_GAMMA_V));
    R tint = P.slot(ES_P_T_INT), teq = P.slot(ES_P_T_EQ);
    R tau = kappa * p / g;
    R q_irr = R(Q_IRR_INF);
    if (m.tp_kind == ES_TP_GUILLOT_MOD) {
        R p_t = dexp10(P.slot(ES_P_LOG_P_T)) * BAR;
        R beta = P.slot(ES_P_BETA);
        R z = dexp(beta * dlog(p / p_t));         // (p/p_t)^beta
        q_irr = Q_IRR_INF + (P.slot(ES_P_Q_IRR0) - Q_IRR_INF) * dexp(-z);
    }
    const double s3 = 1.7320508075688772935;
    R tint2 = tint * tint, teq2 = teq * teq;
    R t4 = 0.75 * (tint2 * tint2) * (Q_INT + tau)
         + 0.75 * (teq2 * teq2) * (4.0 * F_HEM)
               * (q_irr + 1.0 / (gamma * s3) + (gamma / s3 - 1.0 / (gamma * s3)) * dexp(-(gamma * tau * s3)));
    return dsqrt(dsqrt(t4));
}

// Reference radius of the hydrostatic grid: R_p, or for a brown dwarf the
// radius from its mass and gravity, R_bd = sqrt(G M_bd / g) (Sect. 5).
template <class R>
__device__ R reference_radius(const Model &m, const R *th, R g) {
    if (m.emis_flux == ES_FLUX_BROWN_DWARF) return dsqrt((G_GRAV * M_JUP) * th[m.S + ES_P_M_BD] / g);
    return th[m.S + ES_P_R_P] * R_JUP;
}
// Emission output scale: s (R_p/R_*)^2 for Fp/F*, s (R_bd/D)^2 for a brown
// dwarf's flux at distance D (Sect. 5); the ratio is formed before squaring.
template <class R>
__device__ R emission_scale(const Model &m, const R *th, R r_ref) {
    R ratio = (m.emis_flux == ES_FLUX_BROWN_DWARF) ? r_ref / m.distance : r_ref / m.r_star;
    return th[m.S + ES_P_DILUTION] * ratio * ratio;
}

// Non-grey cloud: q_c^eff at pressure p (dyne cm^-2) for the model's profile
// (Sect. 2.5.1). Returns false where the profile is zero; whether p lies in
// the cloud is decided on the FP64 parameter values thv, so that the forward
// and its tangents take the same branch.
template <class R>
__device__ bool cloud_mmr(const Model &m, const R *th, const double *thv, double p, R &q) {
    const int S = m.S;
    if (m.cloud_profile == ES_QC_SLAB_BAND) {
        const double pt = exp10(thv[S + ES_P_LOG_PC_TOP]) * BAR, dp = exp10(thv[S + ES_P_LOG_DPC]) * BAR;
        if (!(p >= pt && p <= pt + dp)) return false;
    } else if (m.cloud_profile == ES_QC_POWER_LAW) {
        if (!(p <= exp10(thv[S + ES_P_LOG_PC_BASE]) * BAR)) return false;
    }
    q = dexp10(th[S + ES_P_LOG_QC]);
    if (m.cloud_profile == ES_QC_POWER_LAW)   // q_base (p / p_base)^alpha_c
        q = q * dexp(th[S + ES_P_ALPHA_C] * dlog(p / (dexp10(th[S + ES_P_LOG_PC_BASE]) * BAR)));
    return true;
}

// Index of the layer whose levels bracket p_ref (clamped to the grid).
__device__ inline int anchor_layer(const Model &m) {
    int j = 0;
    for (int k = 0; k <= m.L; ++k)
        if (m.p_lev[k] <= m.p_ref) j = k;
    return j < 0 ? 0 : (j > m.L - 1 ? m.L - 1 : j);
}

// Hydrostatic level radii with g = g_ref (R_ref/r)^2, isothermal layers:
// 1/r_{k} - 1/r_{k+1} = coef T_k ln(p_k / p_{k+1}), coef = k_B/(mu m_u g R^2),
// anchored at r(p_ref) = R_ref. Writes 1/r into inv_r[L+1]; t_lay[L] given.
template <class R>
__device__ void hydrostatic(const Model &m, const R *t_lay, R mu, R g, R r_ref, R *inv_r) {
    R coef = K_B / (mu * AMU * g * r_ref * r_ref);
    int j = anchor_layer(m);
    R inv_ref = 1.0 / r_ref;
    // ln(p_a / p_b) as differences of the levels' tabulated ln p
    inv_r[j] = inv_ref + coef * t_lay[j] * (m.lnp_lev[j] - m.ln_p_ref);
    inv_r[j + 1] = inv_ref + coef * t_lay[j] * (m.lnp_lev[j + 1] - m.ln_p_ref);
    for (int k = j - 1; k >= 0; --k)
        inv_r[k] = inv_r[k + 1] + coef * t_lay[k] * (m.lnp_lev[k] - m.lnp_lev[k + 1]);
    for (int k = j + 2; k <= m.L; ++k)
        inv_r[k] = inv_r[k - 1] + coef * t_lay[k - 1] * (m.lnp_lev[k] - m.lnp_lev[k - 1]);
}

// Deck level bracket: returns -1 (no deck / at or below the bottom: r_c = r_bot),
// -2 (at or above the top: r_c = r_top) or k with p_lev[k] <= p_c < p_lev[k+1].
__device__ inline int deck_bracket(const Model &m, double p_c) {
    if (m.cloud_kind != ES_CLOUD_DECK || p_c >= m.p_lev[m.L]) return -1;
    if (p_c <= m.p_lev[0]) return -2;
    int k = 0;
    for (int q = 0; q <= m.L; ++q)
        if (m.p_lev[q] <= p_c) k = q;
    return k;
}

// Deck radius by ln p interpolation between the bracketing levels.
template <class R>
__device__ R deck_radius(const Model &m, const R *r_lev, R log10_pc) {
    double p_c = exp10(val(log10_pc)) * BAR;
    int k = deck_bracket(m, p_c);
    if (k == -1) return r_lev[m.L];
    if (k == -2) return r_lev[0];
    R lnpc = log10_pc * LN10 + log(BAR);
    double l0 = m.lnp_lev[k], l1 = m.lnp_lev[k + 1];
    R f = (lnpc - l0) / (l1 - l0);
    return r_lev[k] + f * (r_lev[k + 1] - r_lev[k]);
}

// Bracket of x in an ascending grid: x clamped to [g0, g_last]; i = largest
// index with grid[i] <= x, capped at n-2; w = (x - grid[i])/(grid[i+1]-grid[i]);
// clamped = x outside the open range (no slope there).
__device__ inline void bracket(const double *grid, int n, double x, int &i, double &w, bool &clamped) {
    clamped = false;
    if (x <= grid[0]) { x = grid[0]; clamped = true; }
    if (x >= grid[n - 1]) { x = grid[n - 1]; clamped = true; }
    i = 0;
    for (int q = 0; q < n; ++q)
        if (grid[q] <= x) i = q;
    if (i > n - 2) i = n - 2;
    w = (x - grid[i]) / (grid[i + 1] - grid[i]);
}

}  // namespace es
