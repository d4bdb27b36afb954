"""FP64 CPU oracle for the Exo Skryer forward model and Gaussian log-likelihood.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py may import this module. The product
path (the CUDA library and its Python binding) never calls it.

Plain, slow, obviously correct numpy in float64, one function per stage of the
paper's forward model, in the paper's order and notation:

  T-p profile (Sect. 2.4) -> free-chemistry VMR fill (Sect. 3.1) ->
  hydrostatic altitude grid -> opacity interpolation + extinction (Sect. 3) ->
  transmission chord optical depth via the path matrix (Sect. 4, Eq. P_1D and
  tau_trans = P . dtau_vert) and transit depth, or emission linear-in-tau
  Schwarzschild integration with Gauss-Legendre angles (Sect. 5) ->
  instrument binning -> Gaussian log-likelihood (Sect. 2.3, Eqs. lnL, r_i,
  c_error).

Every function accepts complex input so that the complex-step method
(Squire & Trapp 1998) gives the oracle's own gradient: all branch decisions
(bracket indices, clamps, deck annulus, Taylor switch) are taken on real parts.

Readings taken where the paper is silent:
 - levels log-spaced p_top..p_bot, layer pressure = geometric mean of its levels;
 - hydrostatics with g(r) = g_ref (R_ref/r)^2, each layer isothermal at its
   layer temperature, anchored r(p_ref) = R_p,ref;
 - bilinear interpolation of log10 sigma in (log10 T, log10 p), clamped to the
   table; CIA linear in T of log10 k, clamped;
 - Rayleigh sigma(nu) = sigma_ref (nu/nu_ref)^4 for H2 and He;
 - impact parameter b_i at the radial midpoint of layer i;
 - transit depth = [r_c^2 + sum_i A_i (1 - exp(-tau_i))] / R_*^2 with annulus
   areas (in units of pi) A_i = r_up^2 - max(r_low^2, r_c^2), clipped at 0,
   and r_c the radius of an opaque grey deck (r_bot without a deck);
 - emission: absorption-only linear-in-tau RT with 4 Gauss-Legendre angles on
   [0, 1], or the 4-angle Gauss-Jacobi rule of the flux integral (weight mu:
   "8-stream" read as 4 angles per hemisphere), bottom boundary
   I = B(T_bottom level), F_* = pi B(T_*);
 - modified Milne profile: q_inf fixed at the Hopf function's deep limit;
 - mid-infrared cloud feature: the Q_max = 2 cap applies to Q_ext / Q_1 (Q_1
   folded into q_c^eff); lambda_0 and omega in micron;
 - non-grey cloud: r_eff in micron; each of the three mass-mixing-ratio
   profiles (power law above a base, whole-column slab, slab band with closed
   edges) evaluated at the layer pressures; no grey deck in the same model;
   in emission a clear and a cloudy column mixed by the cloud fraction;
   a brown dwarf's hydrostatic reference radius is its R_bd = sqrt(G M_bd/g);
 - binning: equal-weight mean over native points with lambda in [lo, hi);
 - emission with scattering (Sect. 5 delta-EAA; emission_solver = RT_DELTA_EAA):
   Rayleigh and cloud scattering, the cloud's single-scattering albedo and
   asymmetry parameter constants of the model, delta-M with f = g^2, the
   absorption approximation as the zeroth order and one scattering source
   evaluated on it (emergent_flux_eaa).

Parity status: every stage is pinned by tests/test_oracle_pins.py (closed forms,
brute force, invariants); the complete discretised model (species sums, CIA,
binning together) has no published worked example and rests on those pins.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf, roots_jacobi

# CODATA 2018 (cgs) and nominal radii
K_B = 1.380649e-16          # erg K^-1
H_PLANCK = 6.62607015e-27   # erg s
C_LIGHT = 2.99792458e10     # cm s^-1
AMU = 1.66053906660e-24     # g
R_JUP = 7.1492e9            # cm
BAR = 1.0e6                 # dyn cm^-2
LN10 = np.log(10.0)

# Sect. 3.1: He/H2 ratio of the background gas (Asplund et al. 2021)
HE_TO_H2 = 0.164
M_H2 = 2.01588
M_HE = 4.002602

# Sect. 2.4.4 (modified Guillot): fixed hemispheric factor and Eddington q_int
F_HEM = 0.25
Q_INT = 2.0 / 3.0
Q_IRR_INF = 2.0 / 3.0

INVALID_LNL = -1.0e300      # Sect. 2.3: invalid forward-model output

# canonical slots after the S log-VMR slots
(P_T_ISO, P_T_INT, P_T_EQ, P_LOG_KAPPA, P_LOG_GAMMA, P_Q_IRR0, P_LOG_PT, P_BETA,
 P_LOG_G, P_R_P, P_LOG_PCLOUD, P_C_INFL, P_DILUTION, P_T_RATIO, P_M_BD,
 P_LOG_QC, P_LOG_PC_BASE, P_ALPHA_C, P_LOG_R_EFF, P_A_KH, P_LOG_Q0, P_F_CLD,
 P_LOG_PC_TOP, P_LOG_DPC, P_FEAT_A, P_FEAT_LAM0, P_FEAT_W, P_FEAT_XI) = range(28)
# Sect. 2.5.1 vertical profiles of the cloud mass mixing ratio
QC_POWER_LAW, QC_SLAB, QC_SLAB_BAND = 0, 1, 2
TP_ISOTHERMAL, TP_GUILLOT, TP_GUILLOT_MOD, TP_MILNE = 0, 1, 2, 3
FLUX_PLANET_STAR, FLUX_BROWN_DWARF = 0, 1

# Sect. 2.4.3 (modified Milne): q_inf is not a retrieved parameter; the paper
# quotes the grey solution's deep value as ~0.71. Reading: the Hopf function's
# deep limit q(infinity) = 0.7104460895.
Q_MILNE_INF = 0.7104460895
# Sect. 5 (brown dwarfs): R_bd = sqrt(G M_bd / g); CODATA 2018 G, nominal Jupiter mass
G_GRAV = 6.67430e-8         # cm^3 g^-1 s^-2
M_JUP = 1.89813e30          # g
CLOUD_NONE, CLOUD_DECK, CLOUD_KH18 = 0, 1, 2


def _re(x):
    return np.real(x)


# --------------------------------------------------------------------------
# grids
# --------------------------------------------------------------------------
def pressure_grid(n_layers, p_top_bar, p_bot_bar):
    """Level pressures (L+1, top to bottom) log-spaced between p_top and p_bot,
    and layer pressures as the geometric mean of their two levels [dyn cm^-2]."""
    k = np.arange(n_layers + 1, dtype=np.float64)
    p_lev = p_top_bar * (p_bot_bar / p_top_bar) ** (k / n_layers) * BAR
    p_lay = np.sqrt(p_lev[:-1] * p_lev[1:])
    return p_lev, p_lay


def gauss_legendre_01(n):
    """n-point Gauss-Legendre nodes and weights mapped from [-1, 1] to [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_jacobi_mu_01(n):
    """Sect. 5 (Gauss-Jacobi angles for the intensity-to-flux integral): the
    n-point Gaussian rule for int_0^1 f(mu) mu dmu, i.e. the Gauss-Jacobi rule
    of weight (1 - x)^0 (1 + x)^1 on [-1, 1] mapped by mu = (1 + x)/2 (the
    weight becomes 2 mu, dx = 2 dmu). Returns nodes mu_j and weights W_j with
    sum_j W_j f(mu_j) ~ int_0^1 f(mu) mu dmu."""
    x, w = roots_jacobi(n, 0.0, 1.0)
    return 0.5 * (x + 1.0), 0.25 * w


QUAD_GAUSS_LEGENDRE, QUAD_GAUSS_JACOBI = 0, 1


def flux_quadrature(kind=QUAD_GAUSS_LEGENDRE, n_mu=4):
    """Angles mu_j and flux weights a_j with F = 2 pi sum_j a_j I(mu_j):
    Gauss-Legendre a_j = w_j mu_j, Gauss-Jacobi a_j = W_j."""
    if kind == QUAD_GAUSS_JACOBI:
        return gauss_jacobi_mu_01(n_mu)
    mu, w = gauss_legendre_01(n_mu)
    return mu, w * mu


# --------------------------------------------------------------------------
# Sect. 2.4: temperature-pressure profiles
# --------------------------------------------------------------------------
def temperature_isothermal(t_iso, p):
    """Sect. 2.4.1: T(p) = T_iso."""
    return t_iso * np.ones_like(p, dtype=np.result_type(t_iso, p))


def stretched_hopf(p, q0, q_inf, p_t, beta):
    """Eq. (q) in pressure form: q(p) = q_inf + (q0 - q_inf) exp[-(p/p_t)^beta]."""
    return q_inf + (q0 - q_inf) * np.exp(-(p / p_t) ** beta)


def temperature_guillot(p, t_int, t_eq, kappa_ir, gamma_v, g, q_irr=None):
    """Sect. 2.4.4, modified Guillot with mu_* = 1/sqrt(3), f_hem = 0.25,
    q_int = 2/3 and tau = kappa_ir p / g (Sect. 2.4.3).

    T^4 = 3/4 T_int^4 [q_int + tau]
        + 3/4 T_eq^4 4 f_hem [q_irr + 1/(gamma sqrt3)
                              + (gamma/sqrt3 - 1/(gamma sqrt3)) exp(-gamma tau sqrt3)]
    q_irr = 2/3 everywhere gives the 4-parameter form (Guillot 2010)."""
    tau = kappa_ir * p / g
    if q_irr is None:
        q_irr = Q_IRR_INF
    s3 = np.sqrt(3.0)
    t4 = 0.75 * t_int ** 4 * (Q_INT + tau) \
        + 0.75 * t_eq ** 4 * 4.0 * F_HEM * (q_irr + 1.0 / (gamma_v * s3)
                                           + (gamma_v / s3 - 1.0 / (gamma_v * s3))
                                           * np.exp(-gamma_v * tau * s3))
    return t4 ** 0.25


def temperature_milne(p, t_int, kappa_ir, g, t_ratio, p_t, beta):
    """Sect. 2.4.3, modified Milne: T^4 = 3/4 T_int^4 [tau + q(p)] with
    tau = kappa_ir p / g and the stretched-exponential Hopf function of
    Eq. (q), q0 = 4/3 T_ratio^4 (so T -> T_ratio T_int as p -> 0), q_inf fixed."""
    tau = kappa_ir * p / g
    q0 = 4.0 / 3.0 * t_ratio ** 4
    q = stretched_hopf(p, q0, Q_MILNE_INF, p_t, beta)
    return (0.75 * t_int ** 4 * (tau + q)) ** 0.25


def brown_dwarf_radius(m_bd_jup, g):
    """Sect. 5: R_bd = sqrt(G M_bd / g) [cm], M_bd in Jupiter masses."""
    return np.sqrt(G_GRAV * M_JUP * m_bd_jup / g)


# --------------------------------------------------------------------------
# Sect. 3.1: free chemistry with H2/He background
# --------------------------------------------------------------------------
def background_fill(x_trace):
    """X_H2 = (1 - sum X_i) / (1 + X_He/X_H2), X_He = X_H2 * 0.164."""
    x_h2 = (1.0 - np.sum(x_trace)) / (1.0 + HE_TO_H2)
    return x_h2, HE_TO_H2 * x_h2


def mean_molecular_mass(x_trace, masses_amu, x_h2, x_he):
    return np.sum(x_trace * masses_amu) + x_h2 * M_H2 + x_he * M_HE


# --------------------------------------------------------------------------
# hydrostatic altitude grid
# --------------------------------------------------------------------------
def altitude_grid(p_lev, t_lay, mu_amu, g_ref, r_ref, p_ref):
    """Level radii for hydrostatic balance with g(r) = g_ref (R_ref/r)^2 and
    each layer isothermal at its layer temperature:
        d(1/r) = k_B T / (mu m_u g_ref R_ref^2) d ln p,
    anchored at r(p_ref) = R_ref (exact per layer). Returns (r_lev, inv_r)."""
    n = t_lay.size
    coef = K_B / (mu_amu * AMU * g_ref * r_ref ** 2)
    inv_r = np.empty(n + 1, dtype=np.result_type(t_lay, coef, r_ref))
    j = int(np.clip(np.searchsorted(_re(p_lev), p_ref, side="right") - 1, 0, n - 1))
    inv_r[j] = 1.0 / r_ref + coef * t_lay[j] * np.log(p_lev[j] / p_ref)
    inv_r[j + 1] = 1.0 / r_ref + coef * t_lay[j] * np.log(p_lev[j + 1] / p_ref)
    for k in range(j - 1, -1, -1):                     # upward: layer k spans levels k, k+1
        inv_r[k] = inv_r[k + 1] + coef * t_lay[k] * np.log(p_lev[k] / p_lev[k + 1])
    for k in range(j + 2, n + 1):                      # downward: layer k-1 spans k-1, k
        inv_r[k] = inv_r[k - 1] + coef * t_lay[k - 1] * np.log(p_lev[k] / p_lev[k - 1])
    return 1.0 / inv_r, inv_r


def deck_radius(r_lev, p_lev, p_cloud):
    """Radius of an opaque deck at p_cloud: ln p interpolation between the
    bounding levels, clamped to [r_bot, r_top]."""
    pc = _re(p_cloud)
    if pc >= _re(p_lev[-1]):
        return r_lev[-1]
    if pc <= _re(p_lev[0]):
        return r_lev[0]
    k = int(np.searchsorted(_re(p_lev), pc, side="right") - 1)
    f = (np.log(p_cloud) - np.log(p_lev[k])) / (np.log(p_lev[k + 1]) - np.log(p_lev[k]))
    return r_lev[k] + f * (r_lev[k + 1] - r_lev[k])


# --------------------------------------------------------------------------
# Sect. 4: path distribution matrix
# --------------------------------------------------------------------------
def path_matrix(r_lev):
    """Eq. P_1D with layers l = 0..L-1 counted from the top: r_up,l = r_lev[l],
    r_low,l = r_lev[l+1], Delta r_l = r_up,l - r_low,l, b_i the midpoint
    radius of layer i.
      P_il = 0                                            r_up,l <= b_i
           = 2/dr_l sqrt(r_up,l^2 - b_i^2)                r_low,l < b_i < r_up,l
           = 2/dr_l [sqrt(r_up,l^2-b_i^2) - sqrt(r_low,l^2-b_i^2)]  r_low,l >= b_i
    """
    r_up, r_low = r_lev[:-1], r_lev[1:]
    dr = r_up - r_low
    b = 0.5 * (r_up + r_low)
    n = dr.size
    P = np.zeros((n, n), dtype=r_lev.dtype)
    for i in range(n):
        for l in range(n):
            if _re(r_up[l]) <= _re(b[i]):
                continue
            if _re(r_low[l]) < _re(b[i]):
                P[i, l] = 2.0 / dr[l] * np.sqrt(r_up[l] ** 2 - b[i] ** 2)
            else:
                P[i, l] = 2.0 / dr[l] * (np.sqrt(r_up[l] ** 2 - b[i] ** 2)
                                         - np.sqrt(r_low[l] ** 2 - b[i] ** 2))
    return P, dr, b


# --------------------------------------------------------------------------
# Sect. 3: opacity interpolation and extinction
# --------------------------------------------------------------------------
def bracket(grid, x):
    """Clamp x to [grid[0], grid[-1]]; i = largest index with grid[i] <= x,
    capped at N-2; w = (x - grid[i]) / (grid[i+1] - grid[i])."""
    xr = _re(x)
    if xr <= grid[0]:
        x = grid[0] + 0.0 * x
    elif xr >= grid[-1]:
        x = grid[-1] + 0.0 * x
    i = int(np.searchsorted(grid, _re(x), side="right") - 1)
    i = min(max(i, 0), grid.size - 2)
    w = (x - grid[i]) / (grid[i + 1] - grid[i])
    return i, w


def log10_sigma_bilinear(table, t_grid, p_grid_bar, t, p):
    """Bilinear interpolation of a species table log10 sigma[T, P, nu] in
    (log10 T, log10 p) at one (T, p); returns log10 sigma(nu)."""
    it, wt = bracket(np.log10(t_grid), np.log10(t))
    ip, wp = bracket(np.log10(p_grid_bar), np.log10(p / BAR))
    return ((1 - wt) * (1 - wp) * table[it, ip] + (1 - wt) * wp * table[it, ip + 1]
            + wt * (1 - wp) * table[it + 1, ip] + wt * wp * table[it + 1, ip + 1])


def log10_cia_linear(table, t_grid, t):
    """CIA log10 k linear in T between the bracketing temperatures, clamped."""
    i, w = bracket(t_grid, t)
    return (1 - w) * table[i] + w * table[i + 1]


def rayleigh_sigma(nu, sigma_ref, nu_ref):
    """sigma_R(nu) = sigma_ref (nu / nu_ref)^4."""
    return sigma_ref * (nu / nu_ref) ** 4


def extinction(tabs, model, x_trace, x_h2, x_he, t_lay, p_lay, rayleigh=True):
    """alpha_l(nu) [cm^-1] = n_l sum_s X_s 10^{log10 sigma_s(T_l, p_l, nu)}
       + n_l^2 X_H2 (X_H2 k_H2H2 + X_He k_H2He)(T_l, nu)
       + n_l (X_H2 sigma_R,H2 + X_He sigma_R,He)(nu),   n_l = p_l / (k_B T_l);
    without the Rayleigh term when rayleigh is False."""
    nu = tabs.nu
    ray = x_h2 * rayleigh_sigma(nu, model.ray_h2_cm2, model.ray_nu_ref) \
        + x_he * rayleigh_sigma(nu, model.ray_he_cm2, model.ray_nu_ref)
    alpha = np.zeros((t_lay.size, nu.size), dtype=np.result_type(t_lay, x_h2))
    for l in range(t_lay.size):
        n_l = p_lay[l] / (K_B * t_lay[l])
        for s in range(model.n_species):
            ls = log10_sigma_bilinear(tabs.log10_sigma[s], tabs.t_grid, tabs.p_grid_bar,
                                      t_lay[l], p_lay[l])
            alpha[l] += n_l * x_trace[s] * 10.0 ** ls
        k11 = 10.0 ** log10_cia_linear(tabs.cia_h2h2, tabs.cia_t_grid, t_lay[l])
        k12 = 10.0 ** log10_cia_linear(tabs.cia_h2he, tabs.cia_t_grid, t_lay[l])
        alpha[l] += n_l ** 2 * x_h2 * (x_h2 * k11 + x_he * k12)
        if rayleigh:
            alpha[l] += n_l * ray
    return alpha


def rayleigh_extinction(model, x_h2, x_he, t_lay, p_lay, nu):
    """The Rayleigh term of the extinction alone, n_l (X_H2 sigma_R,H2 + X_He sigma_R,He)(nu)."""
    ray = x_h2 * rayleigh_sigma(nu, model.ray_h2_cm2, model.ray_nu_ref) \
        + x_he * rayleigh_sigma(nu, model.ray_he_cm2, model.ray_nu_ref)
    n_lay = p_lay / (K_B * t_lay)
    return n_lay[:, None] * ray[None, :]


# --------------------------------------------------------------------------
# Sect. 2.5: non-grey aerosol opacity
# --------------------------------------------------------------------------
def cloud_mass_mixing_ratio(p, q_base, p_base, alpha_c):
    """Sect. 2.5.1 (third profile): q_c(p) = q_base (p / p_base)^alpha above
    the cloud base (p <= p_base) and 0 below it."""
    return np.where(_re(p) <= _re(p_base), q_base * (p / p_base) ** alpha_c, 0.0)


def cloud_mmr_slab(p, q_slab):
    """Sect. 2.5.1 (first profile): q_c(p) = q_slab over the whole column."""
    return q_slab * np.ones_like(p)


def cloud_mmr_slab_band(p, q_slab, p_top, dp):
    """Sect. 2.5.1 (second profile): q_c = q_slab for p_top <= p <= p_top + dp,
    0 above and below the band."""
    inside = (_re(p) >= _re(p_top)) & (_re(p) <= _re(p_top) + _re(dp))
    return np.where(inside, q_slab, 0.0)


def cloud_profile(model, theta, p_lay):
    """q_c^eff at the layer pressures for the model's profile choice; pressures
    in the parameter vector are log10 bar."""
    s = model.n_species
    q = 10.0 ** theta[s + P_LOG_QC]
    kind = getattr(model, "cloud_profile", QC_POWER_LAW)
    if kind == QC_SLAB:
        return cloud_mmr_slab(p_lay, q)
    if kind == QC_SLAB_BAND:
        return cloud_mmr_slab_band(p_lay, q, 10.0 ** theta[s + P_LOG_PC_TOP] * BAR,
                                   10.0 ** theta[s + P_LOG_DPC] * BAR)
    return cloud_mass_mixing_ratio(p_lay, q, 10.0 ** theta[s + P_LOG_PC_BASE] * BAR, theta[s + P_ALPHA_C])


def q_ext_kh18(x, q0, a):
    """Eq. Q_ext_KH with Q_1 subsumed into the effective mass mixing ratio:
    Q_ext / Q_1 = 1 / (Q_0 x^-a + x^0.2)."""
    return 1.0 / (q0 * x ** (-a) + x ** 0.2)


# Sect. 2.5.3: the feature window's transition size parameter and the cap of
# the total extinction efficiency
FEAT_X0 = 0.5
Q_MAX = 2.0


def q_feat_skew_normal(lam_um, amp, lam0, width, skew):
    """Eq. Q_ext_feat: Q_feat = 2 A exp(-z^2/2) Phi(xi z), z = (lambda -
    lambda_0)/omega, Phi(t) = [1 + erf(t/sqrt 2)]/2; wavelengths in micron."""
    z = (lam_um - lam0) / width
    return 2.0 * amp * np.exp(-0.5 * z * z) * 0.5 * (1.0 + erf(skew * z / np.sqrt(2.0)))


def q_ext_with_feature(x, lam_um, q0, a, amp, lam0, width, skew):
    """Sect. 2.5.3: Q_ext = min(Q_cont + W(x) Q_feat, Q_max), W = exp(-x/x0),
    Q_cont the KH18 form of q_ext_kh18 (Q_1 folded into q_c^eff, so the cap
    applies to Q_ext / Q_1); the cap's branch on the real part."""
    q = q_ext_kh18(x, q0, a) + np.exp(-x / FEAT_X0) * q_feat_skew_normal(lam_um, amp, lam0, width, skew)
    return np.where(_re(q) > Q_MAX, Q_MAX, q)


def cloud_extinction(nu, rho_a, q_c_eff, r_eff, q0, a, feature=None):
    """Sect. 2.5.2 (modified Fisher & Heng 2018): kappa_ext = 3 q_c^eff Q_ext(x)
    / (4 r_eff) [cm^2 g^-1] with the size parameter x = 2 pi r_eff / lambda =
    2 pi r_eff nu, and the layer extinction alpha_c(l, nu) = rho_a(l) kappa_ext
    [cm^-1]; rho_a is the background gas mass density. feature = (A, lambda_0,
    omega, xi) adds the mid-infrared feature of Sect. 2.5.3."""
    x = 2.0 * np.pi * r_eff * nu
    if feature is None:
        q = q_ext_kh18(x, q0, a)
    else:
        q = q_ext_with_feature(x, 1.0e4 / nu, q0, a, *feature)
    return (3.0 * rho_a * q_c_eff / (4.0 * r_eff))[:, None] * q[None, :]


# --------------------------------------------------------------------------
# transmission (Sect. 4)
# --------------------------------------------------------------------------
def transit_depth(tau, r_lev, r_c, r_star):
    """delta(nu) = [r_c^2 + sum_i A_i (1 - exp(-tau_i(nu)))] / R_*^2 with
    A_i = max(0, r_up,i^2 - max(r_low,i^2, r_c^2)) (the pi cancels)."""
    r_up, r_low = r_lev[:-1], r_lev[1:]
    area = np.zeros(r_up.size, dtype=np.result_type(r_lev, r_c))
    for i in range(r_up.size):
        if _re(r_up[i]) <= _re(r_c):
            continue
        inner = r_low[i] ** 2 if _re(r_low[i]) >= _re(r_c) else r_c ** 2
        area[i] = r_up[i] ** 2 - inner
    return (r_c ** 2 + area @ (1.0 - np.exp(-tau))) / r_star ** 2


# --------------------------------------------------------------------------
# emission (Sect. 5)
# --------------------------------------------------------------------------
def planck_wavenumber(t, nu):
    """B(T, nu) = 2 h c^2 nu^3 / (exp(h c nu / k_B T) - 1), per unit
    wavenumber [erg s^-1 cm^-2 sr^-1 (cm^-1)^-1]."""
    x = H_PLANCK * C_LIGHT * nu / (K_B * t)
    return 2.0 * H_PLANCK * C_LIGHT ** 2 * nu ** 3 / np.expm1(x)


def linear_source_factor(x):
    """(1 - e^-x)/x - e^-x, with its Taylor series x/2 - x^2/3 + x^3/8 below
    x = 1e-4."""
    xr = _re(x)
    small = xr < 1.0e-4
    xs = np.where(small, 1.0, x)          # placeholder argument where the series is used
    exact = (1.0 - np.exp(-xs)) / xs - np.exp(-xs)
    series = x / 2.0 - x ** 2 / 3.0 + x ** 3 / 8.0
    return np.where(small, series, exact)


def emergent_flux(b_lev, dtau, n_mu=4, quadrature=QUAD_GAUSS_LEGENDRE):
    """Top-of-atmosphere flux for absorption-only RT with a source linear in
    optical depth within each layer, integrated from I = B(bottom level)
    upward, for each angle mu_j of the flux quadrature on [0, 1]:
        E = exp(-dtau/mu),
        I <- I E + B_top (1 - E) + (B_bot - B_top) [(mu/dtau)(1 - E) - E],
    F = 2 pi sum_j a_j I_j (a_j = w_j mu_j for Gauss-Legendre, W_j for
    Gauss-Jacobi).   b_lev [L+1, N] top to bottom, dtau [L, N]."""
    mu, a = flux_quadrature(quadrature, n_mu)
    n = dtau.shape[0]
    flux = 0.0
    for j in range(n_mu):
        inten = b_lev[n].copy()
        for l in range(n - 1, -1, -1):
            x = dtau[l] / mu[j]
            e = np.exp(-x)
            inten = inten * e + b_lev[l] * (1.0 - e) + (b_lev[l + 1] - b_lev[l]) * linear_source_factor(x)
        flux = flux + 2.0 * np.pi * a[j] * inten
    return flux


# --------------------------------------------------------------------------
# emission with scattering (Sect. 5: linear-in-tau, delta-M scaled extended
# absorption approximation). The paper names the scheme and cites its source
# without printing its formulas; what follows is this library's reading:
#  - scatterers: H2/He Rayleigh (omega = 1, g = 0) and the non-grey cloud
#    with a single-scattering albedo omega_c and asymmetry parameter g_c that
#    are constants of the model (Sect. 2.5 gives Q_ext alone);
#  - delta-M scaling with the forward-peak fraction f = g^2 of the layer's
#    scattering-weighted g (delta-Eddington truncation of a two-term phase
#    function 1 + 3 g mu mu');
#  - zeroth order (absorption approximation): absorption-only linear-in-tau
#    RT in both directions on the scaled absorption depth (1 - omega') dtau';
#  - extended step: the scattering integral evaluated on that zeroth-order
#    field, J = 1/2 int I dmu and H = 1/2 int mu I dmu over both hemispheres
#    (at the flux angles: H with the flux weights, J with the nodes'
#    interpolatory weights of int_0^1 dmu),
#    gives the source S(mu) = (1 - omega') B + omega' (J + 3 g' mu H) at the
#    levels; one more upward linear-in-tau pass on the full scaled depth dtau'
#    with that source gives the emergent intensity.
# --------------------------------------------------------------------------
RT_ABSORPTION, RT_DELTA_EAA = 0, 1


def mean_intensity_weights(mu):
    """Weights c_j of int_0^1 f(mu) dmu at the flux angles mu_j: the
    interpolatory rule of those nodes (exact for polynomials of degree n-1;
    at Gauss-Legendre nodes these are the Gauss-Legendre weights). The flux
    weights of the Gauss-Jacobi rule divided by mu_j would not do: they
    integrate f(mu) = 1 to 0.96 at 4 nodes."""
    n = len(mu)
    vander = np.vander(mu, n, increasing=True).T
    return np.linalg.solve(vander, 1.0 / np.arange(1, n + 1))


def delta_m_scaling(dtau_abs, dtau_ray, dtau_cld, omega_c, g_c):
    """Layer optical properties and their delta-M scaling (Joseph, Wiscombe &
    Weinman 1976). Inputs are the layer's absorption depth (gas and CIA), its
    Rayleigh depth and its cloud extinction depth. With the scattering depth
    dsca = dtau_ray + omega_c dtau_cld, the total dtau, omega = dsca / dtau,
    the scattering-weighted asymmetry g = omega_c g_c dtau_cld / dsca (0 where
    nothing scatters) and f = g^2:
        dtau' = (1 - omega f) dtau,  omega' = (1 - f) omega / (1 - omega f),
        g' = (g - f) / (1 - f).
    Returns (dtau', omega', g')."""
    dtau = dtau_abs + dtau_ray + dtau_cld
    dsca = dtau_ray + omega_c * dtau_cld
    some = _re(dsca) > 0
    g = np.where(some, omega_c * g_c * dtau_cld / np.where(some, dsca, 1.0), 0.0)
    omega = dsca / dtau
    f = g * g
    dtau_s = (1.0 - omega * f) * dtau
    omega_s = (1.0 - f) * omega / (1.0 - omega * f)
    g_s = (g - f) / (1.0 - f)
    return dtau_s, omega_s, g_s


def linear_in_tau_layer(i_in, s_entry, s_exit, x):
    """Intensity leaving a layer of optical path x (along the ray) entered
    with i_in, for a source linear in optical depth from s_entry (where the
    ray enters) to s_exit (where it leaves):
        i_in e^-x + s_exit (1 - e^-x) + (s_entry - s_exit) [(1 - e^-x)/x - e^-x]."""
    e = np.exp(-x)
    return i_in * e + s_exit * (1.0 - e) + (s_entry - s_exit) * linear_source_factor(x)


def emergent_flux_eaa(b_lev, dtau_abs, dtau_ray, dtau_cld, omega_c, g_c, n_mu=4,
                      quadrature=QUAD_GAUSS_LEGENDRE):
    """Top-of-atmosphere flux of the delta-EAA (reading above). b_lev
    [L+1, N] top to bottom; dtau_abs, dtau_ray, dtau_cld [L, N]. Angles mu_j
    and flux weights a_j of the flux quadrature; mean_intensity_weights c_j
    integrate over mu at the same nodes, so
        J = 1/2 sum_j c_j (I_up,j + I_dn,j),  H = 1/2 sum_j a_j (I_up,j - I_dn,j).
    Boundaries: no downward intensity at the top, I_up = B(bottom level) at
    the bottom (both orders). F = 2 pi sum_j a_j I_j(top)."""
    mu, a = flux_quadrature(quadrature, n_mu)
    c = mean_intensity_weights(mu)
    n = dtau_abs.shape[0]
    dtau_s, om, gs = delta_m_scaling(dtau_abs, dtau_ray, dtau_cld, omega_c, g_c)
    dtau_a = (1.0 - om) * dtau_s
    j_lev = 0.0
    h_lev = 0.0
    for j in range(n_mu):
        up = [None] * (n + 1)
        dn = [None] * (n + 1)
        dn[0] = np.zeros_like(b_lev[0])
        for l in range(n):
            dn[l + 1] = linear_in_tau_layer(dn[l], b_lev[l], b_lev[l + 1], dtau_a[l] / mu[j])
        up[n] = b_lev[n]
        for l in range(n - 1, -1, -1):
            up[l] = linear_in_tau_layer(up[l + 1], b_lev[l + 1], b_lev[l], dtau_a[l] / mu[j])
        up, dn = np.array(up), np.array(dn)
        j_lev = j_lev + 0.5 * c[j] * (up + dn)
        h_lev = h_lev + 0.5 * a[j] * (up - dn)
    flux = 0.0
    for j in range(n_mu):
        inten = b_lev[n]
        for l in range(n - 1, -1, -1):
            s_top = (1.0 - om[l]) * b_lev[l] + om[l] * (j_lev[l] + 3.0 * gs[l] * mu[j] * h_lev[l])
            s_bot = (1.0 - om[l]) * b_lev[l + 1] + om[l] * (j_lev[l + 1] + 3.0 * gs[l] * mu[j] * h_lev[l + 1])
            inten = linear_in_tau_layer(inten, s_bot, s_top, dtau_s[l] / mu[j])
        flux = flux + 2.0 * np.pi * a[j] * inten
    return flux


# --------------------------------------------------------------------------
# instrument binning and Sect. 2.3 likelihood
# --------------------------------------------------------------------------
def bin_members(nu, bin_lo_um, bin_hi_um):
    """Per bin, the indices of the native points with lambda = 1e4/nu in [lo, hi)."""
    lam = 1.0e4 / nu
    return [np.nonzero((lam >= lo) & (lam < hi))[0] for lo, hi in zip(bin_lo_um, bin_hi_um)]


def bin_spectrum(spec, members):
    """Equal-weight mean of the native-resolution model over each bin."""
    return np.array([np.mean(spec[m]) for m in members])


def log_likelihood(y_model, y_obs, sigma, c):
    """ln L = sum_i [-ln sigma_eff - 1/2 ln(2 pi) - 1/2 (r_i/sigma_eff)^2],
    r_i = y_obs - y_model, sigma_eff^2 = sigma^2 + 10^(2c)."""
    sig_eff = np.sqrt(sigma ** 2 + 10.0 ** (2.0 * c))
    r = y_obs - y_model
    return np.sum(-np.log(sig_eff) - 0.5 * np.log(2.0 * np.pi) - 0.5 * (r / sig_eff) ** 2)


# --------------------------------------------------------------------------
# complete forward model for one parameter vector
# --------------------------------------------------------------------------
def atmosphere(model, theta):
    """Profile, chemistry and geometry for one canonical parameter vector.
    Returns a dict, with 'valid' False for the paper's invalid outputs."""
    s = model.n_species
    th = theta
    x_trace = 10.0 ** th[:s]
    p_lev, p_lay = pressure_grid(model.n_layers, model.p_top_bar, model.p_bot_bar)
    g = 10.0 ** th[s + P_LOG_G]
    if model.tp_kind == TP_ISOTHERMAL:
        t_lay = temperature_isothermal(th[s + P_T_ISO], p_lay)
        t_lev = temperature_isothermal(th[s + P_T_ISO], p_lev)
    elif model.tp_kind == TP_MILNE:
        kappa = 10.0 ** th[s + P_LOG_KAPPA]
        p_t = 10.0 ** th[s + P_LOG_PT] * BAR
        t_lay, t_lev = (temperature_milne(p, th[s + P_T_INT], kappa, g, th[s + P_T_RATIO], p_t, th[s + P_BETA])
                        for p in (p_lay, p_lev))
    else:
        kappa = 10.0 ** th[s + P_LOG_KAPPA]
        gamma = 10.0 ** th[s + P_LOG_GAMMA]
        q_lay = q_lev = None
        if model.tp_kind == TP_GUILLOT_MOD:
            p_t = 10.0 ** th[s + P_LOG_PT] * BAR
            q_lay = stretched_hopf(p_lay, th[s + P_Q_IRR0], Q_IRR_INF, p_t, th[s + P_BETA])
            q_lev = stretched_hopf(p_lev, th[s + P_Q_IRR0], Q_IRR_INF, p_t, th[s + P_BETA])
        t_lay = temperature_guillot(p_lay, th[s + P_T_INT], th[s + P_T_EQ], kappa, gamma, g, q_lay)
        t_lev = temperature_guillot(p_lev, th[s + P_T_INT], th[s + P_T_EQ], kappa, gamma, g, q_lev)
    x_h2, x_he = background_fill(x_trace)
    mu = mean_molecular_mass(x_trace, model.masses_amu, x_h2, x_he)
    valid = bool(np.all(np.isfinite(_re(t_lay))) and np.all(_re(t_lay) > 0)
                 and np.all(_re(t_lev) > 0) and _re(np.sum(x_trace)) < 1.0)
    brown_dwarf = getattr(model, "emission_flux", FLUX_PLANET_STAR) == FLUX_BROWN_DWARF
    if brown_dwarf:
        valid = valid and _re(th[s + P_M_BD]) > 0
        r_ref = brown_dwarf_radius(th[s + P_M_BD], g) if valid else 0.0
    else:
        r_ref = th[s + P_R_P] * R_JUP
    out = dict(x_trace=x_trace, x_h2=x_h2, x_he=x_he, mu=mu, g=g, p_lev=p_lev, p_lay=p_lay,
               t_lay=t_lay, t_lev=t_lev, r_ref=r_ref, valid=valid)
    if not valid:
        return out
    r_lev, inv_r = altitude_grid(p_lev, t_lay, mu, g, r_ref, model.p_ref_bar * BAR)
    out["r_lev"] = r_lev
    out["valid"] = bool(np.all(_re(inv_r) > 0))
    return out


def forward(model, tabs, theta, kind, members):
    """Native-resolution spectrum (transit depth or Fp/F*) and binned model
    for one canonical parameter vector. Returns (spec, y) or None if invalid."""
    s = model.n_species
    atm = atmosphere(model, theta)
    if not atm["valid"]:
        return None
    alpha = extinction(tabs, model, atm["x_trace"], atm["x_h2"], atm["x_he"],
                       atm["t_lay"], atm["p_lay"])
    r_lev = atm["r_lev"]
    # Sect. 2.5.2: cloudy and cloud-free spectra mixed by the cloud fraction,
    # Phi = f Phi_cld + (1 - f) Phi_cf
    cloudy = model.cloud_kind == CLOUD_KH18
    if cloudy:
        p_lay, t_lay = atm["p_lay"], atm["t_lay"]
        q_c = cloud_profile(model, theta, p_lay)
        rho_a = atm["mu"] * AMU * p_lay / (K_B * t_lay)
        feature = None
        if getattr(model, "cloud_feature", 0):
            feature = (theta[s + P_FEAT_A], theta[s + P_FEAT_LAM0], theta[s + P_FEAT_W], theta[s + P_FEAT_XI])
        alpha_c = cloud_extinction(tabs.nu, rho_a, q_c, 10.0 ** theta[s + P_LOG_R_EFF] * 1.0e-4,
                                   10.0 ** theta[s + P_LOG_Q0], theta[s + P_A_KH], feature)
        alpha_cld = alpha + alpha_c
        f_cld = theta[s + P_F_CLD]
    if kind == 0:
        P, dr, _ = path_matrix(r_lev)
        dtau_vert = alpha * dr[:, None]
        tau = P @ dtau_vert                               # Sect. 4: tau_trans = P . dtau_vert
        if model.cloud_kind == CLOUD_DECK:
            r_c = deck_radius(r_lev, atm["p_lev"], 10.0 ** theta[s + P_LOG_PCLOUD] * BAR)
        else:
            r_c = r_lev[-1]
        spec = transit_depth(tau, r_lev, r_c, model.r_star_cm)
        if cloudy:
            spec_cld = transit_depth(P @ (alpha_cld * dr[:, None]), r_lev, r_c, model.r_star_cm)
            spec = f_cld * spec_cld + (1.0 - f_cld) * spec
    else:
        dr = r_lev[:-1] - r_lev[1:]
        b_lev = planck_wavenumber(atm["t_lev"][:, None], tabs.nu[None, :])
        quad = getattr(model, "emission_quadrature", QUAD_GAUSS_LEGENDRE)
        if getattr(model, "emission_solver", RT_ABSORPTION) == RT_DELTA_EAA:
            # Sect. 5 delta-EAA: absorption, Rayleigh and cloud depths kept apart
            x_h2, x_he, t_lay, p_lay = atm["x_h2"], atm["x_he"], atm["t_lay"], atm["p_lay"]
            alpha_abs = extinction(tabs, model, atm["x_trace"], x_h2, x_he, t_lay, p_lay, rayleigh=False)
            d_abs = alpha_abs * dr[:, None]
            d_ray = rayleigh_extinction(model, x_h2, x_he, t_lay, p_lay, tabs.nu) * dr[:, None]
            ssa, gc = model.cloud_ssa, model.cloud_g
            f_toa = emergent_flux_eaa(b_lev, d_abs, d_ray, np.zeros_like(d_abs), ssa, gc, quadrature=quad)
            if cloudy:
                d_cld = alpha_c * dr[:, None]
                f_toa = f_cld * emergent_flux_eaa(b_lev, d_abs, d_ray, d_cld, ssa, gc, quadrature=quad) \
                    + (1.0 - f_cld) * f_toa
        else:
            dtau = alpha * dr[:, None]
            f_toa = emergent_flux(b_lev, dtau, quadrature=quad)
            if cloudy:
                f_toa = f_cld * emergent_flux(b_lev, alpha_cld * dr[:, None], quadrature=quad) \
                    + (1.0 - f_cld) * f_toa
        if getattr(model, "emission_flux", FLUX_PLANET_STAR) == FLUX_BROWN_DWARF:
            # Sect. 5: F_bd = s F_toa (R_bd / D)^2
            spec = theta[s + P_DILUTION] * f_toa * (atm["r_ref"] / model.distance_cm) ** 2
        else:
            f_star = np.pi * planck_wavenumber(model.t_star_k, tabs.nu)
            # Sect. 5: Fp/F* = s F_toa / F_* (R_p / R_*)^2
            spec = theta[s + P_DILUTION] * f_toa / f_star * (atm["r_ref"] / model.r_star_cm) ** 2
    if not np.all(np.isfinite(_re(spec))):
        return None
    return spec, bin_spectrum(spec, members)


def loglike(model, tabs, theta, kind, members, y_obs, sigma):
    """ln L for one canonical parameter vector; -1e300 if the model is invalid."""
    out = forward(model, tabs, theta, kind, members)
    if out is None:
        return INVALID_LNL
    return log_likelihood(out[1], y_obs, sigma, theta[model.n_species + P_C_INFL])


def loglike_gradient(model, tabs, theta, kind, members, y_obs, sigma, slots, h=1.0e-30):
    """The oracle's own gradient d lnL / d theta[slots] by the complex step:
    d f/d x = Im f(x + i h) / h, exact to rounding (no subtractive error)."""
    grad = np.zeros(len(slots))
    base = np.asarray(theta, dtype=np.complex128)
    for k, slot in enumerate(slots):
        th = base.copy()
        th[slot] += 1j * h
        val = loglike(model, tabs, th, kind, members, y_obs, sigma)
        grad[k] = 0.0 if np.real(val) == INVALID_LNL else np.imag(val) / h
    return grad


# --------------------------------------------------------------------------
# BF16 table storage (the library's reduced-precision table format)
# --------------------------------------------------------------------------
def bf16_row_dequantized(log10_sigma):
    """Values the BF16-table path interpolates: each (species, T, p) row is
    stored as round-to-nearest-even BF16 of (value - offset) with an FP32
    offset equal to the row mean (mean taken in FP64, rounded to FP32; the
    residual formed in FP32). Returns the dequantized table in float64."""
    tab = np.asarray(log10_sigma, dtype=np.float32)
    off = np.mean(tab.astype(np.float64), axis=-1).astype(np.float32)
    resid = (tab - off[..., None]).astype(np.float32)
    bits = resid.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    q = rounded.astype(np.uint32).view(np.float32)
    return q.astype(np.float64) + off[..., None].astype(np.float64)
