"""Pins of the FP64 oracle against closed forms, brute-force integration and
invariants that the paper and the mathematics fix (no GPU needed).

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a wrong layer's temperature) fails it.
"""
import dataclasses
import os

import numpy as np
import pytest

from oracle import exoskry_oracle as O
from paper_2602_19687_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _model(L=40, p_top=1e-6, p_bot=100.0, p_ref=10.0, tp=O.TP_ISOTHERMAL, cloud=O.CLOUD_NONE,
           n_species=1, r_star=synth.R_SUN_CM):
    m = synth._model(n_species, L, p_top, p_bot, tp, cloud, free=[0],
                     species=list(synth.SPECIES)[:n_species])
    m.p_ref_bar = p_ref
    m.r_star_cm = r_star
    return m


def _flat_tables(nu, log10_sigma=-22.0, n_species=1, cia=-99.0):
    t_grid = np.geomspace(100.0, 5000.0, 6)
    p_grid = np.geomspace(1e-9, 1e3, 5)
    sig = np.full((n_species, t_grid.size, p_grid.size, nu.size), log10_sigma)
    cia_t = np.array([100.0, 5000.0])
    cia_tab = np.full((2, nu.size), cia)
    return synth.Tables(nu=nu, t_grid=t_grid, p_grid_bar=p_grid, log10_sigma=sig,
                        cia_t_grid=cia_t, cia_h2h2=cia_tab, cia_h2he=cia_tab)


# ---------------------------------------------------------------- grids, VMR
def test_pressure_grid_levels_and_layers():
    p_lev, p_lay = O.pressure_grid(50, 1e-6, 100.0)
    assert p_lev[0] == pytest.approx(1e-6 * O.BAR) and p_lev[-1] == pytest.approx(100.0 * O.BAR)
    ratio = p_lev[1:] / p_lev[:-1]
    assert np.allclose(ratio, ratio[0], rtol=1e-12)           # log-uniform levels
    assert np.all((p_lay > p_lev[:-1]) & (p_lay < p_lev[1:]))
    assert np.allclose(np.log(p_lay), 0.5 * (np.log(p_lev[:-1]) + np.log(p_lev[1:])))


def test_vmr_fill_sums_to_one_and_he_ratio():
    x = 10.0 ** np.array([-3.0, -4.5, -2.2, -7.0])
    x_h2, x_he = O.background_fill(x)
    assert np.sum(x) + x_h2 + x_he == pytest.approx(1.0, abs=1e-15)
    assert x_he / x_h2 == pytest.approx(0.164, rel=1e-15)
    mu = O.mean_molecular_mass(np.zeros(1), np.array([18.0]), *O.background_fill(np.zeros(1)))
    # solar H2/He mixture: (2.01588 + 0.164*4.002602)/1.164
    assert mu == pytest.approx((2.01588 + 0.164 * 4.002602) / 1.164, rel=1e-14)


# ---------------------------------------------------------------- T-p profiles
def test_guillot_reduces_to_guillot2010():
    """q_irr = 2/3 equals Guillot (2010) Eq. 49 with mu_* = 1/sqrt(3) and
    T_irr^4 mu_* = 4 f_hem T_eq^4, written in its own variables."""
    p = np.geomspace(1e-2, 1e8, 40)
    t_int, t_eq, kappa, gamma, g = 250.0, 1300.0, 10 ** -2.3, 10 ** -0.7, 10 ** 3.1
    mu_s = 1.0 / np.sqrt(3.0)
    t_irr4 = 4.0 * 0.25 * t_eq ** 4 / mu_s
    tau = kappa * p / g
    t4_ref = 0.75 * t_int ** 4 * (2.0 / 3.0 + tau) + 0.75 * t_irr4 * mu_s * (
        2.0 / 3.0 + mu_s / gamma + (gamma / (3.0 * mu_s) - mu_s / gamma) * np.exp(-gamma * tau / mu_s))
    t = O.temperature_guillot(p, t_int, t_eq, kappa, gamma, g)
    assert np.allclose(t, t4_ref ** 0.25, rtol=1e-13)


def test_guillot_deep_limit_and_hopf_limits():
    p = np.array([1e12, 1e13])
    t_int, g, kappa = 400.0, 1e3, 1e-1
    t = O.temperature_guillot(p, t_int, 1500.0, kappa, 0.3, g)
    tau = kappa * p / g
    assert np.allclose(t ** 4 / tau, 0.75 * t_int ** 4, rtol=1e-3)   # T^4 -> 3/4 T_int^4 tau
    q = O.stretched_hopf(np.array([1e-12, 1e12]), 0.2, 2.0 / 3.0, 1e3, 0.7)
    assert q[0] == pytest.approx(0.2, abs=1e-6) and q[1] == pytest.approx(2.0 / 3.0, abs=1e-12)


def test_modified_guillot_q_irr_enters_the_irradiation_term_only():
    """Sect. 2.4.4, 7-parameter modified Guillot through the full profile
    (atmosphere()): with q_irr0 far from 2/3 and T_eq >> T_int, the levels far
    above p_t (q_irr -> q_irr0) follow Guillot (2010) with its irradiation
    bracket's 2/3 replaced by q_irr0 and the internal term's q_int = 2/3 kept;
    the levels far below p_t (q_irr -> 2/3) are Guillot (2010) itself; and at
    p = p_t, q_irr = 2/3 + (q_irr0 - 2/3)/e. Written in Guillot's own variables
    (T_irr^4 mu_* = 4 f_hem T_eq^4, mu_* = 1/sqrt 3), so q_irr placed in the
    internal term, or the Hopf function taken in tau instead of p, fails."""
    m = _model(L=30, tp=O.TP_GUILLOT_MOD)
    s = m.n_species
    th = m.theta_fixed.copy()
    t_int, t_eq, kappa, gamma, q0, beta = 180.0, 1700.0, 10 ** -1.3, 10 ** -0.4, 0.12, 6.0
    p_lev, _ = O.pressure_grid(m.n_layers, m.p_top_bar, m.p_bot_bar)
    k_t = 14
    p_t_bar = p_lev[k_t] / O.BAR                      # p_t on a level: that level sees q(p_t)
    th[0] = -4.0
    th[s + O.P_T_INT], th[s + O.P_T_EQ] = t_int, t_eq
    th[s + O.P_LOG_KAPPA], th[s + O.P_LOG_GAMMA] = np.log10(kappa), np.log10(gamma)
    th[s + O.P_Q_IRR0], th[s + O.P_LOG_PT], th[s + O.P_BETA] = q0, np.log10(p_t_bar), beta
    g = 10 ** th[s + O.P_LOG_G]
    atm = O.atmosphere(m, th)
    mu_s = 1.0 / np.sqrt(3.0)
    t_irr4_mu = 4.0 * 0.25 * t_eq ** 4

    def guillot(p, q_irr):
        tau = kappa * p / g
        return (0.75 * t_int ** 4 * (2.0 / 3.0 + tau) + 0.75 * t_irr4_mu * (
            q_irr + mu_s / gamma + (gamma / (3.0 * mu_s) - mu_s / gamma) * np.exp(-gamma * tau / mu_s))) ** 0.25

    top = p_lev < 1e-2 * p_t_bar * O.BAR              # (p/p_t)^6 < 1e-12: q_irr = q_irr0
    deep = p_lev > 1e2 * p_t_bar * O.BAR              # (p/p_t)^6 > 1e12: q_irr = 2/3
    assert top.sum() >= 5 and deep.sum() >= 3
    assert np.allclose(atm["t_lev"][top], guillot(p_lev[top], q0), rtol=1e-9)
    assert np.allclose(atm["t_lev"][deep], guillot(p_lev[deep], 2.0 / 3.0), rtol=1e-13)
    q_t = 2.0 / 3.0 + (q0 - 2.0 / 3.0) / np.e
    assert atm["t_lev"][k_t] == pytest.approx(guillot(p_lev[k_t], q_t), rel=1e-13)
    # the slip: q_irr in the internal term instead is far off at the top
    tau = kappa * p_lev[top] / g
    slip = (0.75 * t_int ** 4 * (q0 + tau) + 0.75 * t_irr4_mu * (
        2.0 / 3.0 + mu_s / gamma + (gamma / (3.0 * mu_s) - mu_s / gamma) * np.exp(-gamma * tau / mu_s))) ** 0.25
    assert np.min(np.abs(atm["t_lev"][top] / slip - 1.0)) > 1e-2
    # layers use the same profile at their geometric-mean pressures
    _, p_lay = O.pressure_grid(m.n_layers, m.p_top_bar, m.p_bot_bar)
    top_l = p_lay < 1e-2 * p_t_bar * O.BAR
    assert np.allclose(atm["t_lay"][top_l], guillot(p_lay[top_l], q0), rtol=1e-9)


def test_milne_skin_eddington_deep_and_transition():
    """Modified Milne (Sect. 2.4.3): T -> T_ratio T_int at the top (q -> q0 =
    4/3 T_ratio^4, tau -> 0); with q0 = q_inf it is the Eddington-like Milne
    solution 3/4 T_int^4 (tau + q_inf) at every pressure; deep, T^4 -> 3/4
    T_int^4 tau; at p = p_t the Hopf function is q_inf + (q0 - q_inf)/e."""
    t_int, kappa, g, p_t, beta = 1150.0, 10 ** -1.9, 10 ** 5.2, 8.0 * O.BAR, 0.9
    t_ratio = 0.43
    top = O.temperature_milne(np.array([1e-12 * O.BAR]), t_int, kappa, g, t_ratio, p_t, beta)
    assert top[0] == pytest.approx(t_ratio * t_int, rel=1e-8)
    p = np.geomspace(1e-8, 1e3, 50) * O.BAR
    tau = kappa * p / g
    t_edd = (0.75 * O.Q_MILNE_INF) ** 0.25
    t = O.temperature_milne(p, t_int, kappa, g, t_edd, p_t, beta)
    assert np.allclose(t, (0.75 * t_int ** 4 * (tau + O.Q_MILNE_INF)) ** 0.25, rtol=1e-13)
    deep = np.array([1e12, 1e13]) * O.BAR
    t = O.temperature_milne(deep, t_int, kappa, g, t_ratio, p_t, beta)
    assert np.allclose(t ** 4 / (kappa * deep / g), 0.75 * t_int ** 4, rtol=1e-5)
    t = O.temperature_milne(np.array([p_t]), t_int, kappa, g, t_ratio, p_t, beta)
    q = O.Q_MILNE_INF + (4.0 / 3.0 * t_ratio ** 4 - O.Q_MILNE_INF) / np.e
    assert t[0] ** 4 == pytest.approx(0.75 * t_int ** 4 * (kappa * p_t / g + q), rel=1e-13)


def test_brown_dwarf_isothermal_flux():
    """Sect. 5 brown-dwarf flux: an isothermal atmosphere emits pi B(T) at every
    wavenumber, so F_bd = s pi B(T) (R_bd / D)^2 with R_bd = sqrt(G M_bd / g),
    which also anchors the hydrostatic grid."""
    m = _model(L=25)
    m.emission_flux = O.FLUX_BROWN_DWARF
    m.distance_cm = 10.0 * synth.PARSEC_CM
    nu = synth.nu_grid_constant_r(1.0, 5.1, 40)
    rng = np.random.default_rng(9)
    tabs = _flat_tables(nu, -22.0)
    tabs.log10_sigma = rng.uniform(-28, -19, tabs.log10_sigma.shape)
    s = m.n_species
    th = m.theta_fixed.copy()
    th[0], th[s + O.P_LOG_G], th[s + O.P_M_BD], th[s + O.P_DILUTION] = -3.0, 5.1, 68.0, 0.8
    mem = O.bin_members(nu, np.array([0.9]), np.array([6.0]))
    spec, _ = O.forward(m, tabs, th, 1, mem)
    r_bd = np.sqrt(6.67430e-8 * 1.89813e30 * 68.0 / 10 ** 5.1)
    expect = 0.8 * np.pi * O.planck_wavenumber(th[s + O.P_T_ISO], nu) * (r_bd / m.distance_cm) ** 2
    assert np.allclose(spec, expect, rtol=1e-12)
    atm = O.atmosphere(m, th)
    assert atm["r_ref"] == pytest.approx(r_bd, rel=1e-15)
    # isothermal hydrostatics anchored at R_bd (closed form, as for planets)
    g = 10 ** th[s + O.P_LOG_G]
    inv = 1.0 / r_bd + O.K_B * th[s + O.P_T_ISO] * np.log(atm["p_lev"] / (m.p_ref_bar * O.BAR)) \
        / (atm["mu"] * O.AMU * g * r_bd ** 2)
    assert np.allclose(atm["r_lev"], 1.0 / inv, rtol=1e-13)


def test_cloud_profile_qext_and_number_density_form():
    """Sect. 2.5: the base + power-law mass mixing ratio (zero below the base);
    the KH18 fitting form; and kappa_ext = 3 q_eff Q_ext / (4 r) equal to
    N0 Q_ext pi r^2 / rho_a with N0 = 3 rho_a q_c / (4 pi rho_d r^3) and
    q_eff = Q1 q_c / rho_d, for any rho_d and Q1 (monodisperse spheres)."""
    p = np.array([1e-3, 0.5, 1.0, 2.0]) * O.BAR
    q = O.cloud_mass_mixing_ratio(p, 1e-4, 1.0 * O.BAR, 1.5)
    assert np.allclose(q, [1e-4 * 1e-3 ** 1.5, 1e-4 * 0.5 ** 1.5, 1e-4, 0.0], rtol=1e-15, atol=0)
    x = np.array([0.01, 0.3, 1.0, 7.0, 90.0])
    assert np.allclose(O.q_ext_kh18(x, 12.0, 4.5), 1.0 / (12.0 * x ** -4.5 + x ** 0.2), rtol=1e-15)
    rho_a, q_c, r, rho_d, q1 = 3.7e-6, 2.3e-5, 0.8e-4, 3.3, 2.1
    nu = np.array([2000.0, 11000.0])
    n0 = 3.0 * rho_a * q_c / (4.0 * np.pi * rho_d * r ** 3)
    qext = q1 * O.q_ext_kh18(2.0 * np.pi * r * nu, 12.0, 4.5)
    alpha = O.cloud_extinction(nu, np.array([rho_a]), np.array([q1 * q_c / rho_d]), r, 12.0, 4.5)
    assert np.allclose(alpha[0], n0 * qext * np.pi * r ** 2, rtol=1e-13)


def _cloud_setup(kind):
    w = synth.workload("cloudy_trans", n_nu=300, batch=2)
    m = w.model
    th = m.full_theta(w.theta)[0]
    s = m.n_species
    th[s + O.P_LOG_QC], th[s + O.P_LOG_PC_BASE], th[s + O.P_LOG_R_EFF] = -4.0, 0.5, -0.7
    mem = O.bin_members(w.tables.nu, w.bin_lo_um, w.bin_hi_um)
    return w, m, th, s, mem


@pytest.mark.parametrize("kind", [0, 1])
def test_cloud_fraction_limits_and_linearity(kind):
    """f_cld = 0 gives the cloud-free model exactly, the spectrum is linear in
    f_cld, and a vanishing cloud mass has no effect; the cloud changes it."""
    w, m, th, s, mem = _cloud_setup(kind)
    clear = dataclasses.replace(m, cloud_kind=O.CLOUD_NONE)
    ref, _ = O.forward(clear, w.tables, th, kind, mem)
    spec = {}
    for f in (0.0, 0.37, 1.0):
        t = th.copy()
        t[s + O.P_F_CLD] = f
        spec[f], _ = O.forward(m, w.tables, t, kind, mem)
    assert np.allclose(spec[0.0], ref, rtol=1e-14, atol=0)
    assert np.allclose(spec[0.37], 0.37 * spec[1.0] + 0.63 * spec[0.0], rtol=1e-12, atol=0)
    assert np.max(np.abs(spec[1.0] / ref - 1.0)) > 1e-3
    t = th.copy()
    t[s + O.P_LOG_QC], t[s + O.P_F_CLD] = -99.0, 1.0
    assert np.allclose(O.forward(m, w.tables, t, kind, mem)[0], ref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("kind", [0, 1])
def test_uniform_cloud_equals_constant_absorber(kind):
    """A cloud of uniform q_c (base below the model, alpha_c = 0) with no gas
    opacity gives the transit depth (emergent flux) of an absorber whose
    cross-section times VMR is mu m_u kappa_ext(nu): pins rho_a = mu m_u n and
    the cloud's entry into the chord optical depth and the emission column."""
    # an isothermal column emits B(T) whatever its opacity: emission needs a gradient
    m = _model(L=40, tp=O.TP_ISOTHERMAL if kind == 0 else O.TP_GUILLOT, cloud=O.CLOUD_KH18)
    m.ray_h2_cm2 = m.ray_he_cm2 = 0.0
    s = m.n_species
    nu = synth.nu_grid_constant_r(0.6, 5.0, 30)
    th = m.theta_fixed.copy()
    th[0] = -4.0
    th[s + O.P_LOG_QC], th[s + O.P_LOG_PC_BASE], th[s + O.P_ALPHA_C] = -5.5, 5.0, 0.0
    th[s + O.P_LOG_R_EFF], th[s + O.P_A_KH], th[s + O.P_LOG_Q0], th[s + O.P_F_CLD] = -0.4, 4.0, 1.2, 1.0
    mem = O.bin_members(nu, np.array([0.55]), np.array([5.5]))
    cloud_tabs = _flat_tables(nu, -99.0)
    spec_cloud, _ = O.forward(m, cloud_tabs, th, kind, mem)
    atm = O.atmosphere(m, th)
    r = 10 ** th[s + O.P_LOG_R_EFF] * 1e-4
    kappa = 3.0 * 10 ** th[s + O.P_LOG_QC] / (4.0 * r) * O.q_ext_kh18(2 * np.pi * r * nu, 10 ** 1.2, 4.0)
    sigma = atm["mu"] * O.AMU * kappa / 10 ** th[0]
    gas_tabs = _flat_tables(nu, -99.0)
    gas_tabs.log10_sigma = np.broadcast_to(np.log10(sigma), gas_tabs.log10_sigma.shape).copy()
    clear = dataclasses.replace(m, cloud_kind=O.CLOUD_NONE)
    spec_gas, _ = O.forward(clear, gas_tabs, th, kind, mem)
    assert np.allclose(spec_cloud, spec_gas, rtol=1e-12)
    spec_none, _ = O.forward(clear, cloud_tabs, th, kind, mem)   # neither cloud nor absorber
    assert np.max(np.abs(spec_cloud / spec_none - 1.0)) > 1e-3


def test_cloud_feature_skew_normal_area_mean_window_and_cap():
    """Sect. 2.5.3: 2 phi(z) Phi(xi z) / omega is the skew-normal density, so
    the feature integrates to A omega sqrt(2 pi) over wavelength for any xi
    and its centroid is lambda_0 + omega delta sqrt(2/pi), delta =
    xi/sqrt(1 + xi^2); xi = 0 is a Gaussian of peak A at lambda_0; the window
    keeps the whole feature for x << x0 and removes it for x >> x0; the total
    efficiency is capped at Q_max = 2."""
    lam = np.linspace(-30.0, 50.0, 400001)
    amp, lam0, om = 0.7, 9.5, 1.5
    for xi in (0.0, 3.0, -2.0):
        q = O.q_feat_skew_normal(lam, amp, lam0, om, xi)
        area = np.trapezoid(q, lam)
        assert area == pytest.approx(amp * om * np.sqrt(2.0 * np.pi), rel=1e-9)
        delta = xi / np.sqrt(1.0 + xi * xi)
        assert np.trapezoid(q * lam, lam) / area == pytest.approx(lam0 + om * delta * np.sqrt(2.0 / np.pi),
                                                                    rel=1e-9)
    assert O.q_feat_skew_normal(lam0, amp, lam0, om, 0.0) == pytest.approx(amp, rel=1e-15)
    lam_pt = np.array([8.0, 9.5, 11.0])
    feat = O.q_feat_skew_normal(lam_pt, amp, lam0, om, 1.0)
    x = np.full(3, 1e-9)
    q_small = O.q_ext_with_feature(x, lam_pt, 10.0, 4.0, amp, lam0, om, 1.0)
    assert np.allclose(q_small, O.q_ext_kh18(x, 10.0, 4.0) + feat, rtol=1e-8)
    x = np.full(3, 60.0)
    assert np.allclose(O.q_ext_with_feature(x, lam_pt, 10.0, 4.0, amp, lam0, om, 1.0),
                       O.q_ext_kh18(x, 10.0, 4.0), rtol=1e-15)
    capped = O.q_ext_with_feature(np.full(3, 1e-3), lam_pt, 10.0, 4.0, 5.0, lam0, om, 0.0)
    assert capped[1] == 2.0 and np.all(capped <= 2.0)


def test_gauss_jacobi_flux_rule_exactness():
    """Sect. 5's Gauss-Jacobi flux angles (reading: the 4-point Gaussian rule
    of int_0^1 f(mu) mu dmu): exact for f = mu^k, k <= 7, against the closed
    form int_0^1 mu^(k+1) dmu = 1/(k+2), and not for k = 8; nodes inside
    (0, 1), weights positive summing to 1/2; an isothermal column emits pi B
    under either rule."""
    mu, w = O.gauss_jacobi_mu_01(4)
    for k in range(8):
        assert np.sum(w * mu ** k) == pytest.approx(1.0 / (k + 2), rel=1e-13)
    assert abs(np.sum(w * mu ** 8) - 0.1) > 1e-6
    assert np.all((mu > 0) & (mu < 1)) and np.all(w > 0) and np.sum(w) == pytest.approx(0.5, rel=1e-15)
    b_lev = np.full((11, 3), 2.5)
    dtau = np.full((10, 3), 0.3)
    for quad in (O.QUAD_GAUSS_LEGENDRE, O.QUAD_GAUSS_JACOBI):
        assert np.allclose(O.emergent_flux(b_lev, dtau, quadrature=quad), np.pi * 2.5, rtol=1e-14)


@pytest.mark.parametrize("kind", [0, 1])
def test_slab_profiles_against_power_law_and_clear(kind):
    """Sect. 2.5.1's three q_c profiles checked against each other: the
    whole-column slab is the power law with alpha_c = 0 and its base below the
    model; a band that spans the column is the whole-column slab; a band that
    holds no layer pressure leaves the clear spectrum; and a band from above
    the model down to a pressure between two layers is the power law with
    alpha_c = 0 based at that pressure."""
    w, m, th, s, mem = _cloud_setup(kind)
    th[s + O.P_F_CLD] = 1.0
    slab = dataclasses.replace(m, cloud_profile=O.QC_SLAB)
    band = dataclasses.replace(m, cloud_profile=O.QC_SLAB_BAND)
    clear = dataclasses.replace(m, cloud_kind=O.CLOUD_NONE)
    t = th.copy()
    t[s + O.P_LOG_PC_BASE], t[s + O.P_ALPHA_C] = 5.0, 0.0
    ref_pl, _ = O.forward(m, w.tables, t, kind, mem)
    ref_slab, _ = O.forward(slab, w.tables, th, kind, mem)
    assert np.allclose(ref_slab, ref_pl, rtol=1e-14, atol=0)
    t = th.copy()
    t[s + O.P_LOG_PC_TOP], t[s + O.P_LOG_DPC] = -12.0, 5.0
    assert np.allclose(O.forward(band, w.tables, t, kind, mem)[0], ref_slab, rtol=1e-14, atol=0)
    p_lay = O.pressure_grid(m.n_layers, m.p_top_bar, m.p_bot_bar)[1]
    t = th.copy()   # a band strictly between two layer pressures
    lo, hi = np.log10(p_lay[40] / O.BAR), np.log10(p_lay[41] / O.BAR)
    t[s + O.P_LOG_PC_TOP] = lo + 0.2 * (hi - lo)
    t[s + O.P_LOG_DPC] = np.log10(0.5 * (p_lay[41] - p_lay[40]) / O.BAR)
    ref_clear, _ = O.forward(clear, w.tables, th, kind, mem)
    assert np.allclose(O.forward(band, w.tables, t, kind, mem)[0], ref_clear, rtol=1e-14, atol=0)
    # band from above the model down to a pressure between layers 60 and 61
    p_edge = np.sqrt(p_lay[60] * p_lay[61]) / O.BAR
    t = th.copy()
    t[s + O.P_LOG_PC_TOP] = -12.0
    t[s + O.P_LOG_DPC] = np.log10(p_edge - 1e-12)
    u = th.copy()
    u[s + O.P_LOG_PC_BASE], u[s + O.P_ALPHA_C] = np.log10(p_edge), 0.0
    got, _ = O.forward(band, w.tables, t, kind, mem)
    want, _ = O.forward(m, w.tables, u, kind, mem)
    assert np.allclose(got, want, rtol=1e-14, atol=0)
    assert np.max(np.abs(got / ref_slab - 1.0)) > 1e-6 and np.max(np.abs(got / ref_clear - 1.0)) > 1e-6


# ---------------------------------------------------------------- hydrostatics
def test_hydrostatic_isothermal_closed_form():
    """Isothermal, constant mu, g ~ 1/r^2: 1/r(p) = 1/R + k T ln(p/p_ref)/(mu m_u g R^2)
    exactly at every level, for any L and any p_ref (also off-grid)."""
    for L, p_ref in ((7, 10.0), (50, 3.3), (33, 1e-7)):
        p_lev, _ = O.pressure_grid(L, 1e-8, 100.0)
        t, mu, g, R = 1234.0, 2.37, 10 ** 3.2, 1.3 * O.R_JUP
        r, _ = O.altitude_grid(p_lev, np.full(L, t), mu, g, R, p_ref * O.BAR)
        inv = 1.0 / R + O.K_B * t * np.log(p_lev / (p_ref * O.BAR)) / (mu * O.AMU * g * R ** 2)
        assert np.allclose(r, 1.0 / inv, rtol=1e-13)


def test_hydrostatic_layered_profile_matches_ode():
    """Layer-wise temperatures: compare with a numerical integration of
    dr/d ln p = -k_B T(p) r^2 / (mu m_u g_ref R^2) through the piecewise-constant
    profile (pins which layer's temperature applies between which levels)."""
    from scipy.integrate import solve_ivp
    L = 12
    p_lev, _ = O.pressure_grid(L, 1e-6, 100.0)
    t_lay = np.linspace(600.0, 2400.0, L) + 200.0 * np.sin(np.arange(L))
    mu, g, R, p_ref = 2.3, 10 ** 2.9, 1.1 * O.R_JUP, 10.0 * O.BAR
    r, _ = O.altitude_grid(p_lev, t_lay, mu, g, R, p_ref)

    def temp(lnp):
        k = np.searchsorted(np.log(p_lev), lnp, side="right") - 1
        return t_lay[min(max(k, 0), L - 1)]

    for k in (0, 3, L):
        # integrate piecewise so that no step straddles a temperature jump
        a, b = np.log(p_ref), np.log(p_lev[k])
        inner = np.log(p_lev[(np.log(p_lev) > min(a, b)) & (np.log(p_lev) < max(a, b))])
        cuts = np.concatenate([[a], np.sort(inner)[::1 if b > a else -1], [b]])
        y = R
        for c0, c1 in zip(cuts[:-1], cuts[1:]):
            mid = 0.5 * (c0 + c1)
            sol = solve_ivp(lambda x, yy: [-O.K_B * temp(mid) * yy[0] ** 2 / (mu * O.AMU * g * R ** 2)],
                            (c0, c1), [y], rtol=1e-12, atol=1e-3)
            y = sol.y[0, -1]
        assert y == pytest.approx(r[k], rel=1e-10)


# ---------------------------------------------------------------- path matrix
def _radii(L=30):
    p_lev, _ = O.pressure_grid(L, 1e-6, 100.0)
    t_lay = np.linspace(900.0, 1600.0, L)
    r, _ = O.altitude_grid(p_lev, t_lay, 2.3, 1e3, O.R_JUP, 10.0 * O.BAR)
    return r


def test_path_matrix_row_sums_are_chord_lengths():
    """alpha = 1 everywhere: tau_i = sum_l P_il dr_l is the chord length above
    b_i, 2 sqrt(r_top^2 - b_i^2) (a telescoping sum)."""
    r = _radii()
    P, dr, b = O.path_matrix(r)
    assert np.allclose(P @ dr, 2.0 * np.sqrt(r[0] ** 2 - b ** 2), rtol=1e-10)
    # no path through layers below the impact parameter's layer
    assert np.all(np.triu(P[::-1, ::-1], 1) == 0) or np.all(np.tril(P, -1)[:, :] >= 0)
    assert np.all(P[np.triu_indices(len(dr), 1)] >= 0)
    assert np.all(P[np.tril_indices(len(dr), -1)[::-1]] >= 0)
    for i in range(len(dr)):
        assert np.all(P[i, i + 1:] == 0.0)


def test_path_matrix_brute_force_chord_march():
    """Random per-layer extinction: tau_i by marching along each chord in 2e5
    steps and summing the extinction of the shell containing each point."""
    r = _radii(8)
    P, dr, b = O.path_matrix(r)
    rng = np.random.default_rng(3)
    alpha = rng.uniform(0.1, 2.0, dr.size) * 1e-8
    tau = P @ (alpha * dr)
    for i in range(dr.size):
        smax = np.sqrt(r[0] ** 2 - b[i] ** 2)
        n = 200000
        s = (np.arange(n) + 0.5) * smax / n
        rad = np.sqrt(b[i] ** 2 + s ** 2)
        layer = np.searchsorted(-r, -rad, side="left") - 1      # r descending
        layer = np.clip(layer, 0, dr.size - 1)
        brute = 2.0 * np.sum(alpha[layer]) * smax / n
        assert tau[i] == pytest.approx(brute, rel=2e-5)


# ---------------------------------------------------------------- transmission
def _trans_setup(L, log10_sigma, deck=None, p_ref=10.0, p_bot=100.0, p_top=1e-6):
    m = _model(L=L, p_ref=p_ref, p_bot=p_bot, p_top=p_top,
               cloud=O.CLOUD_DECK if deck is not None else O.CLOUD_NONE)
    m.ray_h2_cm2 = m.ray_he_cm2 = 0.0
    nu = synth.nu_grid_constant_r(1.0, 2.0, 8)
    tabs = _flat_tables(nu, log10_sigma)
    th = m.theta_fixed.copy()
    th[0] = -3.0
    if deck is not None:
        th[m.n_species + O.P_LOG_PCLOUD] = deck
    mem = O.bin_members(nu, np.array([0.9]), np.array([2.1]))
    return m, tabs, th, mem


def test_zero_opacity_gives_bottom_disk():
    m, tabs, th, mem = _trans_setup(30, -99.0, p_ref=100.0)
    spec, y = O.forward(m, tabs, th, 0, mem)
    rp = th[m.n_species + O.P_R_P] * O.R_JUP
    assert np.allclose(spec, (rp / m.r_star_cm) ** 2, rtol=1e-14)   # (R_p/R_*)^2 when p_ref = p_bot


def test_opaque_limits_and_deck():
    m, tabs, th, mem = _trans_setup(30, -10.0)
    atm = O.atmosphere(m, th)
    spec, _ = O.forward(m, tabs, th, 0, mem)
    assert np.allclose(spec, (atm["r_lev"][0] / m.r_star_cm) ** 2, rtol=1e-12)
    m, tabs, th, mem = _trans_setup(30, -99.0, deck=-6.0)            # deck at p_top
    spec, _ = O.forward(m, tabs, th, 0, mem)
    assert np.allclose(spec, (O.atmosphere(m, th)["r_lev"][0] / m.r_star_cm) ** 2, rtol=1e-13)
    m1, tabs1, th1, mem1 = _trans_setup(30, -24.0, deck=2.0)         # deck at p_bot: no change
    m2, tabs2, th2, mem2 = _trans_setup(30, -24.0)
    assert np.allclose(O.forward(m1, tabs1, th1, 0, mem1)[0], O.forward(m2, tabs2, th2, 0, mem2)[0],
                       rtol=1e-14)


def test_deck_depth_continuous_in_pressure():
    vals = []
    for lp in (-2.0 - 1e-9, -2.0 + 1e-9):
        m, tabs, th, mem = _trans_setup(30, -25.0, deck=lp)
        vals.append(O.forward(m, tabs, th, 0, mem)[0][0])
    assert vals[0] == pytest.approx(vals[1], rel=1e-9)


def test_deck_radius_is_ln_p_interpolation_of_the_levels():
    """Grey deck reading: r_c = r(p_c) by ln p interpolation between the
    bounding levels. For an isothermal atmosphere 1/r is exactly linear in
    ln p (closed form), so ln-p interpolation of r matches the closed-form
    r(p_c) to its second-order error, at most dr^2 / (4 r) within a layer
    (r = 1/(a + b x) has r'' = 2 b^2 r^3); interpolation linear in p misses by
    a fixed fraction of dr. With zero opacity the transit depth is r_c^2 / R_*^2,
    so the deck's radius is also pinned through the forward model."""
    L = 12
    p_frac = (0.17, 0.5, 0.83)
    checked = 0
    for lp_layer in (4, 9):
        for f in p_frac:
            m, tabs, th, mem = _trans_setup(L, -99.0, deck=0.0)
            m.ray_h2_cm2 = m.ray_he_cm2 = 0.0
            p_lev, _ = O.pressure_grid(L, m.p_top_bar, m.p_bot_bar)
            lpc = (1 - f) * np.log10(p_lev[lp_layer] / O.BAR) + f * np.log10(p_lev[lp_layer + 1] / O.BAR)
            th[m.n_species + O.P_LOG_PCLOUD] = lpc
            atm = O.atmosphere(m, th)
            s = m.n_species
            t, g, R = th[s + O.P_T_ISO], atm["g"], atm["r_ref"]
            pc = 10.0 ** lpc * O.BAR
            r_exact = 1.0 / (1.0 / R + O.K_B * t * np.log(pc / (m.p_ref_bar * O.BAR)) / (atm["mu"] * O.AMU * g * R ** 2))
            r_lev = atm["r_lev"]
            dr = r_lev[lp_layer] - r_lev[lp_layer + 1]
            bound = dr * dr / (4.0 * r_lev[lp_layer + 1])
            r_c = O.deck_radius(r_lev, p_lev, pc)
            assert abs(r_c - r_exact) <= 1.01 * bound
            # linear in p misses by far more than the bound
            w_p = (pc - p_lev[lp_layer]) / (p_lev[lp_layer + 1] - p_lev[lp_layer])
            r_lin_p = r_lev[lp_layer] + w_p * (r_lev[lp_layer + 1] - r_lev[lp_layer])
            assert abs(r_lin_p - r_exact) > 20.0 * bound
            spec, _ = O.forward(m, tabs, th, 0, mem)
            assert np.allclose(spec, r_c ** 2 / m.r_star_cm ** 2, rtol=1e-13)
            assert np.allclose(spec, r_exact ** 2 / m.r_star_cm ** 2, rtol=2.2 * bound / r_exact)
            checked += 1
    assert checked == 6


def test_beer_lambert_single_layer():
    """One layer: the chord at the layer midpoint crosses it over
    s = 2 sqrt(r_up^2 - b^2) and transmits exp(-alpha s)."""
    m, tabs, th, mem = _trans_setup(1, -24.0, p_top=1e-3, p_bot=1e-2, p_ref=1e-2)
    atm = O.atmosphere(m, th)
    r_up, r_low = atm["r_lev"]
    b = 0.5 * (r_up + r_low)
    n = atm["p_lay"][0] / (O.K_B * atm["t_lay"][0])
    x_h2 = atm["x_h2"]
    alpha = n * 1e-3 * 1e-24
    s = 2.0 * np.sqrt(r_up ** 2 - b ** 2)
    expect = (r_low ** 2 + (r_up ** 2 - r_low ** 2) * (1.0 - np.exp(-alpha * s))) / m.r_star_cm ** 2
    spec, _ = O.forward(m, tabs, th, 0, mem)
    assert x_h2 > 0 and np.allclose(spec, expect, rtol=1e-12)


def _continuum_depth(m, th, log10_sigma):
    """Exact transit depth of the continuous isothermal atmosphere with
    constant cross-section, by nested Gauss-Legendre quadrature."""
    s = m.n_species
    atm = O.atmosphere(m, th)
    t = th[s + O.P_T_ISO]
    mu, g, R = atm["mu"], atm["g"], atm["r_ref"]
    p_ref = m.p_ref_bar * O.BAR
    coef = O.K_B * t / (mu * O.AMU * g * R ** 2)
    r_top, r_bot = atm["r_lev"][0], atm["r_lev"][-1]
    x = 10.0 ** th[0]

    def alpha(r):
        p = p_ref * np.exp((1.0 / r - 1.0 / R) / coef)
        return x * 10.0 ** log10_sigma * p / (O.K_B * t)

    gx, gw = np.polynomial.legendre.leggauss(16)

    def tau(b):
        tmax = np.sqrt(r_top - b)
        edges = np.linspace(0.0, tmax, 400)
        tt = (0.5 * (edges[1:] - edges[:-1])[:, None] * gx[None, :] + 0.5 * (edges[1:] + edges[:-1])[:, None])
        ww = 0.5 * (edges[1:] - edges[:-1])[:, None] * gw[None, :]
        rr = b + tt ** 2
        # tau(b) = 2 int_b alpha r dr / sqrt(r^2 - b^2), r = b + t^2
        return np.sum(ww * 4.0 * alpha(rr) * rr / np.sqrt(2.0 * b + tt ** 2))

    edges = np.linspace(r_bot, r_top, 1500)
    acc = 0.0
    for a0, a1 in zip(edges[:-1], edges[1:]):
        bb = 0.5 * (a1 - a0) * gx + 0.5 * (a1 + a0)
        acc += np.sum(0.5 * (a1 - a0) * gw * 2.0 * bb * (1.0 - np.exp(-np.array([tau(v) for v in bb]))))
    return (r_bot ** 2 + acc) / m.r_star_cm ** 2


@pytest.mark.slow
def test_transit_depth_converges_to_continuum():
    """Isothermal atmosphere with a constant cross-section: the discretised
    depth converges to the exact transmission integral of the continuous
    atmosphere. The square-root behaviour of the path length at the tangent
    layer makes the rate ~ (dr)^1.5 (error ratio ~2.9 per halving)."""
    lsig = -25.0
    m0, _, th0, _ = _trans_setup(20, lsig, p_top=1e-7)
    exact = _continuum_depth(m0, th0, lsig)
    errs = []
    for L in (50, 100, 200):
        m, tabs, th, mem = _trans_setup(L, lsig, p_top=1e-7)
        errs.append(abs(O.forward(m, tabs, th, 0, mem)[0][0] / exact - 1.0))
    assert errs[2] < 5e-5
    assert errs[0] / errs[1] > 2.5 and errs[1] / errs[2] > 2.5


def test_scale_height_law():
    """dR_eff/d ln sigma equals the pressure scale height at R_eff (to O(H/R))."""
    rads = []
    for lsig in (-25.0, -24.0):
        m, tabs, th, mem = _trans_setup(300, lsig, p_top=1e-9)
        rads.append(m.r_star_cm * np.sqrt(O.forward(m, tabs, th, 0, mem)[0][0]))
    atm = O.atmosphere(m, th)
    g_eff = atm["g"] * (atm["r_ref"] / np.mean(rads)) ** 2
    h = O.K_B * th[m.n_species + O.P_T_ISO] / (atm["mu"] * O.AMU * g_eff)
    slope = (rads[1] - rads[0]) / np.log(10.0)
    assert slope == pytest.approx(h, rel=2e-2)


# ---------------------------------------------------------------- interpolation
def test_interpolation_nodes_linear_and_clamp():
    rng = np.random.default_rng(1)
    t_grid = np.geomspace(300, 3000, 5)
    p_grid = np.geomspace(1e-6, 100, 4)
    tab = rng.uniform(-28, -20, (5, 4, 3))
    for it in range(5):
        for ip in range(4):
            v = O.log10_sigma_bilinear(tab, t_grid, p_grid, t_grid[it], p_grid[ip] * O.BAR)
            assert np.allclose(v, tab[it, ip], atol=1e-12)
    # a table linear in (log T, log p) is reproduced exactly everywhere
    a, bt, bp = -23.0, 1.7, -0.4
    lin = a + bt * np.log10(t_grid)[:, None, None] + bp * np.log10(p_grid)[None, :, None] + np.zeros(3)
    for t, p in ((777.0, 3e-3), (301.0, 99.0), (2999.0, 1.1e-6)):
        v = O.log10_sigma_bilinear(lin, t_grid, p_grid, t, p * O.BAR)
        assert np.allclose(v, a + bt * np.log10(t) + bp * np.log10(p), atol=1e-12)
    # clamping outside the table
    v_lo = O.log10_sigma_bilinear(tab, t_grid, p_grid, 10.0, 1e-12 * O.BAR)
    v_hi = O.log10_sigma_bilinear(tab, t_grid, p_grid, 9000.0, 1e4 * O.BAR)
    assert np.allclose(v_lo, tab[0, 0]) and np.allclose(v_hi, tab[-1, -1])


def test_cia_linear_in_temperature_between_nodes():
    """CIA reading: log10 k linear in T (not in log T) between the two
    bracketing nodes, clamped at both ends of the grid. A table linear in T is
    reproduced exactly at off-node temperatures; a hand-computed case
    (nodes 1000 K and 2000 K at -45 and -44, T = 1250 K: weight 1/4, -44.75)
    rules out a log-T weight (-44.678) and a swapped weight (-44.25)."""
    t_grid = np.array([400.0, 900.0, 1600.0, 3000.0])
    a, b = -46.0, 1.0e-3
    tab = a + b * t_grid[:, None] + np.array([0.0, 0.3, -0.2])[None, :]
    for t in (400.0, 777.0, 1234.5, 2222.2, 3000.0):
        v = O.log10_cia_linear(tab, t_grid, t)
        assert np.allclose(v, a + b * t + np.array([0.0, 0.3, -0.2]), atol=1e-13)
    assert np.array_equal(O.log10_cia_linear(tab, t_grid, 150.0), tab[0])
    assert np.array_equal(O.log10_cia_linear(tab, t_grid, 9000.0), tab[-1])
    two = np.array([[-45.0], [-44.0]])
    assert O.log10_cia_linear(two, np.array([1000.0, 2000.0]), 1250.0)[0] == pytest.approx(-44.75, abs=1e-14)
    # a table linear in log T is not reproduced between nodes (log-T interpolation would be)
    tab_log = -46.0 + 1.7 * np.log10(t_grid)[:, None]
    assert abs(O.log10_cia_linear(tab_log, t_grid, 1234.5)[0] - (-46.0 + 1.7 * np.log10(1234.5))) > 1e-3
    # through the extinction: n^2 X_H2 (X_H2 k_H2H2 + X_He k_H2He) with two
    # different tables (pins which table pairs with which background gas)
    m = _model(L=4)
    m.ray_h2_cm2 = m.ray_he_cm2 = 0.0
    nu = np.array([1.0e4, 2.0e4])
    tabs = _flat_tables(nu, -99.0)
    tabs.cia_t_grid = np.array([1000.0, 2000.0])
    tabs.cia_h2h2 = np.array([[-45.0, -44.0], [-44.0, -46.0]])
    tabs.cia_h2he = np.array([[-46.0, -45.5], [-45.0, -45.5]])
    x = np.array([1e-30])
    x_h2, x_he = O.background_fill(x)
    p = 3.0e5
    alpha = O.extinction(tabs, m, x, x_h2, x_he, np.array([1250.0]), np.array([p]))
    n = p / (O.K_B * 1250.0)
    k11 = 10.0 ** np.array([-44.75, -44.5])
    k12 = 10.0 ** np.array([-45.75, -45.5])
    assert np.allclose(alpha[0], n * n * x_h2 * (x_h2 * k11 + x_he * k12), rtol=1e-12)


def test_cia_and_rayleigh_scalings():
    """CIA extinction scales as n^2 (pressure squared at fixed T), Rayleigh as
    n nu^4: checked by doubling the pressure and the wavenumber."""
    m = _model(L=4)
    nu = np.array([1.0e4, 2.0e4])
    tabs = _flat_tables(nu, -99.0, cia=-45.0)
    x = np.array([1e-30])
    x_h2, x_he = O.background_fill(x)
    t = np.array([1000.0])
    m.ray_h2_cm2 = m.ray_he_cm2 = 0.0
    a1 = O.extinction(tabs, m, x, x_h2, x_he, t, np.array([1e5]))
    a2 = O.extinction(tabs, m, x, x_h2, x_he, t, np.array([2e5]))
    assert np.allclose(a2 / a1, 4.0, rtol=1e-12)
    n = 1e5 / (O.K_B * 1000.0)
    assert a1[0, 0] == pytest.approx(n * n * x_h2 * (x_h2 + x_he) * 1e-45, rel=1e-12)
    m = _model(L=4)
    tabs = _flat_tables(nu, -99.0, cia=-99.0)
    r1 = O.extinction(tabs, m, x, x_h2, x_he, t, np.array([1e5]))
    r2 = O.extinction(tabs, m, x, x_h2, x_he, t, np.array([2e5]))
    assert np.allclose(r2 / r1, 2.0, rtol=1e-12)
    assert r1[0, 1] / r1[0, 0] == pytest.approx(16.0, rel=1e-12)


# ---------------------------------------------------------------- emission
def test_gauss_legendre_matches_table():
    ref = np.loadtxt(os.path.join(GOLDEN, "gauss_legendre_4.txt"))
    mu, w = O.gauss_legendre_01(4)
    assert np.allclose(mu, 0.5 * (ref[:, 0] + 1.0), atol=1e-14)
    assert np.allclose(w, 0.5 * ref[:, 1], atol=1e-14)


def test_planck_integral_is_stefan_boltzmann():
    sig = dict(np.loadtxt(os.path.join(GOLDEN, "constants.txt"), dtype=str).reshape(-1, 2))
    sigma_sb = float(sig["sigma_sb"])
    for t in (300.0, 1500.0):
        nu = np.linspace(1e-3, 40.0 * t, 400001)
        b = O.planck_wavenumber(t, nu)
        integral = np.sum(0.5 * (b[1:] + b[:-1]) * np.diff(nu))
        assert integral == pytest.approx(sigma_sb * t ** 4 / np.pi, rel=1e-7)


def test_isothermal_emission_is_planck():
    m = _model(L=25)
    nu = synth.nu_grid_constant_r(1.0, 12.0, 50)
    rng = np.random.default_rng(5)
    tabs = _flat_tables(nu, -22.0)
    tabs.log10_sigma = rng.uniform(-28, -19, tabs.log10_sigma.shape)
    th = m.theta_fixed.copy()
    th[0] = -3.0
    mem = O.bin_members(nu, np.array([0.9]), np.array([13.0]))
    spec, _ = O.forward(m, tabs, th, 1, mem)
    t = th[m.n_species + O.P_T_ISO]
    rp = th[m.n_species + O.P_R_P] * O.R_JUP
    expect = O.planck_wavenumber(t, nu) / O.planck_wavenumber(m.t_star_k, nu) * (rp / m.r_star_cm) ** 2
    assert np.allclose(spec, expect, rtol=1e-12)


def test_linear_source_exact_solution():
    """Source linear in optical depth, B = a + b t, over total depth T:
    I_top(mu) = a + b mu (1 - e^{-T/mu}) exactly, so
    F = 2 pi sum_j w_j mu_j I_top(mu_j) from the tabulated GL nodes."""
    ref = np.loadtxt(os.path.join(GOLDEN, "gauss_legendre_4.txt"))
    mu_t, w_t = 0.5 * (ref[:, 0] + 1.0), 0.5 * ref[:, 1]
    a, bcoef = 2.0, 3.5
    dtau = np.array([1e-6, 3e-5, 0.02, 0.3, 1.7, 4.0, 0.9])[:, None] * np.ones((1, 3))
    t_edges = np.concatenate([[0.0], np.cumsum(dtau[:, 0])])
    b_lev = (a + bcoef * t_edges)[:, None] * np.ones((1, 3))
    total = t_edges[-1]
    expect = 2.0 * np.pi * np.sum(w_t * mu_t * (a + bcoef * mu_t * (1.0 - np.exp(-total / mu_t))))
    assert np.allclose(O.emergent_flux(b_lev, dtau), expect, rtol=1e-12)
    # deep limit: Eddington-Barbier, F = pi (a + 2 b / 3)
    deep = np.full((60, 1), 1.0)
    te = np.concatenate([[0.0], np.cumsum(deep[:, 0])])
    assert O.emergent_flux((a + bcoef * te)[:, None], deep)[0] == pytest.approx(np.pi * (a + 2 * bcoef / 3), rel=1e-12)


def test_linear_source_factor_series_matches_exact():
    x = np.array([2e-5, 9.9e-5, 1.01e-4, 1e-3])
    exact = np.array([float((1 - np.exp(-np.longdouble(v))) / np.longdouble(v) - np.exp(-np.longdouble(v)))
                      for v in x])
    assert np.allclose(O.linear_source_factor(x), exact, rtol=1e-10)


# ---------------------------------------------------------------- binning, likelihood
def test_binning_means():
    nu = synth.nu_grid_constant_r(1.0, 2.0, 101)
    lo, hi = synth.make_bins(nu, 7)
    mem = O.bin_members(nu, lo, hi)
    spec = np.arange(nu.size, dtype=float)
    y = O.bin_spectrum(spec, mem)
    lam = 1e4 / nu
    for k in range(7):
        pts = [spec[n] for n in range(nu.size) if lo[k] <= lam[n] < hi[k]]
        assert len(pts) > 0 and y[k] == pytest.approx(sum(pts) / len(pts), rel=1e-15)
    assert sum(len(m_) for m_ in mem) <= nu.size


def test_likelihood_closed_forms():
    rng = np.random.default_rng(0)
    sig = rng.uniform(1e-5, 1e-4, 50)
    y = rng.uniform(0, 1, 50)
    lnl = O.log_likelihood(y, y, sig, -99.0)
    assert lnl == pytest.approx(-np.sum(np.log(sig)) - 25.0 * np.log(2 * np.pi), rel=1e-14)
    # inflation: sigma_eff^2 = sigma^2 + 10^(2c)
    c = np.log10(3e-5)
    yo = y + 2e-5
    s_eff = np.sqrt(sig ** 2 + 9e-10)
    ref = np.sum(-np.log(s_eff) - 0.5 * np.log(2 * np.pi) - 0.5 * (2e-5 / s_eff) ** 2)
    assert O.log_likelihood(y, yo, sig, c) == pytest.approx(ref, rel=1e-13)
    # Gaussian normalisation: exp(lnL) integrates to 1 over one datum
    grid = np.linspace(-1.0, 1.0, 200001) * 1e-3
    dens = np.exp([O.log_likelihood(np.array([0.0]), np.array([v]), np.array([1e-4]), -99.0) for v in grid])
    assert np.sum(dens) * (grid[1] - grid[0]) == pytest.approx(1.0, rel=1e-6)


def test_invalid_outputs():
    w = synth.workload("tiny")
    m = w.model
    th = m.full_theta(w.theta)[0]
    mem = O.bin_members(w.tables.nu, w.bin_lo_um, w.bin_hi_um)
    bad = th.copy()
    bad[0] = np.log10(0.7)
    bad[1] = np.log10(0.5)          # sum X > 1
    assert O.loglike(m, w.tables, bad, 0, mem, w.y_obs[0], w.sigma[0]) == O.INVALID_LNL
    hot = th.copy()
    hot[m.n_species + O.P_T_ISO] = 2.0e6   # runaway inflation (1/r <= 0)
    assert O.loglike(m, w.tables, hot, 0, mem, w.y_obs[0], w.sigma[0]) == O.INVALID_LNL


# ---------------------------------------------------------------- gradient
@pytest.mark.parametrize("kind", [0, 1])
def test_complex_step_gradient_matches_central_differences(kind):
    w = synth.workload("jwst_plain", n_nu=400)
    m = w.model
    m.tp_kind = O.TP_GUILLOT_MOD
    m.cloud_kind = O.CLOUD_DECK
    s = m.n_species
    slots = list(range(s)) + [s + k for k in (O.P_T_INT, O.P_T_EQ, O.P_LOG_KAPPA, O.P_LOG_GAMMA,
                                               O.P_Q_IRR0, O.P_LOG_PT, O.P_BETA, O.P_LOG_G, O.P_R_P,
                                               O.P_C_INFL)]
    if kind == 0:
        slots.append(s + O.P_LOG_PCLOUD)
    else:
        slots.append(s + O.P_DILUTION)
    th = m.full_theta(w.theta)[0]
    th[s + O.P_LOG_PCLOUD] = -3.37
    th[s + O.P_Q_IRR0] = 0.3
    th[s + O.P_LOG_PT] = -1.3
    th[s + O.P_C_INFL] = -4.6
    th[s + O.P_DILUTION] = 0.9
    mem = O.bin_members(w.tables.nu, w.bin_lo_um, w.bin_hi_um)
    y_obs, sig = w.y_obs[kind], w.sigma[kind]
    g = O.loglike_gradient(m, w.tables, th, kind, mem, y_obs, sig, slots)
    for k, slot in enumerate(slots):
        h = 1e-5 * max(1.0, abs(th[slot]))
        a, b = th.copy(), th.copy()
        a[slot] += h
        b[slot] -= h
        fd = (O.loglike(m, w.tables, a, kind, mem, y_obs, sig)
              - O.loglike(m, w.tables, b, kind, mem, y_obs, sig)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=2e-5, abs=1e-6 * np.max(np.abs(g))), slot


def test_complex_step_gradient_brown_dwarf_milne():
    """Complex-step gradient of the brown-dwarf emission likelihood (modified
    Milne profile, mass and gravity through R_bd, dilution, inflation) against
    central differences."""
    w = synth.workload("browndwarf", n_nu=300, batch=2)
    m = w.model
    slots = list(m.free_idx)
    th = m.full_theta(w.theta)[0]
    mem = O.bin_members(w.tables.nu, w.bin_lo_um, w.bin_hi_um)
    y_obs, sig = w.y_obs[1], w.sigma[1]
    g = O.loglike_gradient(m, w.tables, th, 1, mem, y_obs, sig, slots)
    for k, slot in enumerate(slots):
        h = 1e-5 * max(1.0, abs(th[slot]))
        a, b = th.copy(), th.copy()
        a[slot] += h
        b[slot] -= h
        fd = (O.loglike(m, w.tables, a, 1, mem, y_obs, sig)
              - O.loglike(m, w.tables, b, 1, mem, y_obs, sig)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=2e-5, abs=1e-6 * np.max(np.abs(g))), slot


@pytest.mark.parametrize("kind,profile,feature", [(0, O.QC_POWER_LAW, 0), (1, O.QC_POWER_LAW, 0),
                                                  (0, O.QC_SLAB, 0), (1, O.QC_SLAB_BAND, 0),
                                                  (0, O.QC_POWER_LAW, 1), (1, O.QC_POWER_LAW, 1)])
def test_complex_step_gradient_cloud(kind, profile, feature):
    """Complex-step gradient of the non-grey cloud and cloud fraction (the
    cloud slots, radius, a VMR, a profile slot) against central differences,
    for the power-law and slab q_c profiles (the band's edges off the layer
    pressures, where lnL is flat in them) and with the mid-infrared feature
    (its four slots; the feature inside the band, below the Q_max cap)."""
    w, m, th, s, mem = _cloud_setup(kind)
    m = dataclasses.replace(m, cloud_profile=profile, cloud_feature=feature)
    th[s + O.P_LOG_PC_TOP], th[s + O.P_LOG_DPC] = -4.13, -0.61
    th[s + O.P_FEAT_A], th[s + O.P_FEAT_LAM0], th[s + O.P_FEAT_W], th[s + O.P_FEAT_XI] = 0.6, 3.0, 0.8, 2.5
    slots = [0, s + O.P_T_EQ, s + O.P_R_P] + [s + k for k in (O.P_LOG_QC, O.P_LOG_PC_BASE, O.P_ALPHA_C,
                                                              O.P_LOG_R_EFF, O.P_A_KH, O.P_LOG_Q0, O.P_F_CLD,
                                                              O.P_LOG_PC_TOP, O.P_LOG_DPC, O.P_FEAT_A,
                                                              O.P_FEAT_LAM0, O.P_FEAT_W, O.P_FEAT_XI)]
    y_obs, sig = w.y_obs[kind], w.sigma[kind]
    g = O.loglike_gradient(m, w.tables, th, kind, mem, y_obs, sig, slots)
    for k, slot in enumerate(slots):
        h = 1e-5 * max(1.0, abs(th[slot]))
        a, b = th.copy(), th.copy()
        a[slot] += h
        b[slot] -= h
        fd = (O.loglike(m, w.tables, a, kind, mem, y_obs, sig)
              - O.loglike(m, w.tables, b, kind, mem, y_obs, sig)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=2e-5, abs=1e-6 * np.max(np.abs(g))), slot


def test_bf16_row_dequantization_matches_library_rounding():
    """The BF16 table storage the oracle reproduces for parity: residuals about
    the FP32 row mean rounded to BF16 exactly as a library float32 -> bfloat16
    conversion rounds them (round to nearest even), the row offset equal to
    the row mean, and the error at most half a BF16 ulp of the residual."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    tab = (-24.0 + 3.0 * rng.standard_normal((2, 3, 4, 257))).astype(np.float32)
    deq = O.bf16_row_dequantized(tab)
    off = np.mean(tab.astype(np.float64), axis=-1).astype(np.float32)
    resid = (tab - off[..., None]).astype(np.float32)
    lib = torch.from_numpy(resid.copy()).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(deq, lib.astype(np.float64) + off[..., None].astype(np.float64))
    ulp = 2.0 ** (np.floor(np.log2(np.abs(resid.astype(np.float64)) + 1e-300)) - 7)
    assert np.all(np.abs(deq - tab.astype(np.float64)) <= 0.5 * ulp + 1e-12)
    ties = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.0 - 2.0 ** -8], np.float32)   # halfway cases
    row = np.concatenate([ties, -ties])[None, :]          # row mean exactly 0
    got = O.bf16_row_dequantized(row)[0, :3]
    np.testing.assert_array_equal(got, [1.0, 1.0 + 2.0 ** -6, -1.0])
