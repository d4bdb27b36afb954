"""Pins of the oracle's delta-EAA emission solver (Sect. 5, with scattering)
to results fixed independently of its code: the absorption-only solver where
nothing scatters, the invariants of the delta-M scaling, and the closed-form
first-order field of a homogeneous isothermal slab."""
import dataclasses
import os

import numpy as np
import pytest

from oracle import exoskry_oracle as O
from paper_2602_19687_gb300 import synth

QUADS = [O.QUAD_GAUSS_LEGENDRE, O.QUAD_GAUSS_JACOBI]


def synth_golden(name):
    return os.path.join(os.path.dirname(__file__), "golden", name)


def _column(rng, L=30, N=5):
    """Random layered column: Planck-like level sources and layer depths that
    span thin and thick layers."""
    b_lev = np.cumsum(rng.uniform(0.1, 1.0, (L + 1, N)), axis=0)
    d_abs = 10.0 ** rng.uniform(-5, 0.5, (L, N))
    d_ray = 10.0 ** rng.uniform(-4, -0.5, (L, N))
    d_cld = 10.0 ** rng.uniform(-4, 0.0, (L, N))
    return b_lev, d_abs, d_ray, d_cld


@pytest.mark.parametrize("quad", QUADS)
def test_eaa_without_scattering_is_the_absorption_solver(quad):
    """No scatterer (no Rayleigh depth, no cloud, or a cloud of zero albedo):
    delta-M leaves the depths alone, J and H never enter the source, and the
    delta-EAA flux is the absorption-only solver's on the absorbing depth."""
    rng = np.random.default_rng(3)
    b_lev, d_abs, d_ray, d_cld = _column(rng)
    zero = np.zeros_like(d_abs)
    ref = O.emergent_flux(b_lev, d_abs, quadrature=quad)
    assert np.allclose(O.emergent_flux_eaa(b_lev, d_abs, zero, zero, 0.8, 0.5, quadrature=quad), ref,
                       rtol=1e-13, atol=0)
    ref_c = O.emergent_flux(b_lev, d_abs + d_cld, quadrature=quad)
    assert np.allclose(O.emergent_flux_eaa(b_lev, d_abs, zero, d_cld, 0.0, 0.7, quadrature=quad), ref_c,
                       rtol=1e-13, atol=0)
    # and scattering changes it
    got = O.emergent_flux_eaa(b_lev, d_abs, d_ray, d_cld, 0.9, 0.6, quadrature=quad)
    assert np.max(np.abs(got / O.emergent_flux(b_lev, d_abs + d_ray + d_cld, quadrature=quad) - 1)) > 1e-3


def test_mean_intensity_weights():
    """At the Gauss-Legendre nodes the rule is Gauss-Legendre's (against the
    tabulated weights); at the Gauss-Jacobi nodes it integrates 1, mu, mu^2,
    mu^3 over [0, 1] exactly (the closed forms 1 / (k + 1))."""
    ref = np.loadtxt(synth_golden("gauss_legendre_4.txt"))
    mu_t, w_t = 0.5 * (ref[:, 0] + 1.0), 0.5 * ref[:, 1]
    order = np.argsort(mu_t)
    assert np.allclose(O.mean_intensity_weights(mu_t[order]), w_t[order], rtol=1e-13)
    mu, _ = O.flux_quadrature(O.QUAD_GAUSS_JACOBI, 4)
    c = O.mean_intensity_weights(mu)
    for k in range(4):
        assert np.sum(c * mu ** k) == pytest.approx(1.0 / (k + 1), rel=1e-13)


def test_delta_m_scaling_invariants():
    """delta-M moves the forward-peak fraction f of the scattering into the
    direct beam: the absorption depth (1 - omega) dtau is unchanged, the
    scattering depth becomes (1 - f) omega dtau, and omega dtau (1 - g) (the
    part scattered out of the forward peak, weighted by 1 - g) is unchanged.
    With f = g^2 these fix dtau', omega' and g' = g / (1 + g). Without a
    cloud (Rayleigh alone, g = 0) nothing is scaled."""
    rng = np.random.default_rng(11)
    _, d_abs, d_ray, d_cld = _column(rng)
    for w_c, g_c in [(0.9, 0.6), (0.3, 0.95), (1.0, 0.2)]:
        dts, om, gs = O.delta_m_scaling(d_abs, d_ray, d_cld, w_c, g_c)
        dsca = d_ray + w_c * d_cld
        g = w_c * g_c * d_cld / dsca
        assert np.allclose((1 - om) * dts, d_abs + (1 - w_c) * d_cld, rtol=1e-13)
        assert np.allclose(om * dts, (1 - g ** 2) * dsca, rtol=1e-13)
        assert np.allclose(om * dts * (1 - gs), dsca * (1 - g), rtol=1e-13)
        assert np.all((om >= 0) & (om <= 1)) and np.all((gs >= 0) & (gs < 0.5))
    dts, om, gs = O.delta_m_scaling(d_abs, d_ray, np.zeros_like(d_abs), 0.9, 0.6)
    assert np.allclose(dts, d_abs + d_ray, rtol=1e-15) and np.all(gs == 0)
    assert np.allclose(om, d_ray / (d_abs + d_ray), rtol=1e-14)
    # no scatterer at all: omega = g = 0
    dts, om, gs = O.delta_m_scaling(d_abs, np.zeros_like(d_abs), np.zeros_like(d_abs), 0.9, 0.6)
    assert np.all(om == 0) and np.all(gs == 0)


def _slab_closed_form(b, tau_s, om, gs, quad):
    """Emergent flux of the first-order field of a homogeneous isothermal slab
    (source B everywhere, I_up = B at its base, nothing incident at its top)
    of scaled depth tau_s, albedo om and asymmetry gs, in closed form.
    Zeroth order: I_up = B, I_dn(t, mu_j) = B (1 - exp(-k_j t)) with
    k_j = (1 - om) / mu_j; so J(t) = B - B/2 sum_j c_j e^{-k_j t},
    H(t) = B/2 sum_j a_j e^{-k_j t} and
    S(t, mu) = B - om B/2 sum_j (c_j - 3 gs mu a_j) e^{-k_j t}. Then
    I(0, mu) = B e^{-tau/mu} + int_0^tau S(t, mu) e^{-t/mu} dt / mu
             = B - om B/2 sum_j (c_j - 3 gs mu a_j) (1 - e^{-(k_j + 1/mu) tau}) / (1 + mu k_j)."""
    mu, a = O.flux_quadrature(quad, 4)
    c = O.mean_intensity_weights(mu)
    k = (1.0 - om) / mu
    flux = 0.0
    for i in range(4):
        m = mu[i]
        corr = np.sum((c - 3 * gs * m * a) * (1 - np.exp(-(k + 1 / m) * tau_s)) / (1 + m * k))
        flux += 2 * np.pi * a[i] * (b - 0.5 * om * b * corr)
    return flux


@pytest.mark.parametrize("quad", QUADS)
@pytest.mark.parametrize("case", [(0.4, 1.3, 0.0, 0.9, 0.6), (0.05, 0.2, 2.5, 0.95, 0.8), (1.5, 0.0, 0.8, 0.5, 0.3),
                                  (0.02, 3.0, 0.0, 0.0, 0.0)])
def test_eaa_isothermal_slab_matches_closed_form(quad, case):
    """A homogeneous isothermal slab cut into n equal layers: the solver's
    level values of the zeroth order are exact (constant source), its first
    order interpolates the source linearly in each layer, so it converges to
    the closed form at second order in the layer depth."""
    A, R, C, w_c, g_c = case
    b = 2.7
    dsca = R + w_c * C
    g = w_c * g_c * C / dsca if dsca > 0 else 0.0
    tau_s = (A + (1 - w_c) * C) + (1 - g * g) * dsca
    om = (1 - g * g) * dsca / tau_s
    gs = g / (1 + g)
    expect = _slab_closed_form(b, tau_s, om, gs, quad)
    errs = []
    for n in (200, 400):
        one = np.ones((n, 1)) / n
        got = O.emergent_flux_eaa(np.full((n + 1, 1), b), A * one, R * one, C * one, w_c, g_c, quadrature=quad)[0]
        errs.append(abs(got / expect - 1))
    assert errs[1] < 2e-6
    if errs[0] > 1e-11:   # second-order convergence (the error of the linear source interpolation)
        assert 3.2 < errs[0] / errs[1] < 4.8


def test_eaa_model_without_scatterers_is_the_absorption_model():
    """Model level: with zero Rayleigh cross-sections and a cloud of zero
    albedo the delta-EAA model equals the absorption-only model (clear and
    cloudy columns, cloud fraction, Planck sources, flux ratio)."""
    w = synth.workload("scattering_emis", n_nu=120, batch=2)
    m = dataclasses.replace(w.model, ray_h2_cm2=0.0, ray_he_cm2=0.0, cloud_ssa=0.0)
    th = m.full_theta(w.theta)[1]
    mem = O.bin_members(w.tables.nu, w.bin_lo_um, w.bin_hi_um)
    ref, _ = O.forward(dataclasses.replace(m, emission_solver=O.RT_ABSORPTION), w.tables, th, 1, mem)
    got, _ = O.forward(m, w.tables, th, 1, mem)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)
    # with its scatterers the model differs
    got2, _ = O.forward(w.model, w.tables, th, 1, mem)
    assert np.max(np.abs(got2 / ref - 1)) > 1e-3


def test_complex_step_gradient_eaa_matches_central_differences():
    """Complex-step gradient of the delta-EAA likelihood (VMRs, profile,
    gravity and the cloud slots) against central differences."""
    w = synth.workload("scattering_emis", n_nu=150, batch=2)
    m = w.model
    th = m.full_theta(w.theta)[0]
    s = m.n_species
    th[s + O.P_LOG_QC], th[s + O.P_LOG_PC_BASE], th[s + O.P_LOG_R_EFF] = -4.0, 0.5, -0.7
    mem = O.bin_members(w.tables.nu, w.bin_lo_um, w.bin_hi_um)
    slots = [0, 3, s + O.P_T_EQ, s + O.P_LOG_KAPPA, s + O.P_LOG_G, s + O.P_LOG_QC, s + O.P_ALPHA_C,
             s + O.P_LOG_R_EFF, s + O.P_A_KH, s + O.P_F_CLD]
    y_obs, sig = w.y_obs[1], w.sigma[1]
    g = O.loglike_gradient(m, w.tables, th, 1, mem, y_obs, sig, slots)
    for k, slot in enumerate(slots):
        h = 1e-5 * max(1.0, abs(th[slot]))
        a, b = th.copy(), th.copy()
        a[slot] += h
        b[slot] -= h
        fd = (O.loglike(m, w.tables, a, 1, mem, y_obs, sig) - O.loglike(m, w.tables, b, 1, mem, y_obs, sig)) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=2e-5, abs=1e-6 * np.max(np.abs(g))), slot
