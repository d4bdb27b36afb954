"""Seeded synthetic inputs for the forward model: wavenumber grids, cross-section
and CIA tables, instrument bins, observed spectra and parameter batches.

This module makes up input data only. It contains none of the forward model's
arithmetic (no temperature profile, hydrostatics, opacity interpolation,
radiative transfer, binning or likelihood), so that the FP64 oracle and the
CUDA library can both be fed from it without sharing any of the method.

Shapes follow the paper's workloads (Sect. 3: opacity-sampled tables on
temperature/pressure grids; Sect. 6: 100-layer atmospheres, log-VMR priors
U(-12,-2), Guillot-profile priors of Tables 4 and 6). The observational data
and HELIOS-k tables of the paper are not available; these generators stand in
for them.
"""
from __future__ import annotations

import dataclasses
import numpy as np

# Physical scale constants used to *describe* synthetic setups (units only).
R_JUP_CM = 7.1492e9
R_SUN_CM = 6.957e10

# Canonical parameter slots that follow the S log-VMR slots (same documented
# order as include/exoskry.h and the oracle).
P_T_ISO, P_T_INT, P_T_EQ, P_LOG_KAPPA, P_LOG_GAMMA, P_Q_IRR0, P_LOG_PT, P_BETA, \
    P_LOG_G, P_R_P, P_LOG_PCLOUD, P_C_INFL, P_DILUTION, P_T_RATIO, P_M_BD, \
    P_LOG_QC, P_LOG_PC_BASE, P_ALPHA_C, P_LOG_R_EFF, P_A_KH, P_LOG_Q0, P_F_CLD, \
    P_LOG_PC_TOP, P_LOG_DPC, P_FEAT_A, P_FEAT_LAM0, P_FEAT_W, P_FEAT_XI = range(28)
N_EXTRA = 28

TP_ISOTHERMAL, TP_GUILLOT, TP_GUILLOT_MOD, TP_MILNE = 0, 1, 2, 3
FLUX_PLANET_STAR, FLUX_BROWN_DWARF = 0, 1
PARSEC_CM = 3.0856775814913673e18
CLOUD_NONE, CLOUD_DECK, CLOUD_KH18 = 0, 1, 2
QC_POWER_LAW, QC_SLAB, QC_SLAB_BAND = 0, 1, 2
KIND_TRANSMISSION, KIND_EMISSION = 0, 1

SPECIES = {  # name: mass in amu
    "H2O": 18.015, "CO": 28.010, "CO2": 44.009, "CH4": 16.043,
    "NH3": 17.031, "H2S": 34.08, "SO2": 64.066, "K": 39.098,
}


@dataclasses.dataclass
class Model:
    """Static description of an atmosphere model (mirrors es_model_desc)."""
    n_layers: int
    p_top_bar: float
    p_bot_bar: float
    p_ref_bar: float
    tp_kind: int
    cloud_kind: int
    species: list
    masses_amu: np.ndarray
    r_star_cm: float
    t_star_k: float
    ray_h2_cm2: float
    ray_he_cm2: float
    ray_nu_ref: float
    theta_fixed: np.ndarray       # full canonical vector of defaults
    free_idx: np.ndarray          # canonical slots that the user vector fills
    emission_flux: int = FLUX_PLANET_STAR
    distance_cm: float = 0.0
    cloud_profile: int = QC_POWER_LAW
    cloud_feature: int = 0        # 1: the mid-infrared feature of the non-grey cloud
    emission_quadrature: int = 0  # 0: Gauss-Legendre, 1: Gauss-Jacobi flux angles
    emission_solver: int = 0      # 0: absorption-only RT, 1: delta-EAA with scattering
    cloud_ssa: float = 0.0        # delta-EAA: the cloud's single-scattering albedo
    cloud_g: float = 0.0          # delta-EAA: the cloud's asymmetry parameter

    @property
    def n_species(self):
        return len(self.species)

    @property
    def n_full(self):
        return self.n_species + N_EXTRA

    def full_theta(self, theta_free: np.ndarray) -> np.ndarray:
        """Scatter user (free) parameter rows into canonical full rows."""
        theta_free = np.atleast_2d(np.asarray(theta_free, dtype=np.float64))
        full = np.tile(self.theta_fixed, (theta_free.shape[0], 1))
        full[:, self.free_idx] = theta_free
        return full


@dataclasses.dataclass
class Tables:
    nu: np.ndarray            # [N] cm^-1 ascending
    t_grid: np.ndarray        # [NT] K ascending
    p_grid_bar: np.ndarray    # [NP] bar ascending
    log10_sigma: np.ndarray   # [S, NT, NP, N] float32, log10 cm^2
    cia_t_grid: np.ndarray    # [NTc] K ascending
    cia_h2h2: np.ndarray      # [NTc, N] float32, log10 cm^5
    cia_h2he: np.ndarray      # [NTc, N] float32, log10 cm^5


@dataclasses.dataclass
class Workload:
    name: str
    model: Model
    tables: Tables
    bin_lo_um: np.ndarray
    bin_hi_um: np.ndarray
    y_obs: dict               # kind -> [n_bins]
    sigma: dict               # kind -> [n_bins]
    theta: np.ndarray         # [B, n_free]
    kind: np.ndarray          # [B] int32
    table_dtype: str          # "f32" or "bf16"
    description: str


def nu_grid_constant_r(lam_min_um: float, lam_max_um: float, n: int) -> np.ndarray:
    """Log-uniform (constant resolving power) wavenumber grid, ascending."""
    nu_lo, nu_hi = 1.0e4 / lam_max_um, 1.0e4 / lam_min_um
    return nu_lo * (nu_hi / nu_lo) ** (np.arange(n) / (n - 1.0))


def _line_tables(nu, t_grid, p_grid_bar, species_seed, n_lines):
    """Seeded sums of Lorentzian lines on a -28..-20 log10 cm^2 baseline.

    Lines sit at random grid positions with log-uniform strengths over 5 dex,
    temperature scaling (T/296)^-1.5 exp(-E''(1/T - 1/296)) and a width (in
    grid points) that grows with pressure plus a Doppler-like floor. The
    convolution is done in Fourier space with the transform of a periodised
    Lorentzian, exp(-2 pi w |k| / M).
    """
    rng = np.random.default_rng(species_seed)
    n = nu.size
    centre = rng.integers(0, n, size=n_lines)
    s0 = 10.0 ** rng.uniform(-5.0, 0.0, size=n_lines)
    e_low = rng.uniform(0.0, 4000.0, size=n_lines)
    peak = rng.uniform(-21.2, -20.4)            # log10 of the strongest line peak
    cont = rng.uniform(-26.5, -25.0)            # pseudo-continuum level
    tilt = rng.uniform(-0.6, 0.6)
    m = 1 << int(np.ceil(np.log2(2 * n)))
    freq = np.abs(np.fft.rfftfreq(m) * m)
    x = np.linspace(-1.0, 1.0, n)
    out = np.empty((t_grid.size, p_grid_bar.size, n), dtype=np.float32)
    for it, t in enumerate(t_grid):
        strength = s0 * (t / 296.0) ** -1.5 * np.exp(-e_low * (1.0 / t - 1.0 / 296.0))
        hist = np.bincount(centre, weights=strength, minlength=n)
        hist = hist * (10.0 ** peak / strength.max())
        hk = np.fft.rfft(hist, m)
        cont_t = 10.0 ** (cont + tilt * x + 0.3 * np.log10(t / 1000.0))
        for ip, p in enumerate(p_grid_bar):
            w = 0.8 * p * np.sqrt(296.0 / t) + 0.15 * np.sqrt(t / 296.0)
            prof = np.fft.irfft(hk * np.exp(-2.0 * np.pi * w * freq / m), m)[:n]
            sig = np.maximum(prof, 0.0) + cont_t * (1.0 + 0.1 * np.log10(p + 1e-8) / 8.0)
            out[it, ip] = np.clip(np.log10(1e-28 + sig), -28.0, -20.0)
    return out


def _cia_table(nu, t_grid, seed):
    """Smooth seeded CIA table: log10 k in [-47, -43] cm^5, a few Gaussian
    bumps in wavenumber, linear in temperature."""
    rng = np.random.default_rng(seed)
    x = (nu - nu.min()) / max(nu.max() - nu.min(), 1.0)
    base = -46.2 + 0.6 * x
    for _ in range(3):
        c, w, a = rng.uniform(0.05, 0.95), rng.uniform(0.03, 0.15), rng.uniform(0.8, 2.0)
        base = base + a * np.exp(-0.5 * ((x - c) / w) ** 2)
    slope = rng.uniform(0.3, 0.7)
    tab = base[None, :] + slope * (t_grid[:, None] - 1500.0) / 2000.0
    return np.clip(tab, -47.0, -43.0).astype(np.float32)


def make_tables(nu, n_species, t_grid, p_grid_bar, seed_base=1000, line_frac=0.1):
    n_lines = max(8, int(nu.size * line_frac))
    sig = np.stack([_line_tables(nu, t_grid, p_grid_bar, seed_base + s, n_lines)
                    for s in range(n_species)])
    cia_t = np.geomspace(200.0, 4000.0, 12)
    return Tables(nu=nu, t_grid=np.asarray(t_grid, float), p_grid_bar=np.asarray(p_grid_bar, float),
                  log10_sigma=sig, cia_t_grid=cia_t,
                  cia_h2h2=_cia_table(nu, cia_t, seed_base + 101),
                  cia_h2he=_cia_table(nu, cia_t, seed_base + 102))


def make_bins(nu, n_bins):
    """Contiguous, equal-width-in-log-wavelength bins covering the grid's
    interior (edges in micron)."""
    lam = 1.0e4 / nu
    lo, hi = lam.min(), lam.max()
    pad = 0.25 * (np.log(hi) - np.log(lo)) / (nu.size - 1)
    edges = np.exp(np.linspace(np.log(lo) + pad, np.log(hi) - pad, n_bins + 1))
    return edges[:-1].copy(), edges[1:].copy()


def make_data(n_bins, kind, level, seed=7, rel_sigma=None):
    """Synthetic observed spectrum: a smooth seeded curve around `level`
    with Gaussian noise (30 ppm transmission, 50 ppm of Fp/F* emission, or
    rel_sigma x level for an absolute flux)."""
    rng = np.random.default_rng(seed + kind)
    x = np.linspace(0.0, 1.0, n_bins)
    smooth = sum(rng.uniform(-1, 1) * np.sin((k + 1) * np.pi * x + rng.uniform(0, 6.28))
                 for k in range(4))
    if kind == KIND_TRANSMISSION:
        sigma = np.full(n_bins, 30e-6)
        y = level * (1.0 + 0.004 * smooth)
    else:
        sigma = np.full(n_bins, 50e-6 if rel_sigma is None else rel_sigma * level)
        y = level * (1.0 + 0.3 * smooth / 4.0)
    return y + sigma * rng.standard_normal(n_bins), sigma


def _model(n_species, n_layers, p_top, p_bot, tp_kind, cloud_kind, free, fixed=None,
           species=None, r_star_rsun=1.0, t_star=5000.0, emission_flux=FLUX_PLANET_STAR, distance_pc=0.0):
    names = species or list(SPECIES)[:n_species]
    theta = np.zeros(n_species + N_EXTRA)
    theta[:n_species] = -8.0
    s = n_species
    theta[s + P_T_ISO] = 1000.0
    theta[s + P_T_INT] = 300.0
    theta[s + P_T_EQ] = 1200.0
    theta[s + P_LOG_KAPPA] = -2.0
    theta[s + P_LOG_GAMMA] = -1.0
    theta[s + P_Q_IRR0] = 2.0 / 3.0
    theta[s + P_LOG_PT] = -2.0
    theta[s + P_BETA] = 0.5
    theta[s + P_LOG_G] = 3.0
    theta[s + P_R_P] = 1.0
    theta[s + P_LOG_PCLOUD] = 3.0          # below the model bottom: no deck
    theta[s + P_C_INFL] = -99.0
    theta[s + P_DILUTION] = 1.0
    theta[s + P_T_RATIO] = 0.5
    theta[s + P_M_BD] = 70.0
    theta[s + P_LOG_QC] = -5.0
    theta[s + P_LOG_PC_BASE] = 0.0
    theta[s + P_ALPHA_C] = 1.0
    theta[s + P_LOG_R_EFF] = -0.5
    theta[s + P_A_KH] = 4.0
    theta[s + P_LOG_Q0] = 1.0
    theta[s + P_F_CLD] = 0.5
    theta[s + P_LOG_PC_TOP] = -3.0
    theta[s + P_LOG_DPC] = -1.0
    theta[s + P_FEAT_A] = 0.5
    theta[s + P_FEAT_LAM0] = 9.5
    theta[s + P_FEAT_W] = 1.5
    theta[s + P_FEAT_XI] = 2.0
    for k, v in (fixed or {}).items():
        theta[k] = v
    return Model(n_layers=n_layers, p_top_bar=p_top, p_bot_bar=p_bot, p_ref_bar=10.0,
                 tp_kind=tp_kind, cloud_kind=cloud_kind, species=names,
                 masses_amu=np.array([SPECIES[n] for n in names]),
                 r_star_cm=r_star_rsun * R_SUN_CM, t_star_k=t_star,
                 ray_h2_cm2=1.36e-27, ray_he_cm2=9.0e-29, ray_nu_ref=2.0e4,
                 theta_fixed=theta, free_idx=np.asarray(free, dtype=np.int64),
                 emission_flux=emission_flux, distance_cm=distance_pc * PARSEC_CM)


def _prior_batch(model, batch, seed, ranges):
    """Uniform-prior parameter vectors, one row per free slot of `model`."""
    rng = np.random.default_rng(seed)
    cols = [rng.uniform(*ranges[k], size=batch) for k in model.free_idx]
    return np.stack(cols, axis=1)


def prior_ranges(model):
    s = model.n_species
    r = {k: (-12.0, -2.0) for k in range(s)}
    r.update({s + P_T_ISO: (400.0, 2300.0), s + P_T_INT: (100.0, 600.0),
              s + P_T_EQ: (500.0, 2000.0), s + P_LOG_KAPPA: (-6.0, 2.0),
              s + P_LOG_GAMMA: (-4.0, 2.0), s + P_Q_IRR0: (0.0, 0.66),
              s + P_LOG_PT: (-7.0, 1.0), s + P_BETA: (0.0, 1.0),
              s + P_LOG_G: (2.7, 3.3), s + P_R_P: (0.9, 1.5),
              s + P_LOG_PCLOUD: (-6.0, 2.0), s + P_C_INFL: (-9.0, -4.0),
              s + P_DILUTION: (0.5, 1.0), s + P_T_RATIO: (0.2, 0.9),
              s + P_M_BD: (65.0, 78.0), s + P_LOG_QC: (-8.0, -3.0), s + P_LOG_PC_BASE: (-3.0, 1.0),
              s + P_ALPHA_C: (0.0, 2.0), s + P_LOG_R_EFF: (-2.0, 0.5), s + P_A_KH: (2.0, 6.0),
              s + P_LOG_Q0: (0.0, 2.0), s + P_F_CLD: (0.2, 1.0),
              s + P_LOG_PC_TOP: (-5.0, -1.0), s + P_LOG_DPC: (-3.0, 0.0),
              s + P_FEAT_A: (0.0, 1.5), s + P_FEAT_LAM0: (8.0, 11.0), s + P_FEAT_W: (0.5, 3.0),
              s + P_FEAT_XI: (-5.0, 5.0)})
    return r


def workload(name: str, batch: int | None = None, seed: int = 42,
             n_nu: int | None = None) -> Workload:
    """Named synthetic workloads.

    tiny        1 vector, L=50 (1e-6..100 bar), isothermal, 3 absorbers on
                10 T x 8 P x 2000 nu (0.5-5.5 um), CIA, grey deck, FP32.
    jwst_plain  1 vector, L=100 (1e-8..100 bar), Guillot (4 params),
                6 absorbers on 20 T (400-3000 K) x 15 P x 20000 nu
                (0.5-5.5 um), 300 bins, FP32.
    batched_trans 1024 vectors, 12 free parameters (6 log-VMR, 4 Guillot,
                cloud-deck pressure, radius), L=100, 8 absorbers on
                20 x 15 x 30000 nu, BF16 tables, 300 bins.
    batched_emis 512 emission vectors, 13 free parameters (8 log-VMR,
                4 Guillot, log g), L=100, 8 absorbers, 20000 nu (1-12 um),
                4 Gauss-Legendre angles, 400 bins, BF16 tables.
    highres     64 vectors, 10 free parameters (4 log-VMR, 4 Guillot,
                deck, radius), L=60, 4 absorbers on 12 x 10 x 440000 nu
                (0.9-5.3 um, R~250k), ~4400 bins of 100 points, BF16,
                mixed transmission/emission batch.
    cloudy_trans 1024 transmission vectors as batched_trans with the non-grey
                cloud (modified Fisher & Heng / Kitzmann & Heng Q_ext, base
                + power-law q_c profile) and a cloud fraction instead of the
                grey deck: 18 free parameters (6 log-VMR, 4 Guillot, radius,
                7 cloud).
    cloudy_emis 512 emission vectors as batched_emis with the non-grey cloud
                and cloud fraction: 20 free parameters (8 log-VMR, 4 Guillot,
                log g, 7 cloud); a clear and a cloudy column per wavenumber.
    scattering_emis 512 emission vectors as cloudy_emis solved with the
                delta-EAA (Sect. 5): H2/He Rayleigh and cloud scattering with a
                cloud single-scattering albedo of 0.9 and asymmetry parameter
                of 0.6 (constants of the model).
    browndwarf  256 brown-dwarf emission vectors shaped like the paper's
                Gliese 229 B setup: 15 free parameters (6 log-VMR, T_int,
                log kappa_ir, T_ratio, log p_t, beta of the modified Milne
                profile, log g, M_bd, s, c), L=100 (1e-8..1000 bar), 6
                absorbers on 20 T (300-3500 K) x 16 P x 54240 nu (1.0-5.1 um),
                absolute flux at D = 10 pc, 500 bins, BF16.
    `n_nu` shrinks the spectral grid (same physics) for fast tests.
    """
    S = {"tiny": 3, "jwst_plain": 6, "batched_trans": 8, "batched_emis": 8, "highres": 4,
         "browndwarf": 6, "cloudy_trans": 8, "cloudy_emis": 8, "scattering_emis": 8}[name]
    s = S
    if name == "tiny":
        n = n_nu or 2000
        model = _model(3, 50, 1e-6, 100.0, TP_ISOTHERMAL, CLOUD_DECK,
                       free=[0, 1, 2, s + P_T_ISO, s + P_R_P, s + P_LOG_PCLOUD],
                       species=["H2O", "CO", "CO2"])
        nu = nu_grid_constant_r(0.5, 5.5, n)
        tabs = make_tables(nu, 3, np.geomspace(300.0, 3000.0, 10), np.geomspace(1e-6, 100.0, 8))
        lo, hi = make_bins(nu, max(4, min(100, n // 20)))
        theta = np.array([[-3.0, -4.0, -5.0, 1000.0, 1.0, -2.0]])
        if batch and batch > 1:
            theta = np.vstack([theta, _prior_batch(model, batch - 1, seed, prior_ranges(model))])
        kind = np.zeros(theta.shape[0], np.int32)
        dtype, desc = "f32", "plain transmission, L=50, 3 absorbers, 10x8x2000 FP32, isothermal, deck"
        level = (R_JUP_CM / model.r_star_cm) ** 2
    elif name == "jwst_plain":
        n = n_nu or 20000
        free = list(range(6)) + [s + P_T_INT, s + P_T_EQ, s + P_LOG_KAPPA, s + P_LOG_GAMMA, s + P_R_P]
        model = _model(6, 100, 1e-8, 100.0, TP_GUILLOT, CLOUD_NONE, free=free)
        nu = nu_grid_constant_r(0.5, 5.5, n)
        tabs = make_tables(nu, 6, np.geomspace(400.0, 3000.0, 20), np.geomspace(1e-8, 100.0, 15))
        lo, hi = make_bins(nu, min(300, n // 10))
        rows = batch or 1
        theta = _prior_batch(model, rows, seed, prior_ranges(model))
        theta[0] = [-3.5, -4.0, -5.0, -6.0, -7.0, -5.5, 250.0, 1100.0, -2.5, -0.8, 1.2]
        kind = np.zeros(rows, np.int32)
        dtype, desc = "f32", "plain transmission, L=100, 6 absorbers, 20x15x20000 FP32, Guillot-4, 300 bins"
        level = (1.2 * R_JUP_CM / model.r_star_cm) ** 2
    elif name == "batched_trans":
        n = n_nu or 30000
        free = list(range(6)) + [s + P_T_INT, s + P_T_EQ, s + P_LOG_KAPPA, s + P_LOG_GAMMA,
                                 s + P_LOG_PCLOUD, s + P_R_P]
        model = _model(8, 100, 1e-8, 100.0, TP_GUILLOT, CLOUD_DECK, free=free)
        nu = nu_grid_constant_r(0.5, 5.5, n)
        tabs = make_tables(nu, 8, np.geomspace(400.0, 3000.0, 20), np.geomspace(1e-8, 100.0, 15))
        lo, hi = make_bins(nu, min(300, n // 10))
        rows = batch or 1024
        theta = _prior_batch(model, rows, seed, prior_ranges(model))
        kind = np.zeros(rows, np.int32)
        dtype, desc = "bf16", ("batched transmission likelihood, B=1024, L=100, 8 absorbers, "
                               "20x15x30000 BF16, Guillot-4, deck, 300 bins")
        level = (1.2 * R_JUP_CM / model.r_star_cm) ** 2
    elif name == "batched_emis":
        n = n_nu or 20000
        free = list(range(8)) + [s + P_T_INT, s + P_T_EQ, s + P_LOG_KAPPA, s + P_LOG_GAMMA, s + P_LOG_G]
        model = _model(8, 100, 1e-8, 100.0, TP_GUILLOT, CLOUD_NONE, free=free, r_star_rsun=0.765)
        nu = nu_grid_constant_r(1.0, 12.0, n)
        tabs = make_tables(nu, 8, np.geomspace(400.0, 3000.0, 20), np.geomspace(1e-8, 100.0, 15))
        lo, hi = make_bins(nu, min(400, n // 10))
        rows = batch or 512
        theta = _prior_batch(model, rows, seed, prior_ranges(model))
        kind = np.ones(rows, np.int32)
        dtype, desc = "bf16", ("batched emission with adjoint, B=512, L=100, 8 absorbers, "
                               "20x15x20000 BF16 (1-12 um), 4 GL angles, 400 bins")
        level = 2.0e-3
    elif name in ("cloudy_emis", "scattering_emis"):
        n = n_nu or 20000
        free = list(range(8)) + [s + P_T_INT, s + P_T_EQ, s + P_LOG_KAPPA, s + P_LOG_GAMMA, s + P_LOG_G,
                                 s + P_LOG_QC, s + P_LOG_PC_BASE, s + P_ALPHA_C, s + P_LOG_R_EFF,
                                 s + P_A_KH, s + P_LOG_Q0, s + P_F_CLD]
        model = _model(8, 100, 1e-8, 100.0, TP_GUILLOT, CLOUD_KH18, free=free, r_star_rsun=0.765)
        nu = nu_grid_constant_r(1.0, 12.0, n)
        tabs = make_tables(nu, 8, np.geomspace(400.0, 3000.0, 20), np.geomspace(1e-8, 100.0, 15))
        lo, hi = make_bins(nu, min(400, n // 10))
        rows = batch or 512
        theta = _prior_batch(model, rows, seed, prior_ranges(model))
        kind = np.ones(rows, np.int32)
        dtype, desc = "bf16", ("batched emission with a non-grey cloud and cloud fraction, with adjoint, B=512, "
                               "L=100, 8 absorbers, 20x15x20000 BF16 (1-12 um), 4 GL angles, 400 bins")
        if name == "scattering_emis":
            model.emission_solver, model.cloud_ssa, model.cloud_g = 1, 0.9, 0.6
            desc = ("batched delta-EAA emission (Rayleigh and cloud scattering, omega_c = 0.9, g_c = 0.6) "
                    "with adjoint, B=512, L=100, 8 absorbers, 20x15x20000 BF16 (1-12 um), 4 GL angles, 400 bins")
        level = 2.0e-3
    elif name == "highres":
        n = n_nu or 440000
        free = list(range(4)) + [s + P_T_INT, s + P_T_EQ, s + P_LOG_KAPPA, s + P_LOG_GAMMA,
                                 s + P_LOG_PCLOUD, s + P_R_P]
        model = _model(4, 60, 1e-8, 100.0, TP_GUILLOT, CLOUD_DECK, free=free,
                       species=["H2O", "CO", "CO2", "CH4"])
        nu = nu_grid_constant_r(0.9, 5.3, n)
        tabs = make_tables(nu, 4, np.geomspace(400.0, 3000.0, 12), np.geomspace(1e-8, 100.0, 10),
                           line_frac=0.05)
        lo, hi = make_bins(nu, max(4, n // 100))
        rows = batch or 64
        theta = _prior_batch(model, rows, seed, prior_ranges(model))
        kind = (np.arange(rows) % 2).astype(np.int32)     # mixed batch
        dtype, desc = "bf16", ("high-resolution mixed batch with adjoint, B=64, L=60, 4 absorbers, "
                               "12x10x440000 BF16 (0.9-5.3 um), ~4400 bins")
        level = (1.2 * R_JUP_CM / model.r_star_cm) ** 2
    elif name == "cloudy_trans":
        n = n_nu or 30000
        free = list(range(6)) + [s + P_T_INT, s + P_T_EQ, s + P_LOG_KAPPA, s + P_LOG_GAMMA, s + P_R_P,
                                 s + P_LOG_QC, s + P_LOG_PC_BASE, s + P_ALPHA_C, s + P_LOG_R_EFF,
                                 s + P_A_KH, s + P_LOG_Q0, s + P_F_CLD]
        model = _model(8, 100, 1e-8, 100.0, TP_GUILLOT, CLOUD_KH18, free=free)
        nu = nu_grid_constant_r(0.5, 5.5, n)
        tabs = make_tables(nu, 8, np.geomspace(400.0, 3000.0, 20), np.geomspace(1e-8, 100.0, 15))
        lo, hi = make_bins(nu, min(300, n // 10))
        rows = batch or 1024
        theta = _prior_batch(model, rows, seed, prior_ranges(model))
        kind = np.zeros(rows, np.int32)
        dtype, desc = "bf16", ("batched transmission with a non-grey cloud and cloud fraction, B=1024, L=100, "
                               "8 absorbers, 20x15x30000 BF16, Guillot-4, 300 bins")
        level = (1.2 * R_JUP_CM / model.r_star_cm) ** 2
    elif name == "browndwarf":
        n = n_nu or 54240
        free = list(range(6)) + [s + P_T_INT, s + P_LOG_KAPPA, s + P_T_RATIO, s + P_LOG_PT, s + P_BETA,
                                 s + P_LOG_G, s + P_M_BD, s + P_DILUTION, s + P_C_INFL]
        model = _model(6, 100, 1e-8, 1000.0, TP_MILNE, CLOUD_NONE, free=free,
                       species=["H2O", "CO", "CH4", "NH3", "H2S", "K"],
                       emission_flux=FLUX_BROWN_DWARF, distance_pc=10.0)
        nu = nu_grid_constant_r(1.0, 5.1, n)
        tabs = make_tables(nu, 6, np.geomspace(300.0, 3500.0, 20), np.geomspace(1e-8, 1000.0, 16))
        lo, hi = make_bins(nu, min(500, n // 10))
        rows = batch or 256
        ranges = prior_ranges(model)
        ranges.update({s + P_T_INT: (800.0, 1400.0), s + P_LOG_KAPPA: (-3.0, -1.0),
                       s + P_LOG_PT: (-2.0, 2.0), s + P_BETA: (0.3, 1.0), s + P_LOG_G: (4.8, 5.4),
                       s + P_C_INFL: (-16.0, -15.0)})
        theta = _prior_batch(model, rows, seed, ranges)
        kind = np.ones(rows, np.int32)
        dtype, desc = "bf16", ("brown-dwarf emission with adjoint, B=256, L=100, 6 absorbers, "
                               "20x16x54240 BF16 (1.0-5.1 um), modified Milne, flux at 10 pc, 500 bins")
        level = 2.0e-15
    else:
        raise KeyError(name)
    y_obs, sigma = {}, {}
    nb = lo.size
    emis_only = name in ("batched_emis", "cloudy_emis", "scattering_emis")
    y_obs[KIND_TRANSMISSION], sigma[KIND_TRANSMISSION] = make_data(nb, KIND_TRANSMISSION,
                                                                   0.014 if emis_only else level)
    if name == "browndwarf":
        y_obs[KIND_EMISSION], sigma[KIND_EMISSION] = make_data(nb, KIND_EMISSION, level, rel_sigma=0.05)
    else:
        y_obs[KIND_EMISSION], sigma[KIND_EMISSION] = make_data(nb, KIND_EMISSION, 2.0e-3)
    return Workload(name=name, model=model, tables=tabs, bin_lo_um=lo, bin_hi_um=hi,
                    y_obs=y_obs, sigma=sigma, theta=theta, kind=kind, table_dtype=dtype,
                    description=desc)
