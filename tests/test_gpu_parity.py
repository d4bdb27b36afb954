"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element
by element, on seeded synthetic workloads (several tiles and a ragged tail),
at the full batched size on sampled outputs, and on the edge cases.

Tolerances (FP32 path vs FP64): native transit depth 1e-5 relative; emergent
Fp/F* 1e-4 relative; ln L 1e-5 relative; gradient 1e-3 relative per component
with a floor of 1e-4 of the largest component (the adjoint sums FP32 products
over ~1e4 wavenumbers; measured: at most 2.2e-4 relative on the components
above 1% of the largest). BF16-table workloads are compared with the oracle run
on the same dequantized table values.
"""
import copy
import dataclasses

import numpy as np
import pytest

from oracle import exoskry_oracle as O
from paper_2602_19687_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def oracle_tables(w):
    if w.table_dtype != "bf16":
        return w.tables
    t = copy.copy(w.tables)
    t.log10_sigma = O.bf16_row_dequantized(w.tables.log10_sigma)
    return t


def gpu_eval(ctx, w, theta, kind, backward=True):
    B, N, nb = theta.shape[0], w.tables.nu.size, w.bin_lo_um.size
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    kd = torch.tensor(kind, dtype=torch.int32, device=DEV)
    ctx.es_set_batch(th, kd)
    spec = torch.empty((B, N), dtype=torch.float32, device=DEV)
    binned = torch.empty((B, nb), dtype=torch.float64, device=DEV)
    lnl = torch.empty(B, dtype=torch.float64, device=DEV)
    ctx.es_forward(spectrum=spec, binned=binned, lnl=lnl)
    out = dict(spec=spec.cpu().numpy().astype(np.float64), binned=binned.cpu().numpy(), lnl=lnl.cpu().numpy())
    if backward:
        lnl2 = torch.empty_like(lnl)
        grad = torch.empty_like(th)
        ctx.es_forward_backward(lnl2, grad)
        out["lnl2"] = lnl2.cpu().numpy()
        out["grad"] = grad.cpu().numpy()
    flags = torch.empty(B, dtype=torch.int32, device=DEV)
    ctx.es_get_flags(flags)
    out["flags"] = flags.cpu().numpy()
    torch.cuda.synchronize()
    assert ctx.es_query(11) == 0, "a tensor-core kernel gave up on a bounded wait"
    return out


def oracle_eval(w, tabs, theta_row, kind, grad=False):
    m = w.model
    th = m.full_theta(theta_row)[0]
    mem = O.bin_members(tabs.nu, w.bin_lo_um, w.bin_hi_um)
    out = O.forward(m, tabs, th, kind, mem)
    res = {"valid": out is not None}
    if out is not None:
        res["spec"], res["binned"] = out
    res["lnl"] = O.loglike(m, tabs, th, kind, mem, w.y_obs[kind], w.sigma[kind])
    if grad:
        res["grad"] = O.loglike_gradient(m, tabs, th, kind, mem, w.y_obs[kind], w.sigma[kind],
                                         list(m.free_idx))
    return res


def assert_spec(got, ref, kind):
    if kind == 0:
        np.testing.assert_allclose(got, ref, rtol=1e-5, atol=0)
    else:
        np.testing.assert_allclose(got, ref, rtol=1e-4, atol=1e-7 * np.max(np.abs(ref)))


def assert_grad(got, ref):
    tol = 1e-3 * np.abs(ref) + 1e-4 * np.max(np.abs(ref))
    bad = np.abs(got - ref) > tol
    assert not bad.any(), "gradient mismatch:\n gpu %s\n ref %s" % (got, ref)


def check_sample(out, b, ref, kind, grad=True):
    assert out["flags"][b] == 0
    assert_spec(out["spec"][b], ref["spec"], kind)
    # emission: as for the native flux, an absolute floor of 1e-7 of the largest
    # binned value (cold layers' flux at high wavenumber is far below FP32 range)
    np.testing.assert_allclose(out["binned"][b], ref["binned"], rtol=1e-5 if kind else 1e-6,
                               atol=1e-7 * np.max(np.abs(ref["binned"])) if kind else 0.0)
    np.testing.assert_allclose(out["lnl"][b], ref["lnl"], rtol=1e-5, atol=1e-3)
    np.testing.assert_allclose(out["lnl2"][b], out["lnl"][b], rtol=1e-12)
    if grad:
        assert_grad(out["grad"][b], ref["grad"])


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


# ------------------------------------------------------------------ small workloads
@pytest.mark.parametrize("kind", [0, 1])
def test_tiny_transmission_and_emission(kind):
    w = synth.workload("tiny")
    theta = w.theta.copy()
    theta[0, 5] = -2.37           # deck off a level (no kink at the FD/complex-step point)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, theta, np.array([kind], np.int32))
    ref = oracle_eval(w, w.tables, theta[0], kind, grad=True)
    check_sample(out, 0, ref, kind)


@pytest.mark.parametrize("kind", [0, 1])
def test_temperatures_and_pressures_outside_the_table_grid(kind):
    """Layers beyond the tables' pressure range (the model spans 1e-8..1e3 bar,
    the cross-section tables 1e-6..1e2 bar) and isothermal temperatures above
    and below both temperature grids (cross-sections 300-3000 K, CIA
    200-4000 K): the device clamps every bracket as the oracle does, and the
    gradient has no derivative along a clamped coordinate (the oracle's
    complex step sees none there either)."""
    w = synth.workload("tiny", batch=3)
    w.model = dataclasses.replace(w.model, p_top_bar=1e-8, p_bot_bar=1e3)
    theta = np.array([[-3.0, -4.0, -5.0, t, 1.0, -2.37] for t in (4500.0, 150.0, 1500.0)])
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, theta, np.full(3, kind, np.int32))
    for b in range(3):
        ref = oracle_eval(w, w.tables, theta[b], kind, grad=True)
        check_sample(out, b, ref, kind)


def test_jwst_plain_reduced_grid():
    w = synth.workload("jwst_plain", n_nu=3000)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, np.zeros(1, np.int32))
    ref = oracle_eval(w, w.tables, w.theta[0], 0, grad=True)
    check_sample(out, 0, ref, 0)


def test_batched_transmission_bf16_small():
    w = synth.workload("batched_trans", batch=6, n_nu=2500)
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    kind = np.zeros(6, np.int32)
    out = gpu_eval(ctx, w, w.theta, kind)
    for b in range(6):
        ref = oracle_eval(w, tabs, w.theta[b], 0, grad=(b < 2))
        if not ref["valid"]:
            assert out["lnl"][b] == O.INVALID_LNL and np.all(out["grad"][b] == 0)
            continue
        check_sample(out, b, ref, 0, grad=(b < 2))


def test_batched_emission_bf16_small():
    w = synth.workload("batched_emis", batch=4, n_nu=2000)
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, np.ones(4, np.int32))
    for b in range(4):
        ref = oracle_eval(w, tabs, w.theta[b], 1, grad=(b < 2))
        if not ref["valid"]:
            assert out["lnl"][b] == O.INVALID_LNL
            continue
        check_sample(out, b, ref, 1, grad=(b < 2))


def test_brown_dwarf_milne_emission():
    """Modified Milne profile (Sect. 2.4.3) and the absolute brown-dwarf flux
    at distance D with R_bd = sqrt(G M_bd / g) (Sect. 5): spectra, ln L and the
    gradient with respect to all 15 free parameters of the Gliese 229 B-shaped
    setup."""
    w = synth.workload("browndwarf", batch=4, n_nu=2000)
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, np.ones(4, np.int32))
    for b in range(4):
        ref = oracle_eval(w, tabs, w.theta[b], 1, grad=(b < 2))
        assert ref["valid"]
        check_sample(out, b, ref, 1, grad=(b < 2))


def test_gauss_jacobi_flux_angles():
    """The brown-dwarf setup with the Gauss-Jacobi flux angles of Sect. 5
    (the 4-point rule of the weight mu): spectra, ln L and gradients."""
    w = synth.workload("browndwarf", batch=3, n_nu=2000)
    w.model = dataclasses.replace(w.model, emission_quadrature=1)
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, np.ones(3, np.int32))
    for b in range(3):
        ref = oracle_eval(w, tabs, w.theta[b], 1, grad=(b < 2))
        assert ref["valid"]
        check_sample(out, b, ref, 1, grad=(b < 2))


def test_cloudy_transmission():
    """Non-grey cloud (Sect. 2.5, base + power-law q_c, KH18 Q_ext) and cloud
    fraction: transit depth element by element, binned model, ln L, and the
    gradient with respect to all 18 free parameters (7 of them the cloud's)."""
    w = synth.workload("cloudy_trans", batch=6, n_nu=3000)
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, np.zeros(6, np.int32))
    for b in range(6):
        ref = oracle_eval(w, tabs, w.theta[b], 0, grad=(b < 3))
        assert ref["valid"]
        check_sample(out, b, ref, 0, grad=(b < 3))


def test_cloudy_emission():
    """Non-grey cloud and cloud fraction in emission (Sect. 2.5 with Sect. 5):
    a clear and a cloudy column per wavenumber, mixed by f_cld; Fp/F* element
    by element, binned model, ln L and the gradient with respect to all 20
    free parameters (7 of them the cloud's)."""
    w = synth.workload("cloudy_emis", batch=4, n_nu=2000)
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, np.ones(4, np.int32))
    for b in range(4):
        ref = oracle_eval(w, tabs, w.theta[b], 1, grad=(b < 2))
        if not ref["valid"]:
            assert out["lnl"][b] == O.INVALID_LNL
            continue
        check_sample(out, b, ref, 1, grad=(b < 2))


@pytest.mark.parametrize("kind", [0, 1])
def test_cloud_mid_infrared_feature(kind):
    """The non-grey cloud with the mid-infrared feature of Sect. 2.5.3 (skew-
    normal Q_feat, size window, Q_max cap) placed inside the band: spectra,
    ln L and the gradient with respect to 22 free parameters, the feature's
    four among them."""
    w = synth.workload("cloudy_trans", batch=3, n_nu=2000)
    s = w.model.n_species
    feat = [s + synth.P_FEAT_A, s + synth.P_FEAT_LAM0, s + synth.P_FEAT_W, s + synth.P_FEAT_XI]
    w.model = dataclasses.replace(w.model, cloud_feature=1, free_idx=np.concatenate([w.model.free_idx, feat]))
    rng = np.random.default_rng(5)
    w.theta = np.hstack([w.theta, np.column_stack([rng.uniform(0.2, 1.0, 3), rng.uniform(1.5, 4.5, 3),
                                                   rng.uniform(0.4, 1.2, 3), rng.uniform(-4.0, 4.0, 3)])])
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, np.full(3, kind, np.int32))
    for b in range(3):
        ref = oracle_eval(w, tabs, w.theta[b], kind, grad=True)
        assert ref["valid"]
        check_sample(out, b, ref, kind)


@pytest.mark.parametrize("profile", [synth.QC_SLAB, synth.QC_SLAB_BAND])
def test_cloud_slab_profiles_mixed_batch(profile):
    """The whole-column slab and the slab band of Sect. 2.5.1 on a mixed
    transmission / emission batch with the non-grey cloud: spectra, ln L and
    gradients (zero along the power law's slots, which these profiles do not
    use)."""
    w = synth.workload("cloudy_trans", batch=4, n_nu=2000)
    s = w.model.n_species
    fixed = w.model.theta_fixed.copy()
    fixed[s + synth.P_LOG_PC_TOP], fixed[s + synth.P_LOG_DPC] = -4.13, -0.61
    w.model = dataclasses.replace(w.model, cloud_profile=profile, theta_fixed=fixed)
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    kind = np.array([0, 1, 0, 1], np.int32)
    out = gpu_eval(ctx, w, w.theta, kind)
    for b in range(4):
        ref = oracle_eval(w, tabs, w.theta[b], int(kind[b]), grad=True)
        assert ref["valid"]
        check_sample(out, b, ref, int(kind[b]))


def test_mixed_batch_highres_shape():
    w = synth.workload("highres", batch=4, n_nu=6000)
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, w.kind)
    for b in range(4):
        ref = oracle_eval(w, tabs, w.theta[b], int(w.kind[b]), grad=(b < 2))
        if not ref["valid"]:
            assert out["lnl"][b] == O.INVALID_LNL
            continue
        check_sample(out, b, ref, int(w.kind[b]), grad=(b < 2))


# ------------------------------------------------------------------ edge cases
def test_invalid_samples_get_minus_1e300_and_zero_gradient():
    w = synth.workload("tiny")
    theta = np.repeat(w.theta, 3, axis=0)
    theta[1, 0], theta[1, 1] = np.log10(0.7), np.log10(0.5)     # sum X > 1
    theta[2, 3] = 2.0e6                                         # runaway hydrostatics
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, theta, np.zeros(3, np.int32))
    assert out["flags"].tolist() == [0, 1, 1]
    assert out["lnl"][1] == O.INVALID_LNL and out["lnl"][2] == O.INVALID_LNL
    assert np.all(out["grad"][1:] == 0.0)
    assert np.isfinite(out["lnl"][0])


def test_deck_limits():
    w = synth.workload("tiny")
    theta = np.repeat(w.theta, 2, axis=0)
    theta[0, 5] = -12.0            # deck above the top: the whole atmosphere is opaque
    theta[1, 5] = 5.0              # deck below the bottom: no deck
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, theta, np.zeros(2, np.int32), backward=False)
    atm = O.atmosphere(w.model, w.model.full_theta(theta[0])[0])
    np.testing.assert_allclose(out["spec"][0], (atm["r_lev"][0] / w.model.r_star_cm) ** 2, rtol=1e-7)
    ref = oracle_eval(w, w.tables, theta[1], 0)
    assert_spec(out["spec"][1], ref["spec"], 0)


def test_maximum_layers_and_species():
    w = synth.workload("tiny", n_nu=700)
    m = w.model
    S = 16
    names = (list(synth.SPECIES) * 2)[:S]
    model = synth._model(S, 112, 1e-7, 100.0, synth.TP_GUILLOT_MOD, synth.CLOUD_DECK,
                         free=list(range(S)) + [S + k for k in (synth.P_T_INT, synth.P_T_EQ, synth.P_Q_IRR0,
                                                                synth.P_LOG_PT, synth.P_BETA, synth.P_LOG_G,
                                                                synth.P_R_P, synth.P_LOG_PCLOUD, synth.P_C_INFL)],
                         species=names)
    w.model = model
    w.tables = synth.make_tables(w.tables.nu, S, np.geomspace(300, 3000, 7), np.geomspace(1e-7, 100, 6))
    rng = np.random.default_rng(11)
    theta = np.concatenate([rng.uniform(-8, -4, S), [300.0, 1300.0, 0.3, -1.5, 0.6, 3.1, 1.1, -3.3, -5.0]])[None]
    ctx = binding.context_for(w)
    ref = oracle_eval(w, w.tables, theta[0], 0, grad=True)
    # one vector (the one-vector path) and a batch of two copies (the fused kernels)
    out = gpu_eval(ctx, w, theta, np.zeros(1, np.int32))
    check_sample(out, 0, ref, 0)
    out2 = gpu_eval(ctx, w, np.vstack([theta, theta]), np.zeros(2, np.int32))
    for b in range(2):
        check_sample(out2, b, ref, 0)


def test_bin_grid_errors():
    w = synth.workload("tiny", n_nu=400)
    ctx = binding.Context(w.model)
    ctx.es_load_tables(w.tables)
    lam = 1e4 / w.tables.nu
    with pytest.raises(binding.ExoskryError, match="EINVAL"):       # bin with no native point
        ctx.es_set_grid(np.array([lam.max() + 1.0]), np.array([lam.max() + 2.0]))
    with pytest.raises(binding.ExoskryError, match="EINVAL"):       # overlapping bins
        ctx.es_set_grid(np.array([1.0, 1.5]), np.array([2.0, 2.5]))
    with pytest.raises(binding.ExoskryError, match="ESTATE"):
        ctx.es_set_data(0, np.zeros(3), np.ones(3))


def test_state_errors():
    w = synth.workload("tiny", n_nu=400)
    ctx = binding.Context(w.model)
    lnl = torch.empty(1, dtype=torch.float64, device=DEV)
    with pytest.raises(binding.ExoskryError, match="ESTATE"):
        ctx.es_loglike(lnl)
    ctx.es_load_tables(w.tables)
    ctx.es_set_grid(w.bin_lo_um, w.bin_hi_um)
    ctx.es_set_batch(w.theta, np.array([1], np.int32))
    with pytest.raises(binding.ExoskryError, match="ESTATE"):     # no emission data yet
        ctx.es_loglike(lnl)


def test_host_buffers_match_device_buffers():
    w = synth.workload("tiny")
    ctx = binding.context_for(w)
    ctx.es_set_batch(w.theta)                                     # host theta
    lnl_h = np.zeros(1)
    grad_h = np.zeros((1, w.theta.shape[1]))
    ctx.es_forward_backward(lnl_h, grad_h)
    out = gpu_eval(ctx, w, w.theta, np.zeros(1, np.int32))
    np.testing.assert_allclose(lnl_h, out["lnl"], rtol=1e-12)
    np.testing.assert_allclose(grad_h, out["grad"], rtol=1e-6, atol=1e-9 * np.abs(out["grad"]).max())


def test_autograd_function_matches_adjoint():
    w = synth.workload("tiny")
    ctx = binding.context_for(w)
    th = torch.tensor(np.repeat(w.theta, 2, axis=0), dtype=torch.float64, device=DEV, requires_grad=True)
    lnl = binding.loglikelihood(th, ctx)
    (g,) = torch.autograd.grad((lnl * torch.tensor([1.0, 2.0], dtype=torch.float64, device=DEV)).sum(), th)
    out = gpu_eval(ctx, w, w.theta, np.zeros(1, np.int32))
    np.testing.assert_allclose(g[0].cpu().numpy(), out["grad"][0], rtol=1e-6)
    np.testing.assert_allclose(g[1].cpu().numpy(), 2 * out["grad"][0], rtol=1e-6)


# ------------------------------------------------------------------ full size, sampled
@pytest.mark.slow
def test_full_size_batched_transmission_sampled():
    """The bench workload (1024 vectors, 30000 wavenumbers, BF16 tables) in
    the same launch configuration; a few samples checked against the oracle."""
    w = synth.workload("batched_trans")
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, w.kind)
    valid = np.nonzero(out["flags"] == 0)[0]
    assert len(valid) > 0.5 * len(w.theta)
    for b in (valid[0], valid[len(valid) // 2], valid[-1]):
        ref = oracle_eval(w, tabs, w.theta[b], 0, grad=(b == valid[0]))
        check_sample(out, b, ref, 0, grad=(b == valid[0]))
    assert np.all(np.isfinite(out["grad"][valid]))
