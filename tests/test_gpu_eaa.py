"""GPU parity of the delta-EAA emission solver (Sect. 5 with scattering:
ES_RT_DELTA_EAA) against the FP64 oracle, through the C ABI.

Tolerances as for the absorption-only emission path (FP32 kernels against
FP64): emergent Fp/F* 1e-4 relative (with a floor of 1e-7 of the largest
value), binned model 1e-5, ln L 1e-5, gradient 1e-3 relative per component
with a floor of 1e-4 of the largest. BF16-table workloads are compared with
the oracle run on the same dequantized table values.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def oracle_tables(w):
    if w.table_dtype != "bf16":
        return w.tables
    t = copy.copy(w.tables)
    t.log10_sigma = O.bf16_row_dequantized(w.tables.log10_sigma)
    return t


def gpu_eval(ctx, w, theta, kind, backward=True):
    B, N, nb = theta.shape[0], w.tables.nu.size, w.bin_lo_um.size
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    ctx.es_set_batch(th, torch.tensor(kind, dtype=torch.int32, device=DEV))
    spec = torch.empty((B, N), dtype=torch.float32, device=DEV)
    binned = torch.empty((B, nb), dtype=torch.float64, device=DEV)
    lnl = torch.empty(B, dtype=torch.float64, device=DEV)
    ctx.es_forward(spectrum=spec, binned=binned, lnl=lnl)
    out = dict(spec=spec.cpu().numpy().astype(np.float64), binned=binned.cpu().numpy(), lnl=lnl.cpu().numpy())
    if backward:
        lnl2, grad = torch.empty_like(lnl), torch.empty_like(th)
        ctx.es_forward_backward(lnl2, grad)
        out["lnl2"], out["grad"] = lnl2.cpu().numpy(), grad.cpu().numpy()
    flags = torch.empty(B, dtype=torch.int32, device=DEV)
    ctx.es_get_flags(flags)
    out["flags"] = flags.cpu().numpy()
    torch.cuda.synchronize()
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
        res["grad"] = O.loglike_gradient(m, tabs, th, kind, mem, w.y_obs[kind], w.sigma[kind], list(m.free_idx))
    return res


def assert_grad(got, ref):
    tol = 1e-3 * np.abs(ref) + 1e-4 * np.max(np.abs(ref))
    bad = np.abs(got - ref) > tol
    assert not bad.any(), "gradient mismatch:\n gpu %s\n ref %s" % (got, ref)


def check_sample(out, b, ref, kind, grad=True):
    assert out["flags"][b] == 0
    if kind == 0:
        np.testing.assert_allclose(out["spec"][b], ref["spec"], rtol=1e-5, atol=0)
    else:
        np.testing.assert_allclose(out["spec"][b], ref["spec"], rtol=1e-4, atol=1e-7 * np.max(np.abs(ref["spec"])))
    np.testing.assert_allclose(out["binned"][b], ref["binned"], rtol=1e-5 if kind else 1e-6,
                               atol=1e-7 * np.max(np.abs(ref["binned"])) if kind else 0.0)
    np.testing.assert_allclose(out["lnl"][b], ref["lnl"], rtol=1e-5, atol=1e-3)
    if "lnl2" in out:
        np.testing.assert_allclose(out["lnl2"][b], out["lnl"][b], rtol=1e-12)
    if grad:
        assert_grad(out["grad"][b], ref["grad"])


def _scattering(batch=4, n_nu=2000, **kw):
    w = synth.workload("scattering_emis", batch=batch, n_nu=n_nu)
    if kw:
        w.model = dataclasses.replace(w.model, **kw)
    return w


def test_eaa_cloudy_scattering_matches_oracle():
    """Rayleigh and cloud scattering (omega_c = 0.9, g_c = 0.6), a clear and
    a cloudy column mixed by the cloud fraction: Fp/F* element by element over
    two 1024-wavenumber work items and a ragged tail, binned model, ln L and
    the gradient with respect to all 20 free parameters."""
    w = _scattering()
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, np.ones(4, np.int32))
    checked = 0
    for b in range(4):
        ref = oracle_eval(w, tabs, w.theta[b], 1, grad=(b < 2))
        if not ref["valid"]:
            assert out["lnl"][b] == O.INVALID_LNL
            continue
        check_sample(out, b, ref, 1, grad=(b < 2))
        checked += 1
    assert checked >= 2


@pytest.mark.parametrize("quad", [O.QUAD_GAUSS_LEGENDRE, O.QUAD_GAUSS_JACOBI])
def test_eaa_rayleigh_only_matches_oracle(quad):
    """No cloud: Rayleigh scattering alone (albedo from the H2/He Rayleigh
    share, no delta-M scaling), with Gauss-Legendre and Gauss-Jacobi flux
    angles (the mean intensity with the angles' interpolatory weights)."""
    w = synth.workload("batched_emis", batch=3, n_nu=1500)
    w.model = dataclasses.replace(w.model, emission_solver=O.RT_DELTA_EAA, emission_quadrature=quad)
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, np.ones(3, np.int32))
    for b in range(3):
        ref = oracle_eval(w, tabs, w.theta[b], 1, grad=(b == 0))
        assert ref["valid"]
        check_sample(out, b, ref, 1, grad=(b == 0))


def test_eaa_mixed_batch():
    """Transmission and delta-EAA emission samples in one batch: the
    transmission samples through their fused kernels, the emission samples
    through the delta-EAA kernels; every output against the oracle."""
    w = _scattering(batch=4, n_nu=1200)
    kind = np.array([1, 0, 1, 0], np.int32)
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, kind)
    for b in range(4):
        ref = oracle_eval(w, tabs, w.theta[b], int(kind[b]), grad=(b < 2))
        if not ref["valid"]:
            assert out["lnl"][b] == O.INVALID_LNL
            continue
        check_sample(out, b, ref, int(kind[b]), grad=(b < 2))


def test_eaa_without_scatterers_equals_absorption_kernels():
    """With zero Rayleigh cross-sections and a cloud of zero albedo the
    delta-EAA kernels compute the absorption-only model; against the fused
    absorption-only emission kernels on the same batch (both FP32)."""
    w = _scattering(batch=3, n_nu=1500, ray_h2_cm2=0.0, ray_he_cm2=0.0, cloud_ssa=0.0)
    kind = np.ones(3, np.int32)
    eaa = gpu_eval(binding.context_for(w), w, w.theta, kind)
    w2 = copy.copy(w)
    w2.model = dataclasses.replace(w.model, emission_solver=O.RT_ABSORPTION)
    ref = gpu_eval(binding.context_for(w2), w2, w.theta, kind)
    ok = ref["lnl"] > O.INVALID_LNL
    assert ok.any()
    np.testing.assert_allclose(eaa["spec"][ok], ref["spec"][ok], rtol=2e-5, atol=1e-7 * np.max(np.abs(ref["spec"])))
    np.testing.assert_allclose(eaa["lnl"], ref["lnl"], rtol=1e-6)
    for b in np.nonzero(ok)[0]:
        g, r = eaa["grad"][b], ref["grad"][b]
        assert np.all(np.abs(g - r) <= 2e-4 * np.abs(r) + 2e-5 * np.max(np.abs(r))), (g, r)


def test_eaa_invalid_samples_and_replay():
    """Invalid samples (sum of VMRs above 1) get ln L = -1e300 and a zero
    gradient beside valid ones; graph replays of es_loglike and
    es_forward_backward reproduce the first call (the adjoint's sums are
    atomics: to FP32 rounding)."""
    w = _scattering(batch=4, n_nu=1000)
    theta = w.theta.copy()
    theta[1, :3] = -0.2
    ctx = binding.context_for(w)
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    ctx.es_set_batch(th, torch.ones(4, dtype=torch.int32, device=DEV))
    lnl = [torch.empty(4, dtype=torch.float64, device=DEV) for _ in range(3)]
    grad = [torch.empty_like(th) for _ in range(3)]
    for k in range(3):
        ctx.es_forward_backward(lnl[k], grad[k])
    l0 = lnl[0].cpu().numpy()
    assert l0[1] == O.INVALID_LNL and np.all(grad[0].cpu().numpy()[1] == 0)
    for k in (1, 2):
        np.testing.assert_array_equal(lnl[k].cpu().numpy(), l0)
        np.testing.assert_allclose(grad[k].cpu().numpy(), grad[0].cpu().numpy(), rtol=1e-5, atol=1e-9)
    ll = torch.empty(4, dtype=torch.float64, device=DEV)
    for _ in range(3):
        ctx.es_loglike(ll)
        np.testing.assert_array_equal(ll.cpu().numpy(), l0)
    valid = [b for b in range(4) if b != 1]
    ref = oracle_eval(w, oracle_tables(w), theta[valid[0]], 1)
    np.testing.assert_allclose(l0[valid[0]], ref["lnl"], rtol=1e-5, atol=1e-3)


def test_eaa_brown_dwarf_gauss_jacobi():
    """A brown dwarf's absolute flux at distance D (modified Milne profile,
    mass and gravity through R_bd) by the delta-EAA with Rayleigh scattering
    and the Gauss-Jacobi flux angles: spectra, ln L and all 15 gradient
    components against the oracle."""
    w = synth.workload("browndwarf", batch=2, n_nu=1500)
    w.model = dataclasses.replace(w.model, emission_solver=O.RT_DELTA_EAA,
                                  emission_quadrature=O.QUAD_GAUSS_JACOBI)
    tabs = oracle_tables(w)
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, np.ones(2, np.int32))
    for b in range(2):
        ref = oracle_eval(w, tabs, w.theta[b], 1, grad=(b == 0))
        assert ref["valid"]
        check_sample(out, b, ref, 1, grad=(b == 0))


def test_eaa_autotune_mixed_batch():
    """es_autotune on a mixed batch of a delta-EAA model tunes the
    transmission kernels' shapes only; the results with the tuned shapes equal
    the built-in ones to FP32 rounding of the atomically summed adjoint."""
    w = _scattering(batch=4, n_nu=1500)
    kind = np.array([0, 1, 0, 1], np.int32)
    ctx = binding.context_for(w)
    before = gpu_eval(ctx, w, w.theta, kind)
    shapes = ctx.es_autotune()
    for k, (size, _) in shapes.items():
        assert (size >= 1) == (k in ("trans_fwd", "trans_bwd")), (k, size)
    after = gpu_eval(ctx, w, w.theta, kind)
    np.testing.assert_allclose(after["spec"], before["spec"], rtol=1e-6, atol=0)
    np.testing.assert_allclose(after["lnl"], before["lnl"], rtol=1e-9)
    np.testing.assert_allclose(after["grad"], before["grad"], rtol=1e-5, atol=1e-7 * np.abs(before["grad"]).max())


@pytest.mark.slow
def test_eaa_full_size_sampled():
    """The scattering workload at its full size (512 vectors, 20000
    wavenumbers, the launch configuration bench.py times): Fp/F* and ln L of
    two sampled vectors against the oracle, and every ln L finite or -1e300."""
    w = synth.workload("scattering_emis")
    ctx = binding.context_for(w)
    out = gpu_eval(ctx, w, w.theta, np.ones(w.theta.shape[0], np.int32), backward=True)
    assert np.all((out["lnl"] == O.INVALID_LNL) | np.isfinite(out["lnl"]))
    assert np.all(np.isfinite(out["grad"]))
    tabs = oracle_tables(w)
    for b in (0, 311):
        ref = oracle_eval(w, tabs, w.theta[b], 1)
        if not ref["valid"]:
            assert out["lnl"][b] == O.INVALID_LNL
            continue
        check_sample(out, b, ref, 1, grad=False)
