"""GPU parity of the one-vector (plain per-sample) transmission path.

A batch of a single transmission vector runs the opacity stage (Sect. 3) as a
kernel of its own, which reads the raw table rows that bracket the vector's
layers once and writes the layer extinction, and then the chord kernel
(Sect. 4) on that extinction. Checked here:
- against the FP64 oracle element by element (the parity tolerances of
  test_gpu_parity: transit depth 1e-5 relative, ln L 1e-5, gradient 1e-3),
  on FP32 and BF16 tables, with a ragged last window and tile, the non-grey
  cloud, and layers and temperatures outside the tables' grids;
- against the fused batched path for the same vector (a batch of two
  copies): the two differ only in FP32 rounding order of the extinction;
- the row bytes the stage reports (es_query key 17) against the union of the
  (T, p) nodes bracketing the vector's layers, computed on the host from the
  oracle's temperature profile and brackets.
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


def run(ctx, w, theta):
    B, N, nb = theta.shape[0], w.tables.nu.size, w.bin_lo_um.size
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    ctx.es_set_batch(th, torch.zeros(B, dtype=torch.int32, device=DEV))
    spec = torch.empty((B, N), dtype=torch.float32, device=DEV)
    binned = torch.empty((B, nb), dtype=torch.float64, device=DEV)
    lnl = torch.empty(B, dtype=torch.float64, device=DEV)
    ctx.es_forward(spectrum=spec, binned=binned, lnl=lnl)
    launches = ctx.es_query(7)
    rows = ctx.es_query(17)
    lnl2 = torch.empty_like(lnl)
    grad = torch.empty_like(th)
    ctx.es_forward_backward(lnl2, grad)
    flags = torch.empty(B, dtype=torch.int32, device=DEV)
    ctx.es_get_flags(flags)
    torch.cuda.synchronize()
    assert ctx.es_query(11) == 0
    return dict(spec=spec.cpu().numpy().astype(np.float64), binned=binned.cpu().numpy(), lnl=lnl.cpu().numpy(),
                lnl2=lnl2.cpu().numpy(), grad=grad.cpu().numpy(), flags=flags.cpu().numpy(),
                launches=launches, rows=rows)


def oracle_eval(w, theta_row):
    m, tabs = w.model, oracle_tables(w)
    th = m.full_theta(theta_row)[0]
    mem = O.bin_members(tabs.nu, w.bin_lo_um, w.bin_hi_um)
    out = O.forward(m, tabs, th, 0, mem)
    if out is None:
        return None
    return dict(spec=out[0], binned=out[1],
                lnl=O.loglike(m, tabs, th, 0, mem, w.y_obs[0], w.sigma[0]),
                grad=O.loglike_gradient(m, tabs, th, 0, mem, w.y_obs[0], w.sigma[0], list(m.free_idx)))


def bracket_union_bytes(w, theta_row):
    """Bytes of the raw table rows (all species, all wavenumbers) at the (T, p)
    nodes that bracket any layer, plus the two CIA tables' rows at the CIA
    temperature nodes that bracket any layer."""
    m, tabs = w.model, w.tables
    atm = O.atmosphere(m, m.full_theta(theta_row)[0])
    lt, lp = np.log10(tabs.t_grid), np.log10(tabs.p_grid_bar)
    nodes, cia = set(), set()
    for t, p in zip(atm["t_lay"], atm["p_lay"]):
        it, _ = O.bracket(lt, np.log10(t))
        ip, _ = O.bracket(lp, np.log10(p / O.BAR))
        nodes |= {(it + a, ip + c) for a in (0, 1) for c in (0, 1)}
        ic, _ = O.bracket(tabs.cia_t_grid, t)
        cia |= {ic, ic + 1}
    esz = 2 if w.table_dtype == "bf16" else 4
    return (len(nodes) * m.n_species * esz + 2 * len(cia) * 4) * tabs.nu.size


def _out_of_grid():
    w = synth.workload("tiny", n_nu=1001)
    w.model = dataclasses.replace(w.model, p_top_bar=1e-8, p_bot_bar=1e3)
    return w, np.array([[-3.0, -4.0, -5.0, 4500.0, 1.0, -2.37]])


def _case(name):
    if name == "tiny":
        w = synth.workload("tiny", n_nu=2000)
        th = w.theta.copy()
        th[0, 5] = -2.37   # deck off a level
        return w, th
    if name == "jwst_plain":
        w = synth.workload("jwst_plain", n_nu=3001)
        return w, w.theta[:1]
    if name == "out_of_grid":
        return _out_of_grid()
    w = synth.workload(name, batch=8, n_nu=2501)
    for b in range(w.theta.shape[0]):
        if O.atmosphere(w.model, w.model.full_theta(w.theta[b])[0])["valid"]:
            return w, w.theta[b:b + 1]
    raise AssertionError("no valid vector")


@pytest.mark.parametrize("name", ["tiny", "jwst_plain", "batched_trans", "cloudy_trans", "out_of_grid"])
def test_one_vector_path_matches_the_oracle_and_the_fused_path(name):
    w, theta = _case(name)
    _check(w, theta)


def _check(w, theta):
    ctx = binding.context_for(w)
    one = run(ctx, w, theta)
    # setup, opacity stage, chord kernel, binning
    assert one["launches"] == 4
    assert one["flags"][0] == 0
    ref = oracle_eval(w, theta[0])
    assert ref is not None
    np.testing.assert_allclose(one["spec"][0], ref["spec"], rtol=1e-5, atol=0)
    np.testing.assert_allclose(one["binned"][0], ref["binned"], rtol=1e-6)
    np.testing.assert_allclose(one["lnl"][0], ref["lnl"], rtol=1e-5, atol=1e-3)
    np.testing.assert_allclose(one["lnl2"][0], one["lnl"][0], rtol=1e-12)
    tol = 1e-3 * np.abs(ref["grad"]) + 1e-4 * np.max(np.abs(ref["grad"]))
    assert np.all(np.abs(one["grad"][0] - ref["grad"]) <= tol), (one["grad"][0], ref["grad"])
    # the fused batched path on the same vector
    two = run(ctx, w, np.vstack([theta, theta]))
    assert two["launches"] == 3 and two["rows"] == 0
    for b in range(2):
        np.testing.assert_allclose(two["spec"][b], one["spec"][0], rtol=2e-6, atol=0)
        np.testing.assert_allclose(two["lnl"][b], one["lnl"][0], rtol=1e-6)
        gt = 1e-5 * np.abs(one["grad"][0]) + 1e-6 * np.max(np.abs(one["grad"][0]))
        assert np.all(np.abs(two["grad"][b] - one["grad"][0]) <= gt)
    # the rows it read: the bracketing union, exactly
    assert one["rows"] == bracket_union_bytes(w, theta[0])
    ctx.es_destroy()


def test_one_vector_path_graph_replay_and_profile():
    """The one-vector launch sequence replays from a CUDA graph with the
    same ln L (bit for bit) and gradient, and its two kernels appear in the
    per-kernel profile."""
    w = synth.workload("jwst_plain", n_nu=2000)
    ctx = binding.context_for(w)
    th = torch.tensor(w.theta[:1], dtype=torch.float64, device=DEV)
    ctx.es_set_batch(th, torch.zeros(1, dtype=torch.int32, device=DEV))
    lnl = torch.empty(1, dtype=torch.float64, device=DEV)
    grad = torch.empty_like(th)
    got = []
    for _ in range(4):   # direct, capture, replay, replay
        ctx.es_forward_backward(lnl, grad)
        got.append((lnl.item(), grad.cpu().numpy().copy()))
    for l, g in got[1:]:
        assert l == got[0][0]
        # the adjoint's sums over wavenumber use atomics: their order, and so the
        # gradient's last bits, vary from call to call
        np.testing.assert_allclose(g, got[0][1], rtol=1e-6)
    ctx.es_set_profiling(True)
    ctx.es_forward_backward(lnl, grad)
    torch.cuda.synchronize()
    names = [k for k, _, _ in ctx.es_get_profile()]
    ctx.es_set_profiling(False)
    assert "k_trans_alpha" in names and "k_trans_chord" in names and "k_trans_fwd" not in names
    ctx.es_destroy()


def _custom(n_species, n_t, n_p, n_layers, n_nu, dtype, t_lo=300.0, t_hi=3500.0):
    """A hot Guillot atmosphere (T from ~1800 K to ~3300 K) on a table grid of
    n_t x n_p nodes over t_lo-t_hi K and 1e-8..100 bar."""
    s = n_species
    free = list(range(s)) + [s + synth.P_T_INT, s + synth.P_T_EQ, s + synth.P_LOG_KAPPA,
                             s + synth.P_LOG_GAMMA, s + synth.P_R_P]
    names = (list(synth.SPECIES) * 2)[:s]
    model = synth._model(s, n_layers, 1e-8, 100.0, synth.TP_GUILLOT, synth.CLOUD_NONE, free=free, species=names)
    nu = synth.nu_grid_constant_r(0.5, 5.5, n_nu)
    tabs = synth.make_tables(nu, s, np.geomspace(t_lo, t_hi, n_t), np.geomspace(1e-8, 100.0, n_p))
    lo, hi = synth.make_bins(nu, 20)
    y, sg = synth.make_data(20, 0, 0.0145)
    theta = np.array([[-3.5 - 0.3 * k for k in range(s)] + [600.0, 2000.0, -2.0, -0.5, 1.2]])
    w = synth.Workload(name="custom", model=model, tables=tabs, bin_lo_um=lo, bin_hi_um=hi, y_obs={0: y, 1: y},
                       sigma={0: sg, 1: sg}, theta=theta, kind=np.zeros(1, np.int32), table_dtype=dtype,
                       description="custom")
    return w, theta


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_one_vector_path_species_in_rounds(dtype):
    """12 species: their bracketing rows do not fit one block's shared memory
    at once (12 x ~40 nodes x the window), so the stage runs in rounds of
    species, keeping the running sum in the output buffer between rounds."""
    w, theta = _custom(12, 20, 15, 100, 700, dtype)
    assert bracket_union_bytes(w, theta[0]) // (12 * 700 * (2 if dtype == "bf16" else 4)) >= 30
    _check(w, theta)


def test_one_vector_path_direct_reads():
    """A 64 x 64 table (64 temperatures over 1700-3400 K) and 112 layers: the
    layers bracket ~205 nodes, more rows of 256 bytes than one block's
    staging area holds beside the 64 x 64 node tables (~180), so the stage
    reads its corners straight from global memory."""
    w, theta = _custom(3, 64, 64, 112, 256, "f32", 1700.0, 3400.0)
    nodes = bracket_union_bytes(w, theta[0]) // (3 * 256 * 4)
    assert nodes >= 200, nodes
    _check(w, theta)


def test_one_vector_path_high_resolution_shape():
    """The high-resolution shape (60 layers, 4 absorbers, BF16 tables) at
    44,000 wavenumbers, one transmission vector: against the oracle (spectrum
    and ln L) and against the fused path (spectrum, ln L and gradient)."""
    w = synth.workload("highres", batch=8, n_nu=44000)
    b = next(k for k in range(8) if w.kind[k] == 0
             and O.atmosphere(w.model, w.model.full_theta(w.theta[k])[0])["valid"])
    theta = w.theta[b:b + 1]
    ctx = binding.context_for(w)
    one = run(ctx, w, theta)
    assert one["launches"] == 4 and one["flags"][0] == 0
    m, tabs = w.model, oracle_tables(w)
    th = m.full_theta(theta[0])[0]
    mem = O.bin_members(tabs.nu, w.bin_lo_um, w.bin_hi_um)
    spec, _ = O.forward(m, tabs, th, 0, mem)
    np.testing.assert_allclose(one["spec"][0], spec, rtol=1e-5, atol=0)
    np.testing.assert_allclose(one["lnl"][0], O.loglike(m, tabs, th, 0, mem, w.y_obs[0], w.sigma[0]),
                               rtol=1e-5, atol=1e-3)
    two = run(ctx, w, np.vstack([theta, theta]))
    for k in range(2):
        np.testing.assert_allclose(two["spec"][k], one["spec"][0], rtol=2e-6, atol=0)
        np.testing.assert_allclose(two["lnl"][k], one["lnl"][0], rtol=1e-6)
        gt = 1e-5 * np.abs(one["grad"][0]) + 1e-6 * np.max(np.abs(one["grad"][0]))
        assert np.all(np.abs(two["grad"][k] - one["grad"][0]) <= gt)
    assert one["rows"] == bracket_union_bytes(w, theta[0])
    ctx.es_destroy()


def test_one_vector_path_over_prior_draws():
    """48 draws from the batched transmission prior (BF16 tables, 2501
    wavenumbers), invalid ones included: each vector alone (the one-vector
    path) against the same vector in one fused batch of all 48 -- spectrum,
    ln L and gradient, and the invalid samples' ln L = -1e300 with a zero
    gradient on both paths."""
    w = synth.workload("batched_trans", batch=48, n_nu=2501)
    ctx = binding.context_for(w)
    fused = run(ctx, w, w.theta)
    assert fused["launches"] == 3
    n_valid = 0
    for b in range(w.theta.shape[0]):
        one = run(ctx, w, w.theta[b:b + 1])
        assert one["launches"] == 4
        if fused["flags"][b] != 0:
            assert one["flags"][0] == fused["flags"][b]
            assert one["lnl"][0] == O.INVALID_LNL and np.all(one["grad"][0] == 0)
            continue
        n_valid += 1
        np.testing.assert_allclose(one["spec"][0], fused["spec"][b], rtol=2e-6, atol=0)
        np.testing.assert_allclose(one["lnl"][0], fused["lnl"][b], rtol=1e-6)
        g = fused["grad"][b]
        assert np.all(np.abs(one["grad"][0] - g) <= 1e-5 * np.abs(g) + 1e-6 * np.max(np.abs(g)))
    assert n_valid >= 24
    ctx.es_destroy()
