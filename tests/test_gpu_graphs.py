"""CUDA-graph replay and the work-item autotuner: replayed and tuned calls give
the results of direct launches (and of the oracle), pick up new parameter
values, follow batch-shape changes, and order correctly against the caller's
stream.

lnL is compared bit for bit up to FP64 summation order (rtol 1e-12): the
forward has no atomics. The gradient is compared at rtol 1e-5: the adjoint's
shared-memory and FP64 atomics sum in a run-dependent order, and a different
work-item size regroups the FP32 partial sums across wavenumber tiles.
"""
import copy

import numpy as np
import pytest

from oracle import exoskry_oracle as O
from paper_2602_19687_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _thetas(w, n):
    rng = np.random.default_rng(7)
    out = []
    for i in range(n):
        t = w.theta.copy()
        t += 0.01 * i * rng.standard_normal(t.shape)
        out.append(t)
    return out


def _run(ctx, theta, kind, stream=None, loglike_only=False):
    th = torch.tensor(theta, dtype=torch.float64, device=DEV)
    kd = torch.tensor(kind, dtype=torch.int32, device=DEV)
    lnl = torch.full((theta.shape[0],), 7.0, dtype=torch.float64, device=DEV)
    grad = None if loglike_only else torch.full_like(th, 7.0)
    s = None
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream())    # inputs were written on the current stream
        s = stream.cuda_stream
    ctx.es_set_batch(th, kd, stream=s)
    if loglike_only:
        ctx.es_loglike(lnl, stream=s)
    else:
        ctx.es_forward_backward(lnl, grad, stream=s)
    torch.cuda.synchronize()
    return lnl.cpu().numpy(), (None if grad is None else grad.cpu().numpy())


def _close(a, b):
    (la, ga), (lb, gb) = a, b
    np.testing.assert_allclose(la, lb, rtol=1e-12, atol=0)
    if ga is not None:
        np.testing.assert_allclose(ga, gb, rtol=1e-5, atol=1e-7 * max(1.0, np.abs(gb).max()))


def test_graph_replay_matches_direct_launches_and_oracle():
    w = synth.workload("highres", batch=6, n_nu=4000)       # mixed transmission / emission
    ctx = binding.context_for(w)
    thetas = _thetas(w, 4)
    ctx.es_set_graphs(False)
    direct = [_run(ctx, t, w.kind) for t in thetas]
    direct_ll = [_run(ctx, t, w.kind, loglike_only=True) for t in thetas]
    n_direct = ctx.es_query(7)
    ctx.es_set_graphs(True)
    assert ctx.es_query(10) == 1
    # first call direct, second captured, the rest replayed: all must agree
    for rep in range(2):
        for t, ref in zip(thetas, direct):
            _close(_run(ctx, t, w.kind), ref)
        for t, ref in zip(thetas, direct_ll):
            _close(_run(ctx, t, w.kind, loglike_only=True), ref)
    assert ctx.es_query(7) == n_direct
    # different parameter values really reach the replayed graph
    assert not np.array_equal(direct[0][0], direct[3][0])
    # and the replayed result is the oracle's
    tabs = w.tables
    if w.table_dtype == "bf16":
        tabs = copy.copy(w.tables)
        tabs.log10_sigma = O.bf16_row_dequantized(w.tables.log10_sigma)
    lnl, grad = _run(ctx, thetas[1], w.kind)
    m = w.model
    mem = O.bin_members(tabs.nu, w.bin_lo_um, w.bin_hi_um)
    for b in range(2):
        k = int(w.kind[b])
        th = m.full_theta(thetas[1][b])[0]
        ref = O.loglike(m, tabs, th, k, mem, w.y_obs[k], w.sigma[k])
        np.testing.assert_allclose(lnl[b], ref, rtol=1e-5, atol=1e-3)
        if b == 0 and ref > O.INVALID_LNL:
            g = O.loglike_gradient(m, tabs, th, k, mem, w.y_obs[k], w.sigma[k], list(m.free_idx))
            tol = 1e-3 * np.abs(g) + 1e-4 * np.max(np.abs(g))
            assert np.all(np.abs(grad[b] - g) <= tol), (grad[b], g)


def test_graph_follows_batch_shape_changes():
    w = synth.workload("batched_trans", batch=12, n_nu=2500)
    ctx = binding.context_for(w)
    kind = np.zeros(12, np.int32)
    ctx.es_set_graphs(False)
    ref12 = _run(ctx, w.theta, kind)
    ref5 = _run(ctx, w.theta[:5], kind[:5])
    ctx.es_set_graphs(True)
    for _ in range(3):
        _close(_run(ctx, w.theta, kind), ref12)
    for _ in range(3):
        _close(_run(ctx, w.theta[:5], kind[:5]), ref5)
    _close(_run(ctx, w.theta, kind), ref12)


def test_graph_replay_on_a_side_stream():
    w = synth.workload("batched_trans", batch=8, n_nu=2500)
    ctx = binding.context_for(w)
    kind = np.zeros(8, np.int32)
    ctx.es_set_graphs(False)
    ref = _run(ctx, w.theta, kind)
    ctx.es_set_graphs(True)
    side = torch.cuda.Stream()
    for _ in range(4):
        _close(_run(ctx, w.theta, kind, stream=side), ref)


@pytest.mark.parametrize("kinds", ["trans", "emis", "mixed"])
def test_autotune_keeps_results(kinds):
    """The autotuner picks a work-item size and order for the kernels the
    batch runs (transmission, emission, or the mixed kernel) and the results
    stay those of the built-in shapes."""
    w = synth.workload("highres", batch=12, n_nu=6000)
    kind = {"trans": np.zeros(12, np.int32), "emis": np.ones(12, np.int32),
            "mixed": (np.arange(12) % 2).astype(np.int32)}[kinds]
    ctx = binding.context_for(w)
    assert all(v[0] == 0 for v in ctx.launch_shapes().values())
    ref = _run(ctx, w.theta, kind)
    shapes = ctx.es_autotune()
    tuned = {"trans": ("trans_fwd", "trans_bwd"), "emis": ("emis_fwd", "emis_bwd"),
             "mixed": ("mixed_fwd", "mixed_bwd")}[kinds]
    for k, (size, order) in shapes.items():
        assert (size >= 1) == (k in tuned), (k, size)
        assert order in ("chunk-major", "sample-major")
    if kinds == "mixed":
        assert shapes["mixed_fwd"][0] % 4 == 0 and shapes["mixed_bwd"][0] % 4 == 0
    for _ in range(3):
        _close(_run(ctx, w.theta, kind), ref)


def test_mixed_batch_runs_one_kernel_per_direction_and_matches_single_kind_runs():
    """A batch of both kinds runs setup, one mixed forward kernel and the
    binning (3 launches for ln L; 5 with the adjoint), and each sample's ln L
    and gradient equal those of the same sample in a single-kind batch (the
    transmission-only and emission-only kernels). The transmission-only
    forward runs 24 warps (the transit depth summed over 6 impact-parameter
    chunks), the mixed kernel 16 (4 chunks): FP32 summation order, so ln L is
    compared at 1e-6 relative rather than bit for bit."""
    w = synth.workload("highres", batch=10, n_nu=6000)
    kind = np.array([0, 1, 1, 0, 1, 0, 0, 1, 0, 1], np.int32)
    ctx = binding.context_for(w)
    ctx.es_set_graphs(False)
    lm, gm = _run(ctx, w.theta, kind)
    assert ctx.es_query(7) == 5
    _run(ctx, w.theta, kind, loglike_only=True)
    assert ctx.es_query(7) == 3
    for k in (0, 1):
        sel = np.nonzero(kind == k)[0]
        ls, gs = _run(ctx, w.theta[sel], kind[sel])
        assert ctx.es_query(7) == 5
        np.testing.assert_allclose(lm[sel], ls, rtol=1e-6, atol=0)
        np.testing.assert_allclose(gm[sel], gs, rtol=1e-5, atol=1e-7 * max(1.0, np.abs(gs).max()))
