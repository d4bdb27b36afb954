"""Failure handling through the C ABI, without faulting, trapping or hanging
the GPU:

- bounded waits: with the wait-timeout test hook the tensor-core kernels issue
  no product, so their mbarrier waits run out (milliseconds) with nothing in
  flight; the call returns ES_ETIMEOUT (host buffers) or flags every sample
  (device buffers), and the same context computes normally once the hook is
  cleared;
- allocation failure: a per-context device-memory limit makes an allocation
  fail with ES_ENOMEM before cudaMalloc, and the context stays usable;
- corrupted table descriptions (non-finite values, bad sizes, grids out of
  order, unknown storage) are rejected with ES_EINVAL before any upload.
"""
import ctypes

import numpy as np
import pytest

from paper_2602_19687_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _host_call(ctx, B, backward):
    lnl = np.full(B, np.nan)
    if backward:
        grad = np.full((B, len(ctx.model.free_idx)), np.nan)
        ctx.es_forward_backward(lnl, grad)
        return lnl, grad
    ctx.es_loglike(lnl)
    return lnl, None


@pytest.mark.parametrize("backward", [False, True])
def test_bounded_wait_timeout_then_recovery(backward):
    w = synth.workload("tiny", batch=3)
    ctx = binding.context_for(w)
    ctx.es_set_batch(w.theta)
    ref_l, ref_g = _host_call(ctx, 3, backward)
    assert np.all(np.isfinite(ref_l))
    # each toggle of the hook drops the captured graph: the host-buffer call
    # under the hook runs its kernels directly, the device-buffer call after it
    # is captured into a graph and replayed
    for rep in range(3):
        ctx.es_set_test_hooks(binding.ES_TEST_WAIT_TIMEOUT)
        with pytest.raises(binding.ExoskryError, match="ES_ETIMEOUT"):
            _host_call(ctx, 3, backward)
        flags = np.zeros(3, np.int32)
        ctx.es_get_flags(flags)
        assert np.all(flags == binding.ES_FLAG_INVALID | binding.ES_FLAG_TIMEOUT)
        assert ctx.es_query(11) != 0
        # device buffers: the call returns at once; the samples carry the outcome
        lnl = torch.full((3,), float("nan"), dtype=torch.float64, device=DEV)
        ctx.es_loglike(lnl)
        torch.cuda.synchronize()
        assert np.all(lnl.cpu().numpy() == -1e300)
        ctx.es_set_test_hooks(0)
        got_l, got_g = _host_call(ctx, 3, backward)
        np.testing.assert_allclose(got_l, ref_l, rtol=1e-12)
        if backward:
            # (the adjoint's float atomics add in any order: last-bit differences)
            np.testing.assert_allclose(got_g, ref_g, rtol=1e-5, atol=1e-7 * np.max(np.abs(ref_g)))
        assert ctx.es_query(11) == 0
        ctx.es_get_flags(flags)
        assert np.all(flags == 0)


def test_timeout_gradient_is_zero():
    w = synth.workload("tiny", batch=2)
    ctx = binding.context_for(w)
    ctx.es_set_batch(w.theta)
    ctx.es_set_test_hooks(binding.ES_TEST_WAIT_TIMEOUT)
    th = torch.tensor(w.theta, dtype=torch.float64, device=DEV)
    lnl = torch.empty(2, dtype=torch.float64, device=DEV)
    grad = torch.full_like(th, float("nan"))
    ctx.es_forward_backward(lnl, grad)
    torch.cuda.synchronize()
    assert np.all(lnl.cpu().numpy() == -1e300)
    assert np.all(grad.cpu().numpy() == 0.0)
    ctx.es_set_test_hooks(0)


def test_unknown_test_hook_rejected():
    w = synth.workload("tiny")
    ctx = binding.context_for(w)
    with pytest.raises(binding.ExoskryError, match="ES_EINVAL"):
        ctx.es_set_test_hooks(8)


def test_memory_limit_gives_enomem_and_the_context_recovers():
    w = synth.workload("tiny", batch=4)
    ctx = binding.context_for(w)
    held = ctx.es_query(6)
    assert held > 0
    ctx.es_set_memory_limit(held + 4096)
    with pytest.raises(binding.ExoskryError, match="ES_ENOMEM.*limit"):
        ctx.es_set_batch(w.theta)
    assert ctx.es_query(6) <= held + 4096
    ctx.es_set_memory_limit(0)
    ctx.es_set_batch(w.theta)
    lnl = np.empty(4)
    ctx.es_loglike(lnl)
    assert np.all(np.isfinite(lnl) | (lnl == -1e300))
    # a limit that admits the forward workspace but not the adjoint's
    fwd_held = ctx.es_query(6)
    ctx.es_set_memory_limit(fwd_held + 1024)
    grad = np.empty((4, len(w.model.free_idx)))
    with pytest.raises(binding.ExoskryError, match="ES_ENOMEM"):
        ctx.es_forward_backward(lnl, grad)
    ctx.es_set_memory_limit(0)
    ctx.es_forward_backward(lnl, grad)
    assert np.all(np.isfinite(grad))


def _desc(t, **over):
    arrs = dict(nu=np.ascontiguousarray(t.nu, np.float64), tg=np.ascontiguousarray(t.t_grid, np.float64),
                pg=np.ascontiguousarray(t.p_grid_bar, np.float64),
                sig=np.ascontiguousarray(t.log10_sigma, np.float32),
                ct=np.ascontiguousarray(t.cia_t_grid, np.float64),
                c1=np.ascontiguousarray(t.cia_h2h2, np.float32), c2=np.ascontiguousarray(t.cia_h2he, np.float32))
    arrs.update({k: v for k, v in over.items() if k in arrs})
    d = binding.es_tables_desc()
    dp, fp = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
    d.n_nu, d.nu = over.get("n_nu", arrs["nu"].size), arrs["nu"].ctypes.data_as(dp)
    d.n_t, d.t_grid = over.get("n_t", arrs["tg"].size), arrs["tg"].ctypes.data_as(dp)
    d.n_p, d.p_grid_bar = arrs["pg"].size, arrs["pg"].ctypes.data_as(dp)
    d.log10_sigma = arrs["sig"].ctypes.data_as(fp)
    d.n_t_cia, d.cia_t_grid = arrs["ct"].size, arrs["ct"].ctypes.data_as(dp)
    d.cia_h2h2, d.cia_h2he = arrs["c1"].ctypes.data_as(fp), arrs["c2"].ctypes.data_as(fp)
    d.storage = over.get("storage", binding.ES_TABLE_F32)
    return d, arrs


def test_corrupted_table_descriptions_are_rejected():
    w = synth.workload("tiny")
    ctx = binding.context_for(w)
    lib, t = ctx.lib, w.tables
    sig = np.array(t.log10_sigma, np.float32)
    sig[0, 1, 2, 7] = np.nan
    cia = np.array(t.cia_h2he, np.float32)
    cia[0, 3] = np.inf
    nu_bad = np.array(t.nu, np.float64)
    nu_bad[5] = nu_bad[4]
    cases = [(dict(sig=sig), "not finite"), (dict(c2=cia), "not finite"), (dict(nu=nu_bad), "ascending"),
             (dict(storage=7), "storage"), (dict(n_t=1), "out of range"), (dict(n_nu=1), "out of range")]
    for over, msg in cases:
        d, keep = _desc(t, **over)
        st = lib.es_load_tables(ctx.handle, ctypes.byref(d))
        assert st == binding.ES_EINVAL, over
        assert msg in lib.es_last_error(ctx.handle).decode(), (over, lib.es_last_error(ctx.handle))
    # the tables and grid loaded before the rejections are untouched
    ctx.es_set_batch(w.theta)
    lnl = np.empty(1)
    ctx.es_loglike(lnl)
    assert np.isfinite(lnl[0])


def test_reloading_tables_drops_the_batch():
    """es_load_tables frees the workspace: until a new batch is set, a call is
    ES_ESTATE (never a launch on freed buffers)."""
    w = synth.workload("tiny", batch=2)
    ctx = binding.context_for(w)
    ctx.es_set_batch(w.theta)
    lnl = np.empty(2)
    ctx.es_loglike(lnl)
    ctx.es_load_tables(w.tables, w.table_dtype)
    ctx.es_set_grid(w.bin_lo_um, w.bin_hi_um)
    for kind in (0, 1):
        ctx.es_set_data(kind, w.y_obs[kind], w.sigma[kind])
    with pytest.raises(binding.ExoskryError, match="ESTATE"):
        ctx.es_loglike(lnl)
    ctx.es_set_batch(w.theta)
    ctx.es_loglike(lnl)
    assert np.all(np.isfinite(lnl))
