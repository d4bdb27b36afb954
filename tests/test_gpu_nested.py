"""The batched nested sampler driving the library's likelihood: every sampler
call is one es_set_batch + es_loglike over a whole batch of live-point
replacements (host vectors in, host ln L out), and the ln L it records for
its dead points are the oracle's."""
import numpy as np
import pytest

from oracle import exoskry_oracle as O
from paper_2602_19687_gb300 import binding, nested, synth

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("kind", [0, 1])
def test_nested_sampler_consumes_library_batches(kind):
    w = synth.workload("tiny")
    m = w.model
    ctx = binding.context_for(w)
    like = binding.LogLikeBatch(ctx, kind=kind)
    ranges = synth.prior_ranges(m)
    lo = np.array([ranges[k][0] for k in m.free_idx])
    hi = np.array([ranges[k][1] for k in m.free_idx])
    res = nested.run(like, lambda u: lo + (hi - lo) * u, lo.size, n_live=256, batch=64, walk_steps=4,
                     max_iterations=12, seed=2)
    assert like.calls == res.calls == 1 + res.iterations * 4
    assert res.evaluations == 256 + res.iterations * 4 * 64
    assert np.isfinite(res.log_z)
    # ln L increases along the dead points of one run (up to the batch ties)
    dead = res.log_l[:res.iterations * 64]
    assert np.all(np.diff(dead.reshape(res.iterations, 64).max(axis=1)) >= 0)
    mem = O.bin_members(w.tables.nu, w.bin_lo_um, w.bin_hi_um)
    picks = [0, res.iterations * 32, res.iterations * 64 - 1, res.samples.shape[0] - 1]
    for i in picks:
        th = m.full_theta(res.samples[i])[0]
        ref = O.loglike(m, w.tables, th, kind, mem, w.y_obs[kind], w.sigma[kind])
        if ref == O.INVALID_LNL:
            assert res.log_l[i] == O.INVALID_LNL
        else:
            assert res.log_l[i] == pytest.approx(ref, rel=1e-5, abs=1e-3)
    ctx.es_destroy()
