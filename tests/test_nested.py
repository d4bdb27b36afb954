"""Batched nested sampling (the sampler that consumes the batched likelihood)
against likelihoods whose evidence and posterior are known in closed form."""
import numpy as np
import pytest

from paper_2602_19687_gb300 import nested


def _gauss_loglike(mu, sigma, counter=None):
    mu = np.asarray(mu, dtype=np.float64)

    def f(theta):
        if counter is not None:
            counter.append(theta.shape[0])
        r = (theta - mu) / sigma
        return -0.5 * np.sum(r * r, axis=1) - mu.size * np.log(sigma * np.sqrt(2.0 * np.pi))
    return f


def test_gaussian_evidence_and_posterior():
    """A normalised Gaussian well inside a unit-volume uniform prior: Z = 1
    (ln Z = 0 up to the mass outside the cube, < 1e-20), posterior mean mu and
    standard deviation sigma, information H = -d/2 ln(2 pi e sigma^2)."""
    d, sigma = 3, 0.05
    mu = np.array([0.5, 0.4, 0.6])
    res = nested.run(_gauss_loglike(mu, sigma), lambda u: u, d, n_live=400, batch=40, dlogz=0.01,
                     walk_steps=25, seed=3)
    h_true = -0.5 * d * np.log(2.0 * np.pi * np.e * sigma ** 2)
    assert abs(res.log_z) < 4.0 * res.log_z_err + 0.02, (res.log_z, res.log_z_err)
    assert res.information == pytest.approx(h_true, abs=0.3)
    assert np.allclose(res.posterior_mean(), mu, atol=0.01)
    assert np.allclose(res.posterior_std(), sigma, rtol=0.15)
    assert np.exp(res.log_weights).sum() == pytest.approx(1.0, abs=1e-12)


def test_prior_transform_and_bimodal_mass():
    """Two Gaussians of masses 0.3 and 0.7 in a prior box [-5, 5]^2 (volume
    100): Z = 1/100; the posterior mass near each mode is its weight."""
    centers = np.array([[-2.0, -2.0], [2.0, 1.5]])
    wts, sigma = np.array([0.3, 0.7]), 0.3

    def loglike(theta):
        comp = [np.log(w) - 0.5 * np.sum(((theta - c) / sigma) ** 2, axis=1) - np.log(2 * np.pi * sigma ** 2)
                for w, c in zip(wts, centers)]
        return np.logaddexp(comp[0], comp[1])

    res = nested.run(loglike, lambda u: -5.0 + 10.0 * u, 2, n_live=500, batch=50, dlogz=0.01, walk_steps=25,
                     seed=11)
    assert res.log_z == pytest.approx(np.log(0.01), abs=4.0 * res.log_z_err + 0.02)
    p = np.exp(res.log_weights)
    near0 = np.sum(p[np.linalg.norm(res.samples - centers[0], axis=1) < 1.5])
    assert near0 == pytest.approx(0.3, abs=0.06)


def test_calls_carry_whole_batches():
    """The first call evaluates the live set; every later call carries exactly
    `batch` vectors (one call per walk step per iteration)."""
    sizes = []
    res = nested.run(_gauss_loglike([0.5, 0.5], 0.1, sizes), lambda u: u, 2, n_live=100, batch=20,
                     dlogz=0.5, walk_steps=5, seed=0)
    assert sizes[0] == 100 and set(sizes[1:]) == {20}
    assert res.calls == len(sizes) == 1 + res.iterations * 5
    assert res.evaluations == sum(sizes)
    assert res.samples.shape[0] == res.iterations * 20 + 100


def test_invalid_models_never_enter_the_live_set():
    """Vectors the library flags as invalid get ln L = -1e300: they are
    retired first and never accepted as replacements."""
    base = _gauss_loglike([0.5, 0.5], 0.1)

    def loglike(theta):
        out = base(theta)
        out[theta[:, 0] < 0.2] = -1.0e300
        return out

    res = nested.run(loglike, lambda u: u, 2, n_live=200, batch=20, dlogz=0.05, walk_steps=10, seed=5)
    live = res.samples[-200:]
    assert np.all(live[:, 0] >= 0.2)
    assert np.isfinite(res.log_z)
    with pytest.raises(ValueError):
        nested.run(loglike, lambda u: u, 2, n_live=10, batch=10)


def test_loglike_batch_marshals_host_vectors():
    """binding.LogLikeBatch: one es_set_batch with the host vectors and a kind
    vector of the chosen kind, then one es_loglike into a host buffer, per call."""
    from paper_2602_19687_gb300 import binding

    class FakeContext:
        def __init__(self):
            self.log = []

        def es_set_batch(self, theta, kind=None, stream=None):
            assert isinstance(theta, np.ndarray) and theta.dtype == np.float64 and theta.flags["C_CONTIGUOUS"]
            assert kind.dtype == np.int32 and kind.shape == (theta.shape[0],)
            self.log.append(("set", theta.copy(), kind.copy()))
            self.theta = theta.copy()

        def es_loglike(self, lnl, stream=None):
            assert isinstance(lnl, np.ndarray) and lnl.dtype == np.float64
            lnl[:] = -np.sum(self.theta ** 2, axis=1)
            self.log.append(("loglike",))

    ctx = FakeContext()
    like = binding.LogLikeBatch(ctx, kind=1)
    theta = np.asfortranarray(np.arange(12.0).reshape(4, 3))
    out = like(theta)
    np.testing.assert_array_equal(out, -np.sum(theta ** 2, axis=1))
    assert [e[0] for e in ctx.log] == ["set", "loglike"] and like.calls == 1
    assert np.all(ctx.log[0][2] == 1)
