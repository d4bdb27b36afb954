"""Batched nested sampling: the consumer of the batched likelihood.

The paper's retrievals run nested sampling (Skilling 2004) with 1000 live
points and stop at a remaining-evidence estimate of Delta ln Z = 0.1
(Sect. 2.1, Table of experiments in Sect. 6), and its discussion points to
samplers that work in parallel over live points (Sect. 7). This module is such
a sampler, written so that every likelihood call carries a whole batch of
parameter vectors: each iteration retires the k lowest live points at once and
refills them with k constrained random walks whose proposals are evaluated
together, one call per walk step.

Prior volume. Retiring the k lowest of N live points shrinks ln X by
sum_{j<k} 1/(N - j): removing the lowest of n points multiplies the volume by
the largest of n uniform variates, whose log has mean -1/n (Skilling 2006).
Dead point i has weight w_i = X_{i-1} - X_i; Z = sum_i L_i w_i, and at the end
each remaining live point adds X_end L / N. The run stops once the live points
can add at most `dlogz` to ln Z, ln(Z + X max L_live) - ln Z < dlogz. The
statistical error of ln Z is sqrt(H / N), H the information (Skilling 2006).

Constrained moves. A replacement starts from a copy of a surviving live point
and takes `walk_steps` Metropolis steps in the unit cube (Gaussian steps
reflected at the cube's faces, a symmetric kernel, so the uniform prior needs
no correction), accepting a step whose ln L is above the threshold (the
highest retired ln L); the step scale is the live points' per-dimension
spread times a factor adapted towards a 50% acceptance rate. Every call after
the first carries exactly `batch` vectors, so a library that replays a CUDA
graph per batch shape keeps replaying the same one.

Host-side logic only: the likelihood is a callable on an array of parameter
vectors (for the library: `binding.LogLikeBatch`).
"""
from __future__ import annotations

import dataclasses
from typing import Callable

import numpy as np


@dataclasses.dataclass
class NestedResult:
    log_z: float                 # ln of the evidence
    log_z_err: float             # sqrt(H / N)
    information: float           # H in nats
    samples: np.ndarray          # [M, d] dead points then final live points (parameter space)
    log_weights: np.ndarray      # [M] normalised ln posterior weights
    log_l: np.ndarray            # [M]
    iterations: int
    calls: int                   # batched likelihood calls
    evaluations: int             # parameter vectors evaluated

    def posterior_mean(self):
        w = np.exp(self.log_weights)
        return w @ self.samples

    def posterior_std(self):
        w = np.exp(self.log_weights)
        mu = w @ self.samples
        return np.sqrt(w @ (self.samples - mu) ** 2)


def _reflect(u):
    """Fold a point back into the unit cube by reflection at its faces."""
    u = np.abs(u) % 2.0
    return np.where(u > 1.0, 2.0 - u, u)


def _logaddexp_many(a):
    m = np.max(a)
    return m + np.log(np.sum(np.exp(a - m))) if np.isfinite(m) else m


def run(loglike: Callable[[np.ndarray], np.ndarray], prior_transform: Callable[[np.ndarray], np.ndarray],
        ndim: int, n_live: int = 1000, batch: int = 100, dlogz: float = 0.1, walk_steps: int = 20,
        max_iterations: int = 100000, seed: int = 0) -> NestedResult:
    """Nested sampling with `batch` replacements per iteration.

    loglike(theta[B, d]) -> ln L[B] (float64); prior_transform(u[B, d]) ->
    theta[B, d] maps the unit cube to the prior. Invalid models may return a
    very negative ln L (the library's -1e300): they are never accepted above a
    finite threshold.
    """
    if not 1 <= batch < n_live:
        raise ValueError("batch must be in [1, n_live)")
    rng = np.random.default_rng(seed)
    calls = evals = 0

    def eval_u(u):
        nonlocal calls, evals
        calls += 1
        evals += u.shape[0]
        return np.asarray(loglike(prior_transform(u)), dtype=np.float64)

    u_live = rng.random((n_live, ndim))
    l_live = eval_u(u_live)
    dead_u, dead_l, dead_logw = [], [], []
    log_x = 0.0                      # ln X of the current live set
    log_z = -np.inf
    scale = 0.5
    shrink = 1.0 / (n_live - np.arange(batch))     # E[d ln X] of each retirement in a batch
    it = 0
    for it in range(1, max_iterations + 1):
        order = np.argsort(l_live, kind="stable")
        gone = order[:batch]
        # weights of the retired points: w = X_{i-1} - X_i
        log_x_new = log_x - np.cumsum(shrink)
        log_x_prev = np.concatenate(([log_x], log_x_new[:-1]))
        log_w = log_x_prev + np.log1p(-np.exp(log_x_new - log_x_prev))
        for j, idx in enumerate(gone):
            dead_u.append(u_live[idx].copy())
            dead_l.append(l_live[idx])
            dead_logw.append(log_w[j])
        log_z = _logaddexp_many(np.concatenate(([log_z], log_w + l_live[gone])))
        log_x = log_x_new[-1]
        threshold = l_live[gone[-1]]
        # refill: walkers start from copies of surviving live points
        keep = order[batch:]
        start = rng.choice(keep, size=batch)
        u_w, l_w = u_live[start].copy(), l_live[start].copy()
        spread = np.std(u_live[keep], axis=0) + 1e-12
        acc = 0
        for _ in range(walk_steps):
            prop = _reflect(u_w + scale * spread * rng.standard_normal((batch, ndim)))
            l_p = eval_u(prop)
            ok = l_p > threshold
            u_w[ok], l_w[ok] = prop[ok], l_p[ok]
            acc += int(ok.sum())
        rate = acc / (walk_steps * batch)
        scale *= np.exp(np.clip(rate - 0.5, -0.5, 0.5))
        u_live[gone], l_live[gone] = u_w, l_w
        # stop when the live points can add at most dlogz to ln Z
        if np.isfinite(log_z) and np.logaddexp(log_z, log_x + np.max(l_live)) - log_z < dlogz:
            break
    # the remaining live points share the last volume equally
    log_w_live = np.full(n_live, log_x - np.log(n_live))
    all_u = np.vstack([np.array(dead_u), u_live])
    all_l = np.concatenate([np.array(dead_l), l_live])
    all_logw = np.concatenate([np.array(dead_logw), log_w_live])
    log_z = _logaddexp_many(all_logw + all_l)
    post = all_logw + all_l - log_z
    p = np.exp(post)
    finite = p > 0
    h = float(np.sum(p[finite] * all_l[finite]) - log_z)   # H = sum p ln(L / Z)
    return NestedResult(log_z=float(log_z), log_z_err=float(np.sqrt(max(h, 0.0) / n_live)), information=h,
                        samples=prior_transform(all_u), log_weights=post, log_l=all_l, iterations=it,
                        calls=calls, evaluations=evals)
