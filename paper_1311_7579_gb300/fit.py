"""Toy oscillation fit (Sec. 2.2): Metropolis-Hastings over (sin^2 theta23, dm32)
with flat priors and the binned Poisson likelihood of Eq. (2),
    L(o, f | D) = prod_i p(D_i | o, f),   p = Poisson pmf,
where every step rebuilds the expected spectrum by reweighting the Monte Carlo
sample event by event on the GPU (one osc_set_params + osc_histogram call).
The other parameters stay at their Table 1 values, as in the paper's fit.

The paper's fake data (a Landau spectrum, BAT) are not available; the fake
data here are Poisson draws of the expected spectrum of a synthetic
Gamma-shaped beam sample at the Table 1 point.  All arithmetic of the
reweighting runs in the CUDA library; this module is the host-side driver.
"""
from __future__ import annotations

import math

import numpy as np

from . import api, synth


def log_factorials(data) -> np.ndarray:
    """log(D_i!) of every bin (constant over a fit: computed once)."""
    return np.array([math.lgamma(d + 1.0) for d in np.asarray(data, dtype=np.float64)])


def poisson_loglike(data, expected, lgam=None) -> float:
    """log of Eq. (2): sum_i [D_i log(lam_i) - lam_i - log(D_i!)], with lam_i the
    expected count of bin i (bins with lam_i = 0 contribute only if D_i = 0).
    lgam: log_factorials(data), when the caller has them."""
    data = np.asarray(data, dtype=np.float64)
    lam = np.asarray(expected, dtype=np.float64)
    if lgam is None:
        lgam = log_factorials(data)
    with np.errstate(divide="ignore", invalid="ignore"):
        term = np.where(lam > 0, data * np.log(np.where(lam > 0, lam, 1.0)) - lam, np.where(data > 0, -np.inf, 0.0))
    return float(np.sum(term - lgam))


def metropolis(logpost, x0, sigma, n_steps, rng, lower=None, upper=None):
    """Random-walk Metropolis-Hastings with Gaussian proposals of widths `sigma`
    and flat priors on the box [lower, upper].  The generator is advanced by the
    same draws every step (proposal, then the uniform), so two runs with equal
    seeds and equal log-posteriors follow the same chain.  Returns (chain,
    log-posteriors, acceptance fraction)."""
    x = np.asarray(x0, dtype=np.float64).copy()
    sigma = np.asarray(sigma, dtype=np.float64)
    lp = logpost(x)
    chain = np.empty((n_steps, x.size))
    lps = np.empty(n_steps)
    acc = 0
    for k in range(n_steps):
        y = x + sigma * rng.standard_normal(x.size)
        u = rng.random()
        inside = (lower is None or np.all(y >= lower)) and (upper is None or np.all(y <= upper))
        if inside:
            lpy = logpost(y)
            if math.log(u) < lpy - lp:
                x, lp = y, lpy
                acc += 1
        chain[k] = x
        lps[k] = lp
    return chain, lps, acc / max(1, n_steps)


class ToyFit:
    """Expected spectrum and log-likelihood of (sin^2 theta23, dm32) for one
    resident sample.  exposure scales the MC histogram to expected counts."""

    def __init__(self, ctx, sample_id, data, exposure, lo=0.0, hi=5.0, nbins=100, prec="fp32", base_point=None):
        self.ctx = ctx
        self.sid = sample_id
        self.data = np.asarray(data, dtype=np.float64)
        self.exposure = float(exposure)
        self.lo, self.hi, self.nbins = lo, hi, int(nbins)
        self.prec = prec
        self.base = synth.table1_point() if base_point is None else np.asarray(base_point, dtype=np.float64)
        self.lgam = log_factorials(self.data)
        # one output buffer for every step, page-locked when torch can provide it
        # (the histogram kernel then writes it directly, with no staging copy)
        try:
            import torch
            self.out = torch.zeros((1, 1, self.nbins), dtype=torch.float64).pin_memory().numpy()
        except Exception:
            self.out = np.zeros((1, 1, self.nbins))
        # the step's call with its arguments marshalled once; each step writes
        # the two fitted fields into its point buffer
        self.call = api.PointHistogram(ctx, [sample_id], prec, lo, hi, self.nbins, out=self.out)
        self.call.point[:] = self.base
        self.calls = 0

    def point(self, x):
        row = self.base.copy()
        row[2], row[4] = x[0], x[1]
        return row

    def expected(self, x):
        p = self.call.point
        p[2] = x[0]
        p[4] = x[1]
        self.call()
        self.calls += 1
        return self.exposure * self.out[0, 0]

    def loglike(self, x):
        return poisson_loglike(self.data, self.expected(x), self.lgam)


def fake_data(expected, seed):
    """Poisson draws of an expected spectrum (the toy fit's 'data')."""
    return np.random.default_rng(seed).poisson(np.asarray(expected)).astype(np.float64)


def exposure_for(sample, n_unoscillated, lo=0.0, hi=5.0):
    """Scale so that the unoscillated in-range MC weight corresponds to
    n_unoscillated expected events."""
    er = sample["e_reco"]
    w = sample["w_mc"].astype(np.float64)
    sel = (er >= lo) & (er < hi)
    return float(n_unoscillated) / float(w[sel].sum())
