"""The toy-fit driver's host parts on CPU: the Poisson likelihood of Eq. (2)
against scipy's pmf, and the Metropolis-Hastings sampler against a known
Gaussian target (mean, covariance, bounds, determinism)."""
import math

import numpy as np
import pytest

from paper_1311_7579_gb300 import fit


def test_poisson_loglike_matches_scipy():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(1)
    lam = rng.uniform(0.01, 50.0, 100)
    data = rng.poisson(lam).astype(float)
    ref = float(np.sum(stats.poisson.logpmf(data, lam)))
    assert abs(fit.poisson_loglike(data, lam) - ref) < 1e-9 * abs(ref)
    # an empty expected bin with data is impossible; without data it contributes nothing
    assert fit.poisson_loglike([0.0, 3.0], [0.0, 2.0]) == pytest.approx(float(stats.poisson.logpmf(3, 2.0)))
    assert fit.poisson_loglike([1.0], [0.0]) == -math.inf


def test_metropolis_gaussian_target():
    mu = np.array([0.5, 2.4e-3])
    sd = np.array([0.03, 5e-5])
    rho = 0.4
    cov = np.array([[sd[0] ** 2, rho * sd[0] * sd[1]], [rho * sd[0] * sd[1], sd[1] ** 2]])
    icov = np.linalg.inv(cov)

    def logpost(x):
        d = x - mu
        return -0.5 * float(d @ icov @ d)

    chain, lps, acc = fit.metropolis(logpost, mu, 1.5 * sd, 60000, np.random.default_rng(7))
    burn = chain[5000:]
    assert 0.2 < acc < 0.7
    assert np.all(np.abs(burn.mean(axis=0) - mu) < 0.05 * sd * 10)
    c = np.cov(burn.T)
    assert np.allclose(np.sqrt(np.diag(c)), sd, rtol=0.08)
    assert abs(c[0, 1] / np.sqrt(c[0, 0] * c[1, 1]) - rho) < 0.06


def test_metropolis_bounds_and_determinism():
    def logpost(x):
        return -0.5 * float(np.sum(x * x))

    lo, hi = np.array([-0.5, -0.5]), np.array([0.5, 1.0])
    c1, _, _ = fit.metropolis(logpost, [0.0, 0.0], [0.3, 0.3], 5000, np.random.default_rng(3), lo, hi)
    c2, _, _ = fit.metropolis(logpost, [0.0, 0.0], [0.3, 0.3], 5000, np.random.default_rng(3), lo, hi)
    assert np.array_equal(c1, c2)
    assert np.all(c1 >= lo) and np.all(c1 <= hi)
