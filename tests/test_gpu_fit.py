"""Toy oscillation fit on the GPU (Sec. 2.2): the same Metropolis-Hastings chain
driven by GPU FP64 histograms and by the CPU oracle's histograms (equal seeds)
makes the same decisions -- the paper's CPU-vs-GPU posterior comparison --
and the FP32-bulk chain recovers the generating point."""
import numpy as np
import pytest

import oracle
from paper_1311_7579_gb300 import api, fit, synth

pytestmark = pytest.mark.gpu
LO, HI, NB = 0.0, 5.0, 100
TRUE = np.array([0.5, 2.4e-3])
SIG = np.array([0.02, 3e-5])
LOWER, UPPER = np.array([0.3, 2.0e-3]), np.array([0.7, 3.0e-3])


def _setup(ctx, n_mc, n_data):
    s = synth.table1_sample(n_mc, seed=91)
    sid = api.osc_load_sample(ctx, s)
    expo = fit.exposure_for(s, n_data, LO, HI)
    ftrue = fit.ToyFit(ctx, sid, np.zeros(NB), expo, LO, HI, NB, "fp64")
    data = fit.fake_data(ftrue.expected(TRUE), seed=92)
    return s, sid, expo, data


def test_gpu_chain_equals_oracle_chain():
    with api.Context(0) as c:
        s, sid, expo, data = _setup(c.ptr, 100_000, 3000)
        g = fit.ToyFit(c.ptr, sid, data, expo, LO, HI, NB, "fp64")
        chain_g, lp_g, acc_g = fit.metropolis(g.loglike, TRUE, SIG, 150, np.random.default_rng(5), LOWER, UPPER)

    def oracle_loglike(x):
        row = synth.table1_point()
        row[2], row[4] = x[0], x[1]
        return fit.poisson_loglike(data, expo * oracle.histogram(s, [row], LO, HI, NB)[0])

    chain_o, lp_o, acc_o = fit.metropolis(oracle_loglike, TRUE, SIG, 150, np.random.default_rng(5), LOWER, UPPER)
    assert np.array_equal(chain_g, chain_o)
    assert np.max(np.abs(lp_g - lp_o)) < 1e-6
    assert acc_g == acc_o and acc_g > 0.05


def test_fp32_chain_recovers_generating_point():
    with api.Context(0) as c:
        s, sid, expo, data = _setup(c.ptr, 2_000_000, 20000)
        f32 = fit.ToyFit(c.ptr, sid, data, expo, LO, HI, NB, "fp32")
        chain, lp, acc = fit.metropolis(f32.loglike, [0.45, 2.3e-3], SIG, 3000, np.random.default_rng(6), LOWER,
                                        UPPER)
    post = chain[500:]
    assert 0.05 < acc < 0.8
    m, sd = post.mean(axis=0), post.std(axis=0)
    # sin^2 theta23 is octant-degenerate in nu_mu disappearance: fold about 0.5
    s23 = 0.5 + np.abs(post[:, 0] - 0.5)
    assert abs(np.mean(s23) - 0.5) < 0.05
    assert abs(m[1] - TRUE[1]) < 4 * sd[1] + 2e-5
