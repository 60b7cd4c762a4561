"""Randomized parity over the whole domain osc_set_params accepts (CPU oracle vs
the C ABI), single layer and through random layer profiles:

  * s^2 of the three angles anywhere in (0.001, 0.999) (s^2_13 to 0.6), dm21
    log-uniform in [1e-6, 5e-4] eV^2, |dm32| log-uniform from 1.6 dm21 to 2e-2,
    either ordering, any delta; baselines 1-13000 km, densities 0-13 g/cm^3,
    E_true log-uniform in [0.05, 50] GeV, every channel, nu and nubar.

This is where the eigenvalue cubic has near-double roots and the resonances are
narrow.  Both FP32 precisions must hold the FP32 tolerance |dP| <= 1e-5 for every
event: what FP32 arithmetic cannot resolve runs with FP64 shifts and phases
(FP32_F64EIG) or in FP64, per call or per event (include/osc.h, osc_precision).

FP64: the phases reach ~1e6 rad here, and an FP64 evaluation of the definition
(the GPU's or the oracle's) carries a phase error of order 2^-53 times the
phase.  Each event's bound is therefore 1e-12 + 4 * 2^-52 * Phi, with Phi =
c_L L (|dm31| + dm21 + |A|) / E_true an upper bound of its largest phase (the
reading of Sec. 2.2's 1e-12 over this domain); events with Phi <= 1e3 rad, the
scale of the paper's validation at 295 km, are held to 1e-12 itself.  Through
layers (a generalisation the paper does not have) the FP64 layer update, whose
eigenvector weights divide by the distance of an eigenvalue in matter from a
vacuum eigenvalue, is less well conditioned than the single-layer form, and
its bound is TOL64_LAYERS = 5e-11 (measured 1.55e-11 at worst, at phases
below 1e3 rad).
"""
import numpy as np
import pytest

import oracle
from paper_1311_7579_gb300 import api

pytestmark = pytest.mark.gpu

N = 5000
TRIALS = 40
TOL64 = 1e-12
TOL64_LAYERS = 5e-11
TOL32 = 1e-5
C_L = 2.533865  # rad per (eV^2 km / GeV)
K_A = 1.526493e-4  # eV^2 per GeV per g/cm^3


def _point(rng):
    dm21 = float(np.exp(rng.uniform(np.log(1e-6), np.log(5e-4))))
    adm = float(np.exp(rng.uniform(np.log(1.6 * dm21), np.log(2e-2))))
    return np.array([rng.uniform(0.001, 0.999), rng.uniform(0.001, 0.6), rng.uniform(0.001, 0.999), dm21,
                     rng.choice([-1.0, 1.0]) * adm, rng.uniform(-7, 7), rng.uniform(0.8, 1.2), 1.0])


def _sample(rng):
    e = np.exp(rng.uniform(np.log(0.05), np.log(50.0), N)).astype(np.float32)
    return dict(n=N, e_true=e, e_reco=e.copy(), w_mc=np.ones(N, np.float32),
                flav_in=rng.integers(0, 3, N).astype(np.uint8), flav_out=rng.integers(0, 3, N).astype(np.uint8),
                is_nubar=rng.integers(0, 2, N).astype(np.uint8), baseline_km=float(rng.uniform(1, 13000)),
                density_gcc=float(rng.uniform(0, 13)), ye=float(rng.uniform(0.4, 0.55)))


@pytest.mark.parametrize("layered", [False, True], ids=["single-layer", "layers"])
def test_random_points_over_the_accepted_domain(layered):
    rng = np.random.default_rng(20261204 + int(layered))
    worst = {"fp64": 0.0, "fp32": 0.0, "fp32_f64eig": 0.0}
    worst64_ratio = 0.0   # FP64 |dP| over its phase-conditioned bound
    worst64_small = 0.0   # FP64 |dP| over events with Phi <= 1e3 rad
    with api.Context(0) as c:
        for _ in range(TRIALS):
            pt = _point(rng)
            s = _sample(rng)
            sid = api.osc_load_sample(c.ptr, s)
            if layered:
                layers = [(float(rng.uniform(50, 4000)), float(rng.uniform(0, 13)), float(rng.uniform(0.45, 0.5)))
                          for _ in range(int(rng.integers(2, 6)))]
                api.osc_set_layers(c.ptr, sid, layers)
                ref, _ = oracle.reweight_layers(s, oracle.point_from_row(pt), layers)
                L_tot = sum(x[0] for x in layers)
                ka = max(K_A * x[1] * x[2] for x in layers)
            else:
                ref, _ = oracle.reweight(s, oracle.point_from_row(pt))
                L_tot = s["baseline_km"]
                ka = K_A * s["density_gcc"] * s["ye"]
            E = s["e_true"].astype(np.float64)
            phi = C_L * L_tot * (abs(pt[4] + pt[3]) + pt[3] + ka * E) / E
            bound64 = TOL64 + 4 * 2.0 ** -52 * phi
            api.osc_set_params(c.ptr, pt[None, :])
            for prec in worst:
                p = np.zeros(N)
                api.osc_reweight(c.ptr, sid, 0, prec, out_prob=p)
                assert np.all(np.isfinite(p)), prec
                d = np.abs(p - ref)
                worst[prec] = max(worst[prec], float(np.max(d)))
                if prec == "fp64":
                    worst64_ratio = max(worst64_ratio, float(np.max(d / bound64)))
                    small = phi <= 1e3
                    if small.any():
                        worst64_small = max(worst64_small, float(np.max(d[small])))
            api.osc_unload_sample(c.ptr, sid)
    print("worst |dP|", worst, "fp64 / bound", worst64_ratio, "fp64 at Phi <= 1e3", worst64_small)
    if layered:
        assert worst["fp64"] <= TOL64_LAYERS, worst
    else:
        assert worst64_ratio <= 1.0 and worst64_small <= TOL64, (worst, worst64_ratio, worst64_small)
    assert worst["fp32"] <= TOL32 and worst["fp32_f64eig"] <= TOL32, worst
