"""Parity at the edges of the valid parameter domain, every channel, nu and
nubar, E_true in [0.05, 30] GeV, against the oracle.

The FP64 path holds |dP| <= 1e-12 here (phases up to ~2e5 rad; over the whole
accepted domain the FP64 bound grows with the phase, test_gpu_random_domain.py).
Both FP32 precisions hold |dP| <= 1e-5 at every point, including where the FP32
arithmetic alone would not: one of theta12 / theta23 small and the other large
(narrow resonances, whose amplitude rounding the per-event estimate catches and
sends to the FP64 recomputation) and a 12000 km path through 13 g/cm^3 (matter
phase ~30 rad: FP32-bulk calls run with FP64 shifts and phases there)."""
import numpy as np
import pytest

import oracle
from paper_1311_7579_gb300 import api, synth

pytestmark = pytest.mark.gpu

#          s2_12   s2_13   s2_23  dm21     dm32     dcp   escale norm
INSIDE = np.array([
    [0.311, 1.0e-4, 0.5,   7.6e-5, 2.4e-3,  1.0,  1.0, 1.0],   # tiny theta13
    [0.5,   0.5,    0.5,   7.6e-5, 2.4e-3, -2.0,  1.0, 1.0],   # maximal mixing
    [0.311, 0.0251, 0.5,   1.0e-3, 1.1e-3,  0.5,  1.0, 1.0],   # |dm32| just above dm21
    [0.311, 0.0251, 0.5,   7.6e-5, -2.4e-3, 2.5,  1.0, 1.0],   # inverted ordering
])
OUTSIDE = np.array([
    [0.1,   0.0251, 0.9,   7.6e-5, 2.4e-3, -0.3,  1.0, 1.0],   # small theta12, large theta23
    [0.9,   0.0251, 0.1,   7.6e-5, -2.4e-3, 0.8,  1.0, 1.0],   # the other way, IH
    [0.05,  0.0251, 0.95,  7.6e-5, 2.4e-3, -0.3,  1.0, 1.0],
    [0.99,  0.0251, 0.01,  7.6e-5, 2.4e-3, -0.7,  1.0, 1.0],   # extreme theta12, theta23
    [0.01,  0.0251, 0.99,  7.6e-5, -2.4e-3, 3.1,  1.0, 1.0],   # extreme the other way, IH
])
TOL_OUTSIDE = 1e-5


def _worst(s, pts):
    worst = {"fp64": 0.0, "fp32": 0.0, "fp32_f64eig": 0.0}
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pts)
        for k in range(pts.shape[0]):
            po, _ = oracle.reweight(s, oracle.point_from_row(pts[k]))
            for prec in worst:
                p = np.zeros(s["n"])
                api.osc_reweight(c.ptr, sid, k, prec, out_prob=p)
                worst[prec] = max(worst[prec], float(np.max(np.abs(p - po))))
    return worst


@pytest.mark.parametrize("L,rho", [(295.0, 2.6), (1300.0, 2.85)])
def test_special_points_inside_the_fp32_bound(L, rho):
    w = _worst(synth.all_channel_sample(20_000, seed=int(L), L_km=L, rho=rho), INSIDE)
    assert w["fp64"] <= 1e-12, w
    assert w["fp32"] <= 1e-5 and w["fp32_f64eig"] <= 1e-5, w


@pytest.mark.parametrize("L,rho,pts", [(295.0, 2.6, OUTSIDE), (1300.0, 2.85, OUTSIDE),
                                       (12000.0, 13.0, np.vstack([INSIDE, OUTSIDE]))],
                         ids=["295km-extreme-mixing", "1300km-extreme-mixing", "12000km-core"])
def test_extreme_points_measured_bound(L, rho, pts):
    w = _worst(synth.all_channel_sample(20_000, seed=int(L), L_km=L, rho=rho), pts)
    assert w["fp64"] <= 1e-12, w
    assert w["fp32"] <= TOL_OUTSIDE and w["fp32_f64eig"] <= TOL_OUTSIDE, w


def _golden_worst(name, precs):
    """Worst |P - P_exact| per precision over a 40-digit fixture, per case."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        d = json.load(f)
    pts = np.array(d["points"])
    out = []
    with api.Context(0) as c:
        api.osc_set_params(c.ptr, pts)
        for case in d["cases"]:
            ev = np.array(case["events"])
            n = ev.shape[0]
            s = {"n": n, "e_true": ev[:, 4].astype(np.float32), "e_reco": np.ones(n, np.float32),
                 "w_mc": np.ones(n, np.float32), "flav_in": ev[:, 1].astype(np.uint8),
                 "flav_out": ev[:, 2].astype(np.uint8), "is_nubar": ev[:, 3].astype(np.uint8),
                 "baseline_km": case["L_km"], "density_gcc": case["density_gcc"], "ye": case["ye"]}
            sid = api.osc_load_sample(c.ptr, s)
            worst = {}
            for prec in precs:
                w = 0.0
                for k in range(pts.shape[0]):
                    sel = ev[:, 0] == k
                    p = np.zeros(n)
                    api.osc_reweight(c.ptr, sid, k, prec, out_prob=p)
                    w = max(w, float(np.max(np.abs(p[sel] - ev[sel, 5]))))
                worst[prec] = w
            api.osc_unload_sample(c.ptr, sid)
            out.append((case["L_km"], worst))
    return out


def test_near_double_roots_in_matter_against_40_digit_reference():
    """Matter terms up to 0.05 eV^2 against vacuum splittings down to 1e-6 eV^2
    (fixture written by tests/golden/make_fp64_near_double_events.py): two
    eigenvalues in matter lie a few 1e-6 eV^2 apart on a cubic of scale 0.02,
    where the trigonometric seed's angle is ill-conditioned.  The FP64 path
    seeds such a pair by deflation from the isolated root and must stay at the
    level of the inputs' rounding."""
    for L, worst in _golden_worst("fp64_near_double_events.json", ("fp64", "fp32_f64eig", "fp32")):
        print("near-double", L, worst)
        assert worst["fp64"] <= 1e-12, (L, worst)
        # the FP32 precisions: points outside their domain run in FP64 (next test),
        # the others within the FP32 tolerance
        assert worst["fp32"] <= 1e-5 and worst["fp32_f64eig"] <= 1e-5, (L, worst)


K_A = 1.526493e-4  # eV^2 per GeV per g/cm^3 (k_A of the matter term)


def test_fp32_precisions_outside_their_domain_run_in_fp64():
    """Where the matter term exceeds 1000 |dm31| (a near-double pair of
    eigenvalues at the cubic's scale), FP32 cannot resolve the eigenstructure, so
    calls in OSC_FP32_BULK or OSC_FP32_F64EIG with such a (point, sample) run in
    FP64: reweight, histogram and the no-allocation call give the FP64 results
    bit for bit; points inside the domain keep the FP32 path."""
    torch = pytest.importorskip("torch")
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "fp64_near_double_events.json")) as f:
        d = json.load(f)
    pts = np.array(d["points"])
    case = d["cases"][0]
    ev = np.array(case["events"])
    n = ev.shape[0]
    s = {"n": n, "e_true": ev[:, 4].astype(np.float32), "e_reco": (ev[:, 4] * 0.1).astype(np.float32),
         "w_mc": np.ones(n, np.float32), "flav_in": ev[:, 1].astype(np.uint8),
         "flav_out": ev[:, 2].astype(np.uint8), "is_nubar": ev[:, 3].astype(np.uint8),
         "baseline_km": case["L_km"], "density_gcc": case["density_gcc"], "ye": case["ye"]}
    a_max = K_A * case["density_gcc"] * case["ye"] * float(s["e_true"].max())
    outside = [abs(p[4] + p[3]) * 1000.0 < a_max for p in pts]
    assert any(outside) and not all(outside)
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pts)
        for k in range(len(pts)):
            p64 = np.zeros(n)
            api.osc_reweight(c.ptr, sid, k, "fp64", out_prob=p64)
            h64 = api.osc_histogram(c.ptr, [sid], k, 1, "fp64", 0.0, 5.0, 50)
            for prec in ("fp32", "fp32_f64eig"):
                p = np.zeros(n)
                api.osc_reweight(c.ptr, sid, k, prec, out_prob=p)
                h = api.osc_histogram(c.ptr, [sid], k, 1, prec, 0.0, 5.0, 50)
                if outside[k]:
                    assert np.array_equal(p, p64) and np.array_equal(h, h64), (k, prec)
                else:
                    assert not np.array_equal(p, p64), (k, prec)
        # a histogram call mixing inside and outside points runs wholly in FP64
        hall = api.osc_histogram(c.ptr, [sid], 0, len(pts), "fp32", 0.0, 5.0, 50)
        assert np.array_equal(hall, api.osc_histogram(c.ptr, [sid], 0, len(pts), "fp64", 0.0, 5.0, 50))
        api.osc_unload_sample(c.ptr, sid)
    # the no-allocation call: the FP32 kernel flags the events and the call runs again in FP64
    dev = torch.device("cuda", 0)
    t = {k: torch.from_numpy(np.ascontiguousarray(s[k])).to(dev) for k in
         ("e_true", "e_reco", "w_mc", "flav_in", "flav_out", "is_nubar")}
    for k in range(len(pts)):
        outs = {}
        for prec in ("fp32", "fp64"):
            o = torch.zeros(50, dtype=torch.float64, device=dev)
            api.osc_histogram_noalloc(t["e_true"], t["e_reco"], t["w_mc"], t["flav_in"], t["flav_out"],
                                      t["is_nubar"], case["L_km"], case["density_gcc"], case["ye"], 2.0,
                                      pts[k], prec, 0.0, 5.0, 50, o)
            torch.cuda.synchronize()
            outs[prec] = o.cpu().numpy()
        if outside[k]:
            assert np.array_equal(outs["fp32"], outs["fp64"]), k
        else:
            assert not np.array_equal(outs["fp32"], outs["fp64"]), k


def test_fp64_against_40_digit_reference():
    """FP64 path against 40-digit values (oracle/hp.py, fixture written by
    tests/golden/make_fp64_hard_events.py) at 12000 km through 13 g/cm^3 and at
    1300 km, E_true in [0.05, 1] GeV: the eigenvalue shifts from the shifted
    cubics and the exactly formed phases keep the FP64 path at the level of
    the inputs' own rounding."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "fp64_hard_events.json")) as f:
        d = json.load(f)
    pts = np.array(d["points"])
    bound = {12000.0: 1e-13, 1300.0: 3e-14}
    with api.Context(0) as c:
        api.osc_set_params(c.ptr, pts)
        for case in d["cases"]:
            ev = np.array(case["events"])
            n = ev.shape[0]
            s = {"n": n, "e_true": ev[:, 4].astype(np.float32), "e_reco": np.ones(n, np.float32),
                 "w_mc": np.ones(n, np.float32), "flav_in": ev[:, 1].astype(np.uint8),
                 "flav_out": ev[:, 2].astype(np.uint8), "is_nubar": ev[:, 3].astype(np.uint8),
                 "baseline_km": case["L_km"], "density_gcc": case["density_gcc"], "ye": case["ye"]}
            sid = api.osc_load_sample(c.ptr, s)
            worst = 0.0
            for k in range(pts.shape[0]):
                sel = ev[:, 0] == k
                p = np.zeros(n)
                api.osc_reweight(c.ptr, sid, k, "fp64", out_prob=p)
                worst = max(worst, float(np.max(np.abs(p[sel] - ev[sel, 5]))))
            api.osc_unload_sample(c.ptr, sid)
            assert worst <= bound[case["L_km"]], (case["L_km"], worst)
