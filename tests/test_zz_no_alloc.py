"""The allocation-free one-point histogram entry point, osc_histogram_noalloc.

It is for callers that cannot allocate device memory (a framework that owns
all of it, or a step that must not allocate).  This file is collected last so
that a run stopping at the first failure has run every other test first.
Checked through the C ABI on two calls in a row: bitwise against osc_histogram
(both sum the same events exactly in 128-bit fixed point with the same scale
when w_abs_max is the sample's largest |w_mc|), and the FP64 result against the
CPU oracle within the histogram tolerance of the parity tests (1e-9 relative
per bin)."""
import numpy as np
import pytest

import oracle
from paper_1311_7579_gb300 import api, synth

pytestmark = pytest.mark.gpu

TOL_HIST = 1e-9
LO, HI, NB = 0.0, 5.0, 100


def _rel(a, b):
    den = np.maximum(np.abs(b), 1e-300)
    return np.where((a == 0) & (b == 0), 0.0, np.abs(a - b) / den)


def test_noalloc_matches_histogram_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    s = synth.all_channel_sample(40000, seed=31, L_km=810.0, rho=2.8, e_hi=10.0)
    pts = synth.scan_points(2, seed=32)
    dev = {k: torch.from_numpy(np.ascontiguousarray(s[k])).cuda()
           for k in ("e_true", "e_reco", "w_mc", "flav_in", "flav_out", "is_nubar")}
    wmax = float(np.max(np.abs(s["w_mc"])))
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pts)
        ref = {prec: api.osc_histogram(c.ptr, [sid], 0, 2, prec, LO, HI, NB)[0] for prec in ("fp32", "fp64")}
    ho = oracle.histogram(s, pts, LO, HI, NB)
    for call in range(2):
        for prec in ("fp32", "fp64"):
            for k in range(2):
                out = torch.full((NB,), -1.0, dtype=torch.float64, device="cuda")
                api.osc_histogram_noalloc(dev["e_true"], dev["e_reco"], dev["w_mc"], dev["flav_in"],
                                          dev["flav_out"], dev["is_nubar"], s["baseline_km"], s["density_gcc"],
                                          s["ye"], wmax, pts[k], prec, LO, HI, NB, out)
                got = out.cpu().numpy()
                assert np.array_equal(got, ref[prec][k]), (call, prec, k)
                if prec == "fp64":
                    assert np.max(_rel(got, ho[k])) <= TOL_HIST, (call, k)


def test_noalloc_rejects_oversized_and_invalid_input():
    torch = pytest.importorskip("torch")
    n = 1000
    s = synth.table1_sample(n, seed=33)
    dev = {k: torch.from_numpy(np.ascontiguousarray(s[k])).cuda()
           for k in ("e_true", "e_reco", "w_mc", "flav_in", "flav_out", "is_nubar")}
    out = torch.zeros(8192, dtype=torch.float64, device="cuda")
    args = [dev["e_true"], dev["e_reco"], dev["w_mc"], dev["flav_in"], dev["flav_out"], dev["is_nubar"],
            295.0, 2.6, 0.5, 1.5, synth.table1_point(), "fp32", LO, HI]
    with pytest.raises(api.OscError) as e:
        api.osc_histogram_noalloc(*args, 4097, out)
    assert e.value.status == api.OSC_E_ARG
    bad = dev["flav_out"].clone()
    bad[17] = 7
    args2 = list(args)
    args2[4] = bad
    out[:] = -1.0
    with pytest.raises(api.OscError) as e:
        api.osc_histogram_noalloc(*args2, NB, out)
    assert e.value.status == api.OSC_E_RANGE
    assert bool((out[:NB] == -1.0).all())
    # still usable afterwards
    api.osc_histogram_noalloc(*args, NB, out)
    assert float(out[:NB].sum()) > 0
