"""The debug build (OSC_DEBUG_CHECKS): every kernel checks its work-item ranges,
bin indices and table rows against its buffers and records a violation in an
error word that the host reports.  The same mixed workload -- uneven samples,
one-point and tiled histograms, the bin-centre method, layered matter, FP32 and
FP64 -- must run with no violation and give bitwise the release build's
results."""
import numpy as np
import pytest

from paper_1311_7579_gb300 import api, build, synth

pytestmark = pytest.mark.gpu


def _workload():
    ss = [synth.beam_sample(n, seed=900 + k, L_km=L, rho=rho) for k, (n, L, rho) in
          enumerate([(1, 295.0, 2.6), (31, 810.0, 2.8), (4097, 1300.0, 2.85), (250_001, 295.0, 2.6)])]
    pts = synth.scan_points(20, 9090)
    out = []
    with api.Context(0) as c:
        sids = [api.osc_load_sample(c.ptr, s) for s in ss]
        api.osc_set_params(c.ptr, pts)
        for pt in (1, 4, 16):
            api.osc_set_tile(c.ptr, pt, 0)
            out.append(api.osc_histogram(c.ptr, sids, 0, 20, "fp32", 0.0, 20.0, 100))
        api.osc_set_tile(c.ptr, 0, 0)
        out.append(api.osc_histogram(c.ptr, sids[3:], 0, 1, "fp64", 0.0, 5.0, 100))
        out.append(api.osc_histogram_bin_centre(c.ptr, sids, 0, 20, "fp32", 0.0, 45.0, 180, 0.0, 20.0, 50))
        out.append(api.osc_histogram_bin_centre(c.ptr, sids[3:], 0, 2, "fp64", 0.0, 10.0, 40, 0.0, 5.0, 50))
        api.osc_set_layers(c.ptr, sids[2], [(400.0, 2.6, 0.5), (500.0, 3.3, 0.5), (400.0, 2.6, 0.5)])
        out.append(api.osc_histogram(c.ptr, sids[2:], 0, 20, "fp32", 0.0, 20.0, 100))
        api.osc_sync(c.ptr)  # a recorded violation would raise here
    return out


def test_debug_build_no_violation_and_same_results():
    ref = _workload()
    release = api._lib
    api._lib = api.load_library(build.build(debug_checks=True))
    try:
        dbg = _workload()
    finally:
        api._lib = release
    assert len(dbg) == len(ref)
    for a, b in zip(dbg, ref):
        assert np.array_equal(a, b)
