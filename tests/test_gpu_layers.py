"""Parity of the layered-matter path (osc_set_layers) with the oracle's product
of per-layer constant-density propagators, through the C ABI:
  * per-event probabilities, every channel, nu and nubar: FP64 |dP| <= 1e-12,
    FP32 and FP32_F64EIG |dP| <= 1e-5;
  * histograms: FP64 bins within 1e-9 relative of the oracle; FP32 bins within
    1e-9 relative of the oracle's sum of the GPU's own FP32 weights and within
    1e-5 x sum |w_mc| of the FP64 oracle;
  * one layer set through osc_set_layers equals the load-time constant path,
    and equal-density pieces equal one layer;
  * a layered and a single-layer sample in one launch; the binned method on a
    layered sample; argument checks; served requests on layered samples equal
    the same histograms from osc_histogram, bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_1311_7579_gb300 import api, synth

pytestmark = pytest.mark.gpu

PROFILE = [(300.0, 2.2, 0.5), (700.0, 4.5, 0.49), (300.0, 1.0, 0.47)]
TOL64 = 1e-12
TOL32 = 1e-5
TOL_HIST = 1e-9


def _rel(a, b):
    den = np.maximum(np.abs(b), 1e-300)
    return np.where((a == 0) & (b == 0), 0.0, np.abs(a - b) / den)


def _reweight(ctx, sid, k, prec, n):
    p = np.zeros(n)
    w = np.zeros(n)
    api.osc_reweight(ctx, sid, k, prec, p, w)
    return p, w


@pytest.mark.parametrize("prec,tol", [("fp64", TOL64), ("fp32", TOL32), ("fp32_f64eig", TOL32)])
def test_reweight_matches_oracle_every_channel(prec, tol):
    s = synth.all_channel_sample(40_000, seed=31, L_km=1300.0)
    pts = synth.scan_points(4, 4141)
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_layers(c.ptr, sid, PROFILE)
        api.osc_set_params(c.ptr, pts)
        for k in range(4):
            p, w = _reweight(c.ptr, sid, k, prec, s["n"])
            po, wo = oracle.reweight_layers(s, oracle.point_from_row(pts[k]), PROFILE)
            assert np.max(np.abs(p - po)) <= tol, (k, np.max(np.abs(p - po)))
            # weight = P w_mc norm; the FP32 paths round P w_mc to FP32 once more
            bound = (tol + 1e-7) * np.abs(s["w_mc"]).astype(np.float64) * pts[k][7]
            assert np.all(np.abs(w - wo) <= bound)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_f64eig"])
def test_histogram_matches_oracle(prec):
    s = synth.all_channel_sample(30_001, seed=32, L_km=1300.0)
    pts = synth.scan_points(5, 4242)
    lo, hi, nb = 0.0, 20.0, 60
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_layers(c.ptr, sid, PROFILE)
        api.osc_set_params(c.ptr, pts)
        h = api.osc_histogram(c.ptr, [sid], 0, 5, prec, lo, hi, nb)[0]
        for k in range(5):
            row = pts[k]
            ho = oracle.histogram_layers(s, [row], PROFILE, lo, hi, nb)[0]
            if prec == "fp64":
                assert np.max(_rel(h[k], ho)) <= TOL_HIST
            else:
                _, w = _reweight(c.ptr, sid, k, prec, s["n"])
                hw = oracle.hist_from_weights(s["e_reco"], w, row[6], lo, hi, nb)
                assert np.max(_rel(h[k], hw)) <= TOL_HIST
                wsum = oracle.hist_from_weights(s["e_reco"], np.abs(s["w_mc"]).astype(np.float64), row[6], lo, hi, nb)
                assert np.all(np.abs(h[k] - ho) <= TOL32 * wsum + 1e-12)


def test_one_layer_equals_constant_density_and_split_layers():
    s = synth.beam_sample(50_000, seed=33, L_km=810.0, rho=2.8)
    pts = synth.scan_points(3, 4343)
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pts)
        ref = {p: api.osc_histogram(c.ptr, [sid], 0, 3, p, 0.0, 10.0, 50) for p in ("fp64", "fp32")}
        api.osc_set_layers(c.ptr, sid, [(810.0, 2.8, 0.5)])
        for p in ("fp64", "fp32"):
            assert np.array_equal(api.osc_histogram(c.ptr, [sid], 0, 3, p, 0.0, 10.0, 50), ref[p])
        api.osc_set_layers(c.ptr, sid, [(200.0, 2.8, 0.5), (410.0, 2.8, 0.5), (200.0, 2.8, 0.5)])
        for p, tol in (("fp64", 1e-12), ("fp32", 1e-5)):
            pl, _ = _reweight(c.ptr, sid, 1, p, s["n"])
            po, _ = oracle.reweight(s, oracle.point_from_row(pts[1]))
            assert np.max(np.abs(pl - po)) <= tol


def test_layered_and_single_layer_samples_in_one_launch():
    s1 = synth.all_channel_sample(20_000, seed=34, L_km=1300.0)
    s2 = synth.beam_sample(15_000, seed=35)
    pts = synth.scan_points(8, 4444)
    with api.Context(0) as c:
        a = api.osc_load_sample(c.ptr, s1)
        b = api.osc_load_sample(c.ptr, s2)
        api.osc_set_layers(c.ptr, a, PROFILE)
        api.osc_set_params(c.ptr, pts)
        h = api.osc_histogram(c.ptr, [a, b], 0, 8, "fp64", 0.0, 10.0, 40)
        for k in (0, 7):
            ha = oracle.histogram_layers(s1, [pts[k]], PROFILE, 0.0, 10.0, 40)[0]
            hb = oracle.histogram(s2, [pts[k]], 0.0, 10.0, 40)[0]
            assert np.max(_rel(h[0, k], ha)) <= TOL_HIST
            assert np.max(_rel(h[1, k], hb)) <= TOL_HIST


def test_bin_centre_on_layered_sample():
    s = synth.all_channel_sample(25_000, seed=36, L_km=1300.0)
    row = synth.scan_points(1, 4545)[0]
    tb = (0.0, 30.5, 61)
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_layers(c.ptr, sid, PROFILE)
        api.osc_set_params(c.ptr, row[None, :])
        h = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 1, "fp64", *tb, 0.0, 20.0, 40)[0, 0]
    t = oracle.bins(s["e_true"], 1.0, tb[0], tb[1], tb[2])
    cen = np.array([oracle.true_centre(*tb, k) if k >= 0 else 1.0 for k in t], dtype=np.float32)
    sc = dict(s, e_true=cen)
    _, w = oracle.reweight_layers(sc, oracle.point_from_row(row), PROFILE)
    w[t < 0] = 0.0
    ho = oracle.hist_from_weights(s["e_reco"], w, row[6], 0.0, 20.0, 40)
    assert np.max(_rel(h, ho)) <= TOL_HIST


def test_full_size_uneven_sample_with_layers():
    s = synth.uneven_samples(sizes=(1, 1, 2_000_000))[2]  # 2M events, 1300 km beam shape
    pts = synth.uneven_points(16, 4646)
    layers = [(400.0, 2.6, 0.5), (500.0, 3.3, 0.5), (400.0, 2.6, 0.5)]
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_layers(c.ptr, sid, layers)
        api.osc_set_params(c.ptr, pts)
        h = api.osc_histogram(c.ptr, [sid], 0, 16, "fp32", 0.0, 20.0, 100)[0]
        assert np.isfinite(h).all()
        for k in (0, 13):
            ho = oracle.histogram_layers(s, [pts[k]], layers, 0.0, 20.0, 100)[0]
            wsum = oracle.hist_from_weights(s["e_reco"], np.abs(s["w_mc"]).astype(np.float64), pts[k][6],
                                            0.0, 20.0, 100)
            assert np.all(np.abs(h[k] - ho) <= TOL32 * wsum + 1e-12)


def test_layer_arguments_and_serving_state():
    s = synth.beam_sample(1000, seed=37)
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        for bad in ([], [(100.0, 2.0, 0.5)] * 17, [(-1.0, 2.0, 0.5)], [(100.0, -2.0, 0.5)],
                    [(100.0, 2.0, 1.5)], [(np.inf, 2.0, 0.5)]):
            with pytest.raises(api.OscError):
                api.osc_set_layers(c.ptr, sid, bad)
        with pytest.raises(api.OscError):
            api.osc_set_layers(c.ptr, sid + 99, PROFILE)
        api.osc_set_layers(c.ptr, sid, PROFILE)
        api.osc_set_params(c.ptr, synth.table1_point()[None, :])
        api.osc_serve_start(c.ptr, 4, 0.0, 5.0, 10)
        try:
            # the sample's path cannot change while batches may hold it
            with pytest.raises(api.OscError):
                api.osc_set_layers(c.ptr, sid, [(295.0, 2.6, 0.5)])
        finally:
            api.osc_serve_stop(c.ptr)
        h = api.osc_histogram(c.ptr, [sid], 0, 1, "fp64", 0.0, 5.0, 10)
        assert np.isfinite(h).all()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_serving_layered_and_single_layer_requests(prec):
    """Requests on a layered and a single-layer sample, queued together, each
    give the histogram that osc_histogram gives for the same point (same kernels,
    exact accumulation: bit for bit)."""
    s1 = synth.all_channel_sample(20_000, seed=38, L_km=1300.0)
    s2 = synth.beam_sample(15_000, seed=39)
    pts = synth.scan_points(6, 4747)
    lo, hi, nb = 0.0, 10.0, 20
    with api.Context(0) as c:
        a = api.osc_load_sample(c.ptr, s1)
        b = api.osc_load_sample(c.ptr, s2)
        api.osc_set_layers(c.ptr, a, PROFILE)
        api.osc_set_params(c.ptr, pts)
        ref_a = api.osc_histogram(c.ptr, [a], 0, 6, prec, lo, hi, nb)[0]
        ref_b = api.osc_histogram(c.ptr, [b], 0, 6, prec, lo, hi, nb)[0]
        api.osc_serve_start(c.ptr, 16, lo, hi, nb)
        try:
            tickets = []
            for k in range(6):
                tickets.append((0, k, api.osc_submit(c.ptr, a, pts[k], prec)))
                tickets.append((1, k, api.osc_submit(c.ptr, b, pts[k], prec)))
            for which, k, t in tickets:
                h, _ = api.osc_wait(c.ptr, t, nb, 20000)
                ref = ref_a[k] if which == 0 else ref_b[k]
                assert np.array_equal(h, ref), (which, k)
        finally:
            api.osc_serve_stop(c.ptr)


def test_fp32_domain_uses_the_densest_layer_and_serving_applies_it():
    """The FP32 domain rule (matter term at most 1000 |dm31|, else the call runs in
    FP64) takes a layered sample's densest layer: a tiny-splitting point is
    outside it only because of the dense middle layer, and its FP32 and
    FP32_F64EIG results then equal FP64 bit for bit, through osc_histogram,
    osc_reweight and served requests; a physical point keeps the FP32 path."""
    s = synth.all_channel_sample(20_000, seed=41, L_km=6000.0, rho=1.0, e_lo=2.0, e_hi=40.0)
    tiny = np.array([0.311, 0.0251, 0.5, 1.0e-6, 1.4e-5, 0.7, 1.0, 1.0])   # |dm31| = 1.5e-5 eV^2
    phys = synth.table1_point()
    pts = np.stack([tiny, phys])
    # |A|max = k_A rho Y_e E_max: 1.526e-4 * 1.0 * 0.5 * 40 = 3.1e-3 -> 204 |dm31| for the thin
    # layers, 12 * 204 = 2.4e3 |dm31| for the 12 g/cm^3 middle layer
    layers = [(2000.0, 1.0, 0.5), (2000.0, 12.0, 0.5), (2000.0, 1.0, 0.5)]
    lo, hi, nb = 0.0, 40.0, 20
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pts)
        # one thin layer: inside the domain, FP32 stays FP32
        h32 = api.osc_histogram(c.ptr, [sid], 0, 1, "fp32", lo, hi, nb)
        assert not np.array_equal(h32, api.osc_histogram(c.ptr, [sid], 0, 1, "fp64", lo, hi, nb))
        api.osc_set_layers(c.ptr, sid, layers)
        h64 = api.osc_histogram(c.ptr, [sid], 0, 1, "fp64", lo, hi, nb)
        p64, _ = _reweight(c.ptr, sid, 0, "fp64", s["n"])
        for prec in ("fp32", "fp32_f64eig"):
            assert np.array_equal(api.osc_histogram(c.ptr, [sid], 0, 1, prec, lo, hi, nb), h64), prec
            assert np.array_equal(_reweight(c.ptr, sid, 0, prec, s["n"])[0], p64), prec
        # the physical point through the same layers keeps the FP32 path
        p32 = _reweight(c.ptr, sid, 1, "fp32", s["n"])[0]
        assert not np.array_equal(p32, _reweight(c.ptr, sid, 1, "fp64", s["n"])[0])
        api.osc_serve_start(c.ptr, 8, lo, hi, nb)
        try:
            h, _ = api.osc_wait(c.ptr, api.osc_submit(c.ptr, sid, tiny, "fp32"), nb, 20000)
            assert np.array_equal(h, h64[0, 0])
        finally:
            api.osc_serve_stop(c.ptr)
        api.osc_unload_sample(c.ptr, sid)


def test_fp32_bulk_through_layers_needs_a_resolved_solar_splitting():
    """FP32-bulk through layers also needs dm21 >= 5e-3 |dm31| (the layer update
    divides by the solar gap, which FP32 seeds cannot resolve below that): a
    point with dm21 = 4e-4 |dm31| runs in FP64 on a layered sample, bit for bit,
    while FP32_F64EIG (FP64 shifts) keeps its own path and a single-layer sample
    keeps FP32-bulk."""
    s = synth.all_channel_sample(20_000, seed=43, L_km=3000.0, rho=3.0)
    pt = np.array([[0.311, 0.0251, 0.5, 1.0e-6, 2.5e-3, 0.7, 1.0, 1.0]])
    lo, hi, nb = 0.0, 30.0, 20
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pt)
        single32 = _reweight(c.ptr, sid, 0, "fp32", s["n"])[0]
        assert not np.array_equal(single32, _reweight(c.ptr, sid, 0, "fp64", s["n"])[0])
        api.osc_set_layers(c.ptr, sid, PROFILE)
        p64 = _reweight(c.ptr, sid, 0, "fp64", s["n"])[0]
        assert np.array_equal(_reweight(c.ptr, sid, 0, "fp32", s["n"])[0], p64)
        assert np.array_equal(api.osc_histogram(c.ptr, [sid], 0, 1, "fp32", lo, hi, nb),
                              api.osc_histogram(c.ptr, [sid], 0, 1, "fp64", lo, hi, nb))
        pmix = _reweight(c.ptr, sid, 0, "fp32_f64eig", s["n"])[0]
        assert not np.array_equal(pmix, p64)
        assert np.max(np.abs(pmix - p64)) <= TOL32
        api.osc_unload_sample(c.ptr, sid)
