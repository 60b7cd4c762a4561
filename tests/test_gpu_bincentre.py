"""Parity of the binned (bin-centre) method, osc_histogram_bin_centre, with the
oracle's binned reweighting (Sec. 1.1.1), through the C ABI:
  * FP64 bins within 1e-9 relative of the oracle; FP32 and FP32_F64EIG bins
    within 1e-5 x the bin's sum of |w_mc| (|dP| <= 1e-5 per event);
  * events on true-bin edges, just below them and outside the true range: the
    true-bin choice is the oracle's, or FP64 bins would miss by O(0.1);
  * ragged and tiny samples, several samples and points in one launch, both
    finalize routes (fused for small outputs, separate kernel for large ones);
  * events placed at bin centres: binned == event-by-event histogram;
  * the 25 MeV bin at 0.6 GeV on quadrature nodes of a Gamma spectrum: the
    GPU's binning effect equals the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_1311_7579_gb300 import api, synth

pytestmark = pytest.mark.gpu

TOL_HIST = 1e-9
TOL_FP32 = 1e-5


def _rel(a, b):
    den = np.maximum(np.abs(b), 1e-300)
    return np.where((a == 0) & (b == 0), 0.0, np.abs(a - b) / den)


def _wsum(s, row, lo, hi, nb):
    return oracle.hist_from_weights(s["e_reco"], np.abs(s["w_mc"]).astype(np.float64), row[6], lo, hi, nb)


def _check(h, s, rows, tb, lo, hi, nb, prec):
    ho = oracle.histogram_bin_centre(s, rows, *tb, lo, hi, nb)
    for k, row in enumerate(rows):
        if prec == "fp64":
            assert np.max(_rel(h[k], ho[k])) <= TOL_HIST, k
        else:
            assert np.all(np.abs(h[k] - ho[k]) <= TOL_FP32 * _wsum(s, row, lo, hi, nb) + 1e-12), k


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_f64eig"])
def test_bin_centre_matches_oracle_all_channels(prec):
    s = synth.all_channel_sample(60_001, seed=12)
    pts = synth.scan_points(6, 515)
    tb = (0.0, 30.5, 122)
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pts)
        h = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 6, prec, *tb, 0.0, 20.0, 80)[0]
    _check(h, s, pts, tb, 0.0, 20.0, 80, prec)


def _edge_sample():
    """Events on every true-bin edge, one FP32 ulp below each edge, and outside
    the true range, with wide bins where P changes fast between centres."""
    t_lo, t_hi, T = 0.1, 3.1, 12
    edges = np.array([t_lo + k * (t_hi - t_lo) / T for k in range(T + 1)], dtype=np.float32)
    below = np.nextafter(edges, np.float32(0))
    outside = np.array([0.05, 0.0999, 3.1, 3.2, 7.0], dtype=np.float32)
    e = np.concatenate([edges, below, outside, edges, below])
    n = e.size
    rng = np.random.default_rng(2)
    s = {"n": n, "e_true": e.astype(np.float32), "e_reco": rng.uniform(0.0, 4.0, n).astype(np.float32),
         "w_mc": rng.uniform(0.5, 1.5, n).astype(np.float32),
         "flav_in": np.ones(n, np.uint8), "flav_out": rng.integers(0, 2, n).astype(np.uint8),
         "is_nubar": rng.integers(0, 2, n).astype(np.uint8),
         "baseline_km": 295.0, "density_gcc": 2.6, "ye": 0.5}
    return s, (t_lo, t_hi, T)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_true_bin_edges_and_range(prec):
    s, tb = _edge_sample()
    row = synth.table1_point()
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, row[None, :])
        # one bin holding every event: the bin total is sensitive to each event's P
        h1 = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 1, prec, *tb, 0.0, 4.0, 1)[0]
        h40 = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 1, prec, *tb, 0.0, 4.0, 40)[0]
    _check(h1, s, [row], tb, 0.0, 4.0, 1, prec)
    _check(h40, s, [row], tb, 0.0, 4.0, 40, prec)
    # the events outside the true range contribute nothing
    _, w = oracle.reweight_bin_centre(s, oracle.point_from_row(row), *tb)
    assert (w[np.isin(s["e_true"], np.array([0.05, 0.0999, 3.1, 3.2, 7.0], dtype=np.float32))] == 0).all()


@pytest.mark.parametrize("n", [1, 31, 129, 4097])
def test_tiny_and_ragged_samples(n):
    s = synth.beam_sample(n, seed=100 + n)
    pts = synth.scan_points(3, 9)
    tb = (0.0, 10.25, 410)
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pts)
        for prec in ("fp64", "fp32"):
            h = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 3, prec, *tb, 0.0, 5.0, 100)[0]
            _check(h, s, pts, tb, 0.0, 5.0, 100, prec)


def test_several_samples_and_points_both_finalize_routes():
    ss = [synth.beam_sample(n, seed=300 + k, L_km=L, rho=rho) for k, (n, L, rho) in
          enumerate([(20_000, 295.0, 2.6), (33_333, 810.0, 2.8), (7_777, 1300.0, 2.85)])]
    pts = synth.uneven_points(24, 77)
    tb = (0.0, 40.0, 320)
    with api.Context(0) as c:
        sids = [api.osc_load_sample(c.ptr, s) for s in ss]
        api.osc_set_params(c.ptr, pts)
        for nb in (10, 100):  # 3 x 24 x 10 = 720 bins (fused) and 7200 bins (separate finalize)
            h = api.osc_histogram_bin_centre(c.ptr, sids, 0, 24, "fp64", *tb, 0.0, 20.0, nb)
            h2 = api.osc_histogram_bin_centre(c.ptr, sids, 0, 24, "fp64", *tb, 0.0, 20.0, nb)
            assert np.array_equal(h, h2)
            for j, s in enumerate(ss):
                _check(h[j], s, pts, tb, 0.0, 20.0, nb, "fp64")


def test_events_at_centres_equal_event_by_event():
    tb = (0.0, 5.0, 200)
    cen = np.array([oracle.true_centre(*tb, k) for k in range(tb[2])], dtype=np.float32)
    rng = np.random.default_rng(17)
    s = synth.beam_sample(50_000, seed=18)
    s["e_true"] = rng.choice(cen, s["n"]).astype(np.float32)
    pts = synth.scan_points(4, 19)
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pts)
        for prec, tol in (("fp64", 1e-12), ("fp32", 1e-6)):
            hb = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 4, prec, *tb, 0.0, 5.0, 50)[0]
            he = api.osc_histogram(c.ptr, [sid], 0, 4, prec, 0.0, 5.0, 50)[0]
            assert np.max(_rel(hb, he)) <= tol


def test_25mev_bin_study_on_gpu():
    stats = pytest.importorskip("scipy.stats")
    a, b, K = 0.6, 0.625, 4000
    h = (b - a) / K
    nodes = (a + (np.arange(K) + 0.5) * h).astype(np.float32)
    w = (stats.gamma(3.0, scale=0.25).pdf(nodes.astype(np.float64)) * h).astype(np.float32)
    s = {"n": K, "e_true": nodes, "e_reco": nodes, "w_mc": w, "flav_in": np.ones(K, np.uint8),
         "flav_out": np.ones(K, np.uint8), "is_nubar": np.zeros(K, np.uint8),
         "baseline_km": 295.0, "density_gcc": 2.6, "ye": 0.5}
    row = synth.table1_point()
    tb = (0.0, 10.0, 400)
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, row[None, :])
        he = api.osc_histogram(c.ptr, [sid], 0, 1, "fp64", 0.0, 10.0, 400)[0, 0]
        hb = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 1, "fp64", *tb, 0.0, 10.0, 400)[0, 0]
    assert np.count_nonzero(he) == 1 and he[24] > 0 and hb[24] > 0
    pt = oracle.point_from_row(row)
    _, we = oracle.reweight(s, pt)
    _, wb = oracle.reweight_bin_centre(s, pt, *tb)
    effect_gpu = he[24] / hb[24] - 1
    effect_orc = we.sum() / wb.sum() - 1
    assert abs(effect_gpu - effect_orc) < 1e-9
    assert 0.02 < effect_gpu < 0.05


def test_precision_sample_10M_full_size():
    s = synth.precision_sample()
    row = synth.table1_point()
    tb = (0.0, 10.25, 410)
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, row[None, :])
        h64 = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 1, "fp64", *tb, 0.0, 5.0, 100)[0]
        h32 = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 1, "fp32", *tb, 0.0, 5.0, 100)[0]
    _check(h64, s, [row], tb, 0.0, 5.0, 100, "fp64")
    _check(h32, s, [row], tb, 0.0, 5.0, 100, "fp32")


def test_batched_scan_2M_x_4096_full_size():
    """The bench's scan configuration: 2M events x 4096 points in one
    autotuned bin-centre launch (FP32 and FP64 tables); six sampled points,
    among them the first and last of the table, against the oracle."""
    s = synth.scan_sample()
    pts = synth.scan_points()
    tb = (0.0, 10.25, 410)
    pick = [0, 1, 777, 2048, 3001, 4095]
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pts)
        h32 = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 4096, "fp32", *tb, 0.0, 5.0, 100)[0]
        h64 = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 4096, "fp64", *tb, 0.0, 5.0, 100)[0]
    _check(h32[pick], s, pts[pick], tb, 0.0, 5.0, 100, "fp32")
    _check(h64[pick], s, pts[pick], tb, 0.0, 5.0, 100, "fp64")


def test_bad_arguments_rejected():
    s = synth.beam_sample(100, seed=1)
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, synth.table1_point()[None, :])
        for tb in ((1.0, 1.0, 10), (0.0, 5.0, 0), (0.0, 5.0, 70000), (np.nan, 5.0, 10)):
            with pytest.raises(api.OscError):
                api.osc_histogram_bin_centre(c.ptr, [sid], 0, 1, "fp64", *tb, 0.0, 5.0, 10)
        # the context stays usable
        h = api.osc_histogram_bin_centre(c.ptr, [sid], 0, 1, "fp64", 0.0, 10.0, 40, 0.0, 5.0, 10)
        assert np.isfinite(h).all()
