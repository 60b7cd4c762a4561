"""GPU-vs-oracle parity through the C ABI (needs a GB300).

Tolerances:
  * FP64 path probabilities: |dP| <= 1e-12 (Sec. 2.2 validation residual ~1e-12);
  * FP32-bulk path probabilities: |dP| <= 1e-5;
  * histogram bins: relative 1e-9 (FP64 path against the oracle's FP64 histogram;
    FP32-bulk path against the oracle's sum of the GPU's own returned weights,
    which pins binning and accumulation separately from the probability);
  * bin selection: exact (a misbinned event moves >= 1e-6 of a bin).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1311_7579_gb300 import api, synth

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12
TOL_FP32 = 1e-5
TOL_HIST = 1e-9
LO, HI, NB = 0.0, 5.0, 100


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c.ptr
    c.close()


def _rel_err(a, b):
    den = np.maximum(np.abs(b), 1e-300)
    return np.where((a == 0) & (b == 0), 0.0, np.abs(a - b) / den)


def _gpu_probs(ctx, sid, point, prec, n):
    p = np.zeros(n)
    w = np.zeros(n)
    api.osc_reweight(ctx, sid, point, prec, p, w)
    return p, w


# ------------------------------------------------------------ probabilities
def test_table1_sample_fp64_and_fp32(ctx):
    s = synth.table1_sample()
    sid = api.osc_load_sample(ctx, s)
    api.osc_set_params(ctx, synth.table1_point()[None, :])
    po, wo = oracle.reweight(s, oracle.point_from_row(synth.table1_point()))
    p64, w64 = _gpu_probs(ctx, sid, 0, "fp64", s["n"])
    assert np.max(np.abs(p64 - po)) <= TOL_FP64
    assert np.max(np.abs(w64 - wo)) <= 2 * TOL_FP64
    p32, w32 = _gpu_probs(ctx, sid, 0, "fp32", s["n"])
    assert np.max(np.abs(p32 - po)) <= TOL_FP32
    api.osc_unload_sample(ctx, sid)


@pytest.mark.parametrize("L,rho", [(295.0, 2.6), (810.0, 2.8), (1300.0, 2.85)])
def test_all_channels_random_points(ctx, L, rho):
    """Every (alpha, beta, nu/nubar) channel, both hierarchies, random delta,
    E_true uniform in [0.05, 10 L/295] GeV (crosses both MSW resonances)."""
    s = synth.all_channel_sample(60000, seed=int(L), L_km=L, rho=rho, e_hi=10 * L / 295)
    sid = api.osc_load_sample(ctx, s)
    pts = synth.scan_points(6, seed=int(L) + 1)
    api.osc_set_params(ctx, pts)
    for k in range(pts.shape[0]):
        po, _ = oracle.reweight(s, oracle.point_from_row(pts[k]))
        p64, _ = _gpu_probs(ctx, sid, k, "fp64", s["n"])
        p32, _ = _gpu_probs(ctx, sid, k, "fp32", s["n"])
        pmx, _ = _gpu_probs(ctx, sid, k, "fp32_f64eig", s["n"])
        assert np.max(np.abs(p64 - po)) <= TOL_FP64, (k, np.max(np.abs(p64 - po)))
        assert np.max(np.abs(p32 - po)) <= TOL_FP32, (k, np.max(np.abs(p32 - po)))
        assert np.max(np.abs(pmx - po)) <= TOL_FP32, (k, np.max(np.abs(pmx - po)))
    api.osc_unload_sample(ctx, sid)


def test_delta_in_every_quadrant(ctx):
    """The constants kernel reduces delta_CP by pi/2 and sums Taylor series for
    its sine and cosine; phases on the quadrant edges, past 2 pi and far from the
    origin (up to the ABI limit of 1e6 rad) must match the oracle's libm values."""
    s = synth.all_channel_sample(20000, seed=1300, L_km=1300.0, rho=2.85, e_hi=40.0)
    sid = api.osc_load_sample(ctx, s)
    deltas = [0.0, np.pi / 2, np.pi, -np.pi, -np.pi / 2, 1.5 * np.pi, 2 * np.pi, 0.1 - 2 * np.pi, 7.0, -20.3,
              1e5 + 0.3, -9.99e5]
    pts = np.tile(synth.table1_point(), (len(deltas), 1))
    pts[:, 5] = deltas
    api.osc_set_params(ctx, pts)
    for k, d in enumerate(deltas):
        po, _ = oracle.reweight(s, oracle.point_from_row(pts[k]))
        p64, _ = _gpu_probs(ctx, sid, k, "fp64", s["n"])
        p32, _ = _gpu_probs(ctx, sid, k, "fp32", s["n"])
        assert np.max(np.abs(p64 - po)) <= TOL_FP64, (d, np.max(np.abs(p64 - po)))
        assert np.max(np.abs(p32 - po)) <= TOL_FP32, (d, np.max(np.abs(p32 - po)))
    api.osc_unload_sample(ctx, sid)


def test_validation_residual_10M(ctx, golden_dir):
    """Sec. 2.2: 10 million energies uniform in (0.05, 30] GeV, Table 1 point:
    FP64 GPU vs CPU residual within 1e-12."""
    g = json.load(open(os.path.join(golden_dir, "validation_residual.json")))
    n = g["n_energies"]
    e = synth.validation_energies(n)
    rng = np.random.default_rng(77)
    s = dict(n=n, e_true=e, e_reco=e.copy(), w_mc=np.ones(n, np.float32),
             flav_in=rng.integers(0, 3, n).astype(np.uint8), flav_out=rng.integers(0, 3, n).astype(np.uint8),
             is_nubar=rng.integers(0, 2, n).astype(np.uint8), baseline_km=295.0, density_gcc=2.6, ye=0.5)
    sid = api.osc_load_sample(ctx, s)
    api.osc_set_params(ctx, synth.table1_point()[None, :])
    po, _ = oracle.reweight(s, oracle.point_from_row(synth.table1_point()))
    p64, _ = _gpu_probs(ctx, sid, 0, "fp64", n)
    assert np.max(np.abs(p64 - po)) <= g["residual_fp64"]
    p32, _ = _gpu_probs(ctx, sid, 0, "fp32", n)
    assert np.max(np.abs(p32 - po)) <= TOL_FP32
    api.osc_unload_sample(ctx, sid)


# --------------------------------------------------------------- histograms
def _check_fp64_hist(h_gpu, h_orc):
    assert np.array_equal(h_gpu == 0, h_orc == 0)
    assert np.max(_rel_err(h_gpu, h_orc)) <= TOL_HIST


def test_histograms_multi_point_both_paths(ctx):
    s = synth.table1_sample(200000, seed=11)
    sid = api.osc_load_sample(ctx, s)
    pts = synth.scan_points(37, seed=5)  # ragged against every tile width
    api.osc_set_params(ctx, pts)
    h64 = api.osc_histogram(ctx, [sid], 0, pts.shape[0], "fp64", LO, HI, NB)[0]
    h32 = api.osc_histogram(ctx, [sid], 0, pts.shape[0], "fp32", LO, HI, NB)[0]
    hmx = api.osc_histogram(ctx, [sid], 0, pts.shape[0], "fp32_f64eig", LO, HI, NB)[0]
    for k in range(pts.shape[0]):
        pt = oracle.point_from_row(pts[k])
        _, wo = oracle.reweight(s, pt)
        ho = oracle.hist_from_weights(s["e_reco"], wo, pts[k, 6], LO, HI, NB, compensated=True)
        _check_fp64_hist(h64[k], ho)
        # FP32 path: accumulation and binning pinned with the GPU's own weights
        _, w32 = _gpu_probs(ctx, sid, k, "fp32", s["n"])
        hw = oracle.hist_from_weights(s["e_reco"], w32, pts[k, 6], LO, HI, NB, compensated=True)
        _check_fp64_hist(h32[k], hw)
        # and the FP32 histogram against the FP64 oracle: bounded by |dP| <= 1e-5 per event
        wsum = oracle.hist_from_weights(s["e_reco"], s["w_mc"].astype(np.float64), pts[k, 6], LO, HI, NB)
        assert np.all(np.abs(h32[k] - ho) <= TOL_FP32 * wsum + 1e-12)
        # the FP64-eigen variant the same way
        _, wmx = _gpu_probs(ctx, sid, k, "fp32_f64eig", s["n"])
        _check_fp64_hist(hmx[k], oracle.hist_from_weights(s["e_reco"], wmx, pts[k, 6], LO, HI, NB, compensated=True))
        assert np.all(np.abs(hmx[k] - ho) <= TOL_FP32 * wsum + 1e-12)
    api.osc_unload_sample(ctx, sid)


def test_histograms_of_subnormal_weights(ctx):
    """Every weight below the smallest normal float (max |w_mc| ~ 2^-134, the
    fixed-point scale at its cap F = 190): each FP32 event weight P w_mc is a
    subnormal float, and its fixed-point addend must still be floor(|P w_mc| 2^F),
    so the FP32 bins equal the exact sums of the weights the GPU returns, and the
    FP64 bins the oracle's."""
    s = dict(synth.table1_sample(60000, seed=17))
    s["w_mc"] = (s["w_mc"].astype(np.float64) * 2.0 ** -135).astype(np.float32)
    assert np.all(np.abs(s["w_mc"]) < np.finfo(np.float32).tiny) and np.all(s["w_mc"] > 0)
    sid = api.osc_load_sample(ctx, s)
    pt = synth.table1_point()
    api.osc_set_params(ctx, pt[None, :])
    h32 = api.osc_histogram(ctx, [sid], 0, 1, "fp32", LO, HI, NB)[0, 0]
    _, w32 = _gpu_probs(ctx, sid, 0, "fp32", s["n"])
    assert h32.sum() > 0 and np.all(np.abs(w32) < np.finfo(np.float32).tiny)
    _check_fp64_hist(h32, oracle.hist_from_weights(s["e_reco"], w32, pt[6], LO, HI, NB, compensated=True))
    h64 = api.osc_histogram(ctx, [sid], 0, 1, "fp64", LO, HI, NB)[0, 0]
    _, wo = oracle.reweight(s, oracle.point_from_row(pt))
    _check_fp64_hist(h64, oracle.hist_from_weights(s["e_reco"], wo, pt[6], LO, HI, NB, compensated=True))
    api.osc_unload_sample(ctx, sid)


def test_mixed_sign_weights_sum_exactly(ctx):
    """Weights of both signs in the same bins (an FP32-precision run adds a
    negative addend as its one's complement and counts the missing ones): every
    FP32 bin equals the exact integer sum of floor(|w| 2^F) with the signs of the
    GPU's own per-event weights, scaled by 2^-F, whatever the tile shape, and the
    FP64 bins match the oracle's."""
    import math
    s = dict(synth.table1_sample(40000, seed=71))
    rng = np.random.default_rng(72)
    s["w_mc"] = (s["w_mc"] * np.where(rng.random(s["n"]) < 0.4, -1.0, 1.0)).astype(np.float32)
    sid = api.osc_load_sample(ctx, s)
    pts = synth.scan_points(3, seed=73)
    api.osc_set_params(ctx, pts)
    F = 62 - math.ceil(math.log2(float(np.max(np.abs(s["w_mc"])))))
    ref = {}
    for prec in ("fp32", "fp64"):
        for ppb in (1, 4, 256):
            api.osc_set_tile(ctx, ppb, 0)
            h = api.osc_histogram(ctx, [sid], 0, 3, prec, LO, HI, NB)[0]
            ref.setdefault(prec, h)
            assert np.array_equal(h, ref[prec]), (prec, ppb)
    api.osc_set_tile(ctx, 0, 0)
    for k in range(3):
        _, w = _gpu_probs(ctx, sid, k, "fp32", s["n"])
        b = oracle.bins(s["e_reco"], pts[k, 6], LO, HI, NB)
        exact = [0] * NB
        for bi, wi in zip(b, w):
            if bi >= 0:
                x = math.floor(abs(float(wi)) * 2.0 ** F)
                exact[bi] += -x if wi < 0 else x
        want = np.array([math.ldexp(v, -F) for v in exact]) * pts[k, 7]
        assert np.max(np.abs(ref["fp32"][k] - want) - 1e-15 * np.abs(want)) <= 0.0, k
        _, wo = oracle.reweight(s, oracle.point_from_row(pts[k]))
        ho = oracle.hist_from_weights(s["e_reco"], wo, pts[k, 6], LO, HI, NB, compensated=True)
        assert np.max(np.abs(ref["fp64"][k] - ho)) <= 1e-9 * np.max(np.abs(ho)), k
    api.osc_unload_sample(ctx, sid)


def test_one_point_ticket_modes_give_the_same_bins(ctx):
    """One-point work items are scheduled three ways: few items (one ticket at a
    time), many items (a ticket held one item ahead), and, over the last
    2 x warps tickets of a long list, one ticket at a time again.  64-event items
    over 2M events (31250 items, more than three per warp) run all three; the
    bins equal those of 4096-event items (few items) bitwise, in both
    precisions, through osc_histogram and the fit step."""
    s = synth.precision_sample(2_000_000, seed=29)
    sid = api.osc_load_sample(ctx, s)
    pt = synth.table1_point()
    api.osc_set_params(ctx, pt[None, :])
    for prec in ("fp32", "fp64"):
        api.osc_set_tile(ctx, 1, 4096)
        ref = api.osc_histogram(ctx, [sid], 0, 1, prec, LO, HI, NB)
        api.osc_set_tile(ctx, 1, 64)
        for _ in range(2):
            assert np.array_equal(api.osc_histogram(ctx, [sid], 0, 1, prec, LO, HI, NB), ref), prec
            assert np.array_equal(api.osc_histogram_point(ctx, [sid], pt, prec, LO, HI, NB), ref), prec
        api.osc_set_tile(ctx, 0, 0)
        assert np.array_equal(api.osc_histogram(ctx, [sid], 0, 1, prec, LO, HI, NB), ref), prec
    api.osc_unload_sample(ctx, sid)


def test_histogram_bitwise_independent_of_tile_shape(ctx):
    s = synth.table1_sample(50000, seed=12)
    sid = api.osc_load_sample(ctx, s)
    pts = synth.scan_points(20, seed=6)
    api.osc_set_params(ctx, pts)
    ref = {}
    for prec in ("fp32", "fp64", "fp32_f64eig"):
        for ppb in (1, 4, 16, 64, 256):
            for chunk in (1024, 4096, 0):
                api.osc_set_tile(ctx, ppb, chunk)
                h = api.osc_histogram(ctx, [sid], 0, 20, prec, LO, HI, NB)
                if prec not in ref:
                    ref[prec] = h.copy()
                assert np.array_equal(h, ref[prec]), (prec, ppb, chunk)
        h2 = api.osc_histogram(ctx, [sid], 0, 20, prec, LO, HI, NB)
        assert np.array_equal(h2, ref[prec])
    api.osc_set_tile(ctx, 0, 0)
    api.osc_unload_sample(ctx, sid)


def test_uneven_samples_one_launch(ctx):
    sizes = (1000, 3, 1023, 1025, 20000, 77777)
    ss = synth.uneven_samples(sizes)
    sids = [api.osc_load_sample(ctx, s) for s in ss]
    pts = synth.uneven_points(9, seed=8)
    api.osc_set_params(ctx, pts)
    for prec in ("fp64", "fp32", "fp32_f64eig"):
        h = api.osc_histogram(ctx, sids, 0, 9, prec, LO, 20.0, 80)
        for j, s in enumerate(ss):
            for k in range(9):
                if prec == "fp64":
                    _, w = oracle.reweight(s, oracle.point_from_row(pts[k]))
                else:
                    _, w = _gpu_probs(ctx, sids[j], k, prec, s["n"])
                ho = oracle.hist_from_weights(s["e_reco"], w, pts[k, 6], LO, 20.0, 80, compensated=True)
                _check_fp64_hist(h[j, k], ho)
    for sid in sids:
        api.osc_unload_sample(ctx, sid)


def test_edge_cases(ctx):
    # one event; events outside the range; negative weights and E_reco; norm; nbins = 1; lo != 0
    s = synth.table1_sample(5, seed=13)
    s["e_reco"][1] = -0.3
    s["e_reco"][2] = 7.0
    s["w_mc"][3] = -1.25
    sid = api.osc_load_sample(ctx, s)
    row = synth.table1_point().copy()
    row[7] = 2.5
    pts = np.stack([row, synth.table1_point()])
    api.osc_set_params(ctx, pts)
    for prec in ("fp64", "fp32"):
        for lo, hi, nb in ((0.0, 5.0, 100), (0.1, 1.7, 1), (-1.0, 2.0, 7)):
            h = api.osc_histogram(ctx, [sid], 0, 2, prec, lo, hi, nb)[0]
            for k in range(2):
                _, w = _gpu_probs(ctx, sid, k, prec, s["n"])
                if prec == "fp64":
                    _, wo = oracle.reweight(s, oracle.point_from_row(pts[k]))
                    assert np.max(np.abs(w - wo)) <= 3 * TOL_FP64
                ho = oracle.hist_from_weights(s["e_reco"], w, pts[k, 6], lo, hi, nb)
                assert np.max(np.abs(h[k] - ho)) <= 1e-12 * max(1.0, np.max(np.abs(ho)))
    one = synth.table1_sample(1, seed=14)
    sid1 = api.osc_load_sample(ctx, one)
    h = api.osc_histogram(ctx, [sid1], 1, 1, "fp64", LO, HI, NB)[0, 0]
    _, wo = oracle.reweight(one, oracle.point_from_row(pts[1]))
    assert np.max(np.abs(h - oracle.hist_from_weights(one["e_reco"], wo, 1.0, LO, HI, NB))) <= 1e-12
    api.osc_unload_sample(ctx, sid)
    api.osc_unload_sample(ctx, sid1)


def test_invalid_input_rejected_before_launch(ctx):
    s = synth.table1_sample(100, seed=15)
    bad = dict(s, e_true=s["e_true"].copy())
    bad["e_true"][7] = 0.0
    with pytest.raises(api.OscError) as e:
        api.osc_load_sample(ctx, bad)
    assert e.value.status == api.OSC_E_RANGE
    bad = dict(s, flav_out=s["flav_out"].copy())
    bad["flav_out"][3] = 3
    with pytest.raises(api.OscError):
        api.osc_load_sample(ctx, bad)
    for field, val in ((1, 0.0), (3, 0.0), (4, 5e-5), (6, 0.0), (0, float("nan")), (5, 2e6)):
        row = synth.table1_point().copy()
        row[field] = val
        with pytest.raises(api.OscError) as e:
            api.osc_set_params(ctx, row[None, :])
        assert e.value.status == api.OSC_E_RANGE
    sid = api.osc_load_sample(ctx, s)
    api.osc_set_params(ctx, synth.table1_point()[None, :])
    for args in (([sid], 0, 2), ([sid + 999], 0, 1), ([sid], -1, 1)):
        with pytest.raises(api.OscError) as e:
            api.osc_histogram(ctx, args[0], args[1], args[2], "fp64", LO, HI, NB)
        assert e.value.status == api.OSC_E_ARG
    with pytest.raises(api.OscError):
        api.osc_histogram(ctx, [sid], 0, 1, "fp64", 5.0, 5.0, NB)
    with pytest.raises(api.OscError):
        api.osc_histogram(ctx, [sid], 0, 1, "fp64", LO, HI, 0)
    # the context is still usable afterwards
    h = api.osc_histogram(ctx, [sid], 0, 1, "fp64", LO, HI, NB)
    assert np.isfinite(h).all()
    api.osc_unload_sample(ctx, sid)


def test_workspace_cap_enforced():
    with api.Context(0, workspace_cap_bytes=1 << 20) as c:
        s = synth.table1_sample(200000, seed=16)
        with pytest.raises(api.OscError) as e:
            api.osc_load_sample(c.ptr, s)
        assert e.value.status == api.OSC_E_NOMEM
        small = synth.table1_sample(1000, seed=16)
        sid = api.osc_load_sample(c.ptr, small)
        api.osc_set_params(c.ptr, synth.table1_point()[None, :])
        h = api.osc_histogram(c.ptr, [sid], 0, 1, "fp32", LO, HI, NB)
        assert h.sum() > 0


def test_device_outputs_match_host_outputs(ctx):
    torch = pytest.importorskip("torch")
    s = synth.table1_sample(30000, seed=17)
    sid = api.osc_load_sample(ctx, s)
    pts = synth.scan_points(5, seed=9)
    api.osc_set_params(ctx, pts)
    hh = api.osc_histogram(ctx, [sid], 0, 5, "fp32", LO, HI, NB)
    hd = torch.zeros((1, 5, NB), dtype=torch.float64, device="cuda")
    api.osc_histogram(ctx, [sid], 0, 5, "fp32", LO, HI, NB, out=hd)
    api.osc_sync(ctx)
    assert np.array_equal(hd.cpu().numpy(), hh)
    # page-locked host buffers are written by the kernels directly: same bins, for
    # the fused finalize (5 x NB bins) and the separate finalize kernel (60 x 100)
    hp = torch.zeros((1, 5, NB), dtype=torch.float64).pin_memory().numpy()
    api.osc_histogram(ctx, [sid], 0, 5, "fp32", LO, HI, NB, out=hp)
    assert np.array_equal(hp, hh)
    hb = api.osc_histogram_bin_centre(ctx, [sid], 0, 5, "fp64", 0.0, 10.0, 40, LO, HI, NB)
    hbp = torch.zeros((1, 5, NB), dtype=torch.float64).pin_memory().numpy()
    api.osc_histogram_bin_centre(ctx, [sid], 0, 5, "fp64", 0.0, 10.0, 40, LO, HI, NB, out=hbp)
    assert np.array_equal(hbp, hb)
    pts60 = synth.scan_points(60, seed=10)
    api.osc_set_params(ctx, pts60)
    hl = api.osc_histogram(ctx, [sid], 0, 60, "fp32", LO, HI, 100)
    hlp = torch.zeros((1, 60, 100), dtype=torch.float64).pin_memory().numpy()
    api.osc_histogram(ctx, [sid], 0, 60, "fp32", LO, HI, 100, out=hlp)
    assert np.array_equal(hlp, hl)
    api.osc_set_params(ctx, pts)
    pd = torch.zeros(s["n"], dtype=torch.float64, device="cuda")
    api.osc_reweight(ctx, sid, 2, "fp64", out_prob=pd)
    ph, _ = _gpu_probs(ctx, sid, 2, "fp64", s["n"])
    assert np.array_equal(pd.cpu().numpy(), ph)
    # osc_reweight into page-locked host buffers (written by the kernel directly),
    # one of them pageable (staged): same values
    for prec in ("fp32", "fp64"):
        ph, wh = _gpu_probs(ctx, sid, 2, prec, s["n"])
        pp = torch.zeros(s["n"], dtype=torch.float64).pin_memory().numpy()
        wp = torch.zeros(s["n"], dtype=torch.float64).pin_memory().numpy()
        api.osc_reweight(ctx, sid, 2, prec, out_prob=pp, out_weight=wp)
        assert np.array_equal(pp, ph) and np.array_equal(wp, wh)
        wq = np.zeros(s["n"])
        api.osc_reweight(ctx, sid, 2, prec, out_prob=pp, out_weight=wq)
        assert np.array_equal(wq, wh)
    api.osc_unload_sample(ctx, sid)


def test_histogram_point_is_set_params_plus_histogram(ctx):
    """osc_histogram_point(pt) gives the bins of osc_set_params([pt]) followed by
    osc_histogram over point 0, bitwise, for host, page-locked and device outputs;
    an invalid point is rejected and leaves the table as it was."""
    torch = pytest.importorskip("torch")
    s1 = synth.table1_sample(20000, seed=21)
    s2 = synth.all_channel_sample(15000, seed=22, L_km=810.0, rho=2.8)
    ids = [api.osc_load_sample(ctx, s1), api.osc_load_sample(ctx, s2)]
    pts = synth.scan_points(3, seed=23)
    for k in range(3):
        for prec in ("fp32", "fp64"):
            api.osc_set_params(ctx, pts[k:k + 1])
            ref = api.osc_histogram(ctx, ids, 0, 1, prec, LO, HI, NB)
            got = api.osc_histogram_point(ctx, ids, pts[k], prec, LO, HI, NB)
            assert np.array_equal(got, ref)
            pin = torch.zeros((2, 1, NB), dtype=torch.float64).pin_memory().numpy()
            api.osc_histogram_point(ctx, ids, pts[k], prec, LO, HI, NB, out=pin)
            assert np.array_equal(pin, ref)
            dev = torch.zeros((2, 1, NB), dtype=torch.float64, device="cuda")
            api.osc_histogram_point(ctx, ids, pts[k], prec, LO, HI, NB, out=dev)
            api.osc_sync(ctx)
            assert np.array_equal(dev.cpu().numpy(), ref)
    bad = pts[0].copy()
    bad[3] = -1.0  # dm21 <= 0
    with pytest.raises(api.OscError) as e:
        api.osc_histogram_point(ctx, ids, bad, "fp32", LO, HI, NB)
    assert e.value.status == api.OSC_E_RANGE
    # the table still holds the last valid point
    again = api.osc_histogram(ctx, ids, 0, 1, "fp64", LO, HI, NB)
    api.osc_set_params(ctx, pts[2:3])
    assert np.array_equal(again, api.osc_histogram(ctx, ids, 0, 1, "fp64", LO, HI, NB))
    for sid in ids:
        api.osc_unload_sample(ctx, sid)


def test_fit_step_constants_are_the_constants_kernels(ctx):
    """The FP32-bulk fit step computes its point's constants on the host, passes
    them by value to its histogram kernel and stores them in row 0 of the
    constants tables; they must be bitwise the constants kernel's.  After
    osc_histogram_point(pt) the per-event probabilities of every precision (which
    read the stored row) equal those after osc_set_params([pt]), bit for bit,
    through constant density and through layers, for points across the accepted
    domain: both mass orderings, near-extreme mixing, tiny and large splittings,
    |delta| up to 1e3; and the fit step's bins equal osc_histogram's."""
    s = synth.all_channel_sample(3000, seed=61, L_km=810.0, rho=2.8)
    sl = synth.all_channel_sample(2000, seed=64, L_km=1300.0)
    sid, lid = api.osc_load_sample(ctx, s), api.osc_load_sample(ctx, sl)
    api.osc_set_layers(ctx, lid, [(300.0, 2.2, 0.5), (700.0, 4.5, 0.49), (300.0, 1.0, 0.47)])
    edge = np.array([[0.311, 0.0251, 0.5, 7.6e-5, 2.4e-3, 0.0, 1.0, 1.0],
                     [0.02, 0.001, 0.98, 1.0e-6, -2.0e-3, -1000.0, 1.1, 0.5],
                     [0.97, 0.2, 0.03, 3.0e-4, 3.5e-3, 987.654321, 0.95, 2.0],
                     [0.5, 0.5, 0.5, 2.0e-5, -1.0e-2, 3.14159, 1.0, -1.0]])
    pts = np.concatenate([synth.scan_points(12, seed=63), edge])
    for k, pt in enumerate(pts):
        h = api.osc_histogram_point(ctx, [sid], pt, "fp32", LO, HI, NB)
        step = {(q, prec): _gpu_probs(ctx, q, 0, prec, n)[0]
                for q, n in ((sid, s["n"]), (lid, sl["n"])) for prec in ("fp32", "fp64", "fp32_f64eig")}
        api.osc_set_params(ctx, pt[None, :])
        assert np.array_equal(h, api.osc_histogram(ctx, [sid], 0, 1, "fp32", LO, HI, NB)), k
        for (q, prec), p in step.items():
            n = s["n"] if q == sid else sl["n"]
            assert np.array_equal(p, _gpu_probs(ctx, q, 0, prec, n)[0]), (k, q, prec)
    for q in (sid, lid):
        api.osc_unload_sample(ctx, q)


def test_histogram_point_graph_step_separate_finalize_and_layers(ctx):
    """osc_histogram_point runs the fit step as one CUDA graph (constants,
    histogram, FP64 recomputation pass, finalize, joined by programmatic edges)
    replayed with its parameters refreshed: the bins equal set_params +
    osc_histogram bitwise for a separate finalize kernel (600 bins), a layered
    sample (completion edges) and points alternating between calls; the graph
    launches the kernels the two calls do, less the constants kernel where the
    step passes host-computed constants by value (FP32 bulk through constant
    density)."""
    s1 = synth.table1_sample(30000, seed=24)
    s2 = synth.all_channel_sample(12000, seed=25, L_km=810.0, rho=2.8)
    ids = [api.osc_load_sample(ctx, s1), api.osc_load_sample(ctx, s2)]
    lid = api.osc_load_sample(ctx, synth.all_channel_sample(9000, seed=26, L_km=1300.0, rho=2.85))
    api.osc_set_layers(ctx, lid, [(400.0, 2.6, 0.5), (500.0, 3.3, 0.5), (400.0, 2.6, 0.5)])
    pts = synth.scan_points(4, seed=27)
    for nb in (NB, 300):
        for group in (ids, [lid]):
            for prec in ("fp32", "fp64"):
                api.osc_set_params(ctx, pts[:1])
                api.osc_histogram(ctx, group, 0, 1, prec, LO, HI, nb)  # autotuned here, once
                for k in (0, 1, 0, 2, 3):
                    api.osc_set_params(ctx, pts[k:k + 1])
                    n0 = api.osc_launch_count(ctx)
                    ref = api.osc_histogram(ctx, group, 0, 1, prec, LO, HI, nb)
                    n1 = api.osc_launch_count(ctx)
                    got = api.osc_histogram_point(ctx, group, pts[k], prec, LO, HI, nb)
                    n2 = api.osc_launch_count(ctx)
                    assert np.array_equal(got, ref), (nb, prec, k)
                    by_value = prec == "fp32" and group is ids
                    assert n2 - n1 == (n1 - n0) + (0 if by_value else 1), (nb, prec, k)
    for sid in ids + [lid]:
        api.osc_unload_sample(ctx, sid)


def test_histogram_point_graph_step_runs_the_recomputation_pass(ctx):
    """At extreme mixing angles the FP32-bulk kernels leave events to the FP64
    recomputation pass launched after them (in the fit step's graph, joined by a
    programmatic edge).  The bins agree bitwise across the step, one-point items
    of two sizes and point tiles of 4 and 16, for the fused (100 bins) and
    separate (600 bins) finalize; the per-event probabilities of those points
    stay within the FP32 tolerance."""
    s = synth.all_channel_sample(20000, seed=28, L_km=295.0, rho=2.6, e_lo=0.05, e_hi=3.0)
    sid = api.osc_load_sample(ctx, s)
    pts = np.array([[0.01, 0.0251, 0.99, 7.6e-5, -2.4e-3, 3.1, 1.0, 1.0],
                    [0.99, 0.0251, 0.01, 7.6e-5, 2.4e-3, -0.7, 1.0, 1.0]])
    for k in range(2):
        api.osc_set_params(ctx, pts[k:k + 1])
        po, _ = oracle.reweight(s, oracle.point_from_row(pts[k]))
        p32, _ = _gpu_probs(ctx, sid, 0, "fp32", s["n"])
        assert np.max(np.abs(p32 - po)) <= 1e-5
        for nb in (NB, 600):
            ref = api.osc_histogram(ctx, [sid], 0, 1, "fp32", LO, HI, nb)
            for _ in range(2):
                got = api.osc_histogram_point(ctx, [sid], pts[k], "fp32", LO, HI, nb)
                assert np.array_equal(got, ref), (k, nb)
            for ppb, chunk in ((1, 256), (1, 4096), (4, 0), (16, 0)):
                api.osc_set_tile(ctx, ppb, chunk)
                got = api.osc_histogram(ctx, [sid], 0, 1, "fp32", LO, HI, nb)
                api.osc_set_tile(ctx, 0, 0)
                assert np.array_equal(got, ref), (k, nb, ppb, chunk)
    api.osc_unload_sample(ctx, sid)


def test_prepared_point_histogram_matches_the_plain_call(ctx):
    """api.PointHistogram (arguments marshalled once) gives, bitwise, the bins of
    osc_histogram_point for each point, whether the point is passed to the call
    or written into its point buffer; a rejected point raises and leaves the
    output as it was."""
    torch = pytest.importorskip("torch")
    s1 = synth.table1_sample(20000, seed=31)
    s2 = synth.all_channel_sample(15000, seed=32, L_km=810.0, rho=2.8)
    ids = [api.osc_load_sample(ctx, s1), api.osc_load_sample(ctx, s2)]
    pts = synth.scan_points(4, seed=33)
    for prec in ("fp32", "fp64"):
        pin = torch.zeros((2, 1, NB), dtype=torch.float64).pin_memory().numpy()
        dev = torch.zeros((2, 1, NB), dtype=torch.float64, device="cuda")
        calls = [api.PointHistogram(ctx, ids, prec, LO, HI, NB),
                 api.PointHistogram(ctx, ids, prec, LO, HI, NB, out=pin),
                 api.PointHistogram(ctx, ids, prec, LO, HI, NB, out=dev)]
        for k in range(4):
            ref = api.osc_histogram_point(ctx, ids, pts[k], prec, LO, HI, NB)
            for j, call in enumerate(calls):
                if k % 2:
                    call.point[:] = pts[k]
                    got = call()
                else:
                    got = call(pts[k:k + 1])
                if j == 2:
                    api.osc_sync(ctx)
                    got = got.cpu().numpy()
                assert np.array_equal(got, ref), (prec, k, j)
        before = calls[1].out.copy()
        bad = pts[0].copy()
        bad[4] = 0.0  # dm32 = 0
        with pytest.raises(api.OscError) as e:
            calls[1](bad)
        assert e.value.status == api.OSC_E_RANGE
        assert np.array_equal(calls[1].out, before)
    for sid in ids:
        api.osc_unload_sample(ctx, sid)
