"""Continuous-batching serving loop (needs a GB300): each request's histogram is
the same alone and in a mix of concurrent requests (bitwise: bins are exact
integer sums), and equal to osc_histogram for the same sample and point."""
import threading

import numpy as np
import pytest

from paper_1311_7579_gb300 import api, synth

pytestmark = pytest.mark.gpu
LO, HI, NB = 0.0, 20.0, 100


@pytest.fixture(scope="module")
def served():
    c = api.Context(0)
    ss = synth.uneven_samples((20000, 150000, 3, 600000))
    sids = [api.osc_load_sample(c.ptr, s) for s in ss]
    yield c.ptr, ss, sids
    c.close()


def _direct(ctx, sid, pt, prec):
    api.osc_set_params(ctx, pt[None, :])
    return api.osc_histogram(ctx, [sid], 0, 1, prec, LO, HI, NB)[0, 0]


def test_alone_equals_mix_equals_direct(served):
    ctx, ss, sids = served
    pts = synth.uneven_points(40, seed=41)
    probe = [(sids[3], pts[0], "fp32"), (sids[1], pts[1], "fp64"), (sids[2], pts[2], "fp32")]
    direct = [_direct(ctx, sid, pt, prec) for sid, pt, prec in probe]
    api.osc_serve_start(ctx, 64, LO, HI, NB)
    try:
        alone = []
        for sid, pt, prec in probe:
            t = api.osc_submit(ctx, sid, pt, prec)
            h, lat = api.osc_wait(ctx, t, NB, timeout_ms=60000)
            assert lat > 0
            alone.append(h.copy())
        # the same requests mixed with many others, submitted from two threads
        tickets = {}
        rng = np.random.default_rng(42)

        def submit(tag, items):
            for k, (sid, pt, prec) in enumerate(items):
                tickets[(tag, k)] = api.osc_submit(ctx, sid, pt, prec)

        noise = [(sids[rng.integers(len(sids))], pts[3 + rng.integers(37)], "fp32" if rng.random() < 0.7 else "fp64")
                 for _ in range(150)]
        th = threading.Thread(target=submit, args=("noise", noise))
        th.start()
        submit("probe", probe * 3)
        th.join()
        for k in range(len(probe) * 3):
            h, _ = api.osc_wait(ctx, tickets[("probe", k)], NB, timeout_ms=120000)
            assert np.array_equal(h, alone[k % len(probe)])
        for k in range(len(noise)):
            h, _ = api.osc_wait(ctx, tickets[("noise", k)], NB, timeout_ms=120000)
            assert np.isfinite(h).all()
    finally:
        api.osc_serve_stop(ctx)
    for a, d in zip(alone, direct):
        assert np.array_equal(a, d)


def test_serving_state_and_errors(served):
    ctx, ss, sids = served
    pt = synth.table1_point()
    with pytest.raises(api.OscError) as e:
        api.osc_submit(ctx, sids[0], pt, "fp32")
    assert e.value.status == api.OSC_E_STATE
    api.osc_serve_start(ctx, 8, LO, HI, NB)
    try:
        with pytest.raises(api.OscError) as e:
            api.osc_serve_start(ctx, 8, LO, HI, NB)
        assert e.value.status == api.OSC_E_STATE
        with pytest.raises(api.OscError) as e:
            api.osc_wait(ctx, 10 ** 9, NB, timeout_ms=10)
        assert e.value.status == api.OSC_E_ARG
        bad = pt.copy()
        bad[3] = -1.0
        with pytest.raises(api.OscError) as e:
            api.osc_submit(ctx, sids[0], bad, "fp32")
        assert e.value.status == api.OSC_E_RANGE
        with pytest.raises(api.OscError) as e:
            api.osc_unload_sample(ctx, sids[0])
        assert e.value.status == api.OSC_E_STATE
        t = api.osc_submit(ctx, sids[3], pt, "fp32")
        h, _ = api.osc_wait(ctx, t, NB, timeout_ms=60000)
        assert h.sum() > 0
    finally:
        api.osc_serve_stop(ctx)
    api.osc_serve_stop(ctx)  # idempotent
