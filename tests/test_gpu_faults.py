"""Host-side fault injection: with OSC_FAULT_ALLOC_FAIL_AT=k the k-th device
allocation of a context fails as if the device were out of memory.  Sweeping k
over a whole workflow (load, parameters, autotuned histogram, bin-centre
histogram, reweight, layered path, serving) checks that every allocation site
reports OSC_E_NOMEM with its message, leaves the context usable (a retry
succeeds), leaks nothing (the workspace total ends where the fault-free run
ends) and changes no result (bitwise)."""
import numpy as np
import pytest

from paper_1311_7579_gb300 import api, synth

pytestmark = pytest.mark.gpu

PROFILE = [(300.0, 2.2, 0.5), (700.0, 4.5, 0.49), (300.0, 1.0, 0.47)]


def _workflow(ctx, s, pts, faults):
    c = ctx.ptr

    def call(fn, *args):
        try:
            return fn(*args)
        except api.OscError as e:
            assert e.status == api.OSC_E_NOMEM and "injected" in str(e), str(e)
            faults.append(fn.__name__)
            return fn(*args)  # the injected failure is one-shot: the retry must succeed

    sid = call(api.osc_load_sample, c, s)
    call(api.osc_set_params, c, pts)
    h = call(api.osc_histogram, c, [sid], 0, pts.shape[0], "fp32", 0.0, 5.0, 50)
    hb = call(api.osc_histogram_bin_centre, c, [sid], 0, pts.shape[0], "fp64", 0.0, 10.0, 40, 0.0, 5.0, 50)
    p = np.zeros(s["n"])
    call(api.osc_reweight, c, sid, 1, "fp64", p)
    call(api.osc_set_layers, c, sid, PROFILE)
    hl = call(api.osc_histogram, c, [sid], 0, pts.shape[0], "fp64", 0.0, 5.0, 50)
    call(api.osc_serve_start, c, 8, 0.0, 5.0, 50)
    try:
        hs, _ = api.osc_wait(c, api.osc_submit(c, sid, pts[2], "fp32"), 50, 20000)
    finally:
        api.osc_serve_stop(c)
    return (h, hb, p, hl, hs), api.osc_workspace_used(c)


def test_allocation_failures_everywhere(monkeypatch):
    s = synth.all_channel_sample(5_000, seed=71, L_km=810.0, rho=2.8)
    pts = synth.scan_points(5, 7171)
    monkeypatch.delenv("OSC_FAULT_ALLOC_FAIL_AT", raising=False)
    with api.Context(0) as c:
        ref, used_ref = _workflow(c, s, pts, [])
    # the context's first allocation is its own work counter: creation fails cleanly
    monkeypatch.setenv("OSC_FAULT_ALLOC_FAIL_AT", "1")
    with pytest.raises(api.OscError):
        api.Context(0)
    sites = set()
    for k in range(2, 200):
        monkeypatch.setenv("OSC_FAULT_ALLOC_FAIL_AT", str(k))
        faults = []
        with api.Context(0) as c:
            out, used = _workflow(c, s, pts, faults)
        for a, b in zip(out, ref):
            assert np.array_equal(a, b), k
        assert used == used_ref, (k, used, used_ref)
        if not faults:
            break  # k is past the workflow's last allocation
        assert len(faults) == 1
        sites.add(faults[0])
    else:
        pytest.fail("the workflow never ran out of allocations to fail")
    # the workflow allocates dozens of times (sample, point table, plans of the
    # autotuner candidates, bin-centre table, layered plan, serving buffers)
    assert k > 40, k
    # every kind of call that allocates was hit at least once
    assert {"osc_load_sample", "osc_set_params", "osc_histogram", "osc_histogram_bin_centre",
            "osc_reweight", "osc_set_layers", "osc_serve_start"} <= sites, sites
