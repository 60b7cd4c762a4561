"""OSC_AUTOTUNE_CACHE: the autotuner's choice for a workload class is appended to
the cache file; a new context on the same GPU model reads it back and launches
the chosen shape at once (no tuning launches), with bitwise the same result."""
import numpy as np
import pytest

from paper_1311_7579_gb300 import api, synth

pytestmark = pytest.mark.gpu


def _run(s, pts):
    with api.Context(0) as c:
        sid = api.osc_load_sample(c.ptr, s)
        api.osc_set_params(c.ptr, pts)
        n0 = api.osc_launch_count(c.ptr)
        h = api.osc_histogram(c.ptr, [sid], 0, pts.shape[0], "fp32", 0.0, 5.0, 100)
        return h, api.osc_launch_count(c.ptr) - n0


def test_tuned_shapes_persist_across_contexts(tmp_path, monkeypatch):
    cache = tmp_path / "osc_tune.txt"
    monkeypatch.setenv("OSC_AUTOTUNE_CACHE", str(cache))
    s = synth.scan_sample(300_000, seed=81)
    pts = synth.scan_points(64, 8181)
    h1, launches1 = _run(s, pts)
    lines = cache.read_text().split("\n")
    assert len([x for x in lines if x.strip()]) == 1
    dev, key, pt, chunk = lines[0].split()
    assert int(pt) in (1, 4, 16, 64, 256) and int(chunk) % 64 == 0
    h2, launches2 = _run(s, pts)
    assert launches1 > 4 * launches2  # the first call timed several candidate shapes
    # histogram kernel, the FP64 recomputation pass of the FP32 precisions (+ finalize kernel for this output size)
    assert launches2 <= 3
    assert np.array_equal(h1, h2)
    # a corrupt cache is ignored, not fatal
    cache.write_text("garbage line\nanother\n")
    h3, _ = _run(s, pts)
    assert np.array_equal(h3, h1)
