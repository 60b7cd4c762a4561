"""C-ABI contract checks that need no GPU: the library builds for sm_103a, loads,
and exports every entry point include/osc.h declares; calls fail cleanly (a
status, never a crash) without a device or with null arguments."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1311_7579_gb300 import api, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_entry_points():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", hdr)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(osc_\w+)\s*\(", src, flags=re.M)
    return names


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (osc_\w+)", out))
    declared = _declared_entry_points()
    assert declared, "no declarations parsed"
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    assert sorted(set(declared)) == sorted(set(api.ENTRY_POINTS))
    L = api.lib()
    for n in declared:
        assert hasattr(L, n)


def test_debug_build_exports_the_same_symbols():
    """The debug-check build (OSC_DEBUG_CHECKS) compiles and exports the same ABI."""
    dbg = build.build(debug_checks=True)
    syms = subprocess.run(["nm", "-D", "--defined-only", dbg], capture_output=True, text=True, check=True).stdout
    for name in api.ENTRY_POINTS:
        assert re.search(r"\b%s\b" % name, syms), name


def test_build_targets_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_and_error_strings():
    assert "sm_103a" in api.osc_version()
    assert api.osc_last_error(None) == "no context"


def test_calls_without_context_return_arg_status():
    L = api.lib()
    sid = ctypes.c_int32()
    assert L.osc_load_sample(None, None, ctypes.byref(sid)) == api.OSC_E_ARG
    assert L.osc_set_params(None, None, 1) == api.OSC_E_ARG
    assert L.osc_reweight(None, 0, 0, 0, None, None, 0) == api.OSC_E_ARG
    assert L.osc_histogram(None, None, 1, 0, 1, 0, 0.0, 5.0, 100, None, 0) == api.OSC_E_ARG
    assert L.osc_histogram_bin_centre(None, None, 1, 0, 1, 0, 0.0, 10.0, 40, 0.0, 5.0, 100, None, 0) == api.OSC_E_ARG
    assert L.osc_histogram_point(None, None, 1, None, 0, 0.0, 5.0, 100, None, 0) == api.OSC_E_ARG
    assert L.osc_set_layers(None, 0, 1, None, None, None) == api.OSC_E_ARG
    assert L.osc_sync(None) == api.OSC_E_ARG
    assert L.osc_serve_stop(None) == api.OSC_E_ARG
    assert L.osc_create(0, 0, None, None) == api.OSC_E_ARG
    L.osc_destroy(None)  # no-op


def test_prepared_point_histogram_marshalling_without_a_gpu():
    """api.PointHistogram marshals once: its point buffer is a writable float64[8]
    view that a call with a point overwrites, the output is allocated with the
    call's shape, and the library's status comes back as OscError (a null
    context is rejected before any device work)."""
    import numpy as np
    call = api.PointHistogram(None, [3, 5], "fp32", 0.0, 5.0, 100)
    assert call.point.dtype == np.float64 and call.point.shape == (8,) and call.point.flags.writeable
    assert call.out.shape == (2, 1, 100)
    p = np.arange(1.0, 9.0)
    with pytest.raises(api.OscError) as e:
        call(p)
    assert e.value.status == api.OSC_E_ARG and "no context" in str(e.value)
    assert np.array_equal(call.point, p)
    call.point[4] = -2.5e-3
    with pytest.raises(api.OscError):
        call()
    assert call.point[4] == -2.5e-3
    with pytest.raises(ValueError):
        call(np.zeros(7))


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(api.OscError) as e:
        api.osc_create(0)
    assert e.value.status in (api.OSC_E_CUDA, api.OSC_E_ARG)


def test_oracle_library_builds():
    import oracle
    oracle.build()
    assert oracle.num_threads() >= 1


def test_noalloc_wrapper_rejects_bad_tensors_before_any_call():
    """osc_histogram_noalloc's binding checks the caller's tensors (the library
    only sees pointers): CPU tensors, wrong dtypes, unequal lengths and a short
    or non-float64 output are each rejected with OSC_E_ARG before the library
    is called."""
    torch = pytest.importorskip("torch")
    from paper_1311_7579_gb300 import synth

    n = 64
    f = torch.zeros(n, dtype=torch.float32)
    u = torch.zeros(n, dtype=torch.uint8)
    out = torch.zeros(100, dtype=torch.float64)
    pt = synth.table1_point()

    def call(*arrs, out=out, nbins=100):
        api.osc_histogram_noalloc(*arrs, 295.0, 2.6, 0.5, 1.5, pt, "fp32", 0.0, 5.0, nbins, out)

    cases = [(f, f, f, u, u, u)]  # CPU tensors
    if torch.cuda.is_available():
        fc, uc = f.cuda(), u.cuda()
        cases = [(f, fc, fc, uc, uc, uc), (fc, fc, fc.double(), uc, uc, uc), (fc, fc, fc, uc.int(), uc, uc),
                 (fc, fc[:10], fc, uc, uc, uc), (fc, fc, fc, uc, uc, uc[:-1])]
    for arrs in cases:
        with pytest.raises(api.OscError) as e:
            call(*arrs)
        assert e.value.status == api.OSC_E_ARG
    if torch.cuda.is_available():
        fc, uc = f.cuda(), u.cuda()
        for bad_out in (out, out.cuda().float(), out.cuda()[:50]):
            with pytest.raises(api.OscError) as e:
                call(fc, fc, fc, uc, uc, uc, out=bad_out)
            assert e.value.status == api.OSC_E_ARG
