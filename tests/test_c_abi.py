"""The C ABI driven from a plain C program (tests/c_abi/osc_abi_test.c), built
with gcc against the in-tree library: argument and state checks without a GPU,
and (on a GB300) histograms and probabilities compared with the oracle."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1311_7579_gb300 import build, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    lib = build.build()
    libdir = os.path.dirname(lib)
    out = str(tmp_path_factory.mktemp("c_abi") / "osc_abi_test")
    subprocess.run(["gcc", "-std=c11", "-O2", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi", "osc_abi_test.c"), "-L" + libdir, "-losc_gb300",
                    "-Wl,-rpath," + libdir, "-o", out], check=True)
    return out


def test_c_program_without_gpu(exe):
    import torch
    if torch.cuda.is_available():
        pytest.skip("this part checks the no-GPU behaviour")
    r = subprocess.run([exe, "nogpu"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.gpu
def test_c_program_on_gpu(exe, tmp_path):
    s = synth.all_channel_sample(20_001, seed=61, L_km=810.0, rho=2.8)
    pts = synth.scan_points(3, 6161)
    nbins, lo, hi = 40, 0.0, 20.0
    inp = tmp_path / "in.bin"
    with open(inp, "wb") as f:
        f.write(np.array([s["n"]], np.int64).tobytes())
        f.write(np.array([pts.shape[0], nbins], np.int32).tobytes())
        f.write(np.array([lo, hi, s["baseline_km"], s["density_gcc"], s["ye"]], np.float64).tobytes())
        for k in ("e_true", "e_reco", "w_mc"):
            f.write(np.ascontiguousarray(s[k], np.float32).tobytes())
        for k in ("flav_in", "flav_out", "is_nubar"):
            f.write(np.ascontiguousarray(s[k], np.uint8).tobytes())
        f.write(np.ascontiguousarray(pts, np.float64).tobytes())
    outp = tmp_path / "out.bin"
    r = subprocess.run([exe, "gpu", str(inp), str(outp)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = np.fromfile(outp, dtype=np.float64)
    nh = pts.shape[0] * nbins
    h64 = out[:nh].reshape(pts.shape[0], nbins)
    p64 = out[nh:nh + s["n"]]
    h32 = out[nh + s["n"]:].reshape(pts.shape[0], nbins)
    ho = oracle.histogram(s, pts, lo, hi, nbins)
    rel = np.abs(h64 - ho) / np.maximum(np.abs(ho), 1e-300)
    assert np.max(np.where(ho == 0, np.abs(h64), rel)) <= 1e-9
    po, _ = oracle.reweight(s, oracle.point_from_row(pts[0]))
    assert np.max(np.abs(p64 - po)) <= 1e-12
    for k in range(pts.shape[0]):
        wsum = oracle.hist_from_weights(s["e_reco"], np.abs(s["w_mc"]).astype(np.float64), pts[k][6], lo, hi, nbins)
        assert np.all(np.abs(h32[k] - ho[k]) <= 1e-5 * wsum + 1e-12)


def _write_input(path, s, pts, nbins, lo, hi):
    with open(path, "wb") as f:
        f.write(np.array([s["n"]], np.int64).tobytes())
        f.write(np.array([pts.shape[0], nbins], np.int32).tobytes())
        f.write(np.array([lo, hi, s["baseline_km"], s["density_gcc"], s["ye"]], np.float64).tobytes())
        for k in ("e_true", "e_reco", "w_mc"):
            f.write(np.ascontiguousarray(s[k], np.float32).tobytes())
        for k in ("flav_in", "flav_out", "is_nubar"):
            f.write(np.ascontiguousarray(s[k], np.uint8).tobytes())
        f.write(np.ascontiguousarray(pts, np.float64).tobytes())


@pytest.mark.gpu
def test_c_program_times_fit_steps(exe, tmp_path):
    """The plain C program's timing mode: k fit steps (osc_histogram_point into a
    host buffer) without any Python, reported per step."""
    import json
    s = synth.table1_sample(200_000, seed=62)
    inp = tmp_path / "in.bin"
    _write_input(inp, s, synth.table1_point()[None, :], 100, 0.0, 5.0)
    r = subprocess.run([exe, "time", str(inp), "20"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["steps"] == 20 and res["events"] == s["n"] and res["us_per_step"] > 0
