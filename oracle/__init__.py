"""FP64 CPU oracle for constant-density three-flavour oscillation reweighting.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline / reference leg of ``bench.py``; never by the product
package.  It shares no code with the CUDA path.

The arithmetic lives in ``osc_oracle.c`` (plain C99 complex double, compiled
with ``-O2 -ffp-contract=off``); this module only builds and loads it and
marshals numpy arrays.  What each function computes, and which passage of the
paper it follows (Sec. 1.1 Eq. (1) and the matter term; Sec. 1.1.1 weights,
energy-scale systematic and binning), is stated in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "osc_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


class OrcPoint(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("s2_12", "s2_13", "s2_23", "dm21", "dm32", "dcp", "escale", "norm")]


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (gcc, no contraction, OpenMP)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-std=gnu11", "-shared", "-fPIC",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            u8 = ctypes.POINTER(ctypes.c_uint8)
            i32 = ctypes.POINTER(ctypes.c_int32)
            pt = ctypes.POINTER(OrcPoint)
            i64 = ctypes.c_int64
            d = ctypes.c_double
            sig = {
                "orc_const_c_L": (d, []),
                "orc_const_k_A": (d, []),
                "orc_prob": (d, [pt, d, d, d, d, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
                "orc_prob_matrix_many": (None, [pt, d, d, d, i64, dp, ctypes.c_int, dp]),
                "orc_prob_matrix_A": (None, [pt, d, d, d, ctypes.c_int, dp]),
                "orc_reweight": (None, [i64, fp, fp, u8, u8, u8, d, d, d, pt, dp, dp]),
                "orc_hist_from_weights": (None, [i64, fp, dp, d, d, d, ctypes.c_int, ctypes.c_int, dp]),
                "orc_histogram": (None, [i64, fp, fp, fp, u8, u8, u8, d, d, d, pt, ctypes.c_int,
                                         d, d, ctypes.c_int, ctypes.c_int, dp, dp]),
                "orc_eigh3_flat": (ctypes.c_int, [dp, dp, dp]),
                "orc_hamiltonian_flat": (None, [pt, d, ctypes.c_int, dp]),
                "orc_pmns_flat": (None, [pt, dp]),
                "orc_bin": (ctypes.c_int, [d, ctypes.c_float, d, d, ctypes.c_int]),
                "orc_bin_many": (None, [i64, fp, d, d, d, ctypes.c_int, i32]),
                "orc_num_threads": (ctypes.c_int, []),
                "orc_set_num_threads": (None, [ctypes.c_int]),
                "orc_true_centre": (ctypes.c_float, [d, d, ctypes.c_int, ctypes.c_int]),
                "orc_reweight_bin_centre": (None, [i64, fp, fp, u8, u8, u8, d, d, d, pt, d, d, ctypes.c_int,
                                                   dp, dp]),
                "orc_prob_matrix_layers_many": (None, [pt, ctypes.c_int, dp, dp, dp, i64, dp, ctypes.c_int, dp]),
                "orc_reweight_layers": (None, [i64, fp, fp, u8, u8, u8, ctypes.c_int, dp, dp, dp, pt, dp, dp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def make_point(s2_12=0.311, s2_13=0.0251, s2_23=0.5, dm21=7.6e-5, dm32=2.4e-3, dcp=0.0,
               escale=1.0, norm=1.0) -> OrcPoint:
    return OrcPoint(s2_12, s2_13, s2_23, dm21, dm32, dcp, escale, norm)


def point_from_row(row) -> OrcPoint:
    return OrcPoint(*[float(x) for x in row])


def c_L() -> float:
    return lib().orc_const_c_L()


def k_A() -> float:
    return lib().orc_const_k_A()


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads used by the oracle's parallel loops from now on."""
    lib().orc_set_num_threads(int(n))


def pmns(pt: OrcPoint) -> np.ndarray:
    out = np.zeros(18)
    lib().orc_pmns_flat(ctypes.byref(pt), _ptr(out, ctypes.c_double))
    return (out[0::2] + 1j * out[1::2]).reshape(3, 3)


def hamiltonian(pt: OrcPoint, A_abs: float, nubar: int) -> np.ndarray:
    out = np.zeros(18)
    lib().orc_hamiltonian_flat(ctypes.byref(pt), float(A_abs), int(nubar), _ptr(out, ctypes.c_double))
    return (out[0::2] + 1j * out[1::2]).reshape(3, 3)


def eigh3(M: np.ndarray):
    m = np.empty(18)
    m[0::2] = M.real.ravel()
    m[1::2] = M.imag.ravel()
    lam = np.zeros(3)
    v = np.zeros(18)
    sweeps = lib().orc_eigh3_flat(_ptr(m, ctypes.c_double), _ptr(lam, ctypes.c_double),
                                  _ptr(v, ctypes.c_double))
    return lam, (v[0::2] + 1j * v[1::2]).reshape(3, 3), sweeps


def prob(pt: OrcPoint, L_km, rho, ye, E, alpha, beta, nubar) -> float:
    return lib().orc_prob(ctypes.byref(pt), L_km, rho, ye, E, alpha, beta, nubar)


def prob_matrix_many(pt: OrcPoint, L_km, rho, ye, E, nubar) -> np.ndarray:
    """P[i, beta, alpha] for energies E[i]."""
    E = np.ascontiguousarray(E, dtype=np.float64)
    out = np.zeros((E.size, 3, 3))
    lib().orc_prob_matrix_many(ctypes.byref(pt), L_km, rho, ye, E.size, _ptr(E, ctypes.c_double),
                               int(nubar), _ptr(out, ctypes.c_double))
    return out


def prob_matrix_A(pt: OrcPoint, L_km, A_abs, E, nubar) -> np.ndarray:
    out = np.zeros((3, 3))
    lib().orc_prob_matrix_A(ctypes.byref(pt), L_km, A_abs, E, int(nubar), _ptr(out, ctypes.c_double))
    return out


def reweight(sample, pt: OrcPoint, n=None):
    """Per-event (prob, weight) for the first n events of a sample dict."""
    n = sample["n"] if n is None else int(n)
    prob_out = np.zeros(n)
    w_out = np.zeros(n)
    lib().orc_reweight(n, _ptr(sample["e_true"], ctypes.c_float), _ptr(sample["w_mc"], ctypes.c_float),
                       _ptr(sample["flav_in"], ctypes.c_uint8), _ptr(sample["flav_out"], ctypes.c_uint8),
                       _ptr(sample["is_nubar"], ctypes.c_uint8), sample["baseline_km"],
                       sample["density_gcc"], sample["ye"], ctypes.byref(pt),
                       _ptr(prob_out, ctypes.c_double), _ptr(w_out, ctypes.c_double))
    return prob_out, w_out


def hist_from_weights(e_reco, weight, escale, lo, hi, nbins, compensated=False) -> np.ndarray:
    e_reco = np.ascontiguousarray(e_reco, dtype=np.float32)
    weight = np.ascontiguousarray(weight, dtype=np.float64)
    out = np.zeros(nbins)
    lib().orc_hist_from_weights(e_reco.size, _ptr(e_reco, ctypes.c_float), _ptr(weight, ctypes.c_double),
                                escale, lo, hi, nbins, int(compensated), _ptr(out, ctypes.c_double))
    return out


def histogram(sample, points, lo, hi, nbins, compensated=False, n=None) -> np.ndarray:
    """out[p, b]: event-by-event histogram of the first n events for each point row."""
    n = sample["n"] if n is None else int(n)
    pts = (OrcPoint * len(points))(*[point_from_row(r) if not isinstance(r, OrcPoint) else r
                                     for r in points])
    out = np.zeros((len(points), nbins))
    scratch = np.zeros(n)
    lib().orc_histogram(n, _ptr(sample["e_true"], ctypes.c_float), _ptr(sample["e_reco"], ctypes.c_float),
                        _ptr(sample["w_mc"], ctypes.c_float), _ptr(sample["flav_in"], ctypes.c_uint8),
                        _ptr(sample["flav_out"], ctypes.c_uint8), _ptr(sample["is_nubar"], ctypes.c_uint8),
                        sample["baseline_km"], sample["density_gcc"], sample["ye"], pts, len(points),
                        lo, hi, nbins, int(compensated), _ptr(scratch, ctypes.c_double),
                        _ptr(out, ctypes.c_double))
    return out


def bins(e_reco, escale, lo, hi, nbins) -> np.ndarray:
    e_reco = np.ascontiguousarray(e_reco, dtype=np.float32)
    out = np.zeros(e_reco.size, dtype=np.int32)
    lib().orc_bin_many(e_reco.size, _ptr(e_reco, ctypes.c_float), escale, lo, hi, nbins,
                       _ptr(out, ctypes.c_int32))
    return out


def true_centre(t_lo, t_hi, t_nbins, t) -> float:
    """FP32 centre energy of true-energy bin t (see orc_true_centre)."""
    return lib().orc_true_centre(float(t_lo), float(t_hi), int(t_nbins), int(t))


def reweight_bin_centre(sample, pt: OrcPoint, t_lo, t_hi, t_nbins, n=None):
    """Per-event (prob, weight) of the binned method: P at the centre of the
    event's true-energy bin, 0 outside [t_lo, t_hi)."""
    n = sample["n"] if n is None else int(n)
    prob_out = np.zeros(n)
    w_out = np.zeros(n)
    lib().orc_reweight_bin_centre(n, _ptr(sample["e_true"], ctypes.c_float), _ptr(sample["w_mc"], ctypes.c_float),
                                  _ptr(sample["flav_in"], ctypes.c_uint8), _ptr(sample["flav_out"], ctypes.c_uint8),
                                  _ptr(sample["is_nubar"], ctypes.c_uint8), sample["baseline_km"],
                                  sample["density_gcc"], sample["ye"], ctypes.byref(pt), float(t_lo), float(t_hi),
                                  int(t_nbins), _ptr(prob_out, ctypes.c_double), _ptr(w_out, ctypes.c_double))
    return prob_out, w_out


def histogram_bin_centre(sample, points, t_lo, t_hi, t_nbins, lo, hi, nbins, compensated=False, n=None):
    """out[p, b]: binned-method histograms (weights of reweight_bin_centre binned
    by E_reco under each point's energy scale)."""
    n = sample["n"] if n is None else int(n)
    out = np.zeros((len(points), nbins))
    for k, r in enumerate(points):
        pt = r if isinstance(r, OrcPoint) else point_from_row(r)
        _, w = reweight_bin_centre(sample, pt, t_lo, t_hi, t_nbins, n)
        out[k] = hist_from_weights(sample["e_reco"][:n], w, pt.escale, lo, hi, nbins, compensated)
    return out


def _layers(layers):
    L = np.ascontiguousarray([x[0] for x in layers], dtype=np.float64)
    rho = np.ascontiguousarray([x[1] for x in layers], dtype=np.float64)
    ye = np.ascontiguousarray([x[2] for x in layers], dtype=np.float64)
    return L, rho, ye


def prob_matrix_layers_many(pt: OrcPoint, layers, E, nubar) -> np.ndarray:
    """P[i, beta, alpha] through layers [(L_km, rho, ye), ...] in order of travel."""
    L, rho, ye = _layers(layers)
    E = np.ascontiguousarray(E, dtype=np.float64)
    out = np.zeros((E.size, 3, 3))
    lib().orc_prob_matrix_layers_many(ctypes.byref(pt), L.size, _ptr(L, ctypes.c_double), _ptr(rho, ctypes.c_double),
                                      _ptr(ye, ctypes.c_double), E.size, _ptr(E, ctypes.c_double), int(nubar),
                                      _ptr(out, ctypes.c_double))
    return out


def reweight_layers(sample, pt: OrcPoint, layers, n=None):
    """Per-event (prob, weight) through layers [(L_km, rho, ye), ...]."""
    n = sample["n"] if n is None else int(n)
    L, rho, ye = _layers(layers)
    prob_out = np.zeros(n)
    w_out = np.zeros(n)
    lib().orc_reweight_layers(n, _ptr(sample["e_true"], ctypes.c_float), _ptr(sample["w_mc"], ctypes.c_float),
                              _ptr(sample["flav_in"], ctypes.c_uint8), _ptr(sample["flav_out"], ctypes.c_uint8),
                              _ptr(sample["is_nubar"], ctypes.c_uint8), L.size, _ptr(L, ctypes.c_double),
                              _ptr(rho, ctypes.c_double), _ptr(ye, ctypes.c_double), ctypes.byref(pt),
                              _ptr(prob_out, ctypes.c_double), _ptr(w_out, ctypes.c_double))
    return prob_out, w_out


def histogram_layers(sample, points, layers, lo, hi, nbins, compensated=False, n=None):
    """out[p, b]: event-by-event histograms through a layered path."""
    n = sample["n"] if n is None else int(n)
    out = np.zeros((len(points), nbins))
    for k, r in enumerate(points):
        pt = r if isinstance(r, OrcPoint) else point_from_row(r)
        _, w = reweight_layers(sample, pt, layers, n)
        out[k] = hist_from_weights(sample["e_reco"][:n], w, pt.escale, lo, hi, nbins, compensated)
    return out
