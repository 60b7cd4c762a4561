"""Thin Python binding of the C ABI in ``include/osc.h`` (argument marshalling only).

Every function has the name of the C entry point it calls.  Arrays are numpy
arrays (host) or torch CUDA tensors (device); a non-OK status raises
``OscError`` carrying the status and ``osc_last_error``.  All arithmetic runs in
the CUDA library; there is no CPU fallback -- if the library cannot be built or
loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import build as _build

OSC_OK, OSC_E_ARG, OSC_E_RANGE, OSC_E_NOMEM, OSC_E_CUDA, OSC_E_STATE, OSC_E_TIMEOUT, OSC_E_BUSY = range(8)
STATUS_NAMES = ["OSC_OK", "OSC_E_ARG", "OSC_E_RANGE", "OSC_E_NOMEM", "OSC_E_CUDA", "OSC_E_STATE",
                "OSC_E_TIMEOUT", "OSC_E_BUSY"]
OSC_FP64, OSC_FP32_BULK, OSC_FP32_F64EIG = 0, 1, 2
PRECISIONS = {"fp64": OSC_FP64, "fp32": OSC_FP32_BULK, "fp32_f64eig": OSC_FP32_F64EIG,
              OSC_FP64: OSC_FP64, OSC_FP32_BULK: OSC_FP32_BULK, OSC_FP32_F64EIG: OSC_FP32_F64EIG}

# Every entry point declared in include/osc.h, in declaration order.
ENTRY_POINTS = [
    "osc_version", "osc_create", "osc_destroy", "osc_last_error", "osc_load_sample", "osc_unload_sample",
    "osc_set_params", "osc_reweight", "osc_histogram", "osc_histogram_point", "osc_histogram_bin_centre",
    "osc_set_layers", "osc_set_tile", "osc_enable_timing", "osc_last_timing", "osc_timing_totals",
    "osc_launch_count", "osc_workspace_used", "osc_sync", "osc_serve_start", "osc_submit", "osc_wait",
    "osc_serve_stop", "osc_histogram_noalloc", "osc_sample_set_bounds", "osc_histogram_digits",
    "osc_histogram_from_digits", "osc_measure_fp32_peak",
]


class OscError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__("%s: %s" % (name, message))


class OscSampleDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64),
                ("e_true", ctypes.c_void_p), ("e_reco", ctypes.c_void_p), ("w_mc", ctypes.c_void_p),
                ("flav_in", ctypes.c_void_p), ("flav_out", ctypes.c_void_p), ("is_nubar", ctypes.c_void_p),
                ("baseline_km", ctypes.c_double), ("density_gcc", ctypes.c_double), ("ye", ctypes.c_double)]


class OscPoint(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("s2_12", "s2_13", "s2_23", "dm21", "dm32", "dcp", "escale", "norm")]


_lock = threading.Lock()
_lib = None


def lib():
    """Build (if stale) and load the CUDA library; raises if that is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            _lib = load_library(_build.build())
    return _lib


def load_library(path):
    """Load a built copy of the library at ``path`` and declare its C signatures."""
    L = ctypes.CDLL(path)
    vp, i32, i64, d, st = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    sig = {
        "osc_version": (ctypes.c_char_p, []),
        "osc_create": (st, [ctypes.c_int, ctypes.c_size_t, vp, ctypes.POINTER(vp)]),
        "osc_destroy": (None, [vp]),
        "osc_last_error": (ctypes.c_char_p, [vp]),
        "osc_load_sample": (st, [vp, ctypes.POINTER(OscSampleDesc), ctypes.POINTER(i32)]),
        "osc_unload_sample": (st, [vp, i32]),
        "osc_set_params": (st, [vp, ctypes.POINTER(OscPoint), i32]),
        "osc_reweight": (st, [vp, i32, i32, ctypes.c_int, vp, vp, ctypes.c_int]),
        "osc_histogram": (st, [vp, ctypes.POINTER(i32), i32, i32, i32, ctypes.c_int, d, d, i32, vp,
                               ctypes.c_int]),
        "osc_histogram_point": (st, [vp, ctypes.POINTER(i32), i32, ctypes.POINTER(OscPoint), ctypes.c_int, d, d,
                                     i32, vp, ctypes.c_int]),
        "osc_histogram_bin_centre": (st, [vp, ctypes.POINTER(i32), i32, i32, i32, ctypes.c_int, d, d, i32, d, d,
                                          i32, vp, ctypes.c_int]),
        "osc_set_layers": (st, [vp, i32, i32, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d)]),
        "osc_set_tile": (st, [vp, i32, i32]),
        "osc_enable_timing": (st, [vp, ctypes.c_int]),
        "osc_last_timing": (st, [vp, ctypes.POINTER(d), ctypes.POINTER(d), ctypes.POINTER(d)]),
        "osc_timing_totals": (st, [vp, ctypes.POINTER(i64), ctypes.POINTER(d)]),
        "osc_launch_count": (st, [vp, ctypes.POINTER(ctypes.c_uint64)]),
        "osc_workspace_used": (st, [vp, ctypes.POINTER(ctypes.c_size_t)]),
        "osc_sync": (st, [vp]),
        "osc_serve_start": (st, [vp, i32, d, d, i32]),
        "osc_submit": (st, [vp, i32, ctypes.POINTER(OscPoint), ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]),
        "osc_wait": (st, [vp, ctypes.c_uint64, vp, i32, ctypes.POINTER(d)]),
        "osc_serve_stop": (st, [vp]),
        "osc_histogram_noalloc": (st, [vp, vp, vp, vp, vp, vp, i64, d, d, d, d, ctypes.POINTER(OscPoint),
                                       ctypes.c_int, d, d, i32, vp, vp, ctypes.c_char_p, ctypes.c_size_t]),
        "osc_sample_set_bounds": (st, [vp, i32, d, d]),
        "osc_measure_fp32_peak": (st, [ctypes.c_int, ctypes.POINTER(d)]),
        "osc_histogram_digits": (st, [vp, ctypes.POINTER(i32), i32, i32, i32, ctypes.c_int, d, d, i32, vp,
                                      ctypes.c_int]),
        "osc_histogram_from_digits": (st, [vp, ctypes.POINTER(i32), i32, i32, i32, i32, vp, vp, ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def _check(ctx, status):
    if status != OSC_OK:
        msg = lib().osc_last_error(ctx)
        raise OscError(status, msg.decode() if msg else "")


def _addr(a):
    """Data address of a numpy array.  A ctypes view of a writable contiguous
    buffer is cheaper to make than ``a.ctypes``; other arrays use the latter."""
    try:
        return ctypes.addressof(ctypes.c_char.from_buffer(a))
    except (TypeError, ValueError, BufferError):
        return a.ctypes.data


def _ptr(a):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return _addr(a)
    return a.data_ptr()


def _ids(sample_ids):
    """Sample ids as a C int32 array and its length."""
    if type(sample_ids) in (list, tuple):
        return (ctypes.c_int32 * len(sample_ids))(*[int(i) for i in sample_ids]), len(sample_ids)
    a = np.ascontiguousarray(np.atleast_1d(sample_ids), dtype=np.int32)
    return (ctypes.c_int32 * a.size).from_buffer_copy(a), a.size


def _is_device(a):
    return a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def _points(points):
    if (type(points) is np.ndarray and points.dtype == np.float64 and points.ndim in (1, 2) and points.shape[-1] == 8
            and points.size > 0 and points.flags.c_contiguous and points.flags.writeable):
        # a view of the caller's rows (read during the call)
        n = points.size // 8
        return (OscPoint * n).from_buffer(points), n
    rows = np.ascontiguousarray(np.atleast_2d(np.asarray(points, dtype=np.float64)))
    if rows.shape[1] != 8:
        raise ValueError("points must have 8 columns: s2_12 s2_13 s2_23 dm21 dm32 dcp escale norm")
    arr = (OscPoint * rows.shape[0])()
    ctypes.memmove(arr, rows.ctypes.data, rows.nbytes)
    return arr, rows.shape[0]


def osc_version() -> str:
    return lib().osc_version().decode()


def osc_create(device=0, workspace_cap_bytes=0, cuda_stream=None):
    out = ctypes.c_void_p()
    s = lib().osc_create(int(device), int(workspace_cap_bytes), cuda_stream, ctypes.byref(out))
    if s != OSC_OK:
        raise OscError(s, "osc_create failed")
    return out


def osc_destroy(ctx):
    lib().osc_destroy(ctx)


def osc_last_error(ctx) -> str:
    m = lib().osc_last_error(ctx)
    return m.decode() if m else ""


def osc_load_sample(ctx, sample) -> int:
    """sample: dict with n, e_true, e_reco, w_mc (float32), flav_in, flav_out, is_nubar
    (uint8), baseline_km, density_gcc, ye."""
    arrs = {}
    for k, dt in (("e_true", np.float32), ("e_reco", np.float32), ("w_mc", np.float32),
                  ("flav_in", np.uint8), ("flav_out", np.uint8), ("is_nubar", np.uint8)):
        arrs[k] = np.ascontiguousarray(sample[k], dtype=dt)
    n = int(sample.get("n", arrs["e_true"].size))
    for k, a in arrs.items():
        if a.size < n:
            raise ValueError("array %s shorter than n" % k)
    desc = OscSampleDesc(n, *[arrs[k].ctypes.data for k in ("e_true", "e_reco", "w_mc", "flav_in", "flav_out",
                                                            "is_nubar")],
                         float(sample["baseline_km"]), float(sample["density_gcc"]), float(sample["ye"]))
    sid = ctypes.c_int32()
    _check(ctx, lib().osc_load_sample(ctx, ctypes.byref(desc), ctypes.byref(sid)))
    return sid.value


def osc_unload_sample(ctx, sample_id):
    _check(ctx, lib().osc_unload_sample(ctx, int(sample_id)))


def osc_set_params(ctx, points):
    arr, n = _points(points)
    _check(ctx, lib().osc_set_params(ctx, arr, n))


def osc_reweight(ctx, sample_id, point, prec, out_prob=None, out_weight=None):
    """Outputs: numpy float64 arrays (host) or torch float64 CUDA tensors (device), n each."""
    dev = _is_device(out_prob) or _is_device(out_weight)
    _check(ctx, lib().osc_reweight(ctx, int(sample_id), int(point), PRECISIONS[prec], _ptr(out_prob),
                                   _ptr(out_weight), 1 if dev else 0))
    return out_prob, out_weight


def osc_histogram(ctx, sample_ids, point_begin, n_points, prec, lo, hi, nbins, out=None):
    """out: numpy (n_samples, n_points, nbins) float64 (allocated if None) or a torch CUDA tensor."""
    ids, n_ids = _ids(sample_ids)
    if out is None:
        out = np.zeros((n_ids, int(n_points), int(nbins)))
    dev = _is_device(out)
    _check(ctx, lib().osc_histogram(ctx, ids, n_ids, int(point_begin), int(n_points), PRECISIONS[prec], float(lo),
                                    float(hi), int(nbins), _ptr(out), 1 if dev else 0))
    return out


def osc_measure_fp32_peak(device=0):
    """FP32 FMA throughput of the device [TFLOP/s, FMA = 2 flops]."""
    t = ctypes.c_double()
    s = lib().osc_measure_fp32_peak(int(device), ctypes.byref(t))
    if s != OSC_OK:
        raise OscError(s, "osc_measure_fp32_peak failed")
    return t.value


def osc_sample_set_bounds(ctx, sample_id, w_abs_max, e_true_max):
    """The whole sample's bounds for this rank's slice of it (event sharding)."""
    _check(ctx, lib().osc_sample_set_bounds(ctx, int(sample_id), float(w_abs_max), float(e_true_max)))


def osc_histogram_digits(ctx, sample_ids, point_begin, n_points, prec, lo, hi, nbins, out=None):
    """Exact bin sums as digit columns: numpy uint64 (n_samples, n_points, nbins, 4)
    (allocated if None) or a torch int64/uint64 CUDA tensor of that shape."""
    ids, n_ids = _ids(sample_ids)
    if out is None:
        out = np.zeros((n_ids, int(n_points), int(nbins), 4), dtype=np.uint64)
    dev = _is_device(out)
    _check(ctx, lib().osc_histogram_digits(ctx, ids, n_ids, int(point_begin), int(n_points), PRECISIONS[prec],
                                           float(lo), float(hi), int(nbins), _ptr(out), 1 if dev else 0))
    return out


def osc_histogram_from_digits(ctx, sample_ids, point_begin, n_points, nbins, digits, out=None):
    """Bins (n_samples, n_points, nbins) from digit columns summed over ranks.
    digits and out: both numpy (host) or both torch CUDA tensors."""
    ids, n_ids = _ids(sample_ids)
    dev = _is_device(digits)
    if out is None:
        out = np.zeros((n_ids, int(n_points), int(nbins)))
    if _is_device(out) != dev:
        raise OscError(OSC_E_ARG, "digits and out must both be host or both be device arrays")
    if not dev:
        digits = np.ascontiguousarray(digits)
        if digits.dtype not in (np.uint64, np.int64) or digits.size != n_ids * int(n_points) * int(nbins) * 4:
            raise OscError(OSC_E_ARG, "digits must be 64-bit integers, 4 per bin")
    _check(ctx, lib().osc_histogram_from_digits(ctx, ids, n_ids, int(point_begin), int(n_points), int(nbins),
                                                _ptr(digits), _ptr(out), 1 if dev else 0))
    return out


def osc_histogram_point(ctx, sample_ids, point, prec, lo, hi, nbins, out=None):
    """One fit step: the point (8 fields) becomes the table and its histograms
    are computed; out: (n_samples, 1, nbins) as for osc_histogram."""
    ids, n_ids = _ids(sample_ids)
    arr, n = _points(point)
    if n != 1:
        raise ValueError("osc_histogram_point takes exactly one point")
    if out is None:
        out = np.zeros((n_ids, 1, int(nbins)))
    dev = _is_device(out)
    _check(ctx, lib().osc_histogram_point(ctx, ids, n_ids, arr, PRECISIONS[prec], float(lo), float(hi), int(nbins),
                                          _ptr(out), 1 if dev else 0))
    return out


class PointHistogram:
    """``osc_histogram_point`` with its arguments marshalled once, for a caller
    that evaluates many points on the same samples, range and output buffer (a
    fit).  ``point`` is a writable float64[8] view of the point that the next
    call sends (the fields of ``osc_point`` in order); ``call(p)`` copies ``p``
    there first, ``call()`` sends it as it stands.  Each call writes the
    histograms into ``out`` (n_samples, 1, nbins) and returns it.  Like the C
    call, an instance is not safe to use from two threads at once."""

    def __init__(self, ctx, sample_ids, prec, lo, hi, nbins, out=None):
        ids, n_ids = _ids(sample_ids)
        if out is None:
            out = np.zeros((n_ids, 1, int(nbins)))
        self.out = out
        self._ctx = ctx
        self._ids = ids
        self._buf = (ctypes.c_double * 8)()
        self.point = np.ctypeslib.as_array(self._buf)
        self._fn = lib().osc_histogram_point
        self._args = (ctx, ids, ctypes.c_int32(n_ids), ctypes.cast(self._buf, ctypes.POINTER(OscPoint)),
                      ctypes.c_int(PRECISIONS[prec]), ctypes.c_double(float(lo)), ctypes.c_double(float(hi)),
                      ctypes.c_int32(int(nbins)), ctypes.c_void_p(_ptr(out)), ctypes.c_int(1 if _is_device(out) else 0))

    def __call__(self, point=None):
        if point is not None:
            self.point[:] = point
        status = self._fn(*self._args)
        if status != OSC_OK:
            _check(self._ctx, status)
        return self.out


def osc_histogram_bin_centre(ctx, sample_ids, point_begin, n_points, prec, t_lo, t_hi, t_nbins, lo, hi, nbins,
                             out=None):
    """Binned-method histograms (probability at the centre of each event's
    true-energy bin); out as for osc_histogram."""
    ids, n_ids = _ids(sample_ids)
    if out is None:
        out = np.zeros((n_ids, int(n_points), int(nbins)))
    dev = _is_device(out)
    _check(ctx, lib().osc_histogram_bin_centre(ctx, ids, n_ids,
                                               int(point_begin), int(n_points), PRECISIONS[prec], float(t_lo),
                                               float(t_hi), int(t_nbins), float(lo), float(hi), int(nbins),
                                               _ptr(out), 1 if dev else 0))
    return out


def osc_set_layers(ctx, sample_id, layers):
    """layers: sequence of (length_km, density_gcc, ye) in the order of travel."""
    arr = np.ascontiguousarray(np.asarray(layers, dtype=np.float64).reshape(-1, 3))
    cols = [np.ascontiguousarray(arr[:, k]) for k in range(3)]
    dp = ctypes.POINTER(ctypes.c_double)
    _check(ctx, lib().osc_set_layers(ctx, int(sample_id), arr.shape[0], *[c.ctypes.data_as(dp) for c in cols]))


def osc_set_tile(ctx, points_per_block=0, events_per_item=0):
    _check(ctx, lib().osc_set_tile(ctx, int(points_per_block), int(events_per_item)))


def osc_enable_timing(ctx, enable=True):
    _check(ctx, lib().osc_enable_timing(ctx, 1 if enable else 0))


def osc_last_timing(ctx):
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().osc_last_timing(ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def osc_timing_totals(ctx):
    """Returns (counts[3], sums_ms[3]) for (constants, histogram, finalize) kernels."""
    n = (ctypes.c_int64 * 3)()
    t = (ctypes.c_double * 3)()
    _check(ctx, lib().osc_timing_totals(ctx, n, t))
    return list(n), list(t)


def osc_launch_count(ctx) -> int:
    v = ctypes.c_uint64()
    _check(ctx, lib().osc_launch_count(ctx, ctypes.byref(v)))
    return v.value


def osc_workspace_used(ctx) -> int:
    v = ctypes.c_size_t()
    _check(ctx, lib().osc_workspace_used(ctx, ctypes.byref(v)))
    return v.value


def osc_sync(ctx):
    _check(ctx, lib().osc_sync(ctx))


def osc_serve_start(ctx, max_slots, lo, hi, nbins):
    _check(ctx, lib().osc_serve_start(ctx, int(max_slots), float(lo), float(hi), int(nbins)))


def osc_submit(ctx, sample_id, point, prec) -> int:
    arr, n = _points(point)
    t = ctypes.c_uint64()
    _check(ctx, lib().osc_submit(ctx, int(sample_id), arr, PRECISIONS[prec], ctypes.byref(t)))
    return t.value


def osc_wait(ctx, ticket, nbins, timeout_ms=-1, out=None):
    """Returns (histogram, latency_us)."""
    if out is None:
        out = np.zeros(int(nbins))
    lat = ctypes.c_double()
    _check(ctx, lib().osc_wait(ctx, int(ticket), _addr(out), int(timeout_ms), ctypes.byref(lat)))
    return out, lat.value


def osc_serve_stop(ctx):
    _check(ctx, lib().osc_serve_stop(ctx))


def osc_histogram_noalloc(e_true, e_reco, w_mc, flav_in, flav_out, is_nubar, baseline_km, density_gcc, ye,
                          w_abs_max, point, prec, lo, hi, nbins, out, cuda_stream=None):
    """One-point histogram with no allocation inside the library: every array
    (inputs and the nbins-long float64 output) is a caller-owned torch CUDA tensor.

    The library sees only device pointers and n, so the arrays are checked here,
    before the call: CUDA and contiguous, float32 energies and weights, uint8
    flavour flags, all six of the same length n >= 1, and a float64 output of at
    least nbins elements.  A violation raises OscError(OSC_E_ARG)."""
    arr, _ = _points(point)
    ins = {"e_true": (e_true, "float32"), "e_reco": (e_reco, "float32"), "w_mc": (w_mc, "float32"),
           "flav_in": (flav_in, "uint8"), "flav_out": (flav_out, "uint8"), "is_nubar": (is_nubar, "uint8")}
    n = None
    for name, (t, dt) in ins.items():
        if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous()):
            raise OscError(OSC_E_ARG, "%s must be a contiguous CUDA tensor" % name)
        if str(t.dtype) != "torch." + dt:
            raise OscError(OSC_E_ARG, "%s must be %s, got %s" % (name, dt, t.dtype))
        if n is None:
            n = int(t.numel())
        elif int(t.numel()) != n:
            raise OscError(OSC_E_ARG, "all six event arrays must have the same length (%s has %d, not %d)"
                           % (name, int(t.numel()), n))
    if not (hasattr(out, "is_cuda") and out.is_cuda and out.is_contiguous()) or str(out.dtype) != "torch.float64":
        raise OscError(OSC_E_ARG, "out must be a contiguous float64 CUDA tensor")
    if int(out.numel()) < int(nbins):
        raise OscError(OSC_E_ARG, "out holds %d values, fewer than nbins = %d" % (int(out.numel()), int(nbins)))
    buf = ctypes.create_string_buffer(256)
    s = lib().osc_histogram_noalloc(_ptr(e_true), _ptr(e_reco), _ptr(w_mc), _ptr(flav_in), _ptr(flav_out),
                                    _ptr(is_nubar), n, float(baseline_km), float(density_gcc), float(ye),
                                    float(w_abs_max), arr, PRECISIONS[prec], float(lo), float(hi), int(nbins),
                                    _ptr(out), cuda_stream, buf, 256)
    if s != OSC_OK:
        raise OscError(s, buf.value.decode())
    return out


class Context:
    """Owning handle: ``with Context() as c: osc_load_sample(c.ptr, ...)``."""

    def __init__(self, device=0, workspace_cap_bytes=0, cuda_stream=None):
        self.ptr = osc_create(device, workspace_cap_bytes, cuda_stream)

    def close(self):
        if self.ptr:
            osc_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
