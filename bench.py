"""Benchmark: event-by-event oscillation reweighting on GB300.

Workload (one step = one pass of the whole hot path over one batch): the
precision-study configuration -- 10M events shaped like the paper's beam MC
(Gamma(3, 0.25 GeV) true energies, 295 km, 2.6 g/cm^3, Y_e 0.5, nu_mu -> nu_mu
90 % / nu_mu -> nu_e 10 %, 20 % antineutrinos) at the Table 1 parameter point:
one fit step, osc_histogram_point -- the point by value to the FP64 constants
kernel, then the histogram kernel (probability, weight, bin and exact
accumulation, finalized in place) and the FP32 path's FP64 recomputation pass,
replayed as one CUDA graph whose kernels are joined by programmatic edges --
into a 100-bin E_reco histogram over [0, 5) GeV.  FP32-bulk path; the all-FP64
path is timed on the same workload as the GPU baseline to beat.

Timing: W warm-up steps, then K steps each bracketed by CUDA events on the
launching stream, with a 256 MB write between steps to flush the 129 MB L2
(outside the events); barrier + synchronize around the timed region; the max
over ranks.  Under torchrun every rank reweights its own independent sample
(weak scaling, no data-path collective).

--impl reference times the FP64 CPU oracle on the host cores instead (rank 0
only), on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "event-weights/s FP32-bulk vs all-FP64 at |dP|<=1e-5; p50/p99 reweight latency"
UNIT = "event-weights/s"
N_EVENTS = 10_000_000
NBINS, LO, HI = 100, 0.0, 5.0
FLUSH_BYTES = 256 << 20

# Algorithmic work per (event, point) of the FP32-bulk path.
#  * The method's minimum (the roofline's count): about 95 FP32 operations and 6
#    SFU operations -- the cubic's eigenvalues from a seed and Newton steps, the
#    Sylvester amplitude over three roots, weight and bin.
#  * The kernel's own arithmetic, counted from osc_math.cuh / osc_kernels.cuh
#    (FMA = 2, add/mul = 1; conversions, comparisons, selects and integer work not
#    counted) for the mu -> mu / tau -> tau channels, 90 % of the workload: event
#    terms 11, matter shifts 70 (seed 27, seeds 8, two Newton steps with one shared
#    reciprocal 33, trace 2), gaps and phases 30, amplitude in the mass
#    basis with its error bound 48, weight and bin 4 -- 163 flops; the other
#    channels add the matter and electron terms, about 185.  SFU: 11 (1/E, the
#    seed's rsqrt, sqrt and sin/cos, the Newton steps' shared reciprocal, two
#    sin/cos of half phases, 1/D).  On this GPU the FP32 adds, multiplies and FMAs
#    of an event pair issue as packed pairs (add/mul/fma.f32x2).
ALG_OPS_PER_EVPT = 95
ALG_SFU_PER_EVPT = 6
FP32_FLOP_PER_EVPT = 163
SFU_PER_EVPT = 11
ALG_BYTES_PER_EVENT = 13  # E_true, E_reco, w_mc (FP32) and the channel byte


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


KERNEL_SOURCES = ("osc_internal.h", "osc_math.cuh", "osc_kernels.cuh", "osc_kernels_fp32.cu")
TRAFFIC_PROFILE = os.path.join(ROOT, "profiles", "k_hist_inline_fp32_precision10M_1pt.md")


def _kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1311_7579_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_field(name, kind=int):
    """A numeric field of the bench kernel's committed ncu summary, or None when
    the kernel sources changed since that capture."""
    if not os.path.exists(TRAFFIC_PROFILE):
        return None
    fields = {}
    for line in open(TRAFFIC_PROFILE):
        if ":" in line and not line.startswith("|"):
            k, v = line.split(":", 1)
            fields[k.strip()] = v.split()[0] if v.split() else ""
    if fields.get("kernel_source_sha256_16") != _kernel_source_hash():
        return None
    try:
        return kind(fields[name])
    except (KeyError, ValueError):
        return None


def _profiled_traffic():
    """DRAM bytes per launch of the bench kernel (ncu), or None."""
    return _profile_field("dram_bytes_per_launch")


def _measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")] + [time.perf_counter()])

    def window(self, t0, t1):
        inside = [r for r in self.rows if t0 <= r[-1] <= t1]
        self.rows = inside if inside else self.rows

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def cpu_baseline_leg(sample, point_row, gpu_p32, gpu_p64, n_sample):
    """FP64 oracle on the host cores over the first n_sample events: throughput,
    and the |dP| of both GPU paths on that subsample (precision study)."""
    import oracle
    pt = oracle.point_from_row(point_row)
    sub = {k: (v[:n_sample] if isinstance(v, np.ndarray) else v) for k, v in sample.items()}
    sub["n"] = n_sample
    oracle.reweight(dict(sub, n=min(1000, n_sample)), pt)  # warm (thread pool, pages)
    t0 = time.perf_counter()
    po, wo = oracle.reweight(sub, pt)
    h = oracle.hist_from_weights(sub["e_reco"], wo, point_row[6], LO, HI, NBINS)
    dt = time.perf_counter() - t0
    d32 = np.abs(gpu_p32[:n_sample] - po)
    d64 = np.abs(gpu_p64[:n_sample] - po)
    cores = oracle.num_threads()
    # the same work on one core, over a shorter sample
    n1 = min(n_sample, 300_000)
    oracle.set_num_threads(1)
    t1 = time.perf_counter()
    _, w1 = oracle.reweight(dict(sub, n=n1), pt)
    oracle.hist_from_weights(sub["e_reco"][:n1], w1, point_row[6], LO, HI, NBINS)
    dt1 = time.perf_counter() - t1
    oracle.set_num_threads(cores)
    # the batched-scan shape: the first 16 scan points over the 2M-event scan sample
    from paper_1311_7579_gb300 import synth
    scan = synth.scan_sample()
    t2 = time.perf_counter()
    oracle.histogram(scan, synth.scan_points()[:16], LO, HI, NBINS)
    dt2 = time.perf_counter() - t2
    cpu = {"value": n_sample / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "first %d events of the 10M-event sample, Table 1 point: FP64 Jacobi oracle reweight + "
                     "100-bin histogram, %.2f s wall" % (n_sample, dt),
           "single_core": {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                           "sample": "first %d events, %.2f s wall" % (n1, dt1)},
           "scan_16_points": {"value": 16 * scan["n"] / dt2, "unit": UNIT, "cores": cores,
                              "sample": "2M-event scan sample x first 16 scan points, %.2f s wall" % dt2}}
    prec = {"subsample_events": n_sample, "fp32_max_dP": float(d32.max()), "fp32_rms_dP": float(np.sqrt(np.mean(d32 ** 2))),
            "fp64_max_dP": float(d64.max()), "fp64_rms_dP": float(np.sqrt(np.mean(d64 ** 2)))}
    return cpu, prec, h


_UNEVEN = []


def _uneven_samples(synth):
    """The 8 uneven samples (47.6M events), generated once per run."""
    if not _UNEVEN:
        _UNEVEN.extend(synth.uneven_samples())
    return _UNEVEN


def precision_per_config(api, synth, c):
    """FP32-bulk and FP32_F64EIG |dP| against the FP64 oracle on each workload
    shape (bounded subsets so the oracle finishes in seconds): the Table 1
    sample (100k events), the scan sample at 4 scan points, the first 500k
    events of each uneven sample at one point, and the 10M U(0.05, 30) GeV
    validation energies subsampled to 1M (nu_mu -> nu_mu at Table 1)."""
    import oracle
    cases = []
    cases.append(("table1_100k", synth.table1_sample(), synth.table1_point()[None, :]))
    scan = synth.scan_sample()
    cases.append(("scan_2M_x_4pts", scan, synth.scan_points()[[0, 1, 2047, 4095]]))
    for j, u in enumerate(_uneven_samples(synth)):
        sub = {k: (v[:500_000] if isinstance(v, np.ndarray) else v) for k, v in u.items()}
        sub["n"] = min(u["n"], 500_000)
        cases.append(("uneven_%d_first500k" % j, sub, synth.uneven_points()[[3]]))
    e = synth.validation_energies(1_000_000)
    n = e.size
    val = {"n": n, "e_true": e.astype(np.float32), "e_reco": e.astype(np.float32),
           "w_mc": np.ones(n, np.float32), "flav_in": np.ones(n, np.uint8), "flav_out": np.ones(n, np.uint8),
           "is_nubar": np.zeros(n, np.uint8), "baseline_km": 295.0, "density_gcc": 2.6, "ye": 0.5}
    cases.append(("validation_1M_U(0.05,30)", val, synth.table1_point()[None, :]))
    out = {}
    for name, smp, pts in cases:
        sid = api.osc_load_sample(c, smp)
        api.osc_set_params(c, pts)
        res = {"events": int(smp["n"]), "points": int(pts.shape[0])}
        worst = {"fp32": [0.0, 0.0], "fp32_f64eig": [0.0, 0.0], "fp64": [0.0, 0.0]}
        for k in range(pts.shape[0]):
            po, _ = oracle.reweight(smp, oracle.point_from_row(pts[k]))
            for prec in worst:
                p = np.zeros(smp["n"])
                api.osc_reweight(c, sid, k, prec, out_prob=p)
                d = np.abs(p - po)
                worst[prec][0] = max(worst[prec][0], float(d.max()))
                worst[prec][1] = max(worst[prec][1], float(np.sqrt(np.mean(d ** 2))))
        for prec, (mx, rms) in worst.items():
            res[prec] = {"max_dP": mx, "rms_dP": rms}
        out[name] = res
        api.osc_unload_sample(c, sid)
    return out


SERVE_CAP_BYTES = 8 << 30
SERVE_RATES = (1000, 2000, 5000, 10000, 20000, 50000)  # the serving context's workspace cap (samples, points, batch buffers)


def serving_leg(api, synth, device, rates, seconds, prec="fp32"):
    """Serving workload: requests (sample id uniform over the 8 uneven samples,
    point from the scan distribution) arrive as a Poisson process at each rate for
    `seconds`; a submitter thread follows the arrival schedule, a collector thread
    waits on the tickets.  The serving context has an 8 GB workspace cap: the 8
    resident samples (47.6M events) and every batch buffer are admitted under it.
    Reports achieved request and event-weight throughput and the p50/p99
    submit-to-completion latency measured inside the library."""
    with api.Context(device, workspace_cap_bytes=SERVE_CAP_BYTES) as ctx:
        out = _serving_leg(api, synth, ctx.ptr, rates, seconds, prec)
        out["workspace_cap_bytes"] = SERVE_CAP_BYTES
        return out


def _serving_leg(api, synth, c, rates, seconds, prec):
    import threading
    samples = _uneven_samples(synth)
    sids = [api.osc_load_sample(c, s) for s in samples]
    sizes = np.array([s["n"] for s in samples], dtype=np.float64)
    api.osc_serve_start(c, 256, LO, 20.0, NBINS)
    out = {"samples_events": [int(x) for x in sizes], "max_slots": 256, "prec": prec, "rates": [],
           "seconds_per_rate": seconds, "workspace_used_bytes": int(api.osc_workspace_used(c))}
    try:
        # warm-up
        for k in range(16):
            t = api.osc_submit(c, sids[k % len(sids)], synth.scan_points(1, seed=k)[0], prec)
            api.osc_wait(c, t, NBINS)
        for rate in rates:
            t_arr, sid_idx, pts = synth.serving_requests(seconds, rate, n_samples=len(sids), seed=4004)
            n = len(t_arr)
            tickets = [None] * n
            lat = np.zeros(n)
            done = [0]

            def collect():
                buf = np.zeros(NBINS)
                for i in range(n):
                    while tickets[i] is None:
                        time.sleep(0)
                    if tickets[i] < 0:  # rejected at submission: the queue was full
                        continue
                    _, lat[i] = api.osc_wait(c, tickets[i], NBINS, out=buf)
                    done[0] += 1

            th = threading.Thread(target=collect)
            th.start()
            t0 = time.perf_counter()
            for i in range(n):
                while time.perf_counter() - t0 < t_arr[i]:
                    pass
                try:
                    tickets[i] = api.osc_submit(c, sids[sid_idx[i]], pts[i], prec)
                except api.OscError as err:
                    # above saturation the queue (2^20 requests) fills: the request is
                    # shed, as a server under overload would, and counted
                    if err.status != api.OSC_E_BUSY:
                        for k in range(i, n):
                            tickets[k] = -1
                        th.join()
                        raise
                    tickets[i] = -1
            th.join()
            wall = time.perf_counter() - t0
            ok = np.array([t is not None and t >= 0 for t in tickets])
            evpt = float(sizes[sid_idx[ok]].sum())
            out["rates"].append({"offered_req_s": rate, "requests": n, "rejected_queue_full": int(n - ok.sum()),
                                 "achieved_req_s": float(ok.sum()) / wall, "event_weights_s": evpt / wall,
                                 "p50_us": float(np.percentile(lat[ok], 50)) if ok.any() else None,
                                 "p99_us": float(np.percentile(lat[ok], 99)) if ok.any() else None})
        # saturation: everything queued at once
        nsat = 2000 if prec == "fp32" else 100
        rng = np.random.default_rng(5005)
        sid_idx = rng.integers(0, len(sids), nsat)
        pts = synth.scan_points(nsat, seed=5006)
        t0 = time.perf_counter()
        tk = [api.osc_submit(c, sids[sid_idx[i]], pts[i], prec) for i in range(nsat)]
        buf = np.zeros(NBINS)
        for t in tk:
            api.osc_wait(c, t, NBINS, out=buf)
        wall = time.perf_counter() - t0
        out["saturation"] = {"requests": nsat, "req_s": nsat / wall,
                             "event_weights_s": float(sizes[sid_idx].sum()) / wall}
    finally:
        api.osc_serve_stop(c)
        for sid in sids:
            api.osc_unload_sample(c, sid)
    return out


def mcmc_leg(api, synth, c, sid, sample, n_steps, prec="fp32"):
    """Toy fit (Sec. 2.2): Metropolis-Hastings over (sin^2 theta23, dm32) on the
    bench sample, each step one set_params + histogram + Eq. (2) likelihood on the
    host.  Reports the steps per second of the whole fit loop (wall clock)."""
    from paper_1311_7579_gb300 import fit
    expo = fit.exposure_for(sample, 20000, LO, HI)
    truth = fit.ToyFit(c, sid, np.zeros(NBINS), expo, LO, HI, NBINS, "fp64")
    data = fit.fake_data(truth.expected(np.array([0.5, 2.4e-3])), seed=92)
    f = fit.ToyFit(c, sid, data, expo, LO, HI, NBINS, prec)
    lower, upper = np.array([0.3, 2.0e-3]), np.array([0.7, 3.0e-3])
    fit.metropolis(f.loglike, [0.45, 2.3e-3], [0.02, 3e-5], 20, np.random.default_rng(1), lower, upper)
    t0 = time.perf_counter()
    chain, _, acc = fit.metropolis(f.loglike, [0.45, 2.3e-3], [0.02, 3e-5], n_steps, np.random.default_rng(2),
                                   lower, upper)
    dt = time.perf_counter() - t0
    post = chain[n_steps // 5:]
    return {"prec": prec, "steps": n_steps, "steps_per_s": n_steps / dt, "ms_per_step": 1e3 * dt / n_steps,
            "events_per_step": int(sample["n"]), "acceptance": acc,
            "posterior_mean": [float(x) for x in post.mean(axis=0)],
            "posterior_sd": [float(x) for x in post.std(axis=0)]}


def _event_times(torch, stream, flush, fn, k, w):
    """Per-call device times [ms] of fn() on the library's stream, L2 flushed before each call."""
    for _ in range(w):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
    for i in range(k):
        flush.zero_()
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return np.array([a.elapsed_time(b) for a, b in ev])


def bin_centre_leg(torch, api, synth, c, sid, sample, point, stream, flush, hbm_peak, k=200):
    """Binned (bin-centre) method on the bench workload: P at the centre of each
    event's 25 MeV true-energy bin (410 bins over [0, 10.25) GeV), same E_reco
    histogram.  Times the whole call (table kernel + histogram kernel); the
    event stream (16 B per event) over that time is a lower bound of the
    histogram kernel's bandwidth.  Also the Sec. 1.1.1 25 MeV-bin study."""
    tb = (0.0, 10.25, 410)
    out = torch.zeros((1, 1, NBINS), dtype=torch.float64, device=flush.device)
    api.osc_set_params(c, point)
    res = {"true_bins": {"lo": tb[0], "hi": tb[1], "n": tb[2]}}
    for prec in ("fp32", "fp64"):
        ms = _event_times(torch, stream, flush, lambda: api.osc_histogram_bin_centre(
            c, [sid], 0, 1, prec, *tb, LO, HI, NBINS, out=out), k, 5)
        t = float(np.median(ms))
        res[prec] = {"value": N_EVENTS / (t * 1e-3), "unit": UNIT, "call_ms_p50": t,
                     "event_stream_gbs": 16.0 * N_EVENTS / (t * 1e-3) / 1e9}
        if hbm_peak:
            res[prec]["event_stream_frac_of_measured_hbm"] = res[prec]["event_stream_gbs"] / hbm_peak
    # binned vs event-by-event spectra of the whole sample (FP64)
    hb = api.osc_histogram_bin_centre(c, [sid], 0, 1, "fp64", *tb, LO, HI, NBINS)[0, 0]
    he = api.osc_histogram(c, [sid], 0, 1, "fp64", LO, HI, NBINS)[0, 0]
    nz = he > 0
    res["spectrum_max_rel_diff_vs_event_by_event"] = float(np.max(np.abs(hb[nz] - he[nz]) / he[nz]))
    # the 25 MeV bin from 0.6 GeV: quadrature nodes of the Gamma(3, 0.25 GeV) spectrum as events
    from scipy import stats
    K = 4000
    h = 0.025 / K
    nodes = (0.6 + (np.arange(K) + 0.5) * h).astype(np.float32)
    q = {"n": K, "e_true": nodes, "e_reco": nodes,
         "w_mc": (stats.gamma(3.0, scale=0.25).pdf(nodes.astype(np.float64)) * h).astype(np.float32),
         "flav_in": np.ones(K, np.uint8), "flav_out": np.ones(K, np.uint8), "is_nubar": np.zeros(K, np.uint8),
         "baseline_km": 295.0, "density_gcc": 2.6, "ye": 0.5}
    qid = api.osc_load_sample(c, q)
    ee = api.osc_histogram(c, [qid], 0, 1, "fp64", 0.0, 10.0, 400)[0, 0, 24]
    bb = api.osc_histogram_bin_centre(c, [qid], 0, 1, "fp64", 0.0, 10.0, 400, 0.0, 10.0, 400)[0, 0, 24]
    api.osc_unload_sample(c, qid)
    res["study_25MeV_bin_0.6GeV"] = {"event_by_event_over_bin_centre_minus_1": float(ee / bb - 1.0),
                                     "spectrum": "Gamma(3, 0.25 GeV), nu_mu -> nu_mu, 295 km, 2.6 g/cm^3"}
    return res


def configs_leg(torch, api, synth, c, stream, flush):
    """The other workload configurations, one histogram call each (autotuned):
    the 100k-event Table 1 sample x 1 point in FP64 and FP32, and the 8 uneven
    samples (47.6M events) x 512 points in one FP32 launch."""
    res = {}
    s0 = synth.table1_sample()
    sid = api.osc_load_sample(c, s0)
    api.osc_set_params(c, synth.table1_point()[None, :])
    out = torch.zeros((1, 1, NBINS), dtype=torch.float64, device=flush.device)
    for prec in ("fp64", "fp32"):
        ms = _event_times(torch, stream, flush, lambda: api.osc_histogram(
            c, [sid], 0, 1, prec, LO, HI, NBINS, out=out), 50, 5)
        t = float(np.median(ms))
        res["table1_100k_x_1_%s" % prec] = {"value": s0["n"] / (t * 1e-3), "unit": UNIT, "call_ms_p50": t}
    api.osc_unload_sample(c, sid)
    ss = _uneven_samples(synth)
    sids = [api.osc_load_sample(c, u) for u in ss]
    pts = synth.uneven_points()
    api.osc_set_params(c, pts)
    out = torch.zeros((len(ss), pts.shape[0], NBINS), dtype=torch.float64, device=flush.device)
    ms = _event_times(torch, stream, flush, lambda: api.osc_histogram(
        c, sids, 0, pts.shape[0], "fp32", 0.0, 20.0, NBINS, out=out), 3, 2)
    t = float(np.median(ms))
    ev_pt = sum(u["n"] for u in ss) * pts.shape[0]
    res["uneven_8_samples_x_512_fp32"] = {"value": ev_pt / (t * 1e-3), "unit": UNIT, "call_ms_p50": t,
                                          "event_points": ev_pt}
    for x in sids:
        api.osc_unload_sample(c, x)
    return res


def scan_leg(torch, api, synth, c, stream, flush, k=5):
    """Batched parameter scan: the 2M-event scan sample x 4096 points in one
    launch (autotuned tile), FP32-bulk, event by event and by the bin-centre method."""
    s = synth.scan_sample()
    sid = api.osc_load_sample(c, s)
    pts = synth.scan_points()
    api.osc_set_params(c, pts)
    out = torch.zeros((1, pts.shape[0], NBINS), dtype=torch.float64, device=flush.device)
    ev_pt = s["n"] * pts.shape[0]
    res = {"events": s["n"], "points": int(pts.shape[0])}
    ms = _event_times(torch, stream, flush, lambda: api.osc_histogram(
        c, [sid], 0, pts.shape[0], "fp32", LO, HI, NBINS, out=out), k, 3)
    res["event_by_event_fp32"] = {"value": ev_pt / (float(np.median(ms)) * 1e-3), "unit": UNIT,
                                  "call_ms_p50": float(np.median(ms))}
    ms = _event_times(torch, stream, flush, lambda: api.osc_histogram_bin_centre(
        c, [sid], 0, pts.shape[0], "fp32", 0.0, 10.25, 410, LO, HI, NBINS, out=out), k, 2)
    res["bin_centre_fp32"] = {"value": ev_pt / (float(np.median(ms)) * 1e-3), "unit": UNIT,
                              "call_ms_p50": float(np.median(ms))}
    api.osc_unload_sample(c, sid)
    return res


def scaling_leg(api, synth, c, sample, point):
    """The paper's timing experiment (Sec. 2.2) redone on this GPU: probabilities
    for N events with the results copied back to the host (osc_reweight into a
    host array: wall time of the call, FP64 as in the paper and FP32-bulk), against
    the oracle on one host core and on all of them, for N = 1e2 ... 1e7."""
    import oracle
    api.osc_set_params(c, point)
    cores = oracle.num_threads()
    rows = []
    for n in (100, 1_000, 10_000, 100_000, 1_000_000, 10_000_000):
        sub = {k: (v[:n] if isinstance(v, np.ndarray) else v) for k, v in sample.items()}
        sub["n"] = n
        sid = api.osc_load_sample(c, sub)
        prob = np.zeros(n)
        row = {"n": n}
        for prec in ("fp64", "fp32"):
            api.osc_reweight(c, sid, 0, prec, out_prob=prob)  # warm
            reps = max(3, min(200, 2_000_000 // n))
            t0 = time.perf_counter()
            for _ in range(reps):
                api.osc_reweight(c, sid, 0, prec, out_prob=prob)
            row["gpu_%s_per_s" % prec] = n * reps / (time.perf_counter() - t0)
        api.osc_unload_sample(c, sid)
        pt = oracle.point_from_row(point[0])
        m = min(n, 100_000)  # the oracle's rate from at most 1e5 events
        part = dict(sub, n=m)
        for threads, key in ((1, "cpu_1_core_per_s"), (cores, "cpu_all_cores_per_s")):
            oracle.set_num_threads(threads)
            t0 = time.perf_counter()
            oracle.reweight(part, pt)
            row[key] = m / (time.perf_counter() - t0)
        oracle.set_num_threads(cores)
        row["gpu_fp64_over_cpu_1_core"] = row["gpu_fp64_per_s"] / row["cpu_1_core_per_s"]
        rows.append(row)
    return {"what": "per-event probabilities copied back to the host (osc_reweight), wall time per call",
            "cores": cores, "rows": rows}


def layers_leg(torch, api, synth, c, stream, flush, k=20):
    """Layered matter: a 2M-event 1300 km beam-shaped sample through three layers
    (400 km at 2.6, 500 km at 3.3, 400 km at 2.6 g/cm^3), one point, histogram
    per step, against the same sample at constant density."""
    s = synth.uneven_samples(sizes=(1, 1, 2_000_000))[2]
    sid = api.osc_load_sample(c, s)
    out = torch.zeros((1, 1, NBINS), dtype=torch.float64, device=flush.device)
    api.osc_set_params(c, synth.table1_point()[None, :])
    res = {"events": s["n"], "layers": [[400.0, 2.6, 0.5], [500.0, 3.3, 0.5], [400.0, 2.6, 0.5]]}
    for tag in ("constant_density", "three_layers"):
        if tag == "three_layers":
            api.osc_set_layers(c, sid, res["layers"])
        for prec in ("fp32", "fp64"):
            ms = _event_times(torch, stream, flush, lambda: api.osc_histogram(
                c, [sid], 0, 1, prec, 0.0, 20.0, NBINS, out=out), k, 3)
            t = float(np.median(ms))
            res.setdefault(tag, {})[prec] = {"value": s["n"] / (t * 1e-3), "unit": UNIT, "call_ms_p50": t}
    api.osc_unload_sample(c, sid)
    return res


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    from paper_1311_7579_gb300 import synth
    s = synth.precision_sample(N_EVENTS, seed=1)
    pt = oracle.point_from_row(synth.table1_point())
    # bounded per-step sample so that W + K steps finish in a few minutes
    per_step = int(max(1024, min(N_EVENTS, 4_000_000 // max(1, args.steps + args.warmup))))
    sub = {k: (v[:per_step] if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    sub["n"] = per_step
    for _ in range(args.warmup):
        oracle.histogram(sub, [synth.table1_point()], LO, HI, NBINS)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.histogram(sub, [synth.table1_point()], LO, HI, NBINS)
    dt = time.perf_counter() - t0
    value = per_step * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "precision study: 10M events x 1 point (Table 1), per-step bounded sample of "
                                   "%d events" % per_step, "events": N_EVENTS, "points": 1, "nbins": NBINS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d events per step of the 10M-event sample" % per_step},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1311_7579_gb300 import api, synth

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # a dedicated (non-legacy-default) stream shared by torch and the library, so
    # that torch's CUDA events and flush writes order with the library's kernels
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = api.Context(local, cuda_stream=stream.cuda_stream)
    c = ctx.ptr

    sample = synth.precision_sample(N_EVENTS, seed=1 + 1000 * rank)
    sid = api.osc_load_sample(c, sample)
    point = synth.table1_point()[None, :]
    out = torch.zeros((1, 1, NBINS), dtype=torch.float64, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step(prec):
        # one fit step: the point by value and its histogram in one call, replayed as
        # one CUDA graph (constants -> histogram -> FP64 recomputation pass, joined by
        # programmatic edges); with per-kernel timing on, the library makes the two
        # calls it stands for instead (their kernels bracketed by events)
        api.osc_histogram_point(c, [sid], point[0], prec, LO, HI, NBINS, out=out)

    def timed(prec, k, w, kernel_timing):
        """k steps after w warm-up steps; per-step device times [ms].  With
        kernel_timing the library also brackets each of its kernels with CUDA
        events (its graphs then carry event nodes, which rules out the
        programmatic launch of the histogram kernel after the constants kernel)."""
        for _ in range(w):
            step(prec)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        api.osc_timing_totals(c)  # reset
        api.osc_enable_timing(c, kernel_timing)
        n0 = api.osc_launch_count(c)
        for i in range(k):
            flush.zero_()
            ev[i][0].record(stream)
            step(prec)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        n1 = api.osc_launch_count(c)
        counts, sums = api.osc_timing_totals(c)
        api.osc_enable_timing(c, False)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ms = np.array([a.elapsed_time(b) for a, b in ev])
        return ms, counts, sums, n1 - n0

    # the FP32 FMA peak of this device, measured (the roofline's denominator)
    fp32_peak_meas = api.osc_measure_fp32_peak(local)
    with ClockSampler(local) as clk:
        time.sleep(1.0)  # let nvidia-smi start sampling before the timed region
        t_clk0 = time.perf_counter()
        ms32, _, _, launches = timed("fp32", args.steps, args.warmup, False)
        t_clk1 = time.perf_counter()
        # the same K steps again with per-kernel events: kernel durations for the roofline
        ms32k, counts, sums, _ = timed("fp32", args.steps, 3, True)
    clk.window(t_clk0, t_clk1)
    clocks = clk.summary()
    k64 = max(3, min(args.steps, 40))
    ms64, c64, s64, _ = timed("fp64", k64, max(3, min(args.warmup, 5)), True)
    # the FP64-eigen-solve variant (FP64 eigenvalues and phases, FP32 amplitude) on the same workload
    kmx = max(3, min(args.steps, 200))
    msmx, cmx, smx, _ = timed("fp32_f64eig", kmx, max(3, min(args.warmup, 5)), True)

    tot32 = float(ms32.sum())
    tot64 = float(ms64.sum())
    totmx = float(msmx.sum())
    if ws > 1:
        t = torch.tensor([tot32, tot64, totmx], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot32, tot64, totmx = float(t[0]), float(t[1]), float(t[2])
    value = ws * N_EVENTS * args.steps / (tot32 * 1e-3)
    fp64_value = ws * N_EVENTS * k64 / (tot64 * 1e-3)
    f64eig_value = ws * N_EVENTS * kmx / (totmx * 1e-3)
    k_hist_ms = sums[1] / max(1, counts[1])

    # end-to-end through the public API with host buffers: each step sends the
    # point from pinned host memory and receives the histogram in pinned host
    # memory (osc_histogram_point, arguments marshalled once as a fit does)
    pin_pt = torch.from_numpy(point.copy()).pin_memory()
    host_out = torch.zeros((1, 1, NBINS), dtype=torch.float64).pin_memory()
    pin_np = pin_pt.numpy()
    out_np = host_out.numpy()
    fit_call = api.PointHistogram(c, [sid], "fp32", LO, HI, NBINS, out=out_np)
    for _ in range(3):
        fit_call(pin_np)
    lat = []
    k_e2e = args.steps
    for i in range(k_e2e):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fit_call(pin_np)
        lat.append(time.perf_counter() - t0)
    lat = np.array(lat)
    e2e_tot = float(lat.sum())
    if ws > 1:
        t = torch.tensor([e2e_tot], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_tot = float(t[0])
    e2e_value = ws * N_EVENTS * k_e2e / e2e_tot

    result = None
    if rank == 0:
        peaks, src = _measured_peaks()
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        fp32_peak_nominal = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12  # TFLOP/s, FMA = 2
        fp32_peak = fp32_peak_meas
        achieved = ALG_OPS_PER_EVPT * N_EVENTS / (k_hist_ms * 1e-3) / 1e12
        achieved_recount = FP32_FLOP_PER_EVPT * N_EVENTS / (k_hist_ms * 1e-3) / 1e12
        traffic = _profiled_traffic()
        # issue view: the kernel's warp instructions per launch (ncu) over its live duration,
        # against 4 schedulers x 1 warp instruction per clock per SM
        winst = _profile_field("warp_instructions_per_launch")
        issue_peak = n_sm * 4 * sm_mhz * 1e6 / 1e12  # T warp-instructions/s
        issue = None
        if winst:
            ia = winst / (k_hist_ms * 1e-3) / 1e12
            issue = {"achieved": ia, "peak": issue_peak, "unit": "T warp-instructions/s", "frac": ia / issue_peak,
                     "warp_instructions_per_launch": winst,
                     "thread_instructions_per_evpt": 32.0 * winst / N_EVENTS}
        # per-pipe view: instructions executed by each pipe, % of that pipe's peak over the
        # kernel's active cycles (ncu, the committed summary of this kernel)
        pipes = {k: _profile_field("pipe_%s_pct_of_peak" % k, float) for k in ("fma", "alu", "xu", "fp64")}
        pipes = ({k: v / 100.0 for k, v in pipes.items()} if all(v is not None for v in pipes.values()) else None)
        if pipes is not None:
            pipes["binding"] = "instruction issue (no single pipe saturated)"
            pipes["source"] = "ncu sm__inst_executed_pipe_*, " + os.path.relpath(TRAFFIC_PROFILE, ROOT)
        # precision study + CPU baseline (rank 0, N = 1 semantics: its own sample)
        p32 = np.zeros(N_EVENTS)
        p64 = np.zeros(N_EVENTS)
        api.osc_reweight(c, sid, 0, "fp32", out_prob=p32)
        api.osc_reweight(c, sid, 0, "fp64", out_prob=p64)
        cpu, prec_study, h_orc = (None, None, None)
        if not args.no_cpu_baseline:
            cpu, prec_study, h_orc = cpu_baseline_leg(sample, point[0], p32, p64, args.cpu_events)
        h32 = api.osc_histogram(c, [sid], 0, 1, "fp32", LO, HI, NBINS)[0, 0]
        h64 = api.osc_histogram(c, [sid], 0, 1, "fp64", LO, HI, NBINS)[0, 0]
        if prec_study is not None:
            # bin-wise relative error of the full-sample histograms, FP32 vs FP64 GPU path
            nz = h64 != 0
            prec_study["fp32_vs_fp64_hist_max_rel"] = float(np.max(np.abs(h32[nz] - h64[nz]) / np.abs(h64[nz])))
            prec_study["per_config"] = precision_per_config(api, synth, c)
        mcmc = mcmc_leg(api, synth, c, sid, sample, args.mcmc_steps) if args.mcmc_steps > 0 else None
        binned = bin_centre_leg(torch, api, synth, c, sid, sample, point, stream, flush, peaks.get("hbm_gbs"))
        layered = layers_leg(torch, api, synth, c, stream, flush)
        scaling = scaling_leg(api, synth, c, sample, point) if not args.no_cpu_baseline else None
        configs = {"scan_2M_x_4096": scan_leg(torch, api, synth, c, stream, flush)}
        configs.update(configs_leg(torch, api, synth, c, stream, flush))
        serving = None
        if args.serve_seconds > 0:
            serving = {"fp32": serving_leg(api, synth, local, SERVE_RATES, args.serve_seconds, "fp32"),
                       "fp64": serving_leg(api, synth, local, (100,), args.serve_seconds, "fp64")}
        result = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot32 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp32", "data": "synthetic",
            "config": {"workload": "precision study: 10M events x 1 point (Table 1), FP32-bulk, step = "
                                   "osc_histogram_point (point by value + histogram, one CUDA graph)",
                       "events": N_EVENTS, "points": 1, "nbins": NBINS,
                       "baseline_km": 295.0, "density_gcc": 2.6, "ye": 0.5,
                       "l2": "flushed between steps (256 MB write, outside the timed events)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "fp64_value": fp64_value, "fp32_over_fp64": value / fp64_value,
            "fp32_f64eig_value": f64eig_value,
            "latency_us": {"p50": float(np.percentile(lat, 50) * 1e6), "p99": float(np.percentile(lat, 99) * 1e6),
                           "device_p50": float(np.percentile(ms32, 50) * 1e3),
                           "device_p99": float(np.percentile(ms32, 99) * 1e3)},
            "step_ms_with_kernel_events": float(ms32k.mean()),
            "kernel_ms": {"hist_fp32": k_hist_ms, "final": sums[2] / max(1, counts[2]),
                          "const": sums[0] / max(1, counts[0]), "hist_fp64": s64[1] / max(1, c64[1]),
                          "hist_fp32_f64eig": smx[1] / max(1, cmx[1])},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                         "frac": achieved / fp32_peak, "traffic": traffic,
                         "ops_per_evpt": ALG_OPS_PER_EVPT, "sfu_per_evpt": ALG_SFU_PER_EVPT,
                         "peak_source": "measured on this device: FP32 FMA chains on every SM, CUDA events "
                                        "(osc_measure_fp32_peak); nominal %.1f = %d SMs x 128 lanes x 2 x %.0f MHz"
                                        % (fp32_peak_nominal, n_sm, sm_mhz),
                         "peak_nominal": fp32_peak_nominal,
                         "recount": {"flop_per_evpt": FP32_FLOP_PER_EVPT, "sfu_per_evpt": SFU_PER_EVPT,
                                     "achieved": achieved_recount, "frac": achieved_recount / fp32_peak},
                         "algorithmic_bytes_per_launch": ALG_BYTES_PER_EVENT * N_EVENTS,
                         "traffic_over_algorithmic": (traffic / (ALG_BYTES_PER_EVENT * N_EVENTS)) if traffic else None,
                         "hbm_gbs_event_stream": 16.0 * N_EVENTS / (k_hist_ms * 1e-3) / 1e9,
                         "hbm_peak_gbs": peaks.get("hbm_gbs"),
                         "issue": issue, "pipes": pipes},
            "cpu_baseline": cpu,
            "precision": prec_study,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 64, "d2h_bytes_per_step": 8 * NBINS},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "serving": serving,
            "mcmc": mcmc,
            "bin_centre": binned,
            "layers": layered,
            "configs": configs,
            "scaling_vs_n": scaling,
        }
        print(json.dumps(result), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """Small fixed case for ncu captures: --events events of the beam-shaped
    sample x --points scan points, --launches histogram launches with the given
    points-per-block tile (0 = autotuned) and precision.  --method picks the
    event-by-event histogram (ebe), the fit step of the first point
    (osc_histogram_point: the bench's step), the bin-centre method (bc, 410 true
    bins of 25 MeV) or event-by-event through three layers (layers)."""
    import torch

    from paper_1311_7579_gb300 import api, synth
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = api.Context(0, cuda_stream=stream.cuda_stream)
    c = ctx.ptr
    s = synth.precision_sample(args.events, seed=1)
    sid = api.osc_load_sample(c, s)
    pts = synth.table1_point()[None, :] if args.points == 1 else synth.scan_points(args.points)
    api.osc_set_params(c, pts)
    api.osc_set_tile(c, args.tile, 0)
    if args.method == "layers":
        api.osc_set_layers(c, sid, [(100.0, 2.2, 0.5), (95.0, 3.0, 0.5), (100.0, 2.2, 0.5)])
    out = torch.zeros((1, args.points, NBINS), dtype=torch.float64, device="cuda")
    for _ in range(args.launches):
        if args.method == "step":
            # the fit step: one point by value, its constants computed on the host
            api.osc_histogram_point(c, [sid], pts[0], args.prec, LO, HI, NBINS, out=out)
        elif args.method == "bc":
            api.osc_histogram_bin_centre(c, [sid], 0, args.points, args.prec, 0.0, 10.25, 410, LO, HI, NBINS, out=out)
        else:
            api.osc_histogram(c, [sid], 0, args.points, args.prec, LO, HI, NBINS, out=out)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": {"method": args.method, "events": args.events, "points": args.points,
                                       "prec": args.prec, "tile": args.tile, "launches": args.launches,
                                       "checksum": float(out.sum())}}))
    ctx.close()
    return 0


def run_serving_only(args):
    """The serving workload alone on device 0: FP32-bulk at every offered rate and
    FP64 at 100 req/s, --serve-seconds per rate, under the 8 GB workspace cap."""
    from paper_1311_7579_gb300 import api, synth
    res = {"serving": {"fp32": serving_leg(api, synth, 0, SERVE_RATES, args.serve_seconds, "fp32"),
                       "fp64": serving_leg(api, synth, 0, (100,), args.serve_seconds, "fp64")}}
    print(json.dumps(res), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-events", type=int, default=N_EVENTS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mcmc-steps", type=int, default=2000, help="toy-fit steps (0 skips)")
    ap.add_argument("--serve-seconds", type=float, default=2.0,
                    help="seconds per offered rate of the serving leg (0 skips it)")
    ap.add_argument("--profile", action="store_true", help="run the small ncu profiling case and exit")
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving workload (--serve-seconds per rate) and print its JSON")
    ap.add_argument("--events", type=int, default=2_000_000)
    ap.add_argument("--points", type=int, default=1)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--launches", type=int, default=2)
    ap.add_argument("--method", default="ebe", choices=["ebe", "step", "bc", "layers"])
    args = ap.parse_args()
    if args.profile:
        return run_profile_case(args)
    if args.serving_only:
        return run_serving_only(args)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
