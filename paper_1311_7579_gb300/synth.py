"""Seeded synthetic inputs shaped like the paper's long-baseline workload.

This module only draws random numbers: it holds none of the oscillation
arithmetic, and both the CUDA path and the CPU oracle take its arrays as
inputs.  The paper's own inputs (T2K Monte Carlo, a Landau-sampled toy,
Sec. 2.2 and the acknowledgements) are not available, so Gamma-shaped true
energy spectra with peaks scaled to the baseline stand in for them.

Every array is generated with ``numpy.random.default_rng(seed)`` (PCG64) in a
fixed draw order per sample -- E_true, E_reco smearing, channel, nu/nubar,
MC weight -- and stored as float32 / uint8 so that both sides read the same
exactly representable values.

Workloads (sizes and distributions):
  * ``table1_sample``     100k events, seed 0, 295 km, 2.6 g/cm^3 (Table 1 point)
  * ``precision_sample``  10M events, seed 1, same distributions
  * ``scan_sample``       2M events, seed 2; ``scan_points`` 4096 points, seed 2002
  * ``uneven_samples``    8 samples of 1e4 .. 2e7 events, seeds 1000+j, three
                          baselines/densities; 512 points, seed 3003
  * ``validation_energies`` uniform E in [0.05, 30] GeV (Sec. 2.2 validation)
"""
from __future__ import annotations

import numpy as np

# Table 1 of the paper (normal hierarchy; the table's "dm^2_12" is read as dm21).
TABLE1 = dict(s2_12=0.311, s2_13=0.0251, s2_23=0.5, dm21=7.6e-5, dm32=2.4e-3, dcp=0.0,
              escale=1.0, norm=1.0)
TABLE1_L_KM = 295.0
TABLE1_RHO = 2.6
YE = 0.5
POINT_FIELDS = ("s2_12", "s2_13", "s2_23", "dm21", "dm32", "dcp", "escale", "norm")

# Flavour codes.
NU_E, NU_MU, NU_TAU = 0, 1, 2

BASELINES = ((295.0, 2.6), (810.0, 2.8), (1300.0, 2.85))
UNEVEN_SIZES = (10_000, 100_000, 500_000, 2_000_000, 5_000_000, 8_000_000, 12_000_000, 20_000_000)


def table1_point() -> np.ndarray:
    return np.array([TABLE1[k] for k in POINT_FIELDS], dtype=np.float64)


def _gamma_energies(rng, n, scale, lo, hi):
    e = rng.gamma(3.0, scale, size=n)
    return np.clip(e, lo, hi).astype(np.float32)


def beam_sample(n: int, seed: int, L_km=TABLE1_L_KM, rho=TABLE1_RHO, ye=YE,
                channels=((NU_MU, NU_MU, 0.9), (NU_MU, NU_E, 0.1)), nubar_frac=0.2,
                scale_L=False) -> dict:
    """A nu_mu-beam-like sample: E_true ~ Gamma(3, 0.25 GeV * s), clipped to
    [0.05, 10 s] GeV with s = L/295 when ``scale_L`` (else s = 1);
    E_reco = E_true (1 + N(0, 0.1)); channels drawn with the given fractions;
    nubar with probability ``nubar_frac``; w_mc ~ U(0.5, 1.5)."""
    rng = np.random.default_rng(seed)
    s = (L_km / 295.0) if scale_L else 1.0
    e_true = _gamma_energies(rng, n, 0.25 * s, 0.05, 10.0 * s)
    smear = rng.normal(0.0, 0.1, size=n)
    e_reco = (e_true.astype(np.float64) * (1.0 + smear)).astype(np.float32)
    probs = np.array([c[2] for c in channels], dtype=np.float64)
    ch = rng.choice(len(channels), size=n, p=probs / probs.sum())
    flav_in = np.array([c[0] for c in channels], dtype=np.uint8)[ch]
    flav_out = np.array([c[1] for c in channels], dtype=np.uint8)[ch]
    is_nubar = (rng.random(n) < nubar_frac).astype(np.uint8)
    w_mc = rng.uniform(0.5, 1.5, size=n).astype(np.float32)
    return dict(n=int(n), e_true=e_true, e_reco=e_reco, w_mc=w_mc, flav_in=flav_in,
                flav_out=flav_out, is_nubar=is_nubar, baseline_km=float(L_km),
                density_gcc=float(rho), ye=float(ye))


def table1_sample(n: int = 100_000, seed: int = 0) -> dict:
    return beam_sample(n, seed)


def precision_sample(n: int = 10_000_000, seed: int = 1) -> dict:
    return beam_sample(n, seed)


def scan_sample(n: int = 2_000_000, seed: int = 2) -> dict:
    return beam_sample(n, seed)


def scan_points(n: int = 4096, seed: int = 2002) -> np.ndarray:
    """Rows of POINT_FIELDS: sin^2 t23 ~ U(0.35, 0.65), sin^2 t13 ~ U(0.018, 0.030),
    |dm32| ~ U(2.0e-3, 2.8e-3) with a random hierarchy sign, delta ~ U(-pi, pi),
    sin^2 t12 and dm21 at Table 1, energy scale 1 + N(0, 0.02), norm 1."""
    rng = np.random.default_rng(seed)
    s2_23 = rng.uniform(0.35, 0.65, n)
    s2_13 = rng.uniform(0.018, 0.030, n)
    adm = rng.uniform(2.0e-3, 2.8e-3, n)
    sign = np.where(rng.random(n) < 0.5, 1.0, -1.0)
    dcp = rng.uniform(-np.pi, np.pi, n)
    esc = 1.0 + rng.normal(0.0, 0.02, n)
    pts = np.empty((n, 8))
    pts[:, 0] = TABLE1["s2_12"]
    pts[:, 1] = s2_13
    pts[:, 2] = s2_23
    pts[:, 3] = TABLE1["dm21"]
    pts[:, 4] = sign * adm
    pts[:, 5] = dcp
    pts[:, 6] = esc
    pts[:, 7] = 1.0
    return pts


def uneven_samples(sizes=UNEVEN_SIZES, seed0: int = 1000) -> list:
    """Sample j: baseline/density BASELINES[j % 3], Gamma peak scaled by L/295,
    channels mu->mu 80 %, mu->e 10 %, e->e 10 %, nubar 30 %."""
    out = []
    for j, n in enumerate(sizes):
        L, rho = BASELINES[j % 3]
        out.append(beam_sample(n, seed0 + j, L_km=L, rho=rho,
                               channels=((NU_MU, NU_MU, 0.8), (NU_MU, NU_E, 0.1), (NU_E, NU_E, 0.1)),
                               nubar_frac=0.3, scale_L=True))
    return out


def uneven_points(n: int = 512, seed: int = 3003) -> np.ndarray:
    return scan_points(n, seed)


def all_channel_sample(n: int, seed: int, L_km=1300.0, rho=2.85, ye=YE, e_lo=0.05, e_hi=30.0) -> dict:
    """Every (alpha, beta, nu/nubar) channel uniformly, E_true ~ U(e_lo, e_hi):
    the shape used for unitarity-style and corner-case parity."""
    rng = np.random.default_rng(seed)
    e_true = rng.uniform(e_lo, e_hi, n).astype(np.float32)
    e_true = np.maximum(e_true, np.float32(e_lo))
    smear = rng.normal(0.0, 0.1, size=n)
    e_reco = (e_true.astype(np.float64) * (1.0 + smear)).astype(np.float32)
    flav_in = rng.integers(0, 3, n).astype(np.uint8)
    flav_out = rng.integers(0, 3, n).astype(np.uint8)
    is_nubar = rng.integers(0, 2, n).astype(np.uint8)
    w_mc = rng.uniform(0.5, 1.5, size=n).astype(np.float32)
    return dict(n=int(n), e_true=e_true, e_reco=e_reco, w_mc=w_mc, flav_in=flav_in,
                flav_out=flav_out, is_nubar=is_nubar, baseline_km=float(L_km),
                density_gcc=float(rho), ye=float(ye))


def validation_energies(n: int = 10_000_000, seed: int = 7, lo: float = 0.05, hi: float = 30.0):
    """Sec. 2.2 validation shape: E ~ U(0, 30) GeV, restricted to E >= 0.05 GeV."""
    rng = np.random.default_rng(seed)
    return np.maximum(rng.uniform(lo, hi, n).astype(np.float32), np.float32(lo))


def serving_requests(duration_s: float, rate_hz: float, n_samples: int = 8, seed: int = 4004):
    """Poisson arrivals: (arrival time [s], sample id, point row)."""
    rng = np.random.default_rng(seed)
    n = rng.poisson(rate_hz * duration_s)
    t = np.sort(rng.uniform(0.0, duration_s, n))
    sid = rng.integers(0, n_samples, n)
    pts = scan_points(n, seed + 1) if n else np.zeros((0, 8))
    return t, sid, pts
