"""Writes fp64_near_double_events.json: exact (40-digit) probabilities where the
matter term dwarfs the vacuum splittings, so that two eigenvalues in matter lie
within 1e-4 to 1e-3 of the cubic's scale of each other (a near-double root of the
eigenvalue cubic), together with the Table 1 point and a small |dm32| at the same
high matter terms (A up to 0.05 eV^2).

Calls only the oracle package (its arbitrary-precision module).  Run from the
repository root:  python tests/golden/make_fp64_near_double_events.py
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.getcwd())
from oracle import hp  # noqa: E402

#           s2_12   s2_13   s2_23   dm21      dm32       dcp     escale norm
POINTS = [
    [0.3547, 0.251, 0.4942, 1.769e-6, 4.052e-6, -6.171, 1.0, 1.0],   # splittings ~1e-6 eV^2
    [0.9256, 0.3414, 0.9529, 1.213e-6, 1.269e-5, 2.923, 1.0, 1.0],   # large mixing angles
    [0.7563, 0.2795, 0.6739, 2.55e-6, -1.864e-5, 5.741, 1.0, 1.0],   # inverted ordering
    [0.311, 0.0251, 0.5, 1.0e-6, 5.0e-6, 0.7, 1.0, 1.0],             # Table 1 mixing, tiny splittings
    [0.311, 0.0251, 0.5, 2.0e-6, -8.0e-6, -2.0, 1.0, 1.0],           # the same, inverted
    [0.311, 0.0251, 0.5, 7.6e-5, 2.4e-3, 0.0, 1.0, 1.0],             # Table 1 point
    [0.311, 0.0251, 0.5, 7.6e-5, 2.0e-4, 1.0, 1.0, 1.0],             # small |dm32|
]
CASES = [(12000.0, 13.0, 0.5), (6000.0, 5.0, 0.5)]
PER_CHANNEL = 1  # energies per (alpha, beta, nubar) and point


def main():
    rng = np.random.default_rng(20261204)
    cases = []
    for L, rho, ye in CASES:
        ev = []
        for k, pt in enumerate(POINTS):
            for nubar in (0, 1):
                for a in range(3):
                    for b in range(3):
                        for _ in range(PER_CHANNEL):
                            # log-uniform in [2, 50] GeV, stored as FP32 like event energies
                            E = float(np.float32(2.0 * 25.0 ** rng.uniform()))
                            ev.append([k, a, b, nubar, E, hp.prob_exact(pt, L, rho, ye, E, a, b, nubar)])
        cases.append({"L_km": L, "density_gcc": rho, "ye": ye, "events": ev})
    out = {"source": "Sec. 1.1: constant-density three-flavour probability, evaluated at 40 digits by "
                     "the matrix exponential (oracle/hp.py)",
           "columns": ["point", "alpha", "beta", "nubar", "e_true", "p_exact"],
           "points": POINTS, "cases": cases}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fp64_near_double_events.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(path, sum(len(c["events"]) for c in cases), "events")


if __name__ == "__main__":
    main()
