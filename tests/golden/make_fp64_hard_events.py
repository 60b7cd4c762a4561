"""Writes fp64_hard_events.json: exact (40-digit) probabilities at events where
FP64 is hardest pressed -- a 12000 km path at 13 g/cm^3 and low energies, where
c_L L / E reaches 6e5 eV^-2 and the phases ~1e3 rad -- and at 1300 km, for the
Table 1 point in both orderings and the edge points of the parameter domain.

Calls only the oracle package (its arbitrary-precision module).  Run from the
repository root:  python tests/golden/make_fp64_hard_events.py
"""
import json
import os
import sys

import numpy as np

sys.path.insert(0, os.getcwd())
from oracle import hp  # noqa: E402

#           s2_12   s2_13   s2_23  dm21     dm32     dcp   escale norm
POINTS = [
    [0.311, 0.0251, 0.5, 7.6e-5, 2.4e-3, 0.0, 1.0, 1.0],     # Table 1, normal ordering
    [0.311, 0.0251, 0.5, 7.6e-5, -2.4e-3, -1.5, 1.0, 1.0],   # Table 1 mixing, inverted ordering
    [0.311, 1.0e-4, 0.5, 7.6e-5, 2.4e-3, 1.0, 1.0, 1.0],     # tiny theta13
    [0.5, 0.5, 0.5, 7.6e-5, 2.4e-3, -2.0, 1.0, 1.0],         # maximal mixing
    [0.311, 0.0251, 0.5, 1.0e-3, 1.1e-3, 0.5, 1.0, 1.0],     # |dm32| just above dm21
    [0.1, 0.0251, 0.9, 7.6e-5, 2.4e-3, -0.3, 1.0, 1.0],      # small theta12, large theta23
    [0.01, 0.0251, 0.99, 7.6e-5, -2.4e-3, 3.1, 1.0, 1.0],    # extreme mixing, inverted
]
CASES = [(12000.0, 13.0, 0.5), (1300.0, 2.85, 0.5)]
PER_CHANNEL = 2  # energies per (alpha, beta, nubar) and point


def main():
    rng = np.random.default_rng(20131129)
    cases = []
    for L, rho, ye in CASES:
        ev = []
        for k, pt in enumerate(POINTS):
            for nubar in (0, 1):
                for a in range(3):
                    for b in range(3):
                        for _ in range(PER_CHANNEL):
                            # log-uniform in [0.05, 1] GeV, stored as FP32 like event energies
                            E = float(np.float32(0.05 * 20.0 ** rng.uniform()))
                            ev.append([k, a, b, nubar, E, hp.prob_exact(pt, L, rho, ye, E, a, b, nubar)])
        cases.append({"L_km": L, "density_gcc": rho, "ye": ye,
                      "events": ev})
    out = {"source": "Sec. 1.1: constant-density three-flavour probability, evaluated at 40 digits by "
                     "the matrix exponential (oracle/hp.py)",
           "columns": ["point", "alpha", "beta", "nubar", "e_true", "p_exact"],
           "points": POINTS, "cases": cases}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "fp64_hard_events.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print(path, sum(len(c["events"]) for c in cases), "events")


if __name__ == "__main__":
    main()
