"""Arbitrary-precision constant-density oscillation probability.

TEST INFRASTRUCTURE ONLY: used by ``tests/golden/make_fp64_hard_events.py`` to
write a fixture; neither the product package nor the FP64 oracle uses it.

It evaluates the definition the FP64 oracle implements (Sec. 1.1: Eq. (1)'s
PDG mixing matrix U with U_e3 = s13 e^{-i delta}; M = U diag(0, dm21, dm31)
U^dagger + diag(A, 0, 0) with the matter term A = k_A Y_e rho E;
S = exp(-i c_L M L / E); P(alpha -> beta) = |S_{beta alpha}|^2; antineutrinos
U -> U*, A -> -A) with mpmath at 40 significant digits, by the matrix
exponential of M itself -- no characteristic cubic and no eigendecomposition, so
it shares no algorithm with either FP64 implementation.  The inputs are the
double-precision values both implementations start from: the oracle's constants
c_L and k_A, the double product c_L L (each implementation forms it in double
before dividing by E), and E_true as stored (FP32).
"""
from __future__ import annotations

import mpmath as mp

import oracle

DIGITS = 40


def prob_exact(point, L_km: float, rho: float, ye: float, E: float, alpha: int, beta: int, nubar: int) -> float:
    """P(alpha -> beta) for a point row (s2_12, s2_13, s2_23, dm21, dm32, dcp, ...)."""
    with mp.workdps(DIGITS):
        s12, s13, s23 = (mp.sqrt(mp.mpf(x)) for x in point[:3])
        c12, c13, c23 = (mp.sqrt(1 - mp.mpf(x)) for x in point[:3])
        dm21, dm32, d = mp.mpf(point[3]), mp.mpf(point[4]), mp.mpf(point[5])
        dm31 = dm32 + dm21
        ed = mp.expj(d)
        U = mp.matrix([[c12 * c13, s12 * c13, s13 / ed],
                       [-s12 * c23 - c12 * s23 * s13 * ed, c12 * c23 - s12 * s23 * s13 * ed, s23 * c13],
                       [s12 * s23 - c12 * c23 * s13 * ed, -c12 * s23 - s12 * c23 * s13 * ed, c23 * c13]])
        if nubar:
            U = U.conjugate()
        A = mp.mpf(oracle.k_A()) * mp.mpf(ye) * mp.mpf(rho) * mp.mpf(E)
        if nubar:
            A = -A
        M = U * mp.diag([0, dm21, dm31]) * U.transpose_conj()
        M[0, 0] += A
        cLL = mp.mpf(oracle.c_L() * L_km)  # the double product, as both implementations form it
        S = mp.expm(-1j * (cLL / mp.mpf(E)) * M)
        return float(abs(S[beta, alpha]) ** 2)
