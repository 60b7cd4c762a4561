"""Identities the CUDA path's per-point constants rest on, checked on the CPU
with plain numpy linear algebra (no oracle code, no kernel code).

The constants kernel builds the eigenvalue cubic of M = H0 + A Pe (Sec. 1.1:
H0 = U diag(0, dm21, dm31) U^dagger, Pe the electron projector) from four
numbers: T0 = tr H0, c1(0) = dm21 dm31, smt = H0_mumu + H0_tautau and the ee
cofactor mee = H0_mumu H0_tautau - |H0_mutau|^2, the last two in closed form
from the s^2 inputs:
    smt = T0 - (dm21 |U_e2|^2 + dm31 |U_e3|^2),   mee = dm21 dm31 |U_e1|^2.
The characteristic polynomial of M is then
    lambda^3 - (T0 + A) lambda^2 + (c1(0) + A smt) lambda - A mee.
These tests check both closed forms against the matrix entries and the cubic
against numpy's Hermitian eigenvalues, for neutrinos and antineutrinos
(U -> U*, A -> -A), both mass orderings and the degenerate corners.
"""
import numpy as np
import pytest


def pdg_u(s2_12, s2_13, s2_23, dcp):
    """U in the PDG parametrisation, written out entry by entry."""
    s12, s13, s23 = np.sqrt([s2_12, s2_13, s2_23])
    c12, c13, c23 = np.sqrt([1 - s2_12, 1 - s2_13, 1 - s2_23])
    e = np.exp(1j * dcp)
    return np.array([
        [c12 * c13, s12 * c13, s13 / e],
        [-s12 * c23 - c12 * s23 * s13 * e, c12 * c23 - s12 * s23 * s13 * e, s23 * c13],
        [s12 * s23 - c12 * c23 * s13 * e, -c12 * s23 - s12 * c23 * s13 * e, c23 * c13],
    ])


def points(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        s2 = rng.uniform(1e-4, 1 - 1e-4, 3)
        dm21 = rng.uniform(1e-5, 2e-4)
        dm32 = rng.choice([-1.0, 1.0]) * rng.uniform(1.5e-3, 3.5e-3)
        out.append((s2[0], s2[1], s2[2], dm21, dm32, rng.uniform(-2 * np.pi, 2 * np.pi)))
    # corners: maximal and tiny mixing, delta at 0 and pi, inverted ordering
    out += [(0.5, 0.5, 0.5, 7.5e-5, 2.5e-3, 0.0), (1e-6, 1e-6, 1e-6, 7.5e-5, -2.5e-3, np.pi),
            (0.307, 0.0218, 0.545, 7.53e-5, -2.453e-3, 1.36 * np.pi)]
    return out


@pytest.mark.parametrize("nubar", [False, True])
def test_closed_form_invariants_match_the_matrix(nubar):
    for s2_12, s2_13, s2_23, dm21, dm32, dcp in points(40, seed=7):
        dm31 = dm32 + dm21
        U = pdg_u(s2_12, s2_13, s2_23, dcp)
        if nubar:
            U = U.conj()
        H = U @ np.diag([0.0, dm21, dm31]) @ U.conj().T
        T0 = dm21 + dm31
        smt_matrix = (H[1, 1] + H[2, 2]).real
        mee_matrix = (H[1, 1] * H[2, 2] - abs(H[1, 2]) ** 2).real
        smt = T0 - (dm21 * s2_12 * (1 - s2_13) + dm31 * s2_13)
        mee = dm21 * dm31 * (1 - s2_12) * (1 - s2_13)
        scale = abs(dm31) + dm21
        assert abs(smt - smt_matrix) <= 1e-14 * scale
        assert abs(mee - mee_matrix) <= 1e-14 * scale ** 2
        assert abs(np.trace(H).real - T0) <= 1e-15 * scale


@pytest.mark.parametrize("nubar", [False, True])
def test_cubic_from_invariants_has_the_eigenvalues_in_matter(nubar):
    for s2_12, s2_13, s2_23, dm21, dm32, dcp in points(25, seed=11):
        dm31 = dm32 + dm21
        U = pdg_u(s2_12, s2_13, s2_23, dcp)
        if nubar:
            U = U.conj()
        H = U @ np.diag([0.0, dm21, dm31]) @ U.conj().T
        T0, c10 = dm21 + dm31, dm21 * dm31
        smt = T0 - (dm21 * s2_12 * (1 - s2_13) + dm31 * s2_13)
        mee = c10 * (1 - s2_12) * (1 - s2_13)
        for A in (1e-6, 3e-5, 2e-4, 1e-3, 5e-3, 2e-2):
            a = -A if nubar else A
            M = H + np.diag([a, 0.0, 0.0])
            lam = np.linalg.eigvalsh(M)
            # characteristic polynomial at each eigenvalue: zero up to the rounding of
            # its terms and the eigenvalue's own error (about eps |M| times p'(x))
            c2, c1, c0 = T0 + a, c10 + a * smt, a * mee
            norm = np.abs(lam).max()
            for x in lam:
                terms = abs(x) ** 3 + abs(c2) * x * x + abs(c1 * x) + abs(c0)
                dp = abs(3 * x * x - 2 * c2 * x + c1)
                assert abs(x ** 3 - c2 * x * x + c1 * x - c0) <= 64 * 2.2e-16 * (terms + dp * norm)
            # and the three roots of the cubic are the eigenvalues
            roots = np.sort(np.roots([1.0, -c2, c1, -c0]).real)
            assert np.allclose(roots, lam, rtol=0, atol=1e-12 * (abs(dm31) + abs(a)))


def test_deflation_of_a_depressed_cubic_gives_the_pair_and_its_gap():
    """The FP64 solver's seed for a near-double pair: if mu_i is one root of
    mu^3 + p mu + q (the roots sum to zero), the other two are the roots of
    mu^2 + mu_i mu + (p + mu_i^2), and its discriminant -3 mu_i^2 - 4 p is the
    squared difference of the pair -- for well separated and near-double pairs,
    with the isolated root at the top (cos theta near +1) or at the bottom."""
    rng = np.random.default_rng(99)
    for _ in range(200):
        scale = np.exp(rng.uniform(np.log(1e-6), np.log(1e-1)))
        gap = scale * np.exp(rng.uniform(np.log(1e-6), 0.0))
        centre = rng.choice([-1.0, 1.0]) * scale
        a, b = centre - gap / 2, centre + gap / 2
        mi = -(a + b)                    # the isolated root (depressed: roots sum to zero)
        p = a * b + mi * (a + b)         # mu^3 + p mu + q = (mu - a)(mu - b)(mu - mi)
        q = -a * b * mi
        assert abs(mi ** 3 + p * mi + q) <= 1e-12 * abs(mi) ** 3
        disc = -3 * mi * mi - 4 * p
        assert abs(disc - gap * gap) <= 1e-12 * mi * mi
        lo = (-mi - np.sqrt(max(disc, 0.0))) / 2
        hi = (-mi + np.sqrt(max(disc, 0.0))) / 2
        # the pair's roots to the discriminant's rounding: eps mi^2 / gap
        tol = 1e-15 * abs(mi) + 8e-16 * mi * mi / gap
        assert abs(lo - a) <= tol and abs(hi - b) <= tol, (scale, gap)
