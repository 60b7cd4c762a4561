"""Pins of the oracle's binned (bin-centre) reweighting and of its layered-matter
propagation (CPU only).  Each check is computed here by a route independent of
the oracle function it pins:

Bin-centre method (Sec. 1.1.1, the 25 MeV bin example):
* the true-energy bin and the FP32 centre energy, restated with numpy float32
  arithmetic, and the probability taken there;
* events placed exactly at their bin centres: the binned method equals the
  event-by-event method bit for bit;
* events outside the true-energy range weigh 0;
* the 25 MeV bin at 0.6 GeV: with quadrature nodes as events, the event-by-event
  sum reproduces an adaptive quadrature of spectrum x probability and the
  binned sum reproduces P(centre) x the quadrature of the spectrum.

Layered matter (generalising the constant density of Sec. 1.1):
* one layer equals the constant-density oracle; a layer cut into pieces of
  equal density changes nothing; all-vacuum layers reproduce Eq. (1) at the
  summed length;
* RK4 integration of the Schroedinger equation through an asymmetric
  three-layer profile, layer by layer in the order of travel;
* unitarity; T symmetry with the profile reversed at delta = 0, and its
  breaking at delta != 0 for an asymmetric profile.
"""
import numpy as np
import pytest

import oracle
from paper_1311_7579_gb300 import synth

C_L = 2.5338653588396975  # restated: 1e-6 / (2 * 1.973269804e-7)
K_A = 2 * np.sqrt(2) * 1.1663788e-23 * 6.02214076e23 * 1.973269804e-5 ** 3 * 1e9


def _sample(e_true, alpha=1, beta=1, nubar=0, w=None, L=295.0, rho=2.6, ye=0.5, e_reco=None):
    e_true = np.ascontiguousarray(e_true, dtype=np.float32)
    n = e_true.size
    def u8(v):
        return np.ascontiguousarray(np.broadcast_to(np.asarray(v, dtype=np.uint8), (n,)))
    return {"n": n, "e_true": e_true, "e_reco": np.ascontiguousarray(e_true if e_reco is None else e_reco,
                                                                      dtype=np.float32),
            "w_mc": np.ascontiguousarray(np.ones(n) if w is None else w, dtype=np.float32),
            "flav_in": u8(alpha), "flav_out": u8(beta), "is_nubar": u8(nubar),
            "baseline_km": L, "density_gcc": rho, "ye": ye}


def _bin_np(e, t_lo, t_hi, T):
    """FP32 bin rule restated in numpy float32 (unit scale)."""
    e = np.asarray(e, dtype=np.float32)
    t = (e - np.float32(t_lo)).astype(np.float32)
    u = (t * np.float32(T / (t_hi - t_lo))).astype(np.float32)
    keep = (t >= 0) & (u < np.float32(T))
    return np.where(keep, u.astype(np.int64), -1)


def _centre_np(t_lo, t_hi, T, t):
    return np.float32(t_lo + (t + 0.5) * ((t_hi - t_lo) / T))


# ------------------------------------------------------------- bin centres
def test_true_centre_restated():
    rng = np.random.default_rng(5)
    for _ in range(200):
        lo = float(rng.uniform(0, 1))
        hi = lo + float(rng.uniform(0.5, 20))
        T = int(rng.integers(1, 1000))
        t = int(rng.integers(0, T))
        assert oracle.true_centre(lo, hi, T, t) == float(_centre_np(lo, hi, T, t))
    assert oracle.true_centre(0.0, 10.0, 400, 24) == float(np.float32(0.6125))


@pytest.mark.parametrize("nubar,alpha,beta", [(0, 1, 1), (0, 1, 0), (1, 1, 0), (1, 0, 0)])
def test_bin_centre_probability_at_restated_centre(nubar, alpha, beta):
    rng = np.random.default_rng(11 + nubar)
    s = synth.beam_sample(3000, seed=44)
    s = _sample(s["e_true"], alpha, beta, nubar, w=s["w_mc"])
    t_lo, t_hi, T = 0.0, 10.25, 410
    pt = oracle.point_from_row(synth.scan_points(1, int(rng.integers(1 << 30)))[0])
    p, w = oracle.reweight_bin_centre(s, pt, t_lo, t_hi, T)
    t = _bin_np(s["e_true"], t_lo, t_hi, T)
    assert (t >= 0).all()
    cen = np.array([_centre_np(t_lo, t_hi, T, k) for k in t], dtype=np.float64)
    ref = oracle.prob_matrix_many(pt, 295.0, 2.6, 0.5, cen, nubar)[:, beta, alpha]
    assert np.array_equal(p, ref)
    assert np.array_equal(w, p * s["w_mc"].astype(np.float64) * pt.norm)


def test_bin_centre_equals_event_by_event_at_centres():
    t_lo, t_hi, T = 0.0, 5.0, 200
    cen = np.array([oracle.true_centre(t_lo, t_hi, T, k) for k in range(T)], dtype=np.float32)
    rng = np.random.default_rng(3)
    for nubar, alpha, beta in ((0, 1, 1), (1, 1, 0), (0, 0, 2)):
        e = rng.choice(cen, 2000)
        s = _sample(e, alpha, beta, nubar, w=rng.uniform(0.5, 1.5, e.size))
        pt = oracle.make_point(dcp=0.7, escale=1.03, norm=1.2)
        pb, wb = oracle.reweight_bin_centre(s, pt, t_lo, t_hi, T)
        pe, we = oracle.reweight(s, pt)
        assert np.array_equal(pb, pe) and np.array_equal(wb, we)


def test_bin_centre_drops_events_outside_true_range():
    t_lo, t_hi, T = 0.5, 2.5, 80
    e = np.array([0.1, 0.4999, 0.5, 0.7, 2.4999, 2.5, 2.6, 9.0], dtype=np.float32)
    s = _sample(e)
    p, w = oracle.reweight_bin_centre(s, oracle.make_point(), t_lo, t_hi, T)
    inside = (e >= np.float32(0.5)) & (e < np.float32(2.5))
    assert (p[~inside] == 0).all() and (w[~inside] == 0).all()
    assert (p[inside] > 0).all()
    h = oracle.histogram_bin_centre(s, [synth.table1_point()], t_lo, t_hi, T, 0.0, 10.0, 20)[0]
    assert np.isclose(h.sum(), w.sum(), rtol=1e-15)


def test_25mev_bin_study_against_quadrature():
    """The Sec. 1.1.1 example on a Gamma(3, 0.25 GeV) spectrum: nu_mu survival at
    295 km through 2.6 g/cm^3, one 25 MeV bin from 0.6 to 0.625 GeV."""
    integrate = pytest.importorskip("scipy.integrate")
    stats = pytest.importorskip("scipy.stats")
    pt = oracle.point_from_row(synth.table1_point())
    a, b = 0.6, 0.625
    K = 4000
    h = (b - a) / K
    nodes = a + (np.arange(K) + 0.5) * h
    nodes32 = nodes.astype(np.float32)
    phi = stats.gamma(3.0, scale=0.25).pdf
    w = phi(nodes) * h
    s = _sample(nodes32, 1, 1, 0, w=w)
    # bins of width 25 MeV with an edge at 0.6 GeV
    t_lo, t_hi, T = 0.0, 10.0, 400
    assert set(_bin_np(nodes32, t_lo, t_hi, T)) == {24}
    _, w_ebe = oracle.reweight(s, pt)
    _, w_bc = oracle.reweight_bin_centre(s, pt, t_lo, t_hi, T)

    def P(E):
        return oracle.prob(pt, 295.0, 2.6, 0.5, E, 1, 1, 0)

    I1 = integrate.quad(lambda E: phi(E) * P(E), a, b, epsabs=0, epsrel=1e-12)[0]
    I0 = integrate.quad(phi, a, b, epsabs=0, epsrel=1e-12)[0]
    Pc = P(float(np.float32(0.6125)))
    assert abs(w_ebe.sum() / I1 - 1) < 1e-6
    assert abs(w_bc.sum() / (Pc * I0) - 1) < 1e-6
    effect = w_ebe.sum() / w_bc.sum() - 1
    # the probability is convex around its minimum: the binned method underestimates
    assert 0.02 < effect < 0.05


def test_bin_centre_converges_to_event_by_event():
    s = synth.beam_sample(200_000, seed=9)
    pt = synth.table1_point()
    ebe = oracle.histogram(s, [pt], 0.0, 5.0, 100)[0]
    errs = []
    for T in (50, 100, 200, 400, 800):
        bc = oracle.histogram_bin_centre(s, [pt], 0.0, 10.0, T, 0.0, 5.0, 100)[0]
        errs.append(np.abs(bc - ebe).sum() / ebe.sum())
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < errs[0] / 20


# ---------------------------------------------------------- layered matter
def _hamiltonian_np(row, A_abs, nubar):
    s2_12, s2_13, s2_23, dm21, dm32, dcp = row[:6]
    s12, c12 = np.sqrt(s2_12), np.sqrt(1 - s2_12)
    s13, c13 = np.sqrt(s2_13), np.sqrt(1 - s2_13)
    s23, c23 = np.sqrt(s2_23), np.sqrt(1 - s2_23)
    R23 = np.array([[1, 0, 0], [0, c23, s23], [0, -s23, c23]], dtype=complex)
    U13 = np.array([[c13, 0, s13 * np.exp(-1j * dcp)], [0, 1, 0], [-s13 * np.exp(1j * dcp), 0, c13]])
    R12 = np.array([[c12, s12, 0], [-s12, c12, 0], [0, 0, 1]], dtype=complex)
    U = R23 @ U13 @ R12
    if nubar:
        U = U.conj()
    M = U @ np.diag([0.0, dm21, dm32 + dm21]) @ U.conj().T
    M[0, 0] += -A_abs if nubar else A_abs
    return M


PROFILE = [(300.0, 2.2, 0.5), (700.0, 4.5, 0.49), (300.0, 1.0, 0.47)]


def test_single_layer_equals_constant_density():
    pt = oracle.point_from_row(synth.table1_point())
    E = np.geomspace(0.05, 10, 300)
    for nubar in (0, 1):
        a = oracle.prob_matrix_layers_many(pt, [(295.0, 2.6, 0.5)], E, nubar)
        b = oracle.prob_matrix_many(pt, 295.0, 2.6, 0.5, E, nubar)
        assert np.max(np.abs(a - b)) <= 1e-15


def test_equal_density_split_changes_nothing():
    rng = np.random.default_rng(8)
    pts = synth.scan_points(20, 77)
    E = np.geomspace(0.1, 20, 50)
    for row in pts:
        pt = oracle.point_from_row(row)
        cuts = np.sort(rng.uniform(0, 1300, 3))
        lens = np.diff(np.concatenate([[0], cuts, [1300]]))
        split = [(float(x), 2.85, 0.5) for x in lens]
        for nubar in (0, 1):
            a = oracle.prob_matrix_layers_many(pt, split, E, nubar)
            b = oracle.prob_matrix_many(pt, 1300.0, 2.85, 0.5, E, nubar)
            assert np.max(np.abs(a - b)) < 1e-11


def test_vacuum_layers_reproduce_eq1():
    pt = oracle.make_point(dcp=1.1)
    E = np.geomspace(0.1, 5, 40)
    layers = [(100.0, 0.0, 0.5), (150.0, 0.0, 0.3), (45.0, 0.0, 0.5)]
    P = oracle.prob_matrix_layers_many(pt, layers, E, 0)
    s12, c12 = np.sqrt(0.311), np.sqrt(1 - 0.311)
    s13, c13 = np.sqrt(0.0251), np.sqrt(1 - 0.0251)
    s23, c23 = np.sqrt(0.5), np.sqrt(0.5)
    ed = np.exp(1j * 1.1)
    Um = np.array([[c12 * c13, s12 * c13, s13 / ed],
                   [-s12 * c23 - c12 * s23 * s13 * ed, c12 * c23 - s12 * s23 * s13 * ed, s23 * c13],
                   [s12 * s23 - c12 * c23 * s13 * ed, -c12 * s23 - s12 * c23 * s13 * ed, c23 * c13]])
    m2 = np.array([0.0, 7.6e-5, 2.4e-3 + 7.6e-5])
    for i, e in enumerate(E):
        amp = np.einsum("ai,bi,i->ba", Um.conj(), Um, np.exp(-1j * C_L * m2 * 295.0 / e))
        assert np.max(np.abs(P[i] - np.abs(amp) ** 2)) < 1e-12


@pytest.mark.parametrize("nubar", [0, 1])
def test_rk4_through_layers(nubar):
    rng = np.random.default_rng(31 + nubar)
    n = 60
    E = np.clip(rng.gamma(3.0, 0.9, n), 0.2, 12.0)
    pts = synth.scan_points(n, 91 + nubar)
    alpha = rng.integers(0, 3, n)
    Prk = np.zeros((n, 3))
    for i in range(n):
        psi = np.zeros(3, dtype=complex)
        psi[alpha[i]] = 1.0
        for L, rho, ye in PROFILE:
            M = _hamiltonian_np(pts[i], K_A * ye * rho * E[i], nubar)
            K = -1j * C_L * M / E[i]
            rate = np.max(np.abs(np.linalg.eigvalsh(M))) * C_L / E[i]
            m = int(np.ceil(rate * L / 1e-3))
            hK = (L / m) * K
            for _ in range(m):
                k1 = hK @ psi
                k2 = hK @ (psi + 0.5 * k1)
                k3 = hK @ (psi + 0.5 * k2)
                k4 = hK @ (psi + k3)
                psi = psi + (k1 + 2 * k2 + 2 * k3 + k4) / 6.0
        Prk[i] = np.abs(psi) ** 2
    for i in range(n):
        Po = oracle.prob_matrix_layers_many(oracle.point_from_row(pts[i]), PROFILE, E[i:i + 1], nubar)[0]
        assert np.max(np.abs(Po[:, alpha[i]] - Prk[i])) < 1e-9


def test_layers_unitarity_and_reversal():
    E = np.geomspace(0.1, 30, 200)
    rev = PROFILE[::-1]
    for dcp in (0.0, 1.3):
        pt = oracle.make_point(dcp=dcp)
        for nubar in (0, 1):
            P = oracle.prob_matrix_layers_many(pt, PROFILE, E, nubar)
            assert np.max(np.abs(P.sum(axis=1) - 1)) < 1e-13
            assert np.max(np.abs(P.sum(axis=2) - 1)) < 1e-13
            R = oracle.prob_matrix_layers_many(pt, rev, E, nubar)
            d = np.max(np.abs(P - np.transpose(R, (0, 2, 1))))
            if dcp == 0.0:
                assert d < 1e-12
            else:
                assert d > 1e-3


def test_reweight_layers_matches_prob_matrix():
    s = synth.all_channel_sample(3000, seed=5)
    pt = oracle.point_from_row(synth.scan_points(1, 4)[0])
    p, w = oracle.reweight_layers(s, pt, PROFILE)
    for nb in (0, 1):
        sel = np.nonzero(s["is_nubar"] == nb)[0]
        P = oracle.prob_matrix_layers_many(pt, PROFILE, s["e_true"][sel].astype(np.float64), nb)
        ref = P[np.arange(sel.size), s["flav_out"][sel], s["flav_in"][sel]]
        assert np.array_equal(p[sel], ref)
    assert np.array_equal(w, p * s["w_mc"].astype(np.float64) * pt.norm)
