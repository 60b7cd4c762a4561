"""Pins of the FP64 oracle to what the paper and the mathematics fix (CPU only).

Each check is computed by code written here, independently of the oracle's
Jacobi + exponential route, so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them:

* Sec. 1.1 Eq. (1), rho = 0: amplitude sum and its expanded closed form.
* Unitarity of the propagator: rows and columns of P sum to 1.
* theta13 = 0: exact solar two-flavour MSW; dm21 = 0: exact atmospheric
  two-flavour MSW; both: nu_e decouples, vacuum mu-tau oscillation.
* T symmetry at delta in {0, pi}; antineutrino sign flip; vacuum CPT.
* Signs of delta and of the matter term (well-known physics).
* RK4 brute-force integration of the Schroedinger equation; scipy.linalg.expm;
  numpy.linalg.eigh for the Jacobi eigendecomposition.
* Table 1 / Fig. 1: the nu_mu survival trough near 0.6 GeV at 295 km.
* The FP32 binning rule, restated with numpy float32 arithmetic.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1311_7579_gb300 import synth

C_L = 2.5338653588396975  # restated: 1e-6 / (2 * 1.973269804e-7)
# restated: 2 sqrt(2) G_F N_A (hbar c)^3 * 1e9 with G_F = 1.1663788e-23 eV^-2,
# N_A = 6.02214076e23, hbar c = 1.973269804e-5 eV cm
K_A = 2 * np.sqrt(2) * 1.1663788e-23 * 6.02214076e23 * 1.973269804e-5 ** 3 * 1e9


def _point(**kw):
    return oracle.make_point(**kw)


def _pmns_np(s2_12, s2_13, s2_23, dcp):
    """PDG parametrisation written as R23 * U13(delta) * R12 (independent of the
    oracle's explicit matrix)."""
    s12, c12 = np.sqrt(s2_12), np.sqrt(1 - s2_12)
    s13, c13 = np.sqrt(s2_13), np.sqrt(1 - s2_13)
    s23, c23 = np.sqrt(s2_23), np.sqrt(1 - s2_23)
    R23 = np.array([[1, 0, 0], [0, c23, s23], [0, -s23, c23]], dtype=complex)
    U13 = np.array([[c13, 0, s13 * np.exp(-1j * dcp)], [0, 1, 0],
                    [-s13 * np.exp(1j * dcp), 0, c13]], dtype=complex)
    R12 = np.array([[c12, s12, 0], [-s12, c12, 0], [0, 0, 1]], dtype=complex)
    return R23 @ U13 @ R12


def test_constants_match_textbook(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "textbook_constants.json")))
    # phase of dm^2 L / 4E is (c_L / 2) dm^2 L / E
    assert abs(oracle.c_L() / 2 - g["phase_coeff_dm2L_over_4E"]) / g["phase_coeff_dm2L_over_4E"] < g["rel_tol"]
    # A = 2 E V_cc  ->  k_A = 2 * V_cc[eV] * 1e9
    kA_txt = 2 * g["V_cc_eV_per_rho_ye"] * 1e9
    assert abs(oracle.k_A() - kA_txt) / kA_txt < g["rel_tol"]


def test_golden_table1_matches_generator(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "table1.json")))
    t = synth.TABLE1
    assert t["s2_12"] == g["s2_12"] and t["s2_23"] == g["s2_23"] and t["s2_13"] == g["s2_13"]
    assert t["dm32"] == g["dm32_eV2"] and t["dm21"] == g["dm21_eV2"] and t["dcp"] == g["dcp"]
    assert synth.TABLE1_RHO == g["density_gcc"] and synth.TABLE1_L_KM == g["baseline_km"]


@pytest.mark.parametrize("dcp", [0.0, 1.1, -2.5, np.pi])
def test_pmns_matches_rotation_product(dcp):
    pt = _point(s2_13=0.022, s2_23=0.45, dcp=dcp)
    U = oracle.pmns(pt)
    Uref = _pmns_np(0.311, 0.022, 0.45, dcp)
    assert np.max(np.abs(U - Uref)) < 1e-15
    assert np.max(np.abs(U @ U.conj().T - np.eye(3))) < 1e-15


def test_jacobi_matches_numpy_eigh():
    rng = np.random.default_rng(11)
    for _ in range(200):
        X = rng.normal(size=(3, 3)) + 1j * rng.normal(size=(3, 3))
        M = (X + X.conj().T) * 10.0 ** rng.uniform(-5, 0)
        lam, V, sweeps = oracle.eigh3(M)
        assert sweeps >= 0
        ref = np.linalg.eigvalsh(M)
        assert np.max(np.abs(np.sort(lam) - ref)) < 1e-14 * np.max(np.abs(ref))
        assert np.max(np.abs(V @ np.diag(lam) @ V.conj().T - M)) < 1e-14 * np.max(np.abs(M))
        assert np.max(np.abs(V.conj().T @ V - np.eye(3))) < 1e-14
    # degenerate spectrum (dm21 = 0 reductions rely on it)
    M = np.diag([1.0, 1.0, 3.0]).astype(complex)
    lam, V, sweeps = oracle.eigh3(M)
    assert sweeps == 0 and np.allclose(np.sort(lam), [1, 1, 3])


def _vacuum_amplitude_P(U, m2, L, E, alpha, beta):
    """Eq. (1) with the U*_{alpha i} U_{beta i} product and the unit constant restored."""
    amp = sum(np.conj(U[alpha, i]) * U[beta, i] * np.exp(-1j * C_L * m2[i] * L / E) for i in range(3))
    return abs(amp) ** 2


def _vacuum_closed_form_P(U, m2, L, E, alpha, beta):
    """Expanded form: delta - 4 sum Re K sin^2(D) + 2 sum Im K sin(2D), K_ij =
    U*_ai U_bi U_aj U*_bj, D_ij = c_L (m_i^2 - m_j^2) L / (2E)."""
    P = 1.0 if alpha == beta else 0.0
    for i in range(3):
        for j in range(i):
            K = np.conj(U[alpha, i]) * U[beta, i] * U[alpha, j] * np.conj(U[beta, j])
            D = C_L * (m2[i] - m2[j]) * L / (2 * E)
            P += -4 * K.real * np.sin(D) ** 2 + 2 * K.imag * np.sin(2 * D)
    return P


@pytest.mark.parametrize("dm32,dcp", [(2.4e-3, 0.0), (2.4e-3, -1.3), (-2.5e-3, 2.2)])
def test_vacuum_limit_reproduces_eq1(dm32, dcp):
    pt = _point(dm32=dm32, dcp=dcp, s2_23=0.57)
    U = _pmns_np(0.311, 0.0251, 0.57, dcp)
    m2 = [0.0, 7.6e-5, dm32 + 7.6e-5]
    rng = np.random.default_rng(3)
    E = rng.uniform(0.05, 10.0, 64)
    for L in (295.0, 1300.0):
        for nubar in (0, 1):
            P = oracle.prob_matrix_many(pt, L, 0.0, 0.5, E, nubar)
            Uc = U.conj() if nubar else U
            for k, e in enumerate(E):
                for a in range(3):
                    for b in range(3):
                        amp = _vacuum_amplitude_P(Uc, m2, L, e, a, b)
                        cf = _vacuum_closed_form_P(Uc, m2, L, e, a, b)
                        assert abs(amp - cf) < 1e-13
                        assert abs(P[k, b, a] - amp) < 1e-13


@pytest.mark.parametrize("nubar", [0, 1])
def test_unitarity_rows_and_columns(nubar):
    rng = np.random.default_rng(5)
    for trial in range(6):
        pt = _point(s2_13=rng.uniform(0.018, 0.03), s2_23=rng.uniform(0.35, 0.65),
                    dm32=rng.choice([-1, 1]) * rng.uniform(2e-3, 2.8e-3), dcp=rng.uniform(-np.pi, np.pi))
        E = rng.uniform(0.05, 30.0, 100)
        P = oracle.prob_matrix_many(pt, 1300.0, 2.85, 0.5, E, nubar)
        assert np.max(np.abs(P.sum(axis=1) - 1)) < 1e-13  # sum over beta
        assert np.max(np.abs(P.sum(axis=2) - 1)) < 1e-13  # sum over alpha
        assert P.min() > -1e-15


def _two_flavour(dm2, s2, A, L, E):
    """Exact two-flavour MSW: returns (sin^2 2theta_M, phase argument)."""
    c2 = 1 - 2 * s2
    sin2 = 2 * np.sqrt(s2 * (1 - s2))
    dM = np.sqrt((dm2 * c2 - A) ** 2 + (dm2 * sin2) ** 2)
    return (dm2 * sin2 / dM) ** 2, C_L * dM * L / (2 * E)


def test_theta13_zero_solar_msw():
    pt = _point(s2_13=0.0)
    kA = K_A
    for rho in (0.0, 2.6, 12.0):
        E = np.linspace(0.05, 2.0, 97)
        P = oracle.prob_matrix_many(pt, 295.0, rho, 0.5, E, 0)
        Pb = oracle.prob_matrix_many(pt, 295.0, rho, 0.5, E, 1)
        for k, e in enumerate(E):
            A = kA * 0.5 * rho * e
            s2m, ph = _two_flavour(7.6e-5, 0.311, A, 295.0, e)
            assert abs(P[k, 0, 0] - (1 - s2m * np.sin(ph) ** 2)) < 1e-13
            s2m, ph = _two_flavour(7.6e-5, 0.311, -A, 295.0, e)
            assert abs(Pb[k, 0, 0] - (1 - s2m * np.sin(ph) ** 2)) < 1e-13


def test_dm21_zero_atmospheric_msw():
    kA = K_A
    for s2_23 in (0.5, 0.42):
        pt = _point(dm21=0.0, dm32=2.5e-3, s2_23=s2_23, s2_13=0.025, dcp=0.7)
        E = np.linspace(0.5, 20.0, 80)
        P = oracle.prob_matrix_many(pt, 1300.0, 2.85, 0.5, E, 0)
        for k, e in enumerate(E):
            A = kA * 0.5 * 2.85 * e
            s2m, ph = _two_flavour(2.5e-3, 0.025, A, 1300.0, e)
            assert abs(P[k, 0, 0] - (1 - s2m * np.sin(ph) ** 2)) < 1e-13
            assert abs(P[k, 0, 1] - s2_23 * s2m * np.sin(ph) ** 2) < 1e-13  # mu -> e


def test_both_zero_decouples_nue():
    pt = _point(dm21=0.0, s2_13=0.0, dm32=2.4e-3, s2_23=0.45)
    E = np.linspace(0.1, 5.0, 50)
    for rho in (0.0, 2.6, 50.0):
        P = oracle.prob_matrix_many(pt, 810.0, rho, 0.5, E, 0)
        sin2_2t23 = 4 * 0.45 * 0.55
        ref = 1 - sin2_2t23 * np.sin(C_L * 2.4e-3 * 810.0 / (2 * E)) ** 2
        assert np.max(np.abs(P[:, 0, 0] - 1)) < 1e-13
        assert np.max(np.abs(P[:, 1, 1] - ref)) < 1e-13


@pytest.mark.parametrize("dcp", [0.0, np.pi])
def test_t_symmetry_real_hamiltonian(dcp):
    pt = _point(dcp=dcp, s2_23=0.6)
    E = np.linspace(0.05, 15.0, 60)
    for nubar in (0, 1):
        P = oracle.prob_matrix_many(pt, 1300.0, 2.85, 0.5, E, nubar)
        assert np.max(np.abs(P - np.transpose(P, (0, 2, 1)))) < 1e-13


def test_t_symmetry_broken_by_delta():
    pt = _point(dcp=-np.pi / 2)
    P = oracle.prob_matrix_many(pt, 295.0, 2.6, 0.5, np.array([0.6]), 0)
    assert abs(P[0, 0, 1] - P[0, 1, 0]) > 1e-3


def test_antineutrino_flip_and_vacuum_cpt():
    kA = K_A
    for dcp in (0.4, -2.0):
        for e in (0.3, 1.7, 9.0):
            A = kA * 0.5 * 2.8 * e
            Pbar = oracle.prob_matrix_A(_point(dcp=dcp), 810.0, A, e, 1)
            Pflip = oracle.prob_matrix_A(_point(dcp=-dcp), 810.0, -A, e, 0)
            assert np.max(np.abs(Pbar - Pflip)) < 1e-13
            Pv = oracle.prob_matrix_A(_point(dcp=dcp), 810.0, 0.0, e, 0)
            Pvb = oracle.prob_matrix_A(_point(dcp=dcp), 810.0, 0.0, e, 1)
            assert np.max(np.abs(Pvb - Pv.T)) < 1e-13


def test_sign_of_delta_and_matter():
    # first maximum at 295 km: nu_mu -> nu_e larger for delta = -pi/2 (nu), opposite for nubar
    m = oracle.prob(_point(dcp=-np.pi / 2), 295.0, 2.6, 0.5, 0.6, 1, 0, 0)
    p = oracle.prob(_point(dcp=np.pi / 2), 295.0, 2.6, 0.5, 0.6, 1, 0, 0)
    assert m > p + 0.02
    mb = oracle.prob(_point(dcp=-np.pi / 2), 295.0, 2.6, 0.5, 0.6, 1, 0, 1)
    pb = oracle.prob(_point(dcp=np.pi / 2), 295.0, 2.6, 0.5, 0.6, 1, 0, 1)
    assert pb > mb + 0.01
    # normal-hierarchy matter enhancement of nu_mu -> nu_e at 1300 km
    mat = oracle.prob(_point(), 1300.0, 2.85, 0.5, 2.5, 1, 0, 0)
    vac = oracle.prob(_point(), 1300.0, 0.0, 0.5, 2.5, 1, 0, 0)
    assert mat > vac * 1.2
    # ... and suppression for antineutrinos
    matb = oracle.prob(_point(), 1300.0, 2.85, 0.5, 2.5, 1, 0, 1)
    vacb = oracle.prob(_point(), 1300.0, 0.0, 0.5, 2.5, 1, 0, 1)
    assert matb < vacb


def _hamiltonian_np(s2_12, s2_13, s2_23, dm21, dm32, dcp, A_abs, nubar):
    U = _pmns_np(s2_12, s2_13, s2_23, dcp)
    if nubar:
        U = U.conj()
    M = U @ np.diag([0.0, dm21, dm32 + dm21]) @ U.conj().T
    M[0, 0] += -A_abs if nubar else A_abs
    return M


def _draw_events(rng, n, L, rho, scale):
    e = np.clip(rng.gamma(3.0, 0.25 * scale, n), 0.05, 10 * scale).astype(np.float32).astype(np.float64)
    alpha = rng.integers(0, 3, n)
    nubar = rng.integers(0, 2, n)
    pts = synth.scan_points(n, int(rng.integers(1 << 30)))
    return e, alpha, nubar, pts


def test_rk4_brute_force():
    """i d(psi)/dx = c_L (M / E) psi integrated with RK4 at a step where the
    largest |lambda| c_L h / E <= 1e-3, against the oracle's P for all beta."""
    rng = np.random.default_rng(21)
    kA = K_A
    for L, rho, scale, n in ((295.0, 2.6, 1.0, 120), (1300.0, 2.85, 1300 / 295, 80)):
        e, alpha, nubar, pts = _draw_events(rng, n, L, rho, scale)
        Ms = np.array([_hamiltonian_np(*pts[i, :6], kA * 0.5 * rho * e[i], nubar[i]) for i in range(n)])
        K = -1j * C_L * Ms / e[:, None, None]  # d psi / dx = K psi, x in km
        rate = np.max(np.abs(np.linalg.eigvalsh(Ms)), axis=1) * C_L / e
        nsteps = int(np.ceil(np.max(rate) * L / 1e-3))
        h = L / nsteps
        psi = np.zeros((n, 3), dtype=complex)
        psi[np.arange(n), alpha] = 1.0
        hK = h * K

        def f(y):
            return np.einsum("nij,nj->ni", hK, y)

        for _ in range(nsteps):
            k1 = f(psi)
            k2 = f(psi + 0.5 * k1)
            k3 = f(psi + 0.5 * k2)
            k4 = f(psi + k3)
            psi = psi + (k1 + 2 * k2 + 2 * k3 + k4) / 6.0
        Prk = np.abs(psi) ** 2
        for i in range(n):
            Po = oracle.prob_matrix_many(oracle.point_from_row(pts[i]), L, rho, 0.5, e[i:i + 1], nubar[i])[0]
            assert np.max(np.abs(Po[:, alpha[i]] - Prk[i])) < 1e-9


def test_scipy_expm():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(23)
    kA = K_A
    for L, rho, scale in ((295.0, 2.6, 1.0), (810.0, 2.8, 810 / 295), (1300.0, 2.85, 1300 / 295)):
        e, alpha, nubar, pts = _draw_events(rng, 100, L, rho, scale)
        for i in range(e.size):
            M = _hamiltonian_np(*pts[i, :6], kA * 0.5 * rho * e[i], nubar[i])
            S = scipy_linalg.expm(-1j * C_L * M * L / e[i])
            Po = oracle.prob_matrix_many(oracle.point_from_row(pts[i]), L, rho, 0.5, e[i:i + 1], nubar[i])[0]
            assert np.max(np.abs(Po - np.abs(S) ** 2)) < 1e-12


def test_fig1_trough_position(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "fig1_trough.json")))
    t = json.load(open(os.path.join(golden_dir, "table1.json")))
    pt = _point(s2_12=t["s2_12"], s2_13=t["s2_13"], s2_23=t["s2_23"], dm21=t["dm21_eV2"],
                dm32=t["dm32_eV2"], dcp=t["dcp"])
    E = np.arange(g["scan_GeV"][0], g["scan_GeV"][1] + 1e-12, g["scan_step_GeV"])
    P = oracle.prob_matrix_many(pt, t["baseline_km"], t["density_gcc"], g["ye"], E, 0)[:, 1, 1]
    e_min = E[np.argmin(P)]
    assert g["accept_window_GeV"][0] <= e_min <= g["accept_window_GeV"][1]
    assert P.min() < 1e-2


def test_binning_rule_float32_restatement():
    rng = np.random.default_rng(9)
    e = np.concatenate([rng.uniform(-0.5, 6.0, 20000),
                        np.arange(0, 101) * 0.05, np.nextafter(np.float32(5.0), np.float32(0.0)) * np.ones(1),
                        [0.0, -0.0, 4.9999995, 5.0, 5.0000005, 1e30, -1e30]]).astype(np.float32)
    for escale, lo, hi, nb in ((1.0, 0.0, 5.0, 100), (1.0123, 0.0, 5.0, 100), (0.97, 0.2, 3.7, 37),
                               (1.02, -1.0, 4.0, 7)):
        b = oracle.bins(e, escale, lo, hi, nb)
        sf, lof = np.float32(escale), np.float32(lo)
        invf = np.float32(nb / (hi - lo))
        with np.errstate(over="ignore", invalid="ignore"):
            x = (sf * e).astype(np.float32)
            t = (x - lof).astype(np.float32)
            u = (t * invf).astype(np.float32)
        keep = (t >= 0) & (u < np.float32(nb))
        ref = np.where(keep, np.floor(np.where(keep, u, 0)).astype(np.int64), -1)
        assert np.array_equal(b, ref)
        assert b.max() < nb and b.min() >= -1


def test_histogram_sums_and_compensation():
    s = synth.table1_sample(20000, seed=5)
    pt = oracle.point_from_row(synth.table1_point())
    prob, w = oracle.reweight(s, pt)
    assert np.allclose(w, prob * s["w_mc"].astype(np.float64))
    b = oracle.bins(s["e_reco"], 1.0, 0.0, 5.0, 100)
    ref = np.bincount(b[b >= 0], weights=w[b >= 0], minlength=100)
    h = oracle.hist_from_weights(s["e_reco"], w, 1.0, 0.0, 5.0, 100)
    hc = oracle.hist_from_weights(s["e_reco"], w, 1.0, 0.0, 5.0, 100, compensated=True)
    assert np.allclose(h, ref, rtol=1e-12, atol=0)
    assert np.allclose(hc, ref, rtol=1e-12, atol=0)
    h2 = oracle.histogram(s, [synth.table1_point()], 0.0, 5.0, 100)[0]
    assert np.array_equal(h2, h)
    # norm scales the weights
    row = synth.table1_point().copy()
    row[7] = 2.5
    h3 = oracle.histogram(s, [row], 0.0, 5.0, 100)[0]
    assert np.allclose(h3, 2.5 * h, rtol=1e-15)


def test_reweight_matches_prob_matrix_every_channel():
    """orc_reweight picks, for each event, the (flav_out, flav_in) element of the
    probability matrix at its E_true, for nu and nubar, and weights it by w_mc and
    the point's norm: compared exactly with orc_prob_matrix_many, whose
    orientation P[i, beta, alpha] the delta-sign and T-symmetry pins fix."""
    s = synth.all_channel_sample(6000, seed=11)
    row = synth.scan_points(1, 7)[0].copy()
    row[5] = -1.1   # delta away from 0 and pi: P(a -> b) != P(b -> a), so a swapped flavour pair shows
    row[7] = 0.73   # norm != 1
    pt = oracle.point_from_row(row)
    p, w = oracle.reweight(s, pt)
    seen = set()
    for nb in (0, 1):
        sel = np.nonzero(s["is_nubar"] == nb)[0]
        P = oracle.prob_matrix_many(pt, s["baseline_km"], s["density_gcc"], s["ye"],
                                    s["e_true"][sel].astype(np.float64), nb)
        fi, fo = s["flav_in"][sel], s["flav_out"][sel]
        assert np.array_equal(p[sel], P[np.arange(sel.size), fo, fi])
        seen |= set(zip(fi.tolist(), fo.tolist(), [nb] * sel.size))
        # the transposed element differs for off-diagonal channels: the check above is not vacuous
        off = fi != fo
        assert np.max(np.abs(P[np.arange(sel.size), fo, fi] - P[np.arange(sel.size), fi, fo])[off]) > 1e-3
    assert len(seen) == 18
    assert np.array_equal(w, p * s["w_mc"].astype(np.float64) * 0.73)


def test_histogram_many_points_with_energy_scale_and_norm():
    """orc_histogram over several points: row p uses point p's own energy scale
    (E_reco binned after scaling) and norm, and lands at out[p].  Checked against
    an independent numpy restatement: the FP32 binning rule and weights
    P * w_mc * norm from the probability matrix, summed per bin."""
    s = synth.table1_sample(30000, seed=12)
    rows = np.vstack([synth.table1_point()] * 3)
    rows[:, 7] = (0.6, 1.0, 2.5)          # norm
    rows[:, 6] = (0.93, 1.0, 1.08)        # energy scale
    rows[:, 4] = (2.2e-3, 2.4e-3, 2.6e-3)  # different oscillation too
    lo, hi, nb = 0.0, 5.0, 50
    h = oracle.histogram(s, rows, lo, hi, nb)
    assert h.shape == (3, nb)
    for k in range(3):
        pt = oracle.point_from_row(rows[k])
        P = np.zeros(s["n"])
        for nbar in (0, 1):
            sel = np.nonzero(s["is_nubar"] == nbar)[0]
            M = oracle.prob_matrix_many(pt, s["baseline_km"], s["density_gcc"], s["ye"],
                                        s["e_true"][sel].astype(np.float64), nbar)
            P[sel] = M[np.arange(sel.size), s["flav_out"][sel], s["flav_in"][sel]]
        wt = P * s["w_mc"].astype(np.float64) * rows[k, 7]
        x = (np.float32(rows[k, 6]) * s["e_reco"]).astype(np.float32)
        t = (x - np.float32(lo)).astype(np.float32)
        u = (t * np.float32(nb / (hi - lo))).astype(np.float32)
        keep = (t >= 0) & (u < np.float32(nb))
        ref = np.bincount(np.floor(u[keep]).astype(np.int64), weights=wt[keep], minlength=nb)
        assert np.allclose(h[k], ref, rtol=1e-12, atol=1e-300), k
    # the three rows differ, so a row written to the wrong offset shows
    assert np.min(np.abs(h[0] - h[2]).max()) > 1.0
