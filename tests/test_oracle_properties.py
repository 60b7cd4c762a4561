"""Randomised properties of the FP64 oracle (CPU only, hypothesis), over the
whole valid parameter domain rather than fixed points:

* unitarity of the propagator (rows and columns of P sum to 1);
* antineutrinos: P_nubar(delta, A) is P_nu(-delta, -A) (U -> U*, A -> -A);
* T symmetry P(a->b) = P(b->a) at delta in {0, pi}; vacuum CPT
  P_nubar(a->b) = P_nu(b->a);
* vacuum depends on L/E only; matter on rho * Y_e only;
* a constant-density path cut into random pieces equals one layer.
"""
import numpy as np
import pytest

import oracle

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

s2 = st.floats(0.01, 0.99)


@st.composite
def points(draw, dcp=None):
    dm21 = draw(st.floats(1e-5, 2e-4))
    sign = draw(st.sampled_from([-1.0, 1.0]))
    dm32 = sign * draw(st.floats(1.2, 40.0)) * dm21
    d = draw(st.floats(-np.pi, np.pi)) if dcp is None else dcp
    return oracle.make_point(s2_12=draw(s2), s2_13=draw(s2), s2_23=draw(s2), dm21=dm21, dm32=dm32, dcp=d)


energies = st.floats(0.05, 30.0)
baselines = st.floats(1.0, 13000.0)
densities = st.floats(0.0, 13.0)

SETTINGS = settings(max_examples=60, deadline=None)


@SETTINGS
@given(points(), baselines, densities, energies, st.sampled_from([0, 1]))
def test_unitarity(pt, L, rho, E, nubar):
    P = oracle.prob_matrix_many(pt, L, rho, 0.5, [E], nubar)[0]
    assert np.max(np.abs(P.sum(axis=0) - 1)) < 1e-12
    assert np.max(np.abs(P.sum(axis=1) - 1)) < 1e-12
    assert P.min() > -1e-14


@SETTINGS
@given(points(), baselines, st.floats(0.0, 0.05), energies)
def test_antineutrino_is_conjugate_phase_and_negative_potential(pt, L, A, E):
    flipped = oracle.make_point(pt.s2_12, pt.s2_13, pt.s2_23, pt.dm21, pt.dm32, -pt.dcp)
    a = oracle.prob_matrix_A(pt, L, A, E, 1)
    b = oracle.prob_matrix_A(flipped, L, -A, E, 0)
    assert np.max(np.abs(a - b)) <= 1e-15


@SETTINGS
@given(st.sampled_from([0.0, np.pi]).flatmap(lambda d: points(dcp=d)), baselines, densities, energies,
       st.sampled_from([0, 1]))
def test_t_symmetry_with_real_mixing(pt, L, rho, E, nubar):
    P = oracle.prob_matrix_many(pt, L, rho, 0.5, [E], nubar)[0]
    assert np.max(np.abs(P - P.T)) < 1e-12


@SETTINGS
@given(points(), baselines, energies)
def test_vacuum_cpt(pt, L, E):
    Pn = oracle.prob_matrix_many(pt, L, 0.0, 0.5, [E], 0)[0]
    Pb = oracle.prob_matrix_many(pt, L, 0.0, 0.5, [E], 1)[0]
    assert np.max(np.abs(Pb - Pn.T)) < 1e-12


@SETTINGS
@given(points(), baselines, energies, st.sampled_from([0, 1]))
def test_vacuum_depends_on_l_over_e(pt, L, E, nubar):
    a = oracle.prob_matrix_many(pt, L, 0.0, 0.5, [E], nubar)[0]
    b = oracle.prob_matrix_many(pt, 2.0 * L, 0.0, 0.5, [2.0 * E], nubar)[0]
    assert np.array_equal(a, b)  # doubling both is exact in binary floating point


@SETTINGS
@given(points(), baselines, st.floats(0.1, 13.0), energies, st.sampled_from([0, 1]))
def test_matter_depends_on_rho_times_ye(pt, L, rho, E, nubar):
    a = oracle.prob_matrix_many(pt, L, rho, 0.5, [E], nubar)[0]
    b = oracle.prob_matrix_many(pt, L, 2.0 * rho, 0.25, [E], nubar)[0]
    assert np.max(np.abs(a - b)) <= 1e-15


@SETTINGS
@given(points(), st.floats(10.0, 3000.0), st.floats(0.0, 6.0), energies, st.sampled_from([0, 1]),
       st.lists(st.floats(0.05, 0.95), min_size=1, max_size=4))
def test_cutting_a_constant_layer_changes_nothing(pt, L, rho, E, nubar, cuts):
    edges = np.concatenate([[0.0], np.sort(cuts), [1.0]]) * L
    pieces = [(float(b - a), rho, 0.5) for a, b in zip(edges[:-1], edges[1:]) if b - a > 0]
    a = oracle.prob_matrix_layers_many(pt, pieces, [E], nubar)[0]
    b = oracle.prob_matrix_many(pt, L, rho, 0.5, [E], nubar)[0]
    assert np.max(np.abs(a - b)) < 1e-10
