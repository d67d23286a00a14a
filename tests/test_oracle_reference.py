"""Pins of the oracle's reference data against closed forms (no GPU).

Radau rule (Sec. 3.1, Eq. GF), time matrices (Appendix A, Eq. DefKMC) and the DG(k) stability
function, which for the right-Radau DG(k) method is the (k, k+1) Pade approximant of exp
(Lesaint & Raviart 1974; equivalently Radau IIA), DG(0) = backward Euler.
"""
import math

import numpy as np
import pytest

from oracle.reference import (TimeData, gauss_lobatto_01, pressure_modes, radau_right,
                              SpaceRef, lagrange_eval)


def test_radau_closed_forms():
    t, w = radau_right(0)
    assert np.allclose(t, [1.0]) and np.allclose(w, [2.0])
    t, w = radau_right(1)
    assert np.allclose(t, [-1.0 / 3.0, 1.0], atol=1e-15) and np.allclose(w, [1.5, 0.5], atol=1e-15)
    t, w = radau_right(2)
    s6 = math.sqrt(6.0)
    assert np.allclose(t, [(-1 - s6) / 5, (-1 + s6) / 5, 1.0], atol=1e-14)
    # Radau IIA: c = (4 -+ sqrt6)/10, b = (16 -+ sqrt6)/36 on [0, 1]
    assert np.allclose(w, [(16 - s6) / 18, (16 + s6) / 18, 2.0 / 9.0], atol=1e-14)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_radau_exact_to_2k_not_2k_plus_1(k):
    t, w = radau_right(k)
    for p in range(2 * k + 1):
        exact = (1.0 - (-1.0) ** (p + 1)) / (p + 1)
        assert abs(np.dot(w, t ** p) - exact) < 1e-13
    p = 2 * k + 1
    exact = (1.0 - (-1.0) ** (p + 1)) / (p + 1)
    assert abs(np.dot(w, t ** p) - exact) > 1e-3


def test_gll_closed_forms():
    assert np.allclose(gauss_lobatto_01(3), [0, 0.5, 1])
    s = math.sqrt(5.0) / 10.0
    assert np.allclose(gauss_lobatto_01(4), [0, 0.5 - s, 0.5 + s, 1], atol=1e-15)
    s = math.sqrt(21.0) / 14.0
    assert np.allclose(gauss_lobatto_01(5), [0, 0.5 - s, 0.5, 0.5 + s, 1], atol=1e-15)


def test_time_matrices_k1_closed_form():
    td = TimeData(1, 2.0)
    assert np.allclose(td.K, [[9 / 8, 3 / 8], [-9 / 8, 5 / 8]], atol=1e-15)
    assert np.allclose(td.M, np.diag([1.5, 0.5]), atol=1e-15)
    assert np.allclose(td.C, [1.5, -0.5], atol=1e-15)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_time_matrix_invariants(k):
    tau = 0.37
    td = TimeData(k, tau)
    # a constant in time has zero derivative: K 1 = C (steady state reproduces the jump datum)
    assert np.allclose(td.K @ np.ones(k + 1), td.C, atol=1e-13)
    # M^tau is diagonal with entries tau/2 * omega_a (Radau exactness, Appendix A)
    assert np.allclose(td.M, np.diag(0.5 * tau * td.omega), atol=1e-14)
    assert np.all(td.w > 0)
    # the last node is t_n
    assert td.times(1.0)[-1] == pytest.approx(1.0 + tau)


def _pade_exp(L, M, z):
    num = sum(math.factorial(L + M - j) * math.factorial(L) /
              (math.factorial(L + M) * math.factorial(j) * math.factorial(L - j)) * z ** j
              for j in range(L + 1))
    den = sum(math.factorial(L + M - j) * math.factorial(M) /
              (math.factorial(L + M) * math.factorial(j) * math.factorial(M - j)) * (-z) ** j
              for j in range(M + 1))
    return num / den


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_dg_stability_function_is_pade(k):
    td = TimeData(k, 1.0)
    for z in [-0.3, -2.0, -17.0, 0.4, complex(-1.0, 3.0)]:
        Y = np.linalg.solve(td.K - z * td.M, td.C.astype(complex))
        assert Y[-1] == pytest.approx(_pade_exp(k, k + 1, z), rel=1e-12, abs=1e-14)
    if k == 0:
        assert Y[-1] == pytest.approx(1.0 / (1.0 - complex(-1.0, 3.0)))  # backward Euler


@pytest.mark.parametrize("r,d", [(1, 2), (2, 2), (3, 2), (1, 3), (2, 3)])
def test_pressure_basis_count_and_orthogonality(r, d):
    modes = pressure_modes(r, d)
    assert len(modes) == math.comb(r + d, d) and len(set(modes)) == len(modes)
    assert all(sum(m) <= r for m in modes)
    ref = SpaceRef(d, r, nq=r + 3)
    M = np.einsum("q,qi,qj->ij", ref.qwts, ref.psi, ref.psi)
    expect = np.diag([np.prod([1.0 / (2 * a + 1) for a in m]) for m in modes])
    assert np.allclose(M, expect, atol=1e-14)


def test_velocity_basis_is_nodal_partition_of_unity():
    ref = SpaceRef(3, 2)
    nodes = ref.local_node_multi()
    pts = ref.nodes[nodes]
    phi, dphi = ref.velocity_basis(pts)
    assert np.allclose(phi, np.eye(len(pts)), atol=1e-13)
    assert np.allclose(ref.phi.sum(1), 1.0) and np.allclose(ref.dphi.sum(1), 0.0, atol=1e-12)
    assert np.allclose(lagrange_eval(ref.nodes, ref.nodes), np.eye(ref.n), atol=1e-14)
