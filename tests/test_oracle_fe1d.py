"""Pins of the oracle's 1D quadrature and Lagrange tables against textbook values."""
import math

import numpy as np
import pytest

from oracle import fe1d, space
import synth


def test_radau_iia_nodes_weights():
    # Radau IIA (right Radau) on [0,1]: 2 points {1/3, 1} weights {3/4, 1/4}
    t, w = fe1d.gauss_radau_right(2)
    assert np.allclose(t, [1 / 3, 1.0], atol=1e-15) and np.allclose(w, [0.75, 0.25], atol=1e-15)
    s6 = math.sqrt(6.0)
    t, w = fe1d.gauss_radau_right(3)
    assert np.allclose(t, [(4 - s6) / 10, (4 + s6) / 10, 1.0], atol=1e-14)
    assert np.allclose(w, [(16 - s6) / 36, (16 + s6) / 36, 1 / 9], atol=1e-14)


def test_lobatto_three_points():
    t, w = fe1d.gauss_lobatto(3)
    assert np.allclose(t, [0, 0.5, 1]) and np.allclose(w, [1 / 6, 2 / 3, 1 / 6])


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_exactness_degrees(n):
    # Gauss: 2n-1, Radau: 2n-2, Lobatto: 2n-3; and one degree more must fail (non-trivially)
    rules = [(fe1d.gauss_legendre(n), 2 * n - 1), (fe1d.gauss_radau_right(n), 2 * n - 2)]
    if n >= 2:
        rules.append((fe1d.gauss_lobatto(n), 2 * n - 3))
    for (t, w), deg in rules:
        for d in range(deg + 1):
            assert abs(np.sum(w * t ** d) - 1.0 / (d + 1)) < 1e-13
        assert abs(np.sum(w * t ** (deg + 1)) - 1.0 / (deg + 2)) > 1e-8


def test_lagrange_cardinal_and_derivative():
    x = fe1d.gauss_lobatto(5)[0]
    V, D = fe1d.basis_table(x, x)
    assert np.allclose(V, np.eye(5), atol=1e-14)
    # derivatives reproduce d/dt t^3 exactly
    tt = np.linspace(0, 1, 7)
    _, Dt = fe1d.basis_table(x, tt)
    assert np.allclose(Dt @ x ** 3, 3 * tt ** 2, atol=1e-12)


def _one_d_matrices(p, h):
    g = space.Grid(1, 1, p, np.array([[0.0], [h]]))
    A, M = g.element_matrices(np.ones((1, p + 1)))
    return A[0], M[0]


def test_q1_q2_element_matrices_closed_form():
    h = 0.37
    A, M = _one_d_matrices(1, h)
    assert np.allclose(M, h / 6 * np.array([[2, 1], [1, 2]]), atol=1e-15)
    assert np.allclose(A, 1 / h * np.array([[1, -1], [-1, 1]]), atol=1e-14)
    A, M = _one_d_matrices(2, h)
    assert np.allclose(M, h / 30 * np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]), atol=1e-15)
    assert np.allclose(A, 1 / (3 * h) * np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]), atol=1e-13)


def test_splitmix_reference_values():
    # SplitMix64 published reference outputs for seed 0 (first three draws)
    from synth import splitmix64
    assert splitmix64(0) == 0xE220A8397B1DCDAF
    assert splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
