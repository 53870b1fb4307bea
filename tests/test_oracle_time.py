"""Pins of the oracle's time discretisation (eqs. dg-time-weights, cg-time-weights)."""
import math

import numpy as np
import pytest

from oracle import timeint


def test_dg0_is_backward_euler():
    tw = timeint.dg_weights(0)
    assert np.allclose(tw.Mhat, [[1.0]]) and np.allclose(tw.Ahat, [[1.0]]) and np.allclose(tw.alpha, [1.0])


def test_dg1_closed_form():
    tw = timeint.dg_weights(1)
    assert np.allclose(tw.nodes, [1 / 3, 1])
    assert np.allclose(tw.Mhat, np.diag([0.75, 0.25]), atol=1e-15)
    assert np.allclose(tw.Ahat, [[9 / 8, 3 / 8], [-9 / 8, 5 / 8]], atol=1e-14)
    assert np.allclose(tw.alpha, [1.5, -0.5], atol=1e-14)
    ev = np.sort_complex(np.linalg.eigvals(np.linalg.solve(tw.Mhat, tw.Ahat)))
    assert np.allclose(ev, [2 - 1j * math.sqrt(2), 2 + 1j * math.sqrt(2)], atol=1e-13)


def test_dg2_mass_is_radau_weights():
    s6 = math.sqrt(6)
    tw = timeint.dg_weights(2)
    assert np.allclose(tw.Mhat, np.diag([(16 - s6) / 36, (16 + s6) / 36, 1 / 9]), atol=1e-14)


def test_cgp1_is_crank_nicolson():
    tw = timeint.cgp_weights(1)
    assert np.allclose([tw.Mhat[0, 0], tw.Ahat[0, 0], tw.betahat[0], tw.alpha[0]], [0.5, 1.0, 0.5, -1.0])


def test_cgp2_closed_form():
    tw = timeint.cgp_weights(2)
    assert np.allclose(tw.nodes, [0.5, 1.0])
    assert np.allclose(tw.Mhat, np.diag([2 / 3, 1 / 6]), atol=1e-15)
    assert np.allclose(tw.Ahat, [[4 / 3, 1 / 3], [-4 / 3, 2 / 3]], atol=1e-14)
    assert np.allclose(tw.betahat, [1 / 3, -1 / 6], atol=1e-15)
    assert np.allclose(tw.alpha, [-5 / 3, 2 / 3], atol=1e-14)
    AMA = tw.Ahat @ np.linalg.solve(tw.Mhat, tw.Ahat)
    assert np.allclose(AMA, [[0, 2], [-8, 2]], atol=1e-13)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_dg_invariants(k):
    tw = timeint.dg_weights(k)
    # constants are reproduced: Ahat 1 = alpha (a constant-in-time state has no derivative)
    assert np.allclose(tw.Ahat @ np.ones(k + 1), tw.alpha, atol=1e-12)
    # symmetric part: Ahat + Ahat^T = xi(0) xi(0)^T + xi(1) xi(1)^T  (integration by parts)
    e1 = np.zeros(k + 1)
    e1[-1] = 1.0  # xi_j(1) = delta_{j, last} for right Radau nodes
    assert np.allclose(tw.Ahat + tw.Ahat.T, np.outer(tw.alpha, tw.alpha) + np.outer(e1, e1), atol=1e-12)
    assert np.all(np.linalg.eigvalsh(tw.Ahat + tw.Ahat.T) > -1e-12)
    assert np.isclose(np.sum(tw.Mhat), 1.0)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_cgp_invariants(k):
    tw = timeint.cgp_weights(k)
    assert np.allclose(tw.Ahat @ np.ones(k) + tw.alpha, 0.0, atol=1e-12)
    # int psi_i over the trial constant 1 = sum_j Mhat + betahat
    assert np.isclose(np.sum(tw.Mhat) + np.sum(tw.betahat), 1.0)


def _lumped_scalar_system(scheme, k, lam, tau, u0, n_steps):
    """Scalar ODE u' = -lam u through the slab system with A_h = lam, M_h = 1."""
    s = timeint.slab_system("heat", scheme, k, tau)
    u = u0
    for _ in range(n_steps):
        S = s.TA * lam + s.TM
        rhs = s.RA_u0 * lam * u + s.RM_u0 * u
        u = np.linalg.solve(S, rhs)[-1]
    return u


def test_backward_euler_and_crank_nicolson_scalar():
    lam, tau, u0 = 3.0, 0.1, 1.0
    assert np.isclose(_lumped_scalar_system("dg", 0, lam, tau, u0, 5), (1 / (1 + lam * tau)) ** 5)
    cn = (1 - lam * tau / 2) / (1 + lam * tau / 2)
    assert np.isclose(_lumped_scalar_system("cgp", 1, lam, tau, u0, 5), cn ** 5)


@pytest.mark.parametrize("scheme,k,order", [("dg", 1, 3), ("dg", 2, 5), ("cgp", 2, 4)])
def test_nodal_superconvergence_scalar(scheme, k, order):
    """End-point error of u' = -u: dG(k) is order 2k+1, cGP(k) order 2k (Radau IIA / Lobatto IIIA)."""
    errs = []
    for n in (8, 16):
        u = _lumped_scalar_system(scheme, k, 1.0, 1.0 / n, 1.0, n)
        errs.append(abs(u - math.exp(-1.0)))
    assert abs(math.log2(errs[0] / errs[1]) - order) < 0.3
