"""1D quadrature rules and Lagrange bases on the unit interval [0, 1].

Test infrastructure (see oracle/__init__.py).

Paper: Section 2 uses Lagrange bases at Gauss-Radau points (dG, Section 2.1) and
Gauss-Lobatto points (cGP, Section 2.2) in time; the spatial Q_p space
(eq. fespace) uses a nodal Lagrange basis, taken here at Gauss-Lobatto points,
with (p+1)-point Gauss-Legendre quadrature per direction.

Pins (tests/test_oracle_fe1d.py): textbook Radau IIA nodes/weights, polynomial
exactness of every rule, Lagrange cardinality, 1D Q1/Q2 element matrices.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule mapped to [0, 1] (library primitive leggauss)."""
    x, w = npleg.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def _interpolatory_weights(nodes: np.ndarray) -> np.ndarray:
    """Weights w_j = int_0^1 l_j(t) dt of the interpolatory rule on the given nodes."""
    xq, wq = gauss_legendre(len(nodes) + 2)
    return np.array([np.sum(wq * lagrange(nodes, j, xq)) for j in range(len(nodes))])


def gauss_lobatto(n: int):
    """n-point Gauss-Lobatto rule on [0, 1]: endpoints plus roots of P'_{n-1}."""
    assert n >= 2
    if n == 2:
        nodes = np.array([-1.0, 1.0])
    else:
        c = np.zeros(n)
        c[n - 1] = 1.0  # P_{n-1}
        inner = np.sort(np.real(npleg.legroots(npleg.legder(c))))
        nodes = np.concatenate(([-1.0], inner, [1.0]))
    t = 0.5 * (nodes + 1.0)
    return t, _interpolatory_weights(t)


def gauss_radau_right(n: int):
    """n-point right Gauss-Radau rule on [0, 1] (includes t = 1).

    On [-1, 1] the nodes are the roots of P_{n-1}(x) - P_n(x); x = 1 is one of them.
    """
    assert n >= 1
    if n == 1:
        return np.array([1.0]), np.array([1.0])
    c = np.zeros(n + 1)
    c[n - 1] = 1.0
    c[n] = -1.0
    x = np.sort(np.real(npleg.legroots(c)))
    x[-1] = 1.0
    t = 0.5 * (x + 1.0)
    return t, _interpolatory_weights(t)


def lagrange(nodes: np.ndarray, j: int, t) -> np.ndarray:
    """l_j(t) = prod_{m != j} (t - x_m) / (x_j - x_m)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.ones_like(t)
    for m, xm in enumerate(nodes):
        if m != j:
            out = out * (t - xm) / (nodes[j] - xm)
    return out


def lagrange_deriv(nodes: np.ndarray, j: int, t) -> np.ndarray:
    """l_j'(t) by the product rule: sum_m 1/(x_j - x_m) prod_{l != j, m} (t - x_l)/(x_j - x_l)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.zeros_like(t)
    for m, xm in enumerate(nodes):
        if m == j:
            continue
        term = np.full_like(t, 1.0 / (nodes[j] - xm))
        for l, xl in enumerate(nodes):
            if l != j and l != m:
                term = term * (t - xl) / (nodes[j] - xl)
        out = out + term
    return out


def basis_table(nodes: np.ndarray, t: np.ndarray):
    """(len(t), len(nodes)) tables of values and derivatives of all Lagrange functions."""
    V = np.stack([lagrange(nodes, j, t) for j in range(len(nodes))], axis=1)
    D = np.stack([lagrange_deriv(nodes, j, t) for j in range(len(nodes))], axis=1)
    return V, D


def space_nodes(p: int) -> np.ndarray:
    """Nodes of the 1D Q_p Lagrange basis: the p+1 Gauss-Lobatto points."""
    return gauss_lobatto(p + 1)[0]
