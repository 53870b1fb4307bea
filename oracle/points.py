"""Point values of a continuous Q_p finite-element function on a structured, Q1-mapped grid: the goal
quantities of the paper's structural-health-monitoring example (point evaluations of the
displacement, Section 4.3), FP64.

Test infrastructure (see oracle/__init__.py).

A point x is located in the first cell whose Q1 map x(xi) = sum_v X_v N_v(xi) reaches it with xi in
[0, 1]^dim (Newton on the map, started at the cell centre); the value is the sum over the cell's
nodes of the nodal value times the tensor-product Lagrange basis at xi (Gauss-Lobatto nodes).

Pins (tests/test_oracle_points.py): Q_p polynomials are reproduced at arbitrary points of a
Cartesian grid, linear functions of the physical coordinates at arbitrary points of a jittered
grid (the Q1 map keeps them in Q1 of xi), and a node returns its nodal value.
"""
from __future__ import annotations

import numpy as np

from . import fe1d
from .space import Grid


def locate(grid: Grid, x, tol: float = 1e-12, iters: int = 50):
    """(cell index, reference coordinates xi) of the physical point x."""
    x = np.asarray(x, dtype=np.float64)
    verts = grid.cell_vertices()
    for c in range(grid.n_cells):
        lo, hi = verts[c].min(axis=0), verts[c].max(axis=0)
        if np.any(x < lo - 1e-9) or np.any(x > hi + 1e-9):
            continue
        xi = np.full(grid.dim, 0.5)
        for _ in range(iters):
            val, grad = grid.q1_shape(xi[None, :])
            r = val[0] @ verts[c] - x
            J = np.einsum("ve,vd->de", grad[0], verts[c])
            step = np.linalg.solve(J, r)
            xi = xi - step
            if np.abs(step).max() < 1e-15:
                break
        if np.all(xi >= -tol) and np.all(xi <= 1.0 + tol):
            return c, np.clip(xi, 0.0, 1.0)
    raise ValueError(f"point {x} lies outside the grid")


def basis_at(grid: Grid, xi) -> np.ndarray:
    """Values of the cell's n^dim nodal basis functions at reference point xi."""
    xn = fe1d.space_nodes(grid.p)
    phi = np.ones(len(grid.local))
    for d in range(grid.dim):
        phi = phi * np.array([fe1d.lagrange(xn, j, xi[d]) for j in grid.local[:, d]])
    return phi


def point_values(grid: Grid, u: np.ndarray, points) -> np.ndarray:
    """u: (..., n_nodes) nodal values (any leading shape); returns (npts, ...) point values."""
    dofs = grid.cell_dofs()
    u = np.asarray(u, dtype=np.float64)
    out = []
    for x in points:
        c, xi = locate(grid, x)
        phi = basis_at(grid, xi)
        out.append(np.tensordot(u[..., dofs[c]], phi, axes=([-1], [0])))
    return np.array(out)
