"""Q_p finite elements on structured, Q1-mapped quadrilateral/hexahedral grids, FP64.

Test infrastructure (see oracle/__init__.py).

Paper: eq. space-matrices (M_h = (phi_i, phi_j), A_h = (rho grad phi_i, grad phi_j)),
eq. fespace (continuous Q_p on the mesh), Section 4.1 (perturbed meshes).
Readings where the paper is silent: nodal basis at Gauss-Lobatto points, Q1
(multilinear) geometry map from the 2^dim cell vertices, (p+1)^dim
Gauss-Legendre quadrature, coefficient rho sampled at the quadrature points.

Layouts (shared convention, lexicographic with x fastest):
  global node (gx, gy, gz) -> gx + (pN+1) * (gy + (pN+1) * gz)
  cell-local node a = (ax, ay, az) -> ax + n * (ay + n * az),   n = p + 1
  quadrature point q likewise with n_q = p + 1 points per direction

Pins (tests/test_oracle_space.py): 1D Q1/Q2 closed-form element matrices,
Kronecker structure on Cartesian grids, mass sums to the domain measure,
stiffness annihilates constants, exact energy of linear functions on perturbed grids.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from . import fe1d


def lex_indices(n: int, dim: int) -> np.ndarray:
    """(n^dim, dim) multi-indices, x component first, x fastest."""
    return np.indices((n,) * dim).reshape(dim, -1)[::-1].T.copy()


class Grid:
    """Structured grid of N^dim cells with Q_p nodes; vertices (N+1)^dim x dim."""

    def __init__(self, N: int, dim: int, p: int, vertices: np.ndarray):
        self.N, self.dim, self.p = N, dim, p
        self.n = p + 1
        self.vertices = np.asarray(vertices, dtype=np.float64)
        assert self.vertices.shape == ((N + 1) ** dim, dim)
        self.nn1 = p * N + 1
        self.n_nodes = self.nn1 ** dim
        self.n_cells = N ** dim
        self.cells = lex_indices(N, dim)           # (ncells, dim)
        self.local = lex_indices(self.n, dim)      # (n^dim, dim)
        self.xq, self.wq = fe1d.gauss_legendre(self.n)
        self.qloc = lex_indices(self.n, dim)       # quadrature point multi-indices

    # ---- numbering ----
    def node_id(self, g: np.ndarray) -> np.ndarray:
        """Global node ids of integer node coordinates g (..., dim)."""
        idx = np.zeros(g.shape[:-1], dtype=np.int64)
        for d in reversed(range(self.dim)):
            idx = idx * self.nn1 + g[..., d]
        return idx

    def cell_dofs(self) -> np.ndarray:
        """(ncells, n^dim) global node ids of each cell's local nodes."""
        g = self.cells[:, None, :] * self.p + self.local[None, :, :]
        return self.node_id(g)

    def boundary_mask(self) -> np.ndarray:
        g = lex_indices(self.nn1, self.dim)
        return np.any((g == 0) | (g == self.nn1 - 1), axis=1)

    def vertex_id(self, v: np.ndarray) -> np.ndarray:
        idx = np.zeros(v.shape[:-1], dtype=np.int64)
        for d in reversed(range(self.dim)):
            idx = idx * (self.N + 1) + v[..., d]
        return idx

    # ---- Q1 geometry ----
    def cell_vertices(self, cells=None) -> np.ndarray:
        """(ncells, 2^dim, dim) vertex coordinates, vertex bits lexicographic (x fastest)."""
        bits = lex_indices(2, self.dim)
        cidx = self.cells if cells is None else self.cells[cells]
        vid = self.vertex_id(cidx[:, None, :] + bits[None, :, :])
        return self.vertices[vid]

    def q1_shape(self, xi: np.ndarray):
        """Multilinear shape values (m, 2^dim) and reference gradients (m, 2^dim, dim) at points xi (m, dim)."""
        bits = lex_indices(2, self.dim)
        m = xi.shape[0]
        val = np.ones((m, len(bits)))
        grad = np.ones((m, len(bits), self.dim))
        for v, b in enumerate(bits):
            for d in range(self.dim):
                f = xi[:, d] if b[d] else 1.0 - xi[:, d]
                df = 1.0 if b[d] else -1.0
                val[:, v] *= f
                for e in range(self.dim):
                    grad[:, v, e] *= df if e == d else f
        return val, grad

    def map_points(self, xi: np.ndarray) -> np.ndarray:
        """Physical coordinates (ncells, m, dim) of reference points xi (m, dim) in every cell."""
        val, _ = self.q1_shape(xi)
        return np.einsum("mv,cvd->cmd", val, self.cell_vertices())

    def jacobians(self, xi: np.ndarray, cells=None) -> np.ndarray:
        """J[c, m, d, e] = d x_d / d xi_e at reference points xi."""
        _, grad = self.q1_shape(xi)
        return np.einsum("mve,cvd->cmde", grad, self.cell_vertices(cells))

    def quad_points_ref(self) -> np.ndarray:
        return self.xq[self.qloc]                  # (nq^dim, dim)

    def quad_weights(self) -> np.ndarray:
        return np.prod(self.wq[self.qloc], axis=1)

    def quad_points_phys(self) -> np.ndarray:
        return self.map_points(self.quad_points_ref())

    def node_coords(self) -> np.ndarray:
        """(n_nodes, dim) physical coordinates of all global nodes (Q1 map of Gauss-Lobatto points)."""
        xn = fe1d.space_nodes(self.p)
        ref = xn[self.local]                       # (n^dim, dim)
        X = self.map_points(ref)                   # (ncells, n^dim, dim)
        out = np.zeros((self.n_nodes, self.dim))
        out[self.cell_dofs().reshape(-1)] = X.reshape(-1, self.dim)
        return out

    # ---- reference basis at quadrature points ----
    def ref_basis(self):
        """phi (nq, nb) and reference gradients (nq, nb, dim) of the Q_p basis at Gauss points."""
        xn = fe1d.space_nodes(self.p)
        V, D = fe1d.basis_table(xn, self.xq)       # (q1, j1)
        nq = len(self.qloc)
        nb = len(self.local)
        phi = np.ones((nq, nb))
        dphi = np.ones((nq, nb, self.dim))
        for d in range(self.dim):
            Vd = V[self.qloc[:, d]][:, self.local[:, d]]
            Dd = D[self.qloc[:, d]][:, self.local[:, d]]
            phi *= Vd
            for e in range(self.dim):
                dphi[:, :, e] *= Dd if e == d else Vd
        return phi, dphi

    # ---- element and global matrices ----
    def element_matrices(self, rho_qp: np.ndarray, cells=None):
        """A_e, M_e (ncells, nb, nb) by Gauss quadrature on the Q1-mapped cells (or a subset `cells`).

        A_e[a, b] = sum_q w_q |det J| rho_q (J^-T grad phi_a) . (J^-T grad phi_b)
        M_e[a, b] = sum_q w_q |det J| phi_a phi_b
        """
        phi, dphi = self.ref_basis()
        J = self.jacobians(self.quad_points_ref(), cells)  # (c, q, d, e)
        if cells is not None:
            rho_qp = rho_qp[cells]
        det = np.linalg.det(J)
        Jinv = np.linalg.inv(J)                            # (c, q, e, d)
        w = self.quad_weights()
        jw = np.abs(det) * w[None, :]
        # physical gradients: grad phi = J^-T grad_ref phi -> g[c,q,b,d] = sum_e Jinv[c,q,e,d] dphi[q,b,e]
        g = np.einsum("cqed,qbe->cqbd", Jinv, dphi)
        A = np.einsum("cq,cqad,cqbd->cab", jw * rho_qp, g, g)
        M = np.einsum("cq,qa,qb->cab", jw, phi, phi)
        return A, M

    def assemble(self, rho_qp: np.ndarray):
        """Global sparse A_h, M_h (all nodes, no boundary conditions)."""
        A_e, M_e = self.element_matrices(rho_qp)
        dofs = self.cell_dofs()
        nb = dofs.shape[1]
        rows = np.repeat(dofs, nb, axis=1).reshape(-1)
        cols = np.tile(dofs, (1, nb)).reshape(-1)
        shape = (self.n_nodes, self.n_nodes)
        A = sp.csr_matrix((A_e.reshape(-1), (rows, cols)), shape=shape)
        M = sp.csr_matrix((M_e.reshape(-1), (rows, cols)), shape=shape)
        return A, M


def rho_qp_from_cells(grid: Grid, rho_cell: np.ndarray) -> np.ndarray:
    """Per-cell coefficient broadcast to every quadrature point of the cell."""
    return np.repeat(np.asarray(rho_cell, dtype=np.float64)[:, None], grid.n ** grid.dim, axis=1)


def all_neighbour_offsets(dim: int):
    return list(itertools.product((-1, 0, 1), repeat=dim))
