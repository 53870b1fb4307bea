"""Slab systems on the full node vector, their right-hand sides and direct solves, FP64.

Test infrastructure (see oracle/__init__.py).

Paper: eqs. heat-cg-dg, heat-cg-cg, wave-cg-dg, wave-cg-cg (one slab, n_c = 1),
Section 4.1 eq. norms (L2(L2) error).  Vectors hold all nodes of every time
DoF, layout (N_t, n_nodes); homogeneous Dirichlet nodes are constrained:
  * the operator acts as the identity on constrained rows and ignores
    constrained columns;
  * right-hand sides are zero on constrained rows.
The source enters as its nodal interpolant at the space-time nodes
(reading of eq. heat-cg-dg's f_n: the printed (f, w_j) would count M_h twice).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe1d, timeint
from .space import Grid


def constrain(S: sp.spmatrix, bmask_full: np.ndarray) -> sp.csr_matrix:
    """Zero constrained rows and columns of S and put 1 on their diagonal."""
    keep = sp.diags((~bmask_full).astype(np.float64))
    ident = sp.diags(bmask_full.astype(np.float64))
    return (keep @ S @ keep + ident).tocsr()


class SlabProblem:
    """One slab system S u = rhs on grid `grid` with coefficient rho at quadrature points."""

    def __init__(self, grid: Grid, rho_qp: np.ndarray, pde: str, scheme: str, k: int, tau: float):
        self.grid = grid
        self.sys = timeint.slab_system(pde, scheme, k, tau)
        self.nt = self.sys.tw.nt
        self.A, self.M = grid.assemble(rho_qp)
        self.bmask = grid.boundary_mask()
        self.bmask_full = np.tile(self.bmask, self.nt)
        S = sp.kron(self.sys.TA, self.A) + sp.kron(self.sys.TM, self.M)
        self.S = constrain(S, self.bmask_full)
        self._lu = None

    @property
    def n(self) -> int:
        return self.nt * self.grid.n_nodes

    def apply(self, x: np.ndarray) -> np.ndarray:
        return (self.S @ x.reshape(-1)).reshape(self.nt, -1)

    def rhs(self, f, f0=None, u0=None, v0=None) -> np.ndarray:
        """Right-hand side from nodal source values f (N_t, n_nodes) and previous-slab end values."""
        s = self.sys
        nn = self.grid.n_nodes
        z = np.zeros(nn)
        f0 = z if f0 is None else f0
        u0 = z if u0 is None else u0
        v0 = z if v0 is None else v0
        out = (sp.kron(s.RM_f, self.M) @ np.asarray(f).reshape(-1)).reshape(self.nt, nn)
        out += np.outer(s.RM_f0, self.M @ f0)
        out += np.outer(s.RA_u0, self.A @ u0)
        out += np.outer(s.RM_u0, self.M @ u0)
        out += np.outer(s.RM_v0, self.M @ v0)
        out[:, self.bmask] = 0.0
        return out

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        if self._lu is None:
            self._lu = spla.splu(self.S.tocsc())
        return self._lu.solve(rhs.reshape(-1)).reshape(self.nt, -1)

    def velocity(self, u, u0, v0) -> np.ndarray:
        """Wave only: v = VU u + Vu0 u0 + Vv0 v0 (eqs. wave-cg-dg-ade / wave-cg-cg-ade)."""
        s = self.sys
        return s.VU @ u + np.outer(s.Vu0, u0) + np.outer(s.Vv0, v0)


def time_nodes_for_source(scheme: str, k: int) -> tuple[np.ndarray, bool]:
    """Reference time nodes at which f is sampled: (free nodes, whether f0 at t^=0 is needed)."""
    if scheme == timeint.DG:
        return fe1d.gauss_radau_right(k + 1)[0], False
    return fe1d.gauss_lobatto(k + 1)[0][1:], True


def march(prob: SlabProblem, n_slabs: int, source, u_init=None, v_init=None, t0=0.0):
    """Time marching with direct slab solves; returns list of slab solutions (and velocities for wave).

    source(x, t) -> nodal values (may be None for f = 0).
    """
    g = prob.grid
    X = g.node_coords()
    s = prob.sys
    tnodes, need_f0 = time_nodes_for_source(s.tw.scheme, s.tw.k)
    u_prev = np.zeros(g.n_nodes) if u_init is None else u_init.copy()
    v_prev = np.zeros(g.n_nodes) if v_init is None else v_init.copy()
    sols, vels = [], []
    for n in range(n_slabs):
        ts = t0 + n * s.tau
        if source is None:
            f = np.zeros((prob.nt, g.n_nodes))
            f0 = np.zeros(g.n_nodes)
        else:
            f = np.stack([source(X, ts + s.tau * th) for th in tnodes])
            f0 = source(X, ts)
        rhs = prob.rhs(f, f0 if need_f0 else None, u_prev,
                       v_prev if prob.sys.pde == timeint.WAVE else None)
        u = prob.solve(rhs)
        sols.append(u)
        if prob.sys.pde == timeint.WAVE:
            v = prob.velocity(u, u_prev, v_prev)
            v[:, prob.bmask] = 0.0
            vels.append(v)
            v_prev = v[-1].copy()
        u_prev = u[-1].copy()
    return sols, vels


def l2l2_error(prob: SlabProblem, sols, exact, u_init, t0=0.0) -> float:
    """||u - u_h||_{L2(0,T; L2)} by space-time Gauss quadrature (p+2 per direction, k+2 in time)."""
    g = prob.grid
    s = prob.sys
    # spatial quadrature one order above the discretisation rule
    xq, wq = fe1d.gauss_legendre(g.p + 2)
    from .space import lex_indices
    ql = lex_indices(len(xq), g.dim)
    ref = xq[ql]
    wts = np.prod(wq[ql], axis=1)
    xn = fe1d.space_nodes(g.p)
    V, _ = fe1d.basis_table(xn, xq)
    phi = np.ones((len(ref), g.n ** g.dim))
    for d in range(g.dim):
        phi *= V[ql[:, d]][:, g.local[:, d]]
    J = g.jacobians(ref)
    jw = np.abs(np.linalg.det(J)) * wts[None, :]
    Xq = g.map_points(ref)                       # (c, q, d)
    dofs = g.cell_dofs()
    tq, wtq = fe1d.gauss_legendre(s.tw.k + 3)
    if s.tw.scheme == timeint.DG:
        tn = s.tw.nodes
    else:
        tn = fe1d.gauss_lobatto(s.tw.k + 1)[0]
    Tb, _ = fe1d.basis_table(tn, tq)             # (tq, nodes)
    err2 = 0.0
    u_prev = u_init
    for n, u in enumerate(sols):
        coeffs = u if s.tw.scheme == timeint.DG else np.vstack([u_prev[None, :], u])
        for it, th in enumerate(tq):
            t = t0 + (n + th) * s.tau
            uh_nodal = Tb[it] @ coeffs                 # (n_nodes,)
            uh = np.einsum("qa,ca->cq", phi, uh_nodal[dofs])
            ue = exact(Xq, t)
            err2 += s.tau * wtq[it] * np.sum(jw * (uh - ue) ** 2)
        u_prev = u[-1]
    return float(np.sqrt(err2))


def sampled_rows(grid: Grid, rho_qp: np.ndarray, pde: str, scheme: str, k: int, tau: float,
                 x: np.ndarray, samples) -> np.ndarray:
    """(S x)[t, node] for a list of (t, node) pairs, from the element matrices of the touching cells only.

    Same definition as SlabProblem.S (identity on constrained rows, constrained columns ignored),
    for grids too large to assemble.  x has shape (N_t, n_nodes).
    """
    sysm = timeint.slab_system(pde, scheme, k, tau)
    nn1, p, N, dim = grid.nn1, grid.p, grid.N, grid.dim
    bmask = grid.boundary_mask()
    xm = np.where(bmask[None, :], 0.0, x)
    out = []
    for t, node in samples:
        if bmask[node]:
            out.append(x[t, node])
            continue
        g = [(node // nn1 ** d) % nn1 for d in range(dim)]
        cands = [[] for _ in range(dim)]
        for d in range(dim):
            c0 = g[d] // p
            cands[d] = sorted({c for c in (c0 - 1, c0) if 0 <= c < N and c * p <= g[d] <= (c + 1) * p})
        cells = np.array([sum(c[d] * N ** d for d in range(dim)) for c in itertools.product(*cands)])
        A_e, M_e = grid.element_matrices(rho_qp, cells=cells)
        dofs = grid.node_id(grid.cells[cells][:, None, :] * p + grid.local[None, :, :])
        val = 0.0
        for ci in range(len(cells)):
            a = int(np.nonzero(dofs[ci] == node)[0][0])
            for j in range(sysm.tw.nt):
                xl = xm[j, dofs[ci]]
                val += sysm.TA[t, j] * (A_e[ci, a] @ xl) + sysm.TM[t, j] * (M_e[ci, a] @ xl)
        out.append(val)
    return np.array(out)


def kron_apply(grid: Grid, rho_qp: np.ndarray, TA: np.ndarray, TM: np.ndarray, x: np.ndarray,
               constrained: bool = True, A_e=None, M_e=None) -> np.ndarray:
    """y = (TA (x) A_h + TM (x) M_h) x cell by cell from element matrices (no global assembly).

    TA, TM: (n_out, n_in); x: (n_in, n_nodes).  constrained=True gives the slab operator
    convention (identity on constrained rows, constrained columns ignored, needs n_in == n_out);
    constrained=False applies the plain matrices and zeroes constrained rows (right-hand sides).
    """
    if A_e is None:
        A_e, M_e = grid.element_matrices(rho_qp)
    dofs = grid.cell_dofs()
    bmask = grid.boundary_mask()
    xm = np.where(bmask[None, :], 0.0, x) if constrained else x
    xc = xm[:, dofs]                                    # (n_in, cells, nb)
    yA = np.einsum("cab,jcb->jca", A_e, xc)
    yM = np.einsum("cab,jcb->jca", M_e, xc)
    yc = np.einsum("ij,jca->ica", TA, yA) + np.einsum("ij,jca->ica", TM, yM)
    y = np.zeros((TA.shape[0], grid.n_nodes))
    for i in range(TA.shape[0]):
        y[i] = np.bincount(dofs.reshape(-1), weights=yc[i].reshape(-1), minlength=grid.n_nodes)
    if constrained:
        y[:, bmask] = x[:, bmask]
    else:
        y[:, bmask] = 0.0
    return y
