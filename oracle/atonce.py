"""Several consecutive slabs in one system and tau-multigrid, heat equation, dG(k) in time, FP64.

Test infrastructure (see oracle/__init__.py).

Paper: eq. heat-cg-dg-at-once (Section 2.1).  n_c consecutive slabs form one block
lower-bidiagonal system: the slab operator S on the diagonal and -B below it, where
B = 1_{k+1} (x) alpha (x) M_h couples slab i to the last time DoF of slab i-1 (the jump term that a
single slab takes from its right-hand side).  The first slab's right-hand side keeps the term
alpha (x) M_h u_0 of the previous end value.  Constrained rows and columns of B are zero, as for S.

tau-multigrid (Algorithm mg-sequence, mgType tau): two consecutive slabs of length tau become one
coarse slab of length 2 tau.  The prolongation is the embedding of the coarse dG(k) space: on fine
slab 2j + h (h = 0, 1) a coarse time basis function of slab j is evaluated at the fine Radau nodes
mapped into half h of the coarse reference interval.  Restriction = transpose.

Hierarchy (reading of Algorithm mg-sequence for n_c > 1): space levels as for one slab (p, then h),
then tau levels while the number of slabs is even and at least 2, then k levels.  The additive
Schwarz smoother of an at-once level is block diagonal over the slabs: every space-time cell lies in
one slab, and R_T of the at-once matrix restricted to that cell is the slab block S restricted.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe1d, mg, timeint
from .slab import SlabProblem
from .space import Grid


class AtOnceProblem:
    """n_c slabs of the heat equation with dG(k) in time in one system (eq. heat-cg-dg-at-once)."""

    def __init__(self, grid: Grid, rho_qp: np.ndarray, k: int, tau: float, nc: int):
        self.slab = SlabProblem(grid, rho_qp, timeint.HEAT, timeint.DG, k, tau)
        self.grid, self.nc, self.nt = grid, nc, self.slab.nt
        alpha = self.slab.sys.RM_u0          # heat dG: alpha, the slab's coefficient of M_h u_0
        C = np.zeros((self.nt, self.nt))
        C[:, self.nt - 1] = alpha
        keep = sp.diags((~self.slab.bmask_full).astype(np.float64))
        self.Bc = (keep @ sp.kron(C, self.slab.M) @ keep).tocsr()
        blocks = [[None] * nc for _ in range(nc)]
        for i in range(nc):
            blocks[i][i] = self.slab.S
            if i > 0:
                blocks[i][i - 1] = -self.Bc
        self.S = sp.bmat(blocks, format="csr")
        self.bmask_full = np.tile(self.slab.bmask_full, nc)
        self._lu = None

    @property
    def n(self) -> int:
        return self.nc * self.slab.n

    def rhs(self, fs, u0) -> np.ndarray:
        """fs: (n_c, N_t, n_nodes) nodal source values; u0: end value before the first slab."""
        out = np.stack([self.slab.rhs(fs[i], None, u0 if i == 0 else None) for i in range(self.nc)])
        return out

    def solve(self, rhs: np.ndarray) -> np.ndarray:
        if self._lu is None:
            self._lu = spla.splu(self.S.tocsc())
        return self._lu.solve(rhs.reshape(-1)).reshape(self.nc, self.nt, -1)


def tau_prolongation(k: int) -> np.ndarray:
    """P[h, t, j]: coarse dG(k) basis function j at fine Radau node t of half h of the coarse slab."""
    nodes = fe1d.gauss_radau_right(k + 1)[0]
    P = np.zeros((2, len(nodes), len(nodes)))
    for h in range(2):
        for t, th in enumerate(nodes):
            for j in range(len(nodes)):
                P[h, t, j] = fe1d.lagrange(nodes, j, 0.5 * (h + th))
    return P


@dataclass
class AtOnceSpec:
    p: int
    N: int
    k: int
    nc: int
    tau: float


def level_sequence(p: int, N: int, k: int, nc: int, tau: float) -> list[AtOnceSpec]:
    """Fine-to-coarse levels: space (p, then h), then tau (halving n_c), then k."""
    seq = [AtOnceSpec(s.p, s.N, s.k, nc, tau) for s in mg.level_sequence(p, N, k, timeint.DG)
           if s.k == k]
    while seq[-1].nc % 2 == 0 and seq[-1].nc >= 2:
        s = seq[-1]
        seq.append(AtOnceSpec(s.p, s.N, s.k, s.nc // 2, 2 * s.tau))
    while seq[-1].k > 0:
        s = seq[-1]
        seq.append(AtOnceSpec(s.p, s.N, s.k - 1, s.nc, s.tau))
    return seq


@dataclass
class AtOnceLevel:
    spec: AtOnceSpec
    prob: AtOnceProblem
    omega: float = 1.0
    P: sp.csr_matrix | None = None
    B: sp.csr_matrix | None = None
    coarse_inv: np.ndarray | None = None


class AtOnceHierarchy:
    """V-cycle (Algorithm stmg) for the at-once system, finest level first."""

    def __init__(self, dim, N, p, k, tau, nc, vertices, rho_cell=None, omegas=None, estimate=True, weighted=False):
        self.specs = level_sequence(p, N, k, nc, tau)
        fine = Grid(N, dim, p, vertices)
        rho_cell = np.ones(fine.n_cells) if rho_cell is None else np.asarray(rho_cell, np.float64)
        self.levels: list[AtOnceLevel] = []
        for li, s in enumerate(self.specs):
            if li == 0:
                grid = fine
                rq = np.repeat(rho_cell[:, None], fine.n ** dim, axis=1)
            else:
                grid = Grid(s.N, dim, s.p, mg.coarse_vertices(vertices, N, s.N, dim))
                rq = mg.level_rho_qp(grid, rho_cell, N)
            self.levels.append(AtOnceLevel(s, AtOnceProblem(grid, rq, s.k, s.tau, s.nc)))
        for li in range(len(self.levels) - 1):
            f, c = self.levels[li], self.levels[li + 1]
            fs, cs = f.spec, c.spec
            nnf = f.prob.grid.n_nodes
            if cs.nc != fs.nc:                       # tau level
                Pt = tau_prolongation(fs.k)
                T = np.zeros((fs.nc * f.prob.nt, cs.nc * c.prob.nt))
                for s_ in range(fs.nc):
                    j, h = s_ // 2, s_ % 2
                    T[s_ * f.prob.nt:(s_ + 1) * f.prob.nt, j * c.prob.nt:(j + 1) * c.prob.nt] = Pt[h]
                P = sp.kron(sp.csr_matrix(T), sp.identity(nnf))
            else:
                Px = np.ones((1, 1))
                for _ in range(dim):
                    Px = np.kron(mg.space_prolongation_1d(fs.p, fs.N, cs.p, cs.N), Px)
                Pk = mg.time_prolongation(timeint.DG, fs.k, cs.k)
                P = sp.kron(sp.identity(fs.nc), sp.kron(sp.csr_matrix(Pk), sp.csr_matrix(Px)))
            Df = sp.diags((~f.prob.bmask_full).astype(np.float64))
            Dc = sp.diags((~c.prob.bmask_full).astype(np.float64))
            f.P = (Df @ P @ Dc).tocsr()
        for li, lev in enumerate(self.levels[:-1]):
            lev.B = sp.kron(sp.identity(lev.spec.nc), mg.asm_operator(lev.prob.slab, weighted)).tocsr()
            if omegas is not None:
                lev.omega = float(omegas[li])
            elif estimate:
                lev.omega = mg.estimate_omega(lev.prob, lev.B, key=li)
        self.levels[-1].coarse_inv = np.linalg.inv(self.levels[-1].prob.S.toarray())

    def omegas(self):
        return [lev.omega for lev in self.levels[:-1]]

    def vcycle(self, f: np.ndarray, li: int = 0, nu1: int = 1, nu2: int = 1) -> np.ndarray:
        lev = self.levels[li]
        if li == len(self.levels) - 1:
            return lev.coarse_inv @ f
        S = lev.prob.S
        u = np.zeros_like(f)
        for _ in range(nu1):
            u = u + lev.omega * (lev.B @ (f - S @ u))
        e = self.vcycle(lev.P.T @ (f - S @ u), li + 1, nu1, nu2)
        u = u + lev.P @ e
        for _ in range(nu2):
            u = u + lev.omega * (lev.B @ (f - S @ u))
        return u
