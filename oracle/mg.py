"""Space-time multigrid on one slab: hierarchy, transfers, cell-wise additive Schwarz,
V-cycle, relaxation estimate and FGMRES, FP64, explicit sparse matrices.

Test infrastructure (see oracle/__init__.py).

Paper sections and the readings taken where it is silent:
  * hierarchy (Section 3, Algorithm mg-sequence, caption of Fig. stmg): coarsen
    space first -- p -> p-1 down to Q1, then halve the cells while N is even and
    N/2 >= 2 -- then time: k -> k-1 down to dG(0) / cGP(1); tau is kept (one slab).
  * coarse operators are rediscretised (each level has its own S_l).  The
    coefficient of a coarse level at a quadrature point is the cell mean of the
    finest-level coefficient in the finest cell that contains the point, located
    by logical (reference-grid) coordinates.
  * transfers (Section 3.2): prolongation = embedding of the coarse space in the
    fine one (the L2 projection for nested spaces), taken in reference
    coordinates of the structured grid, as a Kronecker product of 1D matrices in
    space and P_tau in time; for cGP only the free time DoFs take part (the
    constrained u_n^0 has zero correction).  Restriction = P^T.
  * smoother (eqs. vanka0, vanka): blocks = all unconstrained DoFs of one
    space-time cell (one spatial cell x all N_t time DoFs of the slab), local
    matrix = R_T S R_T^T of the global S (neighbour contributions included),
    solved exactly; u <- u + omega * sum_T R_T^T L_T^-1 R_T (f - S u).  Option
    (weighted=True, not in the printed eq. vanka0): each cell's correction at a node is
    divided by the number of cells that contain the node, sum_T R_T^T D_T L_T^-1 R_T
    with sum_T R_T^T D_T R_T = I (a partition of unity).
  * relaxation (eq. relaxation): omega = 2 / (lambda_max + lambda_min), with the
    extreme real parts of the Ritz values of an Arnoldi process on S_l B_l with
    min(20, number of unconstrained DoFs) steps from the counter-based start
    vector synth.splitmix_uniform(n, key=level); capped at 1, since the paper takes
    omega_l in (0, 1) (Section 3.3).
  * coarsest level: exact solve; no smoothing there (Algorithm stmg).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import synth
from . import fe1d, timeint
from .slab import SlabProblem
from .space import Grid


@dataclass
class LevelSpec:
    p: int
    N: int
    k: int


def level_unknowns(s: LevelSpec, dim: int, scheme: str) -> int:
    """Unconstrained space-time DoFs of a level: N_t times the interior nodes."""
    nt = s.k + 1 if scheme == timeint.DG else s.k
    return nt * (s.p * s.N - 1) ** dim


def level_sequence(p: int, N: int, k: int, scheme: str, p_coarsening: bool = True, coarse_max_dofs: int = 0,
                   dim: int = 3) -> list[LevelSpec]:
    """Fine-to-coarse list of (p, N, k): space first, then time (Algorithm mg-sequence).  With
    p_coarsening the space levels lower p one by one down to 1 before halving the cells; without it
    they keep p (h-multigrid only).  coarse_max_dofs > 0 ends the list at the first coarser level
    with at most that many unknowns (the coarsest level is solved exactly)."""
    seq = [LevelSpec(p, N, k)]
    while p_coarsening and seq[-1].p > 1:
        s = seq[-1]
        seq.append(LevelSpec(s.p - 1, s.N, s.k))
    while seq[-1].N % 2 == 0 and seq[-1].N // 2 >= 2:
        s = seq[-1]
        seq.append(LevelSpec(s.p, s.N // 2, s.k))
    kmin = 0 if scheme == timeint.DG else 1
    while seq[-1].k > kmin:
        s = seq[-1]
        seq.append(LevelSpec(s.p, s.N, s.k - 1))
    if coarse_max_dofs > 0:
        for i in range(1, len(seq)):
            if level_unknowns(seq[i], dim, scheme) <= coarse_max_dofs:
                return seq[:i + 1]
    return seq


def coarse_vertices(vertices: np.ndarray, N_f: int, N_c: int, dim: int) -> np.ndarray:
    """Vertices of the level with N_c cells: the fine vertices at every (N_f/N_c)-th index."""
    r = N_f // N_c
    idx = np.indices((N_c + 1,) * dim).reshape(dim, -1)[::-1].T * r
    vid = np.zeros(len(idx), dtype=np.int64)
    for d in reversed(range(dim)):
        vid = vid * (N_f + 1) + idx[:, d]
    return vertices[vid]


def level_rho_qp(grid: Grid, fine_cell_mean: np.ndarray, N_f: int) -> np.ndarray:
    """Coefficient at each quadrature point of `grid` from the finest-level cell means."""
    ref = grid.quad_points_ref()                          # (q, dim)
    s = (grid.cells[:, None, :] + ref[None, :, :]) / grid.N   # logical coordinates in [0,1]
    fc = np.minimum(np.floor(s * N_f).astype(np.int64), N_f - 1)
    fid = np.zeros(fc.shape[:-1], dtype=np.int64)
    for d in reversed(range(grid.dim)):
        fid = fid * N_f + fc[..., d]
    return fine_cell_mean[fid]


def space_prolongation_1d(p_f: int, N_f: int, p_c: int, N_c: int) -> np.ndarray:
    """P1[g_f, g_c] = coarse global 1D Lagrange function g_c at the logical position of fine node g_f."""
    xf = fe1d.space_nodes(p_f)
    xc = fe1d.space_nodes(p_c)
    nf, nc = p_f * N_f + 1, p_c * N_c + 1
    P = np.zeros((nf, nc))
    for cf in range(N_f):
        for a in range(p_f + 1):
            gf = cf * p_f + a
            s = (cf + xf[a]) / N_f                   # logical position in [0, 1]
            cc = min(int(np.floor(s * N_c)), N_c - 1)
            xi = s * N_c - cc
            for b in range(p_c + 1):
                P[gf, cc * p_c + b] = fe1d.lagrange(xc, b, xi)
    P[np.abs(P) < 1e-15] = 0.0
    return P


def time_prolongation(scheme: str, k_f: int, k_c: int) -> np.ndarray:
    """P_tau[i_f, j_c]: coarse time basis function j_c at fine free node i_f."""
    if scheme == timeint.DG:
        nf = fe1d.gauss_radau_right(k_f + 1)[0]
        nc = fe1d.gauss_radau_right(k_c + 1)[0]
        return np.array([[fe1d.lagrange(nc, j, t) for j in range(len(nc))] for t in nf])
    nf = fe1d.gauss_lobatto(k_f + 1)[0][1:]
    nc_all = fe1d.gauss_lobatto(k_c + 1)[0]
    return np.array([[fe1d.lagrange(nc_all, j, t) for j in range(1, len(nc_all))] for t in nf])


@dataclass
class Level:
    spec: LevelSpec
    grid: Grid
    prob: SlabProblem
    omega: float = 1.0
    P: sp.csr_matrix | None = None      # prolongation from the next coarser level into this one
    B: sp.csr_matrix | None = None      # additive Schwarz operator sum_T R_T^T L_T^-1 R_T
    coarse_inv: np.ndarray | None = None
    interior: np.ndarray = field(default=None)


def node_multiplicity(grid: Grid) -> np.ndarray:
    """Number of cells that contain each node."""
    m = np.zeros(grid.n_nodes)
    for c in grid.cell_dofs():
        m[c] += 1.0
    return m


def asm_operator(prob: SlabProblem, weighted: bool = False) -> sp.csr_matrix:
    """sum over spatial cells T of R_T^T [R_T S R_T^T]^-1 R_T  (eq. vanka0), unconstrained DoFs only;
    weighted: rows scaled by the inverse node multiplicity (partition of unity over the cells)."""
    g = prob.grid
    dofs = g.cell_dofs()
    S = prob.S.tocsr()
    nn = g.n_nodes
    rows, cols, vals = [], [], []
    for c in range(g.n_cells):
        nodes = dofs[c][~prob.bmask[dofs[c]]]
        if len(nodes) == 0:
            continue
        idx = (np.arange(prob.nt)[:, None] * nn + nodes[None, :]).reshape(-1)
        L = S[idx][:, idx].toarray()
        Li = np.linalg.inv(L)
        rows.append(np.repeat(idx, len(idx)))
        cols.append(np.tile(idx, len(idx)))
        vals.append(Li.reshape(-1))
    n = prob.n
    B = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    if weighted:
        B = (sp.diags(np.tile(1.0 / node_multiplicity(g), prob.nt)) @ B).tocsr()
    return B


def arnoldi_ritz(matvec, v0: np.ndarray, m: int) -> np.ndarray:
    """Ritz values of an m-step Arnoldi process started at v0.

    Gram-Schmidt is applied twice per step (modified Gram-Schmidt with one full
    reorthogonalisation), so that the basis stays orthonormal to rounding even
    when the Krylov space is exhausted; a single pass can lose orthogonality and
    produce spurious Ritz values.
    """
    n = len(v0)
    m = min(m, n)
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    V[0] = v0 / np.linalg.norm(v0)
    steps = m
    for j in range(m):
        w = matvec(V[j])
        for _ in range(2):
            for i in range(j + 1):
                c = np.dot(V[i], w)
                H[i, j] += c
                w = w - c * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-14 * abs(H[j, j]) + 1e-300:
            steps = j + 1
            break
        V[j + 1] = w / H[j + 1, j]
    return np.linalg.eigvals(H[:steps, :steps])


def estimate_omega(prob: SlabProblem, B: sp.csr_matrix, key: int, steps: int = 20) -> float:
    v0 = synth.splitmix_uniform(prob.n, key=key)
    v0[prob.bmask_full] = 0.0
    # the Krylov space lives on the unconstrained DoFs: at most that many steps
    steps = min(steps, int((~prob.bmask_full).sum()))
    ritz = arnoldi_ritz(lambda v: prob.S @ (B @ v), v0, steps)
    re = np.real(ritz)
    re = re[np.abs(ritz) > 1e-12]
    return float(min(1.0, 2.0 / (re.max() + re.min())))


class Hierarchy:
    """All levels of the STMG V-cycle for one slab problem (finest level first)."""

    def __init__(self, dim, N, p, k, pde, scheme, tau, vertices, rho_cell=None, rho_qp=None,
                 omegas=None, estimate=True, p_coarsening=True, coarse_max_dofs=0, weighted=False):
        self.specs = level_sequence(p, N, k, scheme, p_coarsening, coarse_max_dofs, dim)
        self.pde, self.scheme = pde, scheme
        fine = Grid(N, dim, p, vertices)
        if rho_qp is None:
            rho_cell = np.ones(fine.n_cells) if rho_cell is None else np.asarray(rho_cell, np.float64)
            fine_rho_qp = np.repeat(rho_cell[:, None], fine.n ** dim, axis=1)
            cell_mean = rho_cell
        else:
            fine_rho_qp = np.asarray(rho_qp, np.float64)
            cell_mean = fine_rho_qp.mean(axis=1)
        self.levels: list[Level] = []
        for li, s in enumerate(self.specs):
            if li == 0:
                grid, rq = fine, fine_rho_qp
            else:
                grid = Grid(s.N, dim, s.p, coarse_vertices(vertices, N, s.N, dim))
                rq = level_rho_qp(grid, cell_mean, N)
            prob = SlabProblem(grid, rq, pde, scheme, s.k, tau)
            lev = Level(s, grid, prob)
            lev.interior = ~prob.bmask_full
            self.levels.append(lev)
        # transfers: level li is prolongated from level li+1
        for li in range(len(self.levels) - 1):
            f, c = self.levels[li], self.levels[li + 1]
            Px = np.ones((1, 1))
            for _ in range(dim):
                Px = np.kron(space_prolongation_1d(f.spec.p, f.spec.N, c.spec.p, c.spec.N), Px)
            Pt = time_prolongation(scheme, f.spec.k, c.spec.k)
            P = sp.kron(sp.csr_matrix(Pt), sp.csr_matrix(Px))
            Df = sp.diags(f.interior.astype(np.float64))
            Dc = sp.diags(c.interior.astype(np.float64))
            f.P = (Df @ P @ Dc).tocsr()
        for li, lev in enumerate(self.levels[:-1]):
            lev.B = asm_operator(lev.prob, weighted)
            if omegas is not None:
                lev.omega = float(omegas[li])
            elif estimate:
                lev.omega = estimate_omega(lev.prob, lev.B, key=li)
        last = self.levels[-1]
        Si = last.prob.S.toarray()
        last.coarse_inv = np.linalg.inv(Si)

    def omegas(self):
        return [lev.omega for lev in self.levels[:-1]]

    def smooth(self, li: int, f: np.ndarray, u: np.ndarray, sweeps: int) -> np.ndarray:
        lev = self.levels[li]
        for _ in range(sweeps):
            u = u + lev.omega * (lev.B @ (f - lev.prob.S @ u))
        return u

    def vcycle(self, f: np.ndarray, li: int = 0, nu1: int = 1, nu2: int = 1) -> np.ndarray:
        """Algorithm stmg with zero initial guess; f and the result are flat vectors."""
        lev = self.levels[li]
        if li == len(self.levels) - 1:
            return lev.coarse_inv @ f
        u = self.smooth(li, f, np.zeros_like(f), nu1)
        r = f - lev.prob.S @ u
        e = self.vcycle(lev.P.T @ r, li + 1, nu1, nu2)
        u = u + lev.P @ e
        return self.smooth(li, f, u, nu2)


@dataclass
class FgmresResult:
    x: np.ndarray
    iterations: int
    rel_residual: float
    history: list


def fgmres(matvec, precond, b: np.ndarray, x0: np.ndarray, rtol: float = 1e-10, restart: int = 30,
           max_it: int = 200) -> FgmresResult:
    """Right-preconditioned flexible GMRES (Saad 1993) with modified Gram-Schmidt.

    Stops when ||b - A x||_2 <= rtol ||b||_2 (true residual checked at every restart/exit).
    """
    x = x0.astype(np.float64).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return FgmresResult(np.zeros_like(b), 0, 0.0, [0.0])
    its = 0
    hist = []
    while True:
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta <= rtol * bnorm or its >= max_it:
            return FgmresResult(x, its, beta / bnorm, hist)
        m = restart
        V = np.zeros((m + 1, len(b)))
        Z = np.zeros((m, len(b)))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        g = np.zeros(m + 1)
        g[0] = beta
        cs, sn = np.zeros(m), np.zeros(m)
        j_end = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) <= rtol * bnorm or its >= max_it:
                break
        y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        x = x + Z[:j_end].T @ y
