"""Pins of the oracle's multigrid pieces: transfers, additive Schwarz, V-cycle, relaxation, FGMRES."""
import numpy as np
import scipy.sparse as sp
import pytest

import synth
from oracle import fe1d, mg, slab, space, timeint


def test_level_sequence_space_then_time():
    seq = [(s.p, s.N, s.k) for s in mg.level_sequence(2, 32, 2, "dg")]
    assert seq == [(2, 32, 2), (1, 32, 2), (1, 16, 2), (1, 8, 2), (1, 4, 2), (1, 2, 2), (1, 2, 1), (1, 2, 0)]
    seq = [(s.p, s.N, s.k) for s in mg.level_sequence(3, 24, 2, "cgp")]
    assert seq == [(3, 24, 2), (2, 24, 2), (1, 24, 2), (1, 12, 2), (1, 6, 2), (1, 3, 2), (1, 3, 1)]
    # spatial levels that keep p (h-multigrid only), then time
    seq = [(s.p, s.N, s.k) for s in mg.level_sequence(2, 32, 2, "dg", p_coarsening=False)]
    assert seq == [(2, 32, 2), (2, 16, 2), (2, 8, 2), (2, 4, 2), (2, 2, 2), (2, 2, 1), (2, 2, 0)]
    # shallower hierarchy: ends at the first coarser level with <= 1500 unknowns (Q1 8^3 dG(2): 3 * 7^3)
    seq = [(s.p, s.N, s.k) for s in mg.level_sequence(2, 32, 2, "dg", coarse_max_dofs=1500)]
    assert seq == [(2, 32, 2), (1, 32, 2), (1, 16, 2), (1, 8, 2)]
    assert mg.level_unknowns(mg.LevelSpec(1, 8, 2), 3, "dg") == 1029
    # the finest level never becomes the coarsest
    seq = [(s.p, s.N, s.k) for s in mg.level_sequence(1, 4, 0, "dg", coarse_max_dofs=4096)]
    assert seq == [(1, 4, 0), (1, 2, 0)]


@pytest.mark.parametrize("pf,Nf,pc,Nc", [(2, 4, 1, 4), (3, 3, 2, 3), (1, 8, 1, 4), (2, 4, 2, 2)])
def test_space_prolongation_reproduces_coarse_polynomials(pf, Nf, pc, Nc):
    P = mg.space_prolongation_1d(pf, Nf, pc, Nc)
    # coarse nodal values of a polynomial of degree pc (piecewise exact) -> fine nodal values
    xf = np.concatenate([(c + fe1d.space_nodes(pf)[:-1]) / Nf for c in range(Nf)] + [[1.0]])
    xc = np.concatenate([(c + fe1d.space_nodes(pc)[:-1]) / Nc for c in range(Nc)] + [[1.0]])
    q = lambda x: 0.3 + x - 2.0 * x ** pc
    assert np.allclose(P @ q(xc), q(xf), atol=1e-13)
    assert np.allclose(P.sum(axis=1), 1.0)


@pytest.mark.parametrize("scheme,kf,kc", [("dg", 2, 1), ("dg", 1, 0), ("cgp", 2, 1), ("cgp", 3, 2)])
def test_time_prolongation_reproduces_polynomials(scheme, kf, kc):
    Pt = mg.time_prolongation(scheme, kf, kc)
    if scheme == "dg":
        tf = fe1d.gauss_radau_right(kf + 1)[0]
        tc = fe1d.gauss_radau_right(kc + 1)[0]
        q = lambda t: sum((0.5 + j) * t ** j for j in range(kc + 1))
        assert np.allclose(Pt @ q(tc), q(tf))
    else:
        # corrections vanish at t^=0 (the constrained DoF): reproduce t * poly of degree kc-1
        tf = fe1d.gauss_lobatto(kf + 1)[0][1:]
        tc = fe1d.gauss_lobatto(kc + 1)[0][1:]
        q = lambda t: t * (1.0 + 0.5 * t ** (kc - 1))
        assert np.allclose(Pt @ q(tc), q(tf))


def _explicit_asm_by_coordinates(prob):
    """ASM built from scratch: blocks = unconstrained nodes inside each closed cell (by logical node coords)."""
    g = prob.grid
    gl = space.lex_indices(g.nn1, g.dim)
    S = prob.S.toarray()
    n = prob.n
    B = np.zeros((n, n))
    for c in g.cells:
        inside = np.all((gl >= c * g.p) & (gl <= (c + 1) * g.p), axis=1) & ~prob.bmask
        nodes = np.nonzero(inside)[0]
        R = np.zeros((prob.nt * len(nodes), n))
        for t in range(prob.nt):
            for a, node in enumerate(nodes):
                R[t * len(nodes) + a, t * g.n_nodes + node] = 1.0
        B += R.T @ np.linalg.solve(R @ S @ R.T, R)
    return B


def test_asm_operator_brute_force_and_closed_form():
    V = synth.jittered_vertices(3, 2)
    g = space.Grid(3, 2, 2, V)
    prob = slab.SlabProblem(g, space.rho_qp_from_cells(g, synth.block_coefficient(3, 2, blocks=3)), "heat", "dg", 1, 0.1)
    B = mg.asm_operator(prob).toarray()
    assert np.abs(B - _explicit_asm_by_coordinates(prob)).max() < 1e-12 * np.abs(B).max()
    # Q1 on 2x2 cells: one unconstrained node shared by all four cells -> B S = 4 I on it (dG(0))
    g = space.Grid(2, 2, 1, synth.jittered_vertices(2, 2))
    prob = slab.SlabProblem(g, space.rho_qp_from_cells(g, np.ones(4)), "heat", "dg", 0, 0.1)
    B = mg.asm_operator(prob)
    c = 4  # centre node of the 3x3 node grid
    assert np.isclose((B @ prob.S)[c, c], 4.0)


def _multiplicity_by_coordinates(g):
    """cells containing each node, from logical coordinates: a factor 2 per direction in which the
    node lies on an interior cell face (index a multiple of p, not on the domain boundary)"""
    gl = space.lex_indices(g.nn1, g.dim)
    shared = (gl % g.p == 0) & (gl > 0) & (gl < g.nn1 - 1)
    return np.prod(np.where(shared, 2.0, 1.0), axis=1)


@pytest.mark.parametrize("dim,N,p", [(2, 3, 2), (3, 2, 2), (2, 4, 1)])
def test_weighted_asm_is_a_partition_of_unity_and_matches_brute_force(dim, N, p):
    g = space.Grid(N, dim, p, synth.jittered_vertices(N, dim))
    prob = slab.SlabProblem(g, space.rho_qp_from_cells(g, synth.block_coefficient(N, dim, blocks=1)), "heat", "dg",
                            1, 0.1)
    m = _multiplicity_by_coordinates(g)
    inner = ~prob.bmask
    assert np.array_equal(mg.node_multiplicity(g)[inner], m[inner])
    # sum_T R_T^T D_T R_T = I on the unconstrained nodes
    pu = np.zeros(g.n_nodes)
    for c in g.cell_dofs():
        pu[c] += 1.0 / m[c]
    assert np.allclose(pu[inner], 1.0)
    Bw = mg.asm_operator(prob, weighted=True).toarray()
    ref = np.tile(1.0 / m, prob.nt)[:, None] * _explicit_asm_by_coordinates(prob)
    assert np.abs(Bw - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("dim,k", [(2, 0), (3, 1), (2, 2)])
def test_weighted_asm_is_exact_when_every_cell_holds_all_unknowns(dim, k):
    """Q1 on 2^dim cells: the one unconstrained node lies in every cell, each cell block is the whole
    unconstrained system, and the weighted sum is its inverse: B S = I there (the plain sum gives 2^dim I)."""
    g = space.Grid(2, dim, 1, synth.jittered_vertices(2, dim))
    prob = slab.SlabProblem(g, space.rho_qp_from_cells(g, np.ones(2 ** dim)), "heat", "dg", k, 0.1)
    inner = ~prob.bmask_full
    BS = (mg.asm_operator(prob, weighted=True) @ prob.S).toarray()[np.ix_(inner, inner)]
    assert np.allclose(BS, np.eye(inner.sum()), atol=1e-12)
    BS0 = (mg.asm_operator(prob) @ prob.S).toarray()[np.ix_(inner, inner)]
    assert np.allclose(BS0, 2 ** dim * np.eye(inner.sum()), atol=1e-11)


def test_asm_symmetric_positive_for_symmetric_operator():
    g = space.Grid(3, 2, 2, synth.jittered_vertices(3, 2))
    prob = slab.SlabProblem(g, space.rho_qp_from_cells(g, np.ones(9)), "heat", "dg", 0, 0.1)
    B = mg.asm_operator(prob).toarray()
    inner = ~prob.bmask_full
    Bi = B[np.ix_(inner, inner)]
    assert np.allclose(Bi, Bi.T, atol=1e-12) and np.linalg.eigvalsh(Bi).min() > 0


def test_coarse_coefficient_follows_blocks():
    V = synth.jittered_vertices(8, 3)
    rho = synth.block_coefficient(8, 3, blocks=2)
    H = mg.Hierarchy(3, 8, 1, 0, "heat", "dg", 0.1, V, rho_cell=rho, estimate=False)
    lev = H.levels[1]  # 4^3 cells: every cell inside one block
    g = lev.grid
    from oracle.space import rho_qp_from_cells
    assert g.N == 4
    blocks = synth.block_coefficient(4, 3, blocks=2)
    assert np.allclose(mg.level_rho_qp(g, rho, 8), rho_qp_from_cells(g, blocks))


def test_vcycle_contracts_and_fgmres_reaches_direct_solution():
    V = synth.jittered_vertices(4, 3)
    rho = synth.block_coefficient(4, 3, blocks=2)
    H = mg.Hierarchy(3, 4, 2, 2, "heat", "dg", 1.0 / 32, V, rho_cell=rho)
    prob = H.levels[0].prob
    # omega estimate is close to the exact eigenvalue rule on the finest level
    lev = H.levels[0]
    inner = lev.interior
    ev = np.linalg.eigvals((lev.B @ prob.S).toarray()[np.ix_(inner, inner)])
    assert abs(lev.omega - 2.0 / (ev.real.max() + ev.real.min())) < 0.05 * lev.omega
    b = synth.random_vector(prob.n)
    b[prob.bmask_full] = 0.0
    # the stationary V-cycle iteration contracts (rate about 0.6 with the eq. relaxation omega)
    x = np.zeros_like(b)
    r0 = np.linalg.norm(b)
    for _ in range(10):
        x = x + H.vcycle(b - prob.S @ x)
    assert np.linalg.norm(b - prob.S @ x) < 0.8 ** 10 * r0
    res = mg.fgmres(lambda v: prob.S @ v, H.vcycle, b, np.zeros_like(b), rtol=1e-11)
    xd = prob.solve(b).reshape(-1)
    assert res.rel_residual < 1e-11
    assert np.linalg.norm(res.x - xd) < 1e-9 * np.linalg.norm(xd)


def test_relaxation_estimate_is_capped_at_one():
    """eq. relaxation with omega_l in (0, 1) (Section 3.3): the weighted Schwarz sum has lambda_max near 1,
    so the raw estimate 2 / (lambda_max + lambda_min) exceeds 1 and is capped; the plain sum stays below."""
    V = synth.jittered_vertices(4, 2)
    Hw = mg.Hierarchy(2, 4, 2, 1, "heat", "dg", 0.05, V, weighted=True)
    Hp = mg.Hierarchy(2, 4, 2, 1, "heat", "dg", 0.05, V)
    assert all(0.0 < w <= 1.0 for w in Hw.omegas()) and max(Hw.omegas()) == 1.0
    assert all(0.0 < w < 1.0 for w in Hp.omegas())
    # the coarse level with one unconstrained node: weighted B S = I, so lambda = 1 and omega = 1
    assert Hw.omegas()[-1] == 1.0
