"""Pins of the oracle's at-once system for several slabs (heat, dG(k); eq. heat-cg-dg-at-once) and of
its tau-multigrid (Algorithm mg-sequence with mgType tau)."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import atonce, fe1d, mg, slab, timeint


def _problem(dim=2, N=3, p=2, k=1, tau=0.05, nc=4, jitter=True):
    from oracle.space import Grid
    V = synth.jittered_vertices(N, dim) if jitter else synth.cartesian_vertices(N, dim)
    g = Grid(N, dim, p, V)
    rq = np.repeat(synth.block_coefficient(N, dim, blocks=1)[:, None], g.n ** dim, axis=1)
    return atonce.AtOnceProblem(g, rq, k, tau, nc)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_at_once_solution_equals_slab_by_slab_marching(k):
    """The block lower-bidiagonal system has the same solution as solving its slabs one after the
    other with the previous end value in the right-hand side (the marching of eq. heat-cg-dg)."""
    prob = _problem(k=k, nc=4)
    g = prob.grid
    X = g.node_coords()
    src = lambda x, t: np.cos(3.0 * t) * np.prod(np.sin(np.pi * x), axis=1) + t * x[:, 0]
    u0 = np.prod(np.sin(np.pi * X), axis=1)
    u0[g.boundary_mask()] = 0.0
    sols, _ = slab.march(prob.slab, prob.nc, src, u_init=u0)
    tn = fe1d.gauss_radau_right(k + 1)[0]
    fs = np.stack([np.stack([src(X, prob.slab.sys.tau * (i + th)) for th in tn]) for i in range(prob.nc)])
    u = prob.solve(prob.rhs(fs, u0))
    assert np.abs(u - np.stack(sols)).max() <= 1e-12 * np.abs(u).max()


def test_at_once_with_one_slab_is_the_slab_system():
    prob = _problem(nc=1)
    assert abs(prob.S - prob.slab.S).max() == 0.0


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_tau_prolongation_reproduces_coarse_polynomials(k):
    P = atonce.tau_prolongation(k)
    tc = fe1d.gauss_radau_right(k + 1)[0]
    q = lambda t: sum((0.3 + j) * (t - 0.4) ** j for j in range(k + 1))
    for h in range(2):
        # a polynomial on the coarse reference interval [0, 1], sampled at the fine nodes of half h
        assert np.allclose(P[h] @ q(tc), q(0.5 * (h + tc)), atol=1e-13)
    # the last fine node of the second half is the coarse end point (Radau node 1)
    assert np.allclose(P[1][-1], np.eye(k + 1)[-1])


@pytest.mark.parametrize("k,nc", [(0, 2), (1, 2), (2, 4)])
def test_tau_coarse_operator_is_the_galerkin_product(k, nc):
    """dG in time is nested under tau -> 2 tau: on embedded functions the jumps between the two fine
    halves vanish, so P^T S_tau P equals the at-once operator rediscretised with 2 tau and n_c / 2
    slabs (checks the sign and the column of the coupling, the tau scaling and P_tau)."""
    H = atonce.AtOnceHierarchy(2, 2, 1, k, 0.1, nc, synth.jittered_vertices(2, 2), estimate=False)
    li = [i for i in range(len(H.levels) - 1) if H.levels[i + 1].spec.nc != H.levels[i].spec.nc][0]
    f, c = H.levels[li], H.levels[li + 1]
    assert c.spec.tau == 2 * f.spec.tau and c.spec.nc * 2 == f.spec.nc
    G = (f.P.T @ f.prob.S @ f.P).toarray()
    keep = ~c.prob.bmask_full
    Sc = c.prob.S.toarray()
    assert np.abs(G[np.ix_(keep, keep)] - Sc[np.ix_(keep, keep)]).max() <= 1e-13 * np.abs(Sc).max()


def test_level_sequence_space_then_tau_then_k():
    seq = [(s.p, s.N, s.k, s.nc) for s in atonce.level_sequence(2, 8, 2, 8, 0.01)]
    assert seq == [(2, 8, 2, 8), (1, 8, 2, 8), (1, 4, 2, 8), (1, 2, 2, 8), (1, 2, 2, 4), (1, 2, 2, 2),
                   (1, 2, 2, 1), (1, 2, 1, 1), (1, 2, 0, 1)]
    assert [s.tau for s in atonce.level_sequence(1, 2, 0, 6, 0.1)] == [0.1, 0.2]  # 6 -> 3 slabs, odd


def test_at_once_smoother_is_the_cellwise_inverse_of_the_at_once_matrix():
    """Brute force: invert the at-once matrix restricted to each space-time cell (one slab, all its
    time DoFs, the unconstrained nodes of one spatial cell) and add up (eq. vanka0)."""
    H = atonce.AtOnceHierarchy(2, 2, 2, 1, 0.05, 3, synth.jittered_vertices(2, 2), estimate=False)
    lev = H.levels[0]
    S = lev.prob.S.toarray()
    g = lev.prob.grid
    nn, nt = g.n_nodes, lev.prob.nt
    B = np.zeros_like(S)
    for i in range(lev.prob.nc):
        for cell in g.cell_dofs():
            nodes = cell[~g.boundary_mask()[cell]]
            idx = (i * nt * nn + np.arange(nt)[:, None] * nn + nodes[None, :]).reshape(-1)
            B[np.ix_(idx, idx)] += np.linalg.inv(S[np.ix_(idx, idx)])
    assert np.abs(lev.B.toarray() - B).max() <= 1e-12 * np.abs(B).max()


@pytest.mark.parametrize("nc", [2, 4])
def test_at_once_vcycle_in_fgmres_reaches_the_direct_solution(nc):
    H = atonce.AtOnceHierarchy(2, 4, 2, 1, 0.1, nc, synth.jittered_vertices(4, 2),
                               rho_cell=synth.block_coefficient(4, 2, blocks=2))
    prob = H.levels[0].prob
    b = synth.random_vector(prob.n, seed=5)
    b[prob.bmask_full] = 0.0
    res = mg.fgmres(lambda v: prob.S @ v, H.vcycle, b, np.zeros_like(b), rtol=1e-10)
    x = prob.solve(b).reshape(-1)
    assert np.linalg.norm(res.x - x) <= 1e-8 * np.linalg.norm(x)
    assert res.iterations <= 20
    # the V-cycle contracts the error
    e0 = x.copy()
    e1 = e0 - H.vcycle(prob.S @ e0)
    assert np.linalg.norm(e1) < 0.5 * np.linalg.norm(e0)


def test_weighted_at_once_smoother_brute_force_and_fewer_iterations():
    """Weighted Schwarz sum on the at-once system: each cell block's inverse rows divided by the number
    of cells containing the node, built here from the at-once matrix; the weighted V-cycle needs no
    more FGMRES iterations than the plain one."""
    from oracle import space
    V = synth.jittered_vertices(2, 2)
    H = atonce.AtOnceHierarchy(2, 2, 2, 1, 0.05, 3, V, estimate=False, weighted=True)
    lev = H.levels[0]
    S = lev.prob.S.toarray()
    g = lev.prob.grid
    nn, nt = g.n_nodes, lev.prob.nt
    gl = space.lex_indices(g.nn1, g.dim)
    shared = (gl % g.p == 0) & (gl > 0) & (gl < g.nn1 - 1)
    mult = np.prod(np.where(shared, 2.0, 1.0), axis=1)
    B = np.zeros_like(S)
    for i in range(lev.prob.nc):
        for cell in g.cell_dofs():
            nodes = cell[~g.boundary_mask()[cell]]
            idx = (i * nt * nn + np.arange(nt)[:, None] * nn + nodes[None, :]).reshape(-1)
            w = np.tile(1.0 / mult[nodes], nt)
            B[np.ix_(idx, idx)] += w[:, None] * np.linalg.inv(S[np.ix_(idx, idx)])
    assert np.abs(lev.B.toarray() - B).max() <= 1e-12 * np.abs(B).max()
    # iterations: weighted (capped omega) against plain, same problem
    Vj = synth.jittered_vertices(4, 2)
    rho = synth.block_coefficient(4, 2, blocks=2)
    its = {}
    for wt in (False, True):
        Hw = atonce.AtOnceHierarchy(2, 4, 2, 1, 0.1, 4, Vj, rho_cell=rho, weighted=wt)
        prob = Hw.levels[0].prob
        b = synth.random_vector(prob.n, seed=6)
        b[prob.bmask_full] = 0.0
        res = mg.fgmres(lambda v: prob.S @ v, Hw.vcycle, b, np.zeros_like(b), rtol=1e-10)
        x = prob.solve(b).reshape(-1)
        assert np.linalg.norm(res.x - x) <= 1e-8 * np.linalg.norm(x)
        its[wt] = res.iterations
    assert its[True] <= its[False], its
