"""Pins of the oracle's slab solves: convergence orders and the wave condensation."""
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import pytest

import synth
from oracle import slab, space, timeint


def _heat_error(N, n_slabs, p, k, scheme, dim=2, jitter=False):
    V = synth.jittered_vertices(N, dim) if jitter else synth.cartesian_vertices(N, dim)
    g = space.Grid(N, dim, p, V)
    prob = slab.SlabProblem(g, space.rho_qp_from_cells(g, np.ones(g.n_cells)), "heat", scheme, k, 1.0 / n_slabs)
    sols, _ = slab.march(prob, n_slabs, synth.heat_sine_source)
    return slab.l2l2_error(prob, sols, synth.heat_sine_solution, np.zeros(g.n_nodes))


def test_heat_dg1_q2_space_order_3():
    e = [_heat_error(N, 64, 2, 1, "dg") for N in (4, 8)]
    assert abs(math.log2(e[0] / e[1]) - 3.0) < 0.25


def test_heat_dg1_time_order_2():
    e = [_heat_error(12, n, 4, 1, "dg") for n in (4, 8)]
    assert abs(math.log2(e[0] / e[1]) - 2.0) < 0.2


def test_heat_cgp2_time_order_3_on_perturbed_mesh():
    e = [_heat_error(12, n, 4, 2, "cgp", jitter=True) for n in (4, 8)]
    assert abs(math.log2(e[0] / e[1]) - 3.0) < 0.25


def _coupled_wave_solution(prob, f, f0, u0, v0):
    """Solve the un-condensed (u, v) system of eq. var-wave-dg / the cGP wave form directly."""
    s, A, M = prob.sys, prob.A, prob.M
    tw = s.tw
    Mt, At = s.tau * tw.Mhat, tw.Ahat
    beta, alpha = s.tau * tw.betahat, tw.alpha
    nt, nn = prob.nt, prob.grid.n_nodes
    if tw.scheme == timeint.DG:
        # (1) At u - alpha u_prev - Mt v = 0 ; (2) At v - alpha v_prev + Mt A u = Mt M f
        K = sp.bmat([[sp.kron(At, M), -sp.kron(Mt, M)], [sp.kron(Mt, A), sp.kron(At, M)]])
        r1 = np.outer(alpha, M @ u0).reshape(-1)
        r2 = (sp.kron(Mt, M) @ f.reshape(-1)) + np.outer(alpha, M @ v0).reshape(-1)
    else:
        # (1) At u + alpha u0 - Mt v - beta v0 = 0 ; (2) At v + alpha v0 + Mt A u + beta A u0 = Mt M f + beta M f0
        K = sp.bmat([[sp.kron(At, M), -sp.kron(Mt, M)], [sp.kron(Mt, A), sp.kron(At, M)]])
        r1 = (-np.outer(alpha, M @ u0) + np.outer(beta, M @ v0)).reshape(-1)
        r2 = (sp.kron(Mt, M) @ f.reshape(-1) + np.outer(beta, M @ f0).reshape(-1)
              - np.outer(alpha, M @ v0).reshape(-1) - np.outer(beta, A @ u0).reshape(-1))
    bm = np.tile(prob.bmask, 2 * nt)
    K = slab.constrain(K, bm)
    rhs = np.concatenate([r1, r2])
    rhs[bm] = 0.0
    x = spla.spsolve(K.tocsc(), rhs)
    return x[: nt * nn].reshape(nt, nn), x[nt * nn:].reshape(nt, nn)


@pytest.mark.parametrize("scheme,k", [("cgp", 2), ("dg", 1)])
def test_wave_condensation_matches_coupled_system(scheme, k):
    N, p, dim = 3, 2, 2
    g = space.Grid(N, dim, p, synth.jittered_vertices(N, dim))
    rho = synth.layer_coefficient(N, dim, 1.0, 16.0)
    prob = slab.SlabProblem(g, space.rho_qp_from_cells(g, rho), "wave", scheme, k, 0.05)
    rng = np.random.default_rng(3)
    f = rng.standard_normal((prob.nt, g.n_nodes))
    f0, u0, v0 = (rng.standard_normal(g.n_nodes) for _ in range(3))
    u0[prob.bmask] = 0.0
    v0[prob.bmask] = 0.0
    u = prob.solve(prob.rhs(f, f0 if scheme == "cgp" else None, u0, v0))
    v = prob.velocity(u, u0, v0)
    v[:, prob.bmask] = 0.0
    uc, vc = _coupled_wave_solution(prob, f, f0, u0, v0)
    assert np.abs(u - uc).max() < 1e-10 * np.abs(uc).max()
    assert np.abs(v - vc).max() < 1e-10 * np.abs(vc).max()


def test_wave_cgp2_time_order():
    """Standing wave u = sin(pi x) sin(pi y) cos(sqrt(2) pi t): L2(L2) error order 3 in tau."""
    dim, N, p = 2, 10, 4
    w = math.sqrt(2) * math.pi
    exact = lambda X, t: np.sin(math.pi * X[..., 0]) * np.sin(math.pi * X[..., 1]) * math.cos(w * t)
    errs = []
    for n in (8, 16):
        g = space.Grid(N, dim, p, synth.cartesian_vertices(N, dim))
        prob = slab.SlabProblem(g, space.rho_qp_from_cells(g, np.ones(g.n_cells)), "wave", "cgp", 2, 1.0 / n)
        u_init = exact(g.node_coords(), 0.0)
        sols, _ = slab.march(prob, n, None, u_init=u_init)
        errs.append(slab.l2l2_error(prob, sols, exact, u_init))
    assert abs(math.log2(errs[0] / errs[1]) - 3.0) < 0.3


def test_matrix_free_and_sampled_rows_equal_assembled_operator():
    g = space.Grid(4, 3, 2, synth.jittered_vertices(4, 3))
    rho = space.rho_qp_from_cells(g, synth.block_coefficient(4, 3, blocks=2))
    prob = slab.SlabProblem(g, rho, "heat", "dg", 2, 0.1)
    x = synth.random_vector((3, g.n_nodes))
    ref = prob.apply(x)
    assert np.abs(slab.kron_apply(g, rho, prob.sys.TA, prob.sys.TM, x) - ref).max() < 1e-12 * np.abs(ref).max()
    rng = np.random.default_rng(1)
    samples = [(int(rng.integers(3)), int(rng.integers(g.n_nodes))) for _ in range(30)] + [(0, 0)]
    got = slab.sampled_rows(g, rho, "heat", "dg", 2, 0.1, x, samples)
    assert np.abs(got - np.array([ref[t, n] for t, n in samples])).max() < 1e-12 * np.abs(ref).max()
    f = synth.random_vector((3, g.n_nodes))
    u0 = synth.random_vector(g.n_nodes)
    u0[prob.bmask] = 0.0
    rhs = slab.kron_apply(g, rho, np.zeros((3, 3)), prob.sys.RM_f, f, constrained=False)
    rhs += slab.kron_apply(g, rho, np.zeros((3, 1)), prob.sys.RM_u0[:, None], u0[None, :], constrained=False)
    assert np.abs(rhs - prob.rhs(f, None, u0)).max() < 1e-13
