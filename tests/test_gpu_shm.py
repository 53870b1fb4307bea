"""Goal quantities of the structural-health-monitoring example (Section 4.3), reduced: point values of the
GPU solution against the oracle's point evaluation, and a wave run on [-1, 1]^3 with the highly
heterogeneous coefficient (layers 1 / 9 / 16 times c ~ U[0.4, 1.6] per cell of a 5^3 coarse grid)
marched slab by slab on the GPU and by direct solves in the oracle."""
import numpy as np
import pytest

import synth
from gpu_cases import rel_err, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def test_point_values_match_the_oracle_on_a_jittered_grid(env):
    torch, stmg = env
    from oracle import points, space
    N, p = 4, 2
    V = synth.jittered_vertices(N, 3)
    ctx = stmg.Context(3, N, p, 1, 0.1, vertices=V, omega=[0.2] * 8)
    g = space.Grid(N, 3, p, V)
    u = synth.random_vector((ctx.nt, g.n_nodes), seed=41)
    pts = np.random.default_rng(42).uniform(0.03, 0.97, size=(7, 3))
    got = ctx.point_values(torch.from_numpy(u.reshape(-1)).cuda(), pts)
    ref = points.point_values(g, u, pts)                     # (npts, nt)
    assert got.shape == ref.shape and np.abs(got - ref).max() <= 1e-13 * np.abs(u).max()
    with pytest.raises(stmg.StmgError):
        ctx.point_values(torch.from_numpy(u.reshape(-1)).cuda(), [[1.5, 0.5, 0.5]])
    ctx.close()


def test_reduced_shm_wave_goal_quantities(env):
    torch, stmg = env
    from oracle import points, slab, space
    N, p, k, tau, nsl = 10, 2, 2, 0.1, 4
    V = synth.cartesian_vertices(N, 3, lo=-1.0, hi=1.0)
    rho = synth.shm_coefficient(N, rough=True)
    g = space.Grid(N, 3, p, V)
    X = g.node_coords()
    u0 = synth.shm_initial(X, s=0.15)
    u0[g.boundary_mask()] = 0.0
    prob = slab.SlabProblem(g, space.rho_qp_from_cells(g, rho), "wave", "cgp", k, tau)
    sols, _ = slab.march(prob, nsl, None, u_init=u0, v_init=np.zeros(g.n_nodes))
    ref = np.stack([points.point_values(g, s, synth.SHM_POINTS) for s in sols])   # (slab, pt, nt)
    ctx = stmg.Context(3, N, p, k, tau, pde=stmg.WAVE, scheme=stmg.CGP, vertices=V, coeff=rho, rtol=1e-12,
                       max_it=300)
    nt, nn = ctx.nt, ctx.n_nodes
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
    rhs = torch.empty(nt * nn, dtype=torch.float64, device="cuda")
    u = torch.empty_like(rhs)
    v = torch.empty_like(rhs)
    zero_f, zero_n = dev(np.zeros(nt * nn)), dev(np.zeros(nn))
    u_prev, v_prev = dev(u0), dev(np.zeros(nn))
    got, its = [], []
    for s in range(nsl):
        ctx.rhs(zero_f, rhs, f0=zero_n, u0=u_prev, v0=v_prev)
        ctx.guess_previous(u_prev, u)
        st = ctx.solve(rhs, u)
        assert st["converged"], st
        its.append(st["iterations"])
        got.append(ctx.point_values(u, synth.SHM_POINTS))
        ctx.wave_velocity(u, u_prev, v_prev, v)
        u_prev, v_prev = u[(nt - 1) * nn:].clone(), v[(nt - 1) * nn:].clone()
    got = np.stack(got)
    scale = np.abs(ref).max()
    assert scale > 1e-6                                    # the pulse has reached the goal points
    assert np.abs(got - ref).max() <= 1e-8 * scale, (np.abs(got - ref).max(), scale)
    # the marching solution itself, slab by slab
    assert rel_err(u.cpu().numpy(), sols[-1].reshape(-1)) < 1e-8
    print(f"\nreduced SHM (10^3 cells, Q2, cGP(2), rough coefficient): iterations {its}, "
          f"point values at the last slab end {got[-1, :, -1]}")
    ctx.close()
