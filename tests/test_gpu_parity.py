"""GPU path (C ABI via the Python binding) against the FP64 oracle, element by element.

Tolerances: FP64 kernels 1e-10 relative (max-norm over the vector, scaled by its
largest entry), FP32 kernels 2e-5 relative (float rounding of O(100) terms),
double-float kernels 1e-11 relative (about 44 significand bits: 6e-14 per operation
over O(100) operations), solutions 1e-8 relative L2 after FGMRES to rtol 1e-12.
"""
import numpy as np
import pytest

import synth
from gpu_cases import CASES, make_context, oracle_hierarchy, rel_err, require_gpu

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5
TOLDF = 1e-11


def _rand(n, seed, bmask=None):
    x = synth.random_vector(n, seed=seed)
    if bmask is not None:
        x[bmask] = 0.0
    return x


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_apply_every_level(env, case):
    torch, stmg = env
    H = oracle_hierarchy(case)
    ctx = make_context(stmg, case, H)
    for li, lev in enumerate(H.levels):
        prob = lev.prob
        x = _rand(prob.n, 100 + li)  # constrained entries nonzero on purpose: identity rows
        ref = prob.S @ x
        for dt, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
            xd = torch.from_numpy(x).to("cuda", dt)
            yd = torch.empty_like(xd)
            ctx.apply(xd, yd, level=li)
            assert rel_err(yd.cpu().numpy(), ref) < tol, (case.name, li, dt)
        # residual r = f - S u
        f = _rand(prob.n, 200 + li)
        fd = torch.from_numpy(f).cuda()
        ud = torch.from_numpy(x).cuda()
        rd = torch.empty_like(fd)
        ctx.residual(fd, ud, rd, level=li)
        assert rel_err(rd.cpu().numpy(), f - ref) < TOL64
    ctx.close()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_double_float_apply_on_fp32_vectors(env, case):
    """The FGMRES apply on V-cycle outputs: FP32 input, double-float arithmetic, FP64 output."""
    torch, stmg = env
    H = oracle_hierarchy(case)
    ctx = make_context(stmg, case, H)
    prob = H.levels[0].prob
    for seed in (300, 301):
        x32 = _rand(prob.n, seed).astype(np.float32)   # constrained entries nonzero: identity rows
        ref = prob.S @ x32.astype(np.float64)
        y = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        ctx.apply_df(torch.from_numpy(x32).cuda(), y)
        assert rel_err(y.cpu().numpy(), ref) < TOLDF, case.name
    ctx.close()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_rhs_and_velocity(env, case):
    torch, stmg = env
    H = oracle_hierarchy(case)
    ctx = make_context(stmg, case, H)
    prob = H.levels[0].prob
    nn = prob.grid.n_nodes
    f = _rand(prob.n, 7).reshape(prob.nt, nn)
    f0, u0, v0 = (_rand(nn, s, prob.bmask) for s in (8, 9, 10))
    ref = prob.rhs(f, f0, u0, v0 if case.pde == "wave" else None)
    dev = "cuda"
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(dev)
    rhs = torch.empty(prob.n, dtype=torch.float64, device=dev)
    ctx.rhs(t(f), rhs, f0=t(f0), u0=t(u0), v0=t(v0) if case.pde == "wave" else None)
    assert rel_err(rhs.cpu().numpy(), ref) < TOL64
    if case.pde == "wave":
        u = _rand(prob.n, 11).reshape(prob.nt, nn)
        u[:, prob.bmask] = 0.0
        vref = prob.velocity(u, u0, v0)
        vref[:, prob.bmask] = 0.0
        v = torch.empty(prob.n, dtype=torch.float64, device=dev)
        ctx.wave_velocity(t(u), t(u0), t(v0), v)
        assert rel_err(v.cpu().numpy(), vref) < TOL64
    ctx.close()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_smoother_and_transfers(env, case):
    torch, stmg = env
    H = oracle_hierarchy(case)
    ctx = make_context(stmg, case, H, vcycle_precision=stmg.FP64)
    for li, lev in enumerate(H.levels[:-1]):
        prob = lev.prob
        f = _rand(prob.n, 300 + li, prob.bmask_full)
        u = _rand(prob.n, 400 + li, prob.bmask_full)
        ref = u + lev.omega * (lev.B @ (f - prob.S @ u))
        fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u).cuda()
        ctx.smooth(fd, ud, sweeps=1, level=li)
        assert rel_err(ud.cpu().numpy(), ref) < 1e-9, (case.name, li)
        # FP32 storage/arithmetic
        u32 = torch.from_numpy(u).to("cuda", torch.float32)
        ctx.smooth(fd.float(), u32, sweeps=1, level=li)
        assert rel_err(u32.cpu().numpy(), ref) < 1e-4
        # restriction and prolongation
        c = H.levels[li + 1]
        rc_ref = lev.P.T @ f
        rcd = torch.empty(c.prob.n, dtype=torch.float64, device="cuda")
        ctx.restrict(fd, rcd, level=li)
        assert rel_err(rcd.cpu().numpy(), rc_ref) < 1e-13
        e = _rand(c.prob.n, 500 + li, c.prob.bmask_full)
        uf = torch.from_numpy(u).cuda()
        ctx.prolongate_add(torch.from_numpy(e).cuda(), uf, level=li)
        assert rel_err(uf.cpu().numpy(), u + lev.P @ e) < 1e-13
    ctx.close()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_vcycle(env, case):
    torch, stmg = env
    H = oracle_hierarchy(case)
    prob = H.levels[0].prob
    r = _rand(prob.n, 600, prob.bmask_full)
    ref = H.vcycle(r)
    for prec, dt, tol in ((stmg.FP64, torch.float64, 1e-9), (stmg.FP32, torch.float32, 2e-4)):
        ctx = make_context(stmg, case, H, vcycle_precision=prec)
        for _ in range(3):  # first call eager, then captured graph, then replay
            e = torch.empty(prob.n, dtype=dt, device="cuda")
            ctx.vcycle(torch.from_numpy(r).to("cuda", dt), e)
            assert rel_err(e.cpu().numpy(), ref) < tol, (case.name, prec)
        ctx.close()


@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: c.name)
def test_vcycle_with_h_coarsening_only(env, case):
    """Algorithm mg-sequence with spatial levels that keep p (h-multigrid), then time levels."""
    torch, stmg = env
    from oracle import mg
    H = mg.Hierarchy(case.dim, case.N, case.p, case.k, case.pde, case.scheme, case.tau, case.vertices(),
                     rho_cell=case.rho_cell(), p_coarsening=False)
    prob = H.levels[0].prob
    r = _rand(prob.n, 610, prob.bmask_full)
    ref = H.vcycle(r)
    ctx = make_context(stmg, case, H, vcycle_precision=stmg.FP64, space_coarsening=stmg.COARSEN_H)
    assert ctx.n_levels == len(H.levels)
    for li, lev in enumerate(H.levels[:-1]):
        assert ctx.level_info(li)["p"] == case.p
    e = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.from_numpy(r).cuda(), e)
    assert rel_err(e.cpu().numpy(), ref) < 1e-9, case.name
    ctx.close()


@pytest.mark.parametrize("case,max_dofs", [(CASES[0], 5), (CASES[1], 10), (CASES[2], 20), (CASES[5], 30)],
                         ids=lambda v: v.name if hasattr(v, "name") else str(v))
def test_shallow_hierarchy_vcycle_and_solve(env, case, max_dofs):
    """Hierarchy ending at the first coarser level with at most max_dofs unknowns (dense coarse solve)."""
    torch, stmg = env
    from oracle import mg
    H = mg.Hierarchy(case.dim, case.N, case.p, case.k, case.pde, case.scheme, case.tau, case.vertices(),
                     rho_cell=case.rho_cell(), coarse_max_dofs=max_dofs)
    full = mg.level_sequence(case.p, case.N, case.k, case.scheme, dim=case.dim)
    assert 2 <= len(H.levels) < len(full)
    prob = H.levels[0].prob
    r = _rand(prob.n, 620, prob.bmask_full)
    ref = H.vcycle(r)
    for prec, dt, tol in ((stmg.FP64, torch.float64, 1e-9), (stmg.FP32, torch.float32, 2e-4)):
        ctx = make_context(stmg, case, H, vcycle_precision=prec, coarse_max_dofs=max_dofs, rtol=1e-12, max_it=300)
        assert ctx.n_levels == len(H.levels)
        for _ in range(3):
            e = torch.empty(prob.n, dtype=dt, device="cuda")
            ctx.vcycle(torch.from_numpy(r).to("cuda", dt), e)
            assert rel_err(e.cpu().numpy(), ref) < tol, (case.name, prec)
        b = _rand(prob.n, 630, prob.bmask_full)
        u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        st = ctx.solve(torch.from_numpy(b).cuda(), u)
        assert st["converged"]
        xd = prob.solve(b).reshape(-1)
        assert np.linalg.norm(u.cpu().numpy() - xd) / np.linalg.norm(xd) < 1e-8
        ctx.close()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_solve_matches_direct_solution(env, case):
    torch, stmg = env
    H = oracle_hierarchy(case)
    prob = H.levels[0].prob
    b = _rand(prob.n, 700, prob.bmask_full)
    xd = prob.solve(b).reshape(-1)
    # plain FP64; mixed with the double-float outer apply (default); mixed with the FP64 outer apply
    for prec, outer in ((stmg.FP64, 0), (stmg.FP32, 0), (stmg.FP32, stmg.FP64)):
        ctx = make_context(stmg, case, H, vcycle_precision=prec, rtol=1e-12, max_it=300, outer_apply=outer)
        u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        st = ctx.solve(torch.from_numpy(b).cuda(), u)
        assert st["converged"] and st["rel_residual"] <= 1e-12
        err = np.linalg.norm(u.cpu().numpy() - xd) / np.linalg.norm(xd)
        assert err < 1e-8, (case.name, prec, outer, err, st)
        ctx.close()
    # rtol 1e-9: the stopping test runs on the double-float residual (default outer apply); it agrees
    # with the oracle's FP64 residual of the returned solution
    ctx = make_context(stmg, case, H, rtol=1e-9, max_it=300)
    u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st = ctx.solve(torch.from_numpy(b).cuda(), u)
    un = u.cpu().numpy()
    rres = np.linalg.norm(b - prob.S @ un) / np.linalg.norm(b)
    assert st["converged"] and rres <= 1e-9, (case.name, rres, st)
    assert abs(rres - st["rel_residual"]) <= 0.01 * rres + 1e-13, (case.name, rres, st)
    ctx.close()


@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: c.name)
def test_relaxation_estimate_matches_oracle(env, case):
    torch, stmg = env
    H = oracle_hierarchy(case)
    for prec, tol in ((stmg.FP64, 1e-3), (stmg.FP32, 1e-2)):
        ctx = make_context(stmg, case, H, omega=None, vcycle_precision=prec)
        for li, om in enumerate(H.omegas()):
            assert abs(ctx.level_info(li)["omega"] - om) < tol * om, (case.name, li, prec)
        ctx.close()


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name)
def test_smoother_fp64_vectors_with_fp32_and_bf16_inverses(env, case):
    torch, stmg = env
    H = oracle_hierarchy(case)
    for inv, tol in ((stmg.FP32, 1e-5), (stmg.BF16, 2e-2)):
        ctx = make_context(stmg, case, H, vcycle_precision=stmg.FP32, inverse_precision=inv)
        for li, lev in enumerate(H.levels[:-1]):
            prob = lev.prob
            f = _rand(prob.n, 800 + li, prob.bmask_full)
            ref = lev.omega * (lev.B @ f)
            u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
            ctx.smooth(torch.from_numpy(f).cuda(), u, sweeps=1, level=li)
            assert rel_err(u.cpu().numpy(), ref) < tol, (case.name, li, inv)
        ctx.close()


def test_node_coordinates_match_oracle(env):
    torch, stmg = env
    case = CASES[1]
    H = oracle_hierarchy(case)
    ctx = make_context(stmg, case, H)
    assert np.abs(ctx.node_coords() - H.levels[0].grid.node_coords()).max() < 1e-14
    assert np.abs(ctx.qpoint_coords() - H.levels[0].grid.quad_points_phys()).max() < 1e-14
    ctx.close()


def test_fast_diagonalisation_as_approximate_solver_for_variable_coefficient(env):
    """Cartesian grid, coefficient varying inside cells: forced FD uses cell means; FGMRES still
    reaches the exact discrete solution (the smoother only changes the iteration count)."""
    torch, stmg = env
    from oracle import mg
    N, p, k = 4, 2, 1
    V = synth.cartesian_vertices(N, 3)
    a, phi = synth.smooth_coefficient_params(3)
    from oracle import space
    g = space.Grid(N, 3, p, V)
    rho_qp = synth.smooth_coefficient_at(g.quad_points_phys(), a, phi)
    H = mg.Hierarchy(3, N, p, k, "heat", "dg", 1 / 16, V, rho_qp=rho_qp, estimate=False, omegas=[0.2] * 8)
    prob = H.levels[0].prob
    b = _rand(prob.n, 990, prob.bmask_full)
    xd = prob.solve(b).reshape(-1)
    ctx = stmg.Context(3, N, p, k, 1 / 16, vertices=V, coeff=rho_qp.reshape(-1), coeff_mode=stmg.COEFF_PER_QPOINT,
                       smoother_kind=stmg.SMOOTHER_FD, rtol=1e-12, max_it=300)
    u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st = ctx.solve(torch.from_numpy(b).cuda(), u)
    assert st["converged"]
    assert np.linalg.norm(u.cpu().numpy() - xd) < 1e-8 * np.linalg.norm(xd)
    # the operator itself follows the per-quadrature-point coefficient exactly
    x = _rand(prob.n, 991)
    y = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ctx.apply(torch.from_numpy(x).cuda(), y)
    assert rel_err(y.cpu().numpy(), prob.S @ x) < TOL64
    ctx.close()


_HW = {}


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[2], CASES[7]], ids=lambda c: c.name)
def test_weighted_smoother_vcycle_and_solve(env, case):
    """Option asm_weighting = 1: each cell's correction divided by the node's cell count (dense
    inverses, TMA-fed and row-streamed, and fast diagonalisation), against the weighted oracle."""
    torch, stmg = env
    from oracle import mg
    if case.name not in _HW:
        _HW[case.name] = mg.Hierarchy(case.dim, case.N, case.p, case.k, case.pde, case.scheme, case.tau,
                                      case.vertices(), rho_cell=case.rho_cell(), weighted=True)
    H = _HW[case.name]
    assert all(0.0 < w <= 1.0 for w in H.omegas())
    ctx = make_context(stmg, case, H, vcycle_precision=stmg.FP64, asm_weighting=1)
    for li, lev in enumerate(H.levels[:-1]):
        prob = lev.prob
        f = _rand(prob.n, 800 + li, prob.bmask_full)
        u = _rand(prob.n, 900 + li, prob.bmask_full)
        ref = u + lev.omega * (lev.B @ (f - prob.S @ u))
        ud = torch.from_numpy(u).cuda()
        ctx.smooth(torch.from_numpy(f).cuda(), ud, sweeps=1, level=li)
        assert rel_err(ud.cpu().numpy(), ref) < 1e-9, (case.name, li)
        u32 = torch.from_numpy(u).to("cuda", torch.float32)
        ctx.smooth(torch.from_numpy(f).to("cuda", torch.float32), u32, sweeps=1, level=li)
        assert rel_err(u32.cpu().numpy(), ref) < 1e-4, (case.name, li)
    prob = H.levels[0].prob
    r = _rand(prob.n, 1000, prob.bmask_full)
    e = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.from_numpy(r).cuda(), e)
    assert rel_err(e.cpu().numpy(), H.vcycle(r)) < 1e-9, case.name
    ctx.close()
    # the library's own relaxation estimate (capped at 1) and a mixed-precision solve
    ctx = stmg.Context(case.dim, case.N, case.p, case.k, case.tau,
                       pde=stmg.HEAT if case.pde == "heat" else stmg.WAVE,
                       scheme=stmg.DG if case.scheme == "dg" else stmg.CGP, vertices=case.vertices(),
                       coeff=case.rho_cell(), asm_weighting=1, rtol=1e-12, max_it=200)
    for li in range(ctx.n_levels - 1):
        assert 0.0 < ctx.level_info(li)["omega"] <= 1.0
    b = _rand(prob.n, 1001, prob.bmask_full)
    u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st = ctx.solve(torch.from_numpy(b).cuda(), u)
    assert st["converged"]
    xd = prob.solve(b).reshape(-1)
    assert np.linalg.norm(u.cpu().numpy() - xd) / np.linalg.norm(xd) < 1e-8
    ctx.close()


@pytest.mark.parametrize("case", [CASES[1], CASES[2], CASES[6]], ids=lambda c: c.name)
def test_relaxed_outer_apply_reaches_the_same_solution(env, case):
    """outer_relax = 1 (inexact Krylov): once the residual estimate is below 1e5 x the target, the
    FGMRES apply runs in FP32; the stopping test stays on the accurate residual, so the solution and
    its true residual are as without relaxation."""
    torch, stmg = env
    H = oracle_hierarchy(case)
    prob = H.levels[0].prob
    b = _rand(prob.n, 710, prob.bmask_full)
    xd = prob.solve(b).reshape(-1)
    for rtol in (1e-9, 1e-12):
        ctx = make_context(stmg, case, H, rtol=rtol, max_it=300, outer_relax=1)
        u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        st = ctx.solve(torch.from_numpy(b).cuda(), u)
        un = u.cpu().numpy()
        rres = np.linalg.norm(b - prob.S @ un) / np.linalg.norm(b)
        assert st["converged"] and rres <= 1.05 * rtol, (case.name, rtol, rres, st)
        assert st["relaxed_iterations"] >= 1, st
        if rtol == 1e-12:
            assert np.linalg.norm(un - xd) / np.linalg.norm(xd) < 1e-8, (case.name, st)
        ctx.close()


@pytest.mark.parametrize("case", [CASES[1], CASES[2]], ids=lambda c: c.name)
def test_fp8_inverses(env, case):
    """inverse_precision = FP8 (e4m3, one FP32 scale per plane, weighted sum): one smoothing sweep
    differs from the oracle's exact one by the rounding of 4 significant bits (2^-4 relative per
    stored plane entry; the planes are time modes, so the bound passes through the time transforms:
    10 % norm-wise), and FGMRES reaches the same solution (the smoother's precision does not enter
    the solution, only the iteration count)."""
    torch, stmg = env
    from oracle import mg
    H = mg.Hierarchy(case.dim, case.N, case.p, case.k, case.pde, case.scheme, case.tau, case.vertices(),
                     rho_cell=case.rho_cell(), weighted=True)
    ctx = make_context(stmg, case, H, inverse_precision=stmg.FP8, asm_weighting=1, rtol=1e-12, max_it=300)
    lev = H.levels[0]
    prob = lev.prob
    f = _rand(prob.n, 820, prob.bmask_full)
    u = np.zeros(prob.n)
    corr = lev.omega * (lev.B @ f)
    u32 = torch.zeros(prob.n, dtype=torch.float32, device="cuda")
    ctx.smooth(torch.from_numpy(f).to("cuda", torch.float32), u32, sweeps=1, level=0)
    rel = np.linalg.norm(u32.cpu().numpy() - corr) / np.linalg.norm(corr)
    assert 1e-4 < rel < 0.1, (case.name, rel)  # FP8 rounding is visible, and bounded
    b = _rand(prob.n, 821, prob.bmask_full)
    ud = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st = ctx.solve(torch.from_numpy(b).cuda(), ud)
    xd = prob.solve(b).reshape(-1)
    assert st["converged"] and np.linalg.norm(ud.cpu().numpy() - xd) / np.linalg.norm(xd) < 1e-8, st
    ctx.close()


def test_smoother_row_streaming_fallback(env):
    """3D Q3, dG(3) (N_t = 4), FP64 inverses: two stages of one cell's planes exceed the shared memory
    of the bulk-copy kernel, so the row-streaming smoother runs; one sweep and the V-cycle against the
    oracle."""
    torch, stmg = env
    from gpu_cases import Case
    case = Case("heat3d_q3_dg3_jit", 3, 2, 3, 3, "heat", "dg", 0.1, True, "blocks")
    H = oracle_hierarchy(case)
    ctx = make_context(stmg, case, H, vcycle_precision=stmg.FP64)
    lev = H.levels[0]
    prob = lev.prob
    f = _rand(prob.n, 830, prob.bmask_full)
    u = _rand(prob.n, 831, prob.bmask_full)
    ref = u + lev.omega * (lev.B @ (f - prob.S @ u))
    ud = torch.from_numpy(u).cuda()
    ctx.smooth(torch.from_numpy(f).cuda(), ud, sweeps=1, level=0)
    assert rel_err(ud.cpu().numpy(), ref) < 1e-9
    r = _rand(prob.n, 832, prob.bmask_full)
    e = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.from_numpy(r).cuda(), e)
    assert rel_err(e.cpu().numpy(), H.vcycle(r)) < 1e-9
    ctx.close()
