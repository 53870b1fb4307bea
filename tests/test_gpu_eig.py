"""Additive Schwarz local solves through the per-cell generalized eigendecomposition (smoother_kind
EIG): against the oracle's explicit block inverses (eq. vanka0 as printed and the weighted sum), in
every storage precision, inside the V-cycle and in a solve to the direct solution.

Tolerances: FP64 storage and arithmetic 1e-9 (the eigendecomposition converges to 1e-15 of the
cell matrix; the smoother's condition number on these meshes stays below 1e5); FP32 vectors 1e-4;
FP32 storage with FP64 vectors 1e-5; BF16 storage 2e-2 (8-bit mantissa of Q, amplified by the
square root of the condition number of the local mass matrix, measured up to about 5).
"""
import numpy as np
import pytest

from gpu_cases import CASES, make_context, oracle_hierarchy, rel_err, require_gpu

pytestmark = pytest.mark.gpu

EIG_CASES = [c for c in CASES if not (c.dim == 3 and c.p > 3)]


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _rand(n, seed, mask=None):
    v = np.random.default_rng(seed).standard_normal(n)
    if mask is not None:
        v[mask] = 0.0
    return v


_HW = {}


def _weighted(case):
    from oracle import mg
    if case.name not in _HW:
        _HW[case.name] = mg.Hierarchy(case.dim, case.N, case.p, case.k, case.pde, case.scheme, case.tau,
                                      case.vertices(), rho_cell=case.rho_cell(), weighted=True)
    return _HW[case.name]


@pytest.mark.parametrize("weighted", [0, 1])
@pytest.mark.parametrize("case", EIG_CASES, ids=lambda c: c.name)
def test_eig_smoother_matches_oracle_blocks(env, case, weighted):
    torch, stmg = env
    H = _weighted(case) if weighted else oracle_hierarchy(case)
    ctx = make_context(stmg, case, H, vcycle_precision=stmg.FP64, smoother_kind=stmg.SMOOTHER_EIG,
                       asm_weighting=weighted)
    for li, lev in enumerate(H.levels[:-1]):
        prob = lev.prob
        f = _rand(prob.n, 300 + li, prob.bmask_full)
        u = _rand(prob.n, 400 + li, prob.bmask_full)
        ref = u + lev.omega * (lev.B @ (f - prob.S @ u))
        ud = torch.from_numpy(u).cuda()
        ctx.smooth(torch.from_numpy(f).cuda(), ud, sweeps=1, level=li)
        assert rel_err(ud.cpu().numpy(), ref) < 1e-9, (case.name, li)
        u32 = torch.from_numpy(u).to("cuda", torch.float32)
        ctx.smooth(torch.from_numpy(f).to("cuda", torch.float32), u32, sweeps=1, level=li)
        assert rel_err(u32.cpu().numpy(), ref) < 1e-4, (case.name, li)
    prob = H.levels[0].prob
    r = _rand(prob.n, 600, prob.bmask_full)
    e = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.from_numpy(r).cuda(), e)
    assert rel_err(e.cpu().numpy(), H.vcycle(r)) < 1e-9, case.name
    ctx.close()


@pytest.mark.parametrize("case", EIG_CASES, ids=lambda c: c.name)
def test_eig_smoother_reduced_storage(env, case):
    torch, stmg = env
    H = oracle_hierarchy(case)
    for inv, tol in ((stmg.FP32, 1e-5), (stmg.BF16, 2e-2)):
        ctx = make_context(stmg, case, H, vcycle_precision=stmg.FP32, inverse_precision=inv,
                           smoother_kind=stmg.SMOOTHER_EIG)
        for li, lev in enumerate(H.levels[:-1]):
            prob = lev.prob
            f = _rand(prob.n, 800 + li, prob.bmask_full)
            ref = lev.omega * (lev.B @ f)
            u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
            ctx.smooth(torch.from_numpy(f).cuda(), u, sweeps=1, level=li)
            assert rel_err(u.cpu().numpy(), ref) < tol, (case.name, li, inv)
        ctx.close()


@pytest.mark.parametrize("case", [CASES[1], CASES[2]], ids=lambda c: c.name)
def test_eig_smoother_solve_reaches_direct_solution(env, case):
    """Mixed precision (FP32 V-cycle, BF16 Q) with the weighted sum: FGMRES reaches the direct solution."""
    torch, stmg = env
    H = oracle_hierarchy(case)
    prob = H.levels[0].prob
    b = _rand(prob.n, 1001, prob.bmask_full)
    xd = prob.solve(b).reshape(-1)
    ctx = make_context(stmg, case, H, omega=None, vcycle_precision=stmg.FP32, inverse_precision=stmg.BF16,
                       smoother_kind=stmg.SMOOTHER_EIG, asm_weighting=1, rtol=1e-12, max_it=200)
    u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st = ctx.solve(torch.from_numpy(b).cuda(), u)
    assert st["converged"], st
    assert np.linalg.norm(u.cpu().numpy() - xd) < 1e-8 * np.linalg.norm(xd)
    ctx.close()


def test_eig_smoother_several_slabs_in_one_system(env):
    """Heat dG, four slabs in one system: the block-diagonal smoother serves every slab."""
    torch, stmg = env
    import synth
    from oracle import atonce
    dim, N, p, k, tau, nc = 3, 4, 2, 1, 1 / 32, 4
    V = synth.jittered_vertices(N, dim)
    rho = synth.block_coefficient(N, dim, blocks=2)
    H = atonce.AtOnceHierarchy(dim, N, p, k, tau, nc, V, rho_cell=rho, estimate=False, omegas=[0.5] * 16)
    ctx = stmg.Context(dim, N, p, k, tau, vertices=V, coeff=rho, n_slabs=nc, omega=H.omegas(),
                       vcycle_precision=stmg.FP64, smoother_kind=stmg.SMOOTHER_EIG)
    for li, lev in enumerate(H.levels[:-1]):
        prob = lev.prob
        f = _rand(prob.n, 700 + li, prob.bmask_full)
        u = _rand(prob.n, 710 + li, prob.bmask_full)
        ref = u + lev.omega * (lev.B @ (f - prob.S @ u))
        ud = torch.from_numpy(u).cuda()
        ctx.smooth(torch.from_numpy(f).cuda(), ud, sweeps=1, level=li)
        assert rel_err(ud.cpu().numpy(), ref) < 1e-9, li
    ctx.close()


def test_eig_smoother_refuses_q4_in_3d(env):
    torch, stmg = env
    with pytest.raises(stmg.StmgError) as err:
        stmg.Context(3, 2, 4, 1, 0.1, smoother_kind=stmg.SMOOTHER_EIG, omega=[0.3] * 16)
    assert err.value.status == 9  # STMG_ERR_UNSUPPORTED


# ---- tensor-core variant (smoother_kind EIG_TC): BF16 Q images, both products on tcgen05 ----
TC_CASES = [c for c in CASES if (c.p + 1) ** c.dim <= 64]


@pytest.mark.parametrize("weighted", [0, 1])
@pytest.mark.parametrize("case", TC_CASES, ids=lambda c: c.name)
def test_eig_tensor_core_smoother_matches_oracle_blocks(env, case, weighted):
    """FP32 vectors, Q in BF16 (2e-2 as for the BF16 plane storage); the right-hand sides enter the
    tensor cores as two BF16 parts, so the only coarse rounding is that of Q."""
    torch, stmg = env
    H = _weighted(case) if weighted else oracle_hierarchy(case)
    ctx = make_context(stmg, case, H, vcycle_precision=stmg.FP32, smoother_kind=stmg.SMOOTHER_EIG_TC,
                       asm_weighting=weighted)
    for li, lev in enumerate(H.levels[:-1]):
        prob = lev.prob
        f = _rand(prob.n, 300 + li, prob.bmask_full)
        # one sweep from u = 0 is omega B f: the smoother's own error, without the cancellation of
        # u - omega B S u that a sweep from a random u adds on levels where B S is close to I
        ref = lev.omega * (lev.B @ f)
        for call in range(2):  # the operand buffers and tensor memory are reused call after call
            u32 = torch.zeros(prob.n, dtype=torch.float32, device="cuda")
            ctx.smooth(torch.from_numpy(f).to("cuda", torch.float32), u32, sweeps=1, level=li)
            assert rel_err(u32.cpu().numpy(), ref) < 2e-2, (case.name, li, call)
        # FP64 vectors are refused
        with pytest.raises(stmg.StmgError):
            ctx.smooth(torch.from_numpy(f).cuda(), torch.zeros(prob.n, dtype=torch.float64, device="cuda"), sweeps=1,
                       level=li)
    prob = H.levels[0].prob
    r = _rand(prob.n, 600, prob.bmask_full)
    e = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    ctx.vcycle(torch.from_numpy(r).to("cuda", torch.float32), e)
    assert rel_err(e.cpu().numpy(), H.vcycle(r)) < 3e-2, case.name
    ctx.close()


@pytest.mark.parametrize("case", [CASES[1], CASES[2], CASES[6]], ids=lambda c: c.name)
def test_eig_tensor_core_solve_reaches_direct_solution(env, case):
    torch, stmg = env
    H = oracle_hierarchy(case)
    prob = H.levels[0].prob
    b = _rand(prob.n, 1002, prob.bmask_full)
    xd = prob.solve(b).reshape(-1)
    ctx = make_context(stmg, case, H, omega=None, vcycle_precision=stmg.FP32, smoother_kind=stmg.SMOOTHER_EIG_TC,
                       asm_weighting=1, rtol=1e-12, max_it=200)
    u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st = ctx.solve(torch.from_numpy(b).cuda(), u)
    assert st["converged"], st
    assert np.linalg.norm(u.cpu().numpy() - xd) < 1e-8 * np.linalg.norm(xd)
    ctx.close()


@pytest.mark.parametrize("k,nc", [(1, 4), (2, 8)])
def test_eig_tensor_core_smoother_several_slabs(env, k, nc):
    """Heat dG slabs in one system (4 slabs of dG(1), 8 of dG(2): 16 and 48 right-hand-side rows per cell):
    all slabs' right-hand sides share one pass over each Q image."""
    torch, stmg = env
    import synth
    from oracle import atonce
    dim, N, p, tau = 3, 4, 2, 1 / 32
    V = synth.jittered_vertices(N, dim)
    rho = synth.block_coefficient(N, dim, blocks=2)
    H = atonce.AtOnceHierarchy(dim, N, p, k, tau, nc, V, rho_cell=rho, estimate=False, omegas=[0.5] * 16)
    ctx = stmg.Context(dim, N, p, k, tau, vertices=V, coeff=rho, n_slabs=nc, omega=H.omegas(),
                       vcycle_precision=stmg.FP32, smoother_kind=stmg.SMOOTHER_EIG_TC)
    for li, lev in enumerate(H.levels[:-1]):
        prob = lev.prob
        f = _rand(prob.n, 720 + li, prob.bmask_full)
        ref = lev.omega * (lev.B @ f)
        u32 = torch.zeros(prob.n, dtype=torch.float32, device="cuda")
        ctx.smooth(torch.from_numpy(f).to("cuda", torch.float32), u32, sweeps=1, level=li)
        assert rel_err(u32.cpu().numpy(), ref) < 2e-2, li
    ctx.close()
