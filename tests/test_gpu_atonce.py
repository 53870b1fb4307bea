"""Several heat dG slabs in one system (eq. heat-cg-dg-at-once) with tau-multigrid levels: the GPU
path against oracle/atonce.py, element by element (tolerances as in test_gpu_parity.py)."""
from dataclasses import dataclass

import numpy as np
import pytest

import synth
from gpu_cases import rel_err, require_gpu

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5
TOLDF = 1e-11


@dataclass(frozen=True)
class ACase:
    name: str
    dim: int
    N: int
    p: int
    k: int
    nc: int
    tau: float
    jitter: bool
    blocks: bool

    def vertices(self):
        return synth.jittered_vertices(self.N, self.dim) if self.jitter else synth.cartesian_vertices(self.N, self.dim)

    def rho_cell(self):
        if self.blocks:
            return synth.block_coefficient(self.N, self.dim, blocks=2 if self.N % 2 == 0 else 1)
        return np.ones(self.N ** self.dim)


ACASES = [
    ACase("heat2d_q2_dg1_4slabs", 2, 4, 2, 1, 4, 0.05, True, True),
    ACase("heat3d_q2_dg2_2slabs_jit", 3, 4, 2, 2, 2, 1 / 32, True, True),
    # Cartesian, constant coefficient: fast diagonalisation; 3 slabs (odd): no tau-levels
    ACase("heat3d_q2_dg1_3slabs_cart_fd", 3, 4, 2, 1, 3, 1 / 16, False, False),
    # N_t = 4: the tau-transfer acts on blocks of 8 fine time components
    ACase("heat2d_q2_dg3_4slabs", 2, 2, 2, 3, 4, 0.1, True, True),
    ACase("heat2d_q1_dg0_8slabs", 2, 4, 1, 0, 8, 0.02, True, True),
]

_H = {}


def hierarchy(case):
    from oracle import atonce
    if case.name not in _H:
        _H[case.name] = atonce.AtOnceHierarchy(case.dim, case.N, case.p, case.k, case.tau, case.nc, case.vertices(),
                                               rho_cell=case.rho_cell())
    return _H[case.name]


def context(stmg, case, H, **kw):
    kw.setdefault("omega", H.omegas())
    return stmg.Context(case.dim, case.N, case.p, case.k, case.tau, pde=stmg.HEAT, scheme=stmg.DG,
                        vertices=case.vertices(), coeff=case.rho_cell(), n_slabs=case.nc, **kw)


def _rand(n, seed, bmask=None):
    x = synth.random_vector(n, seed=seed)
    if bmask is not None:
        x[bmask] = 0.0
    return x


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.mark.parametrize("case", ACASES, ids=lambda c: c.name)
def test_levels_and_apply_every_level(env, case):
    torch, stmg = env
    H = hierarchy(case)
    ctx = context(stmg, case, H)
    assert ctx.n_levels == len(H.levels)
    for li, lev in enumerate(H.levels):
        info = ctx.level_info(li)
        s = lev.spec
        assert (info["p"], info["n_cells"], info["k"], info["n_slabs"]) == (s.p, s.N, s.k, s.nc), li
        assert abs(info["tau"] - s.tau) <= 1e-15 * s.tau
        prob = lev.prob
        x = _rand(prob.n, 100 + li)  # constrained entries nonzero on purpose: identity rows, zero columns of B
        ref = prob.S @ x
        for dt, tol in ((torch.float64, TOL64), (torch.float32, TOL32)):
            xd = torch.from_numpy(x).to("cuda", dt)
            yd = torch.empty_like(xd)
            ctx.apply(xd, yd, level=li)
            assert rel_err(yd.cpu().numpy(), ref) < tol, (case.name, li, dt)
        f = _rand(prob.n, 200 + li)
        rd = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        ctx.residual(torch.from_numpy(f).cuda(), torch.from_numpy(x).cuda(), rd, level=li)
        assert rel_err(rd.cpu().numpy(), f - ref) < TOL64, (case.name, li)
    # FGMRES apply on V-cycle outputs: slab blocks in double-float, coupling in FP64
    prob = H.levels[0].prob
    x32 = _rand(prob.n, 300).astype(np.float32)
    y = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ctx.apply_df(torch.from_numpy(x32).cuda(), y)
    assert rel_err(y.cpu().numpy(), prob.S @ x32.astype(np.float64)) < TOLDF
    ctx.close()


@pytest.mark.parametrize("case", ACASES, ids=lambda c: c.name)
def test_smoother_and_transfers_including_tau_levels(env, case):
    torch, stmg = env
    H = hierarchy(case)
    ctx = context(stmg, case, H, vcycle_precision=stmg.FP64)
    for li, lev in enumerate(H.levels[:-1]):
        prob = lev.prob
        f = _rand(prob.n, 300 + li, prob.bmask_full)
        u = _rand(prob.n, 400 + li, prob.bmask_full)
        ref = u + lev.omega * (lev.B @ (f - prob.S @ u))
        fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u).cuda()
        ctx.smooth(fd, ud, sweeps=1, level=li)
        assert rel_err(ud.cpu().numpy(), ref) < 1e-9, (case.name, li)
        c = H.levels[li + 1]
        rcd = torch.empty(c.prob.n, dtype=torch.float64, device="cuda")
        ctx.restrict(fd, rcd, level=li)
        assert rel_err(rcd.cpu().numpy(), lev.P.T @ f) < 1e-13, (case.name, li)
        e = _rand(c.prob.n, 500 + li, c.prob.bmask_full)
        uf = torch.from_numpy(u).cuda()
        ctx.prolongate_add(torch.from_numpy(e).cuda(), uf, level=li)
        assert rel_err(uf.cpu().numpy(), u + lev.P @ e) < 1e-13, (case.name, li)
        for dt, tol in ((torch.float32, 1e-5),):
            rc32 = torch.empty(c.prob.n, dtype=dt, device="cuda")
            ctx.restrict(fd.to(dt), rc32, level=li)
            assert rel_err(rc32.cpu().numpy(), lev.P.T @ f) < tol
    ctx.close()


@pytest.mark.parametrize("case", ACASES, ids=lambda c: c.name)
def test_vcycle(env, case):
    torch, stmg = env
    H = hierarchy(case)
    prob = H.levels[0].prob
    r = _rand(prob.n, 600, prob.bmask_full)
    ref = H.vcycle(r)
    for prec, dt, tol in ((stmg.FP64, torch.float64, 1e-9), (stmg.FP32, torch.float32, 2e-4)):
        ctx = context(stmg, case, H, vcycle_precision=prec)
        for _ in range(3):  # eager, captured, replayed
            e = torch.empty(prob.n, dtype=dt, device="cuda")
            ctx.vcycle(torch.from_numpy(r).to("cuda", dt), e)
            assert rel_err(e.cpu().numpy(), ref) < tol, (case.name, prec)
        ctx.close()


@pytest.mark.parametrize("case", ACASES, ids=lambda c: c.name)
def test_solve_equals_slab_by_slab_marching(env, case):
    """Right-hand side from a source and the previous end value, one FGMRES solve of the whole system:
    equal to the direct at-once solution and to marching the slabs one by one."""
    torch, stmg = env
    from oracle import fe1d, slab
    H = hierarchy(case)
    prob = H.levels[0].prob
    g = prob.grid
    X = g.node_coords()
    src = lambda x, t: np.cos(5.0 * t) * np.prod(np.sin(np.pi * x), axis=1) + (1.0 + t) * x[:, 0] * (1.0 - x[:, 0])
    u0 = np.prod(np.sin(np.pi * X), axis=1) * (1.0 + X[:, 0])
    u0[g.boundary_mask()] = 0.0
    tn = fe1d.gauss_radau_right(case.k + 1)[0]
    fs = np.stack([np.stack([src(X, case.tau * (i + th)) for th in tn]) for i in range(case.nc)])
    sols, _ = slab.march(prob.slab, case.nc, src, u_init=u0)
    xm = np.stack(sols).reshape(-1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).cuda()
    for kw in (dict(), dict(vcycle_precision=stmg.FP64)):
        ctx = context(stmg, case, H, rtol=1e-12, max_it=300, **kw)
        rhs = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        ctx.rhs(t(fs), rhs, u0=t(u0))
        assert rel_err(rhs.cpu().numpy(), prob.rhs(fs, u0)) < TOL64
        u = torch.empty_like(rhs)
        ctx.guess_previous(t(u0), u)
        assert rel_err(u.cpu().numpy(), np.tile(u0, case.nc * prob.nt)) == 0.0
        st = ctx.solve(rhs, u)
        assert st["converged"], st
        assert np.linalg.norm(u.cpu().numpy() - xm) / np.linalg.norm(xm) < 1e-8, (case.name, kw)
        ctx.close()


def test_several_slabs_need_heat_dg(env):
    torch, stmg = env
    with pytest.raises(stmg.StmgError) as ei:
        stmg.Context(2, 4, 1, 1, 0.1, pde=stmg.WAVE, scheme=stmg.DG, n_slabs=2)
    assert ei.value.status == 1
    with pytest.raises(stmg.StmgError):
        stmg.Context(2, 4, 1, 1, 0.1, pde=stmg.HEAT, scheme=stmg.CGP, n_slabs=2)


@pytest.mark.parametrize("k,nc", [(2, 12), (1, 4)])
def test_bf16_smoother_several_slabs_in_batches(env, k, nc):
    """FP32 vectors and BF16 inverses (the stored rows kept in registers, slabs in batches of eight): one
    sweep from u = 0 on every level of the hierarchy (12, 6, 3 slabs; Q2 and Q1 cells) against the
    oracle's omega B f, and two sweeps on level 0, at 2e-2 (the BF16 tolerance of the plane store; measured
    3.6e-3).  dG(2) has one real and one complex time mode, dG(1) a complex pair only.  The V-cycle is
    compared with the FP64-arithmetic V-cycle over the same BF16 inverses (measured 2.7e-6): against the
    oracle's exact inverses the BF16 V-cycle of the 12-slab hierarchy differs by 0.146 in either
    arithmetic (5.9e-3 for one slab), an effect of the storage, not of the kernel."""
    torch, stmg = env
    from oracle import atonce
    dim, N, p, tau = 3, 4, 2, 1 / 32
    V = synth.jittered_vertices(N, dim)
    rho = synth.block_coefficient(N, dim, blocks=2)
    H = atonce.AtOnceHierarchy(dim, N, p, k, tau, nc, V, rho_cell=rho, estimate=False, omegas=[0.5] * 16)
    kw = dict(vertices=V, coeff=rho, n_slabs=nc, omega=H.omegas(), inverse_precision=stmg.BF16)
    ctx = stmg.Context(dim, N, p, k, tau, vcycle_precision=stmg.FP32, **kw)
    for li, lev in enumerate(H.levels[:-1]):
        prob = lev.prob
        f = _rand(prob.n, 730 + li, prob.bmask_full)
        ref = lev.omega * (lev.B @ f)
        for _ in range(2):  # stages and registers reused call after call
            u32 = torch.zeros(prob.n, dtype=torch.float32, device="cuda")
            ctx.smooth(torch.from_numpy(f).to("cuda", torch.float32), u32, sweeps=1, level=li)
            assert rel_err(u32.cpu().numpy(), ref) < 2e-2, (k, nc, li)
    lev = H.levels[0]
    prob = lev.prob
    f = _rand(prob.n, 731, prob.bmask_full)
    u1 = lev.omega * (lev.B @ f)
    u2 = u1 + lev.omega * (lev.B @ (f - prob.S @ u1))
    u32 = torch.zeros(prob.n, dtype=torch.float32, device="cuda")
    ctx.smooth(torch.from_numpy(f).to("cuda", torch.float32), u32, sweeps=2, level=0)
    assert rel_err(u32.cpu().numpy(), u2) < 2e-2, (k, nc)
    r = _rand(prob.n, 740, prob.bmask_full)
    e = torch.empty(prob.n, dtype=torch.float32, device="cuda")
    ctx.vcycle(torch.from_numpy(r).to("cuda", torch.float32), e)
    ctx.close()
    ctx64 = stmg.Context(dim, N, p, k, tau, vcycle_precision=stmg.FP64, **kw)
    e64 = torch.empty(prob.n, dtype=torch.float64, device="cuda")
    ctx64.vcycle(torch.from_numpy(r).cuda(), e64)
    ctx64.close()
    assert rel_err(e.cpu().numpy(), e64.cpu().numpy()) < 1e-5, (k, nc)
