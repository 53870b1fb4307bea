"""GMRES iteration counts of the paper's heat-equation convergence test (Cartesian, CG(k)-DG(k),
p = k) against the table the paper prints (tests/golden/iter_heat_dg_cartesian.txt).

The absolute counts depend on details the paper leaves to cited work (the eigenvalue estimator
behind eq. relaxation, the GMRES variant), so parity is not claimed for them. What is checked:
the counts do not grow under refinement (the paper's grid independence), they stay within a
factor 2 of the printed values (measured on GB300: about 1.5-1.7 times the printed counts), and
the error converges at least at the order k + 1 the paper reports."""
import os

import numpy as np
import pytest

from gpu_cases import require_gpu
from oracle import fe1d

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "iter_heat_dg_cartesian.txt")


def _table():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = line.split()
        rows[int(v[0])] = dict(zip((2, 3, 4, 5, 6), map(float, v[1:])))
    return rows


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def _mean_iterations(torch, stmg, k, r):
    f = 2.0
    w = 2.0 * np.pi * f
    N, nsl = 2 ** (r + 1), 4 * 2 ** r
    tau = 1.0 / nsl
    ctx = stmg.Context(3, N, k, k, tau, rtol=1e-12, atol=1e-12, max_it=400)
    nt, nn = ctx.nt, ctx.n_nodes
    X = ctx.node_coords()
    S = np.prod(np.sin(w * X), axis=1)
    tn = fe1d.gauss_radau_right(k + 1)[0]
    rhs = torch.empty(nt * nn, dtype=torch.float64, device="cuda")
    u = torch.empty_like(rhs)
    uprev = torch.zeros(nn, dtype=torch.float64, device="cuda")
    its = []
    for s in range(nsl):
        # u = sin(w t) S(x): source u_t - lap u = (w cos(w t) + 3 w^2 sin(w t)) S(x)
        fs = np.stack([(w * np.cos(w * tau * (s + th)) + 3 * w * w * np.sin(w * tau * (s + th))) * S for th in tn])
        ctx.rhs(torch.from_numpy(fs.reshape(-1)).cuda(), rhs, u0=uprev)
        ctx.guess_previous(uprev, u)
        st = ctx.solve(rhs, u)
        assert st["converged"]
        its.append(st["iterations"])
        uprev = u[(nt - 1) * nn:].clone()
    # the exact solution vanishes at t = 1 (sin(2 pi f) = 0): the nodal values there are the error
    err = float(uprev.abs().max())
    assert err < 1e-3
    ctx.close()
    return float(np.mean(its)), err


@pytest.mark.parametrize("k", [2, 3])
def test_iterations_grid_independent_and_near_the_paper(env, k):
    torch, stmg = env
    table = _table()
    res = {r: _mean_iterations(torch, stmg, k, r) for r in (2, 3)}
    its = {r: v[0] for r, v in res.items()}
    for r, v in its.items():
        assert v <= 2.0 * table[k][r], (k, r, v, table[k][r])
        assert v >= 0.5 * table[k][r], (k, r, v, table[k][r])
    assert its[3] <= its[2] + 1.0, its
    # convergence under refinement of h and tau together: at least the order k + 1 the paper reports
    # (Figure conv-heat); measured on GB300 the nodal error at t = 1 falls by about 14 (k = 2) and 31 (k = 3)
    assert res[2][1] / res[3][1] >= 0.8 * 2 ** (k + 1), res
