"""Failure detection without a GPU fault: a bounded device wait that cannot complete gives up,
records the timeout in the context's status word, and the host reports STMG_ERR_TIMEOUT; the
CUDA context stays usable (a new STMG context on the same GPU solves normally)."""
import time

import numpy as np
import pytest

import synth
from gpu_cases import CASES, make_context, oracle_hierarchy, require_gpu

pytestmark = pytest.mark.gpu

STMG_ERR_TIMEOUT = 6


@pytest.fixture(scope="module")
def env():
    return require_gpu()


def test_bounded_wait_reports_timeout_and_gpu_stays_usable(env):
    torch, stmg = env
    case = CASES[1]
    H = oracle_hierarchy(case)
    prob = H.levels[0].prob
    b = synth.random_vector(prob.n, seed=31)
    b[prob.bmask_full] = 0.0
    ctx = make_context(stmg, case, H, rtol=1e-10, max_it=50)
    t0 = time.perf_counter()
    assert ctx.selftest_device_timeout() == STMG_ERR_TIMEOUT
    waited = time.perf_counter() - t0
    assert 0.5 < waited < 30.0, waited  # the wait bound is one second of device time
    # every later bulk-copy kernel of this context sees the status word and skips its work
    u = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    with pytest.raises(stmg.StmgError) as ei:
        ctx.solve(torch.from_numpy(b).cuda(), u)
    assert ei.value.status == STMG_ERR_TIMEOUT
    ctx.close()
    # the CUDA context is intact: a fresh STMG context solves to the direct solution
    ctx2 = make_context(stmg, case, H, rtol=1e-10, max_it=100)
    u2 = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    st = ctx2.solve(torch.from_numpy(b).cuda(), u2)
    assert st["converged"]
    xd = prob.solve(b).reshape(-1)
    assert np.linalg.norm(u2.cpu().numpy() - xd) / np.linalg.norm(xd) < 1e-7
    ctx2.close()
