"""stmg_smooth_noalloc: smoothing for callers that may not allocate device memory.

The entry point keeps its residual in a fixed buffer inside the library's
device image, so the call itself allocates nothing.  It must give the same
result as stmg_smooth, call after call, and refuse levels whose residual does
not fit the buffer before doing any device work.  Collected last on purpose.
"""
import numpy as np
import pytest

import synth
from gpu_cases import CASES, make_context, oracle_hierarchy, rel_err, require_gpu

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 16 * 1024 * 1024  # STMG_NOALLOC_SCRATCH_BYTES in include/stmg.h


@pytest.fixture(scope="module")
def env():
    return require_gpu()


@pytest.mark.parametrize("prec_name,tol", [("FP64", 1e-10), ("FP32", 2e-5)])
def test_noalloc_smoother_matches_stmg_smooth_on_consecutive_calls(env, prec_name, tol):
    torch, stmg = env
    case = CASES[1]  # 3D Q2 dG(2), jittered grid, block coefficient
    H = oracle_hierarchy(case)
    prec = getattr(stmg, prec_name)
    dt = torch.float64 if prec == stmg.FP64 else torch.float32
    ctx = make_context(stmg, case, H, vcycle_precision=prec)
    for li in (0, 1):
        prob = H.levels[li].prob
        f = synth.random_vector(prob.n, seed=900 + li)
        u0 = synth.random_vector(prob.n, seed=950 + li)
        f[prob.bmask_full] = 0.0
        u0[prob.bmask_full] = 0.0
        fd = torch.from_numpy(f).to("cuda", dt)
        u_ref = torch.from_numpy(u0).to("cuda", dt)
        u_new = u_ref.clone()
        for call in range(2):  # two calls in a row: the fixed buffer keeps the last call's contents
            ctx.smooth(fd, u_ref, sweeps=1, level=li)
            ctx.smooth_noalloc(fd, u_new, sweeps=1, level=li)
            torch.cuda.synchronize()
            assert rel_err(u_new.cpu().numpy(), u_ref.cpu().numpy()) < tol, (li, call)
        # several sweeps in one call
        ctx.smooth(fd, u_ref, sweeps=2, level=li)
        ctx.smooth_noalloc(fd, u_new, sweeps=2, level=li)
        assert rel_err(u_new.cpu().numpy(), u_ref.cpu().numpy()) < tol
    ctx.close()


def test_noalloc_smoother_rejects_levels_larger_than_the_fixed_buffer(env):
    torch, stmg = env
    # 2D, Q2 on 512^2 cells, dG(2): 3 * 1025^2 values -> 25.2 MB in FP64 (too big), 12.6 MB in FP32 (fits)
    N, p, k = 512, 2, 2
    ctx = stmg.Context(2, N, p, k, 0.01, omega=[0.3] * 16, vcycle_precision=stmg.FP32)
    n = ctx.nt * ctx.n_nodes
    assert n * 8 > SCRATCH_BYTES >= n * 4
    f64 = torch.zeros(n, dtype=torch.float64, device="cuda")
    u64 = torch.zeros_like(f64)
    with pytest.raises(stmg.StmgError) as err:
        ctx.smooth_noalloc(f64, u64, sweeps=1, level=0)
    assert err.value.status == 1 and "bytes" in str(err.value)
    # the context stays usable, and the FP32 level fits
    f32 = torch.from_numpy(synth.random_vector(n, seed=5).astype(np.float32)).cuda()
    u_a = torch.zeros(n, dtype=torch.float32, device="cuda")
    u_b = torch.zeros_like(u_a)
    ctx.smooth(f32, u_a, sweeps=1, level=0)
    ctx.smooth_noalloc(f32, u_b, sweeps=1, level=0)
    assert rel_err(u_b.cpu().numpy(), u_a.cpu().numpy()) < 2e-5
    ctx.close()


_FRESH_PROCESS = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import paper_2408_04372_gb300 as stmg
torch.cuda.set_device(0)
N, p, k = 6, 2, 2  # 3D Q2 dG(2): 3 * 13^3 values
ctx = stmg.Context(3, N, p, k, 0.05, omega=[0.3] * 8, vcycle_precision=stmg.FP32)
n = ctx.nt * ctx.n_nodes
f = torch.ones(n, dtype=torch.float32, device="cuda")
u = torch.zeros_like(f)
u_ref = torch.zeros_like(f)
ctx.smooth(f, u_ref, sweeps=1, level=0)  # loads the smoother kernels; allocates the context's own scratch
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
ctx.smooth_noalloc(f, u, sweeps=1, level=0)  # first call of the process
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
err = float((u - u_ref).abs().max() / u_ref.abs().max())
print(free0, free1, err)
"""


def test_first_noalloc_call_takes_no_device_memory(env):
    """In a fresh process the first call must not take the fixed buffer: stmg_create already did."""
    import subprocess
    import sys

    from gpu_cases import ROOT
    res = subprocess.run([sys.executable, "-c", _FRESH_PROCESS, ROOT], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    free0, free1, err = res.stdout.split()[-3:]
    drop = int(free0) - int(free1)
    assert drop < SCRATCH_BYTES // 4, f"free device memory fell by {drop} bytes at the first call"
    assert float(err) < 2e-5
