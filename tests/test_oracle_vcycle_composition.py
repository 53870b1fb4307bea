"""Pin of the oracle's V-cycle composition (Algorithm stmg, Section 3) by its error propagation.

One V-cycle with zero initial guess is a linear map f -> V f.  Algorithm stmg fixes it through the
error propagation E = I - V S of the iteration u <- u + V (f - S u), level by level:

    E_L = 0                                                     (coarsest level: exact solve)
    E_l = (I - w_l B_l S_l)^nu2 (I - P_l (I - E_{l+1}) S_{l+1}^-1 P_l^T S_l) (I - w_l B_l S_l)^nu1

(pre-smoothing nu1 times from the zero guess, the coarse correction from the restricted residual,
solved by one V-cycle on the next level, then nu2 post-smoothing sweeps).  The recursion below is
built from dense per-level matrices on the unconstrained DoFs only (constrained rows are identity
rows of S and carry no correction), with the coarsest inverse taken afresh; it shares nothing with
oracle.mg.Hierarchy.vcycle but the level matrices, which other pins fix (Kronecker identity,
brute-force Schwarz operator, polynomial reproduction of the transfers).  Each test compares
I - V S, with V assembled column by column from the oracle's vcycle on unit vectors, against E to
1e-12, and checks that planted mistakes (no post-smoothing, nu1 and nu2 swapped, pre-smoothing
from the right-hand side instead of zero) are caught.
"""
import numpy as np
import pytest

import synth
from oracle import atonce, mg


def _dense(A, idx_r, idx_c):
    A = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    return A[np.ix_(idx_r, idx_c)]


def _error_propagation(levels, interiors, nu1, nu2):
    """E on the unconstrained DoFs of level 0 by the recursion of the module docstring."""
    L = len(levels) - 1
    E = np.zeros((interiors[L].sum(),) * 2)      # E_L = 0
    S_next = _dense(levels[L].prob.S, interiors[L], interiors[L])
    for li in range(L - 1, -1, -1):
        lev, I_f, I_c = levels[li], interiors[li], interiors[li + 1]
        S = _dense(lev.prob.S, I_f, I_f)
        B = _dense(lev.B, I_f, I_f)
        P = _dense(lev.P, I_f, I_c)
        n = S.shape[0]
        Id = np.eye(n)
        G = Id - lev.omega * B @ S
        coarse = Id - P @ (np.eye(len(E)) - E) @ np.linalg.inv(S_next) @ P.T @ S
        E = np.linalg.matrix_power(G, nu2) @ coarse @ np.linalg.matrix_power(G, nu1)
        S_next = S
    return E


def _vcycle_matrix(vcycle, n, interior):
    cols = []
    for j in np.flatnonzero(interior):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(vcycle(e)[interior])
    return np.array(cols).T


def _mismatch(vcycle, levels, interiors, nu1, nu2):
    lev0 = levels[0]
    I0 = interiors[0]
    V = _vcycle_matrix(vcycle, lev0.prob.n, I0)
    S = _dense(lev0.prob.S, I0, I0)
    E = _error_propagation(levels, interiors, nu1, nu2)
    return np.abs(np.eye(len(S)) - V @ S - E).max() / max(np.abs(E).max(), 1.0)


SLAB_CASES = [
    # (dim, N, p, k, pde, scheme, tau, jitter, weighted)
    (2, 4, 2, 1, "heat", "dg", 0.05, True, False),
    (2, 4, 2, 2, "wave", "cgp", 0.05, True, False),
    (2, 4, 2, 1, "heat", "cgp", 0.05, False, True),
    (3, 2, 2, 1, "heat", "dg", 0.1, True, False),
]


def _slab_hierarchy(dim, N, p, k, pde, scheme, tau, jitter, weighted):
    V = synth.jittered_vertices(N, dim) if jitter else synth.cartesian_vertices(N, dim)
    rho = synth.block_coefficient(N, dim, blocks=2)
    return mg.Hierarchy(dim, N, p, k, pde, scheme, tau, V, rho_cell=rho, weighted=weighted)


@pytest.mark.parametrize("case", SLAB_CASES, ids=lambda c: f"{c[4]}{c[0]}d_q{c[2]}_{c[5]}{c[3]}_w{int(c[8])}")
@pytest.mark.parametrize("nu1,nu2", [(1, 1), (1, 2), (2, 0)])
def test_slab_vcycle_equals_its_error_propagation(case, nu1, nu2):
    H = _slab_hierarchy(*case)
    assert len(H.levels) >= 3  # at least two coarse-grid corrections nested
    interiors = [lev.interior for lev in H.levels]
    err = _mismatch(lambda f: H.vcycle(f, nu1=nu1, nu2=nu2), H.levels, interiors, nu1, nu2)
    assert err < 1e-12, err


def test_slab_vcycle_pin_catches_planted_mistakes():
    H = _slab_hierarchy(*SLAB_CASES[0])
    interiors = [lev.interior for lev in H.levels]

    # 1. post-smoothing dropped
    assert _mismatch(lambda f: H.vcycle(f, nu1=1, nu2=0), H.levels, interiors, 1, 1) > 1e-3
    # 2. nu1 and nu2 swapped
    assert _mismatch(lambda f: H.vcycle(f, nu1=2, nu2=1), H.levels, interiors, 1, 2) > 1e-3

    # 3. pre-smoothing started from the right-hand side instead of the zero guess
    class WrongStart(mg.Hierarchy):
        def vcycle(self, f, li=0, nu1=1, nu2=1):
            lev = self.levels[li]
            if li == len(self.levels) - 1:
                return lev.coarse_inv @ f
            u = self.smooth(li, f, f.copy(), nu1)
            e = self.vcycle(lev.P.T @ (f - lev.prob.S @ u), li + 1, nu1, nu2)
            return self.smooth(li, f, u + lev.P @ e, nu2)

    Hw = _slab_hierarchy(*SLAB_CASES[0])
    Hw.__class__ = WrongStart
    assert _mismatch(lambda f: Hw.vcycle(f), Hw.levels, interiors, 1, 1) > 1e-3

    # 4. coarse correction added without prolongation weights (P replaced by its pattern)
    class PatternP(mg.Hierarchy):
        def vcycle(self, f, li=0, nu1=1, nu2=1):
            lev = self.levels[li]
            if li == len(self.levels) - 1:
                return lev.coarse_inv @ f
            u = self.smooth(li, f, np.zeros_like(f), nu1)
            e = self.vcycle(lev.P.T @ (f - lev.prob.S @ u), li + 1, nu1, nu2)
            Pp = lev.P.copy()
            Pp.data = np.sign(Pp.data)
            return self.smooth(li, f, u + Pp @ e, nu2)

    Hp = _slab_hierarchy(*SLAB_CASES[0])
    Hp.__class__ = PatternP
    assert _mismatch(lambda f: Hp.vcycle(f), Hp.levels, interiors, 1, 1) > 1e-3


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (2, 1)])
@pytest.mark.parametrize("weighted", [False, True])
def test_at_once_vcycle_equals_its_error_propagation(nu1, nu2, weighted):
    """Several slabs in one system (eq. heat-cg-dg-at-once): space, tau and k levels nested."""
    dim, N, p, k, tau, nc = 2, 4, 2, 1, 0.05, 4
    V = synth.jittered_vertices(N, dim)
    rho = synth.block_coefficient(N, dim, blocks=2)
    H = atonce.AtOnceHierarchy(dim, N, p, k, tau, nc, V, rho_cell=rho, weighted=weighted)
    assert any(a.spec.nc != b.spec.nc for a, b in zip(H.levels, H.levels[1:]))  # a tau level is nested
    interiors = [~lev.prob.bmask_full for lev in H.levels]
    err = _mismatch(lambda f: H.vcycle(f, nu1=nu1, nu2=nu2), H.levels, interiors, nu1, nu2)
    assert err < 1e-12, err
    # planted mistake: post-smoothing dropped
    assert _mismatch(lambda f: H.vcycle(f, nu1=nu1, nu2=0), H.levels, interiors, nu1, nu2) > 1e-3
