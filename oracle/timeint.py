"""Time discretisation weights and slab systems, FP64.

Test infrastructure (see oracle/__init__.py).

dG(k) (Section 2.1, eq. dg-time-weights), basis = Lagrange at the k+1 right
Gauss-Radau points of [0, 1], N_t = k+1:
    Mhat_ij = int xi_j xi_i,   Ahat_ij = int xi_j' xi_i + xi_j(0) xi_i(0),   alpha_i = xi_i(0)
  Reading of the garbled print: the jump term of eq. var-heat-dg tests with
  w_{n-1}^+, i.e. the values at t^ = 0, so the upwind term is xi_j(0) xi_i(0) and
  alpha_i = xi_i(0); the previous slab's end value is the last DoF (node t^ = 1).

cGP(k) (Section 2.2, eq. cg-time-weights), trial = Lagrange at the k+1
Gauss-Lobatto points, test psi_i = Lagrange of degree k-1 at the last k
Gauss-Lobatto points, N_t = k:
    Mhat[i, j-1] = int xi_j psi_i,  Ahat[i, j-1] = int xi_j' psi_i   (j = 2..k+1)
    betahat_i = int xi_1 psi_i,     alpha_i = int xi_1' psi_i
Scaling with the step tau: M_tau = tau Mhat, beta = tau betahat, A_tau = Ahat.

Slab systems (all of the form S = T_A (x) A_h + T_M (x) M_h):
  heat dG   eq. heat-cg-dg : T_A = M_tau, T_M = A_tau,
            rhs = M_tau(x)M_h f + alpha(x)M_h u_prev
  heat cGP  eq. heat-cg-cg : same S; rhs signs derived from the variational form
            (the printed signs of the known-data terms disagree with it):
            rhs = M_tau(x)M_h f + beta(x)M_h f0 - (beta(x)A_h + alpha(x)M_h) u0
  wave dG   eq. wave-cg-dg : T_A = M_tau, T_M = A_tau M_tau^-1 A_tau,
            rhs = M_tau(x)M_h f + alpha(x)M_h v_prev + A_tau M_tau^-1 alpha (x) M_h u_prev,
            v = M_tau^-1 (A_tau u - alpha u_prev)
  wave cGP  eq. wave-cg-cg : T_A = M_tau, T_M = A_tau M_tau^-1 A_tau,
            rhs = M_tau(x)M_h f + beta(x)M_h f0 - (beta(x)A_h + A_tau M_tau^-1 alpha (x) M_h) u0
                  - (alpha - A_tau M_tau^-1 beta)(x)M_h v0,
            v = M_tau^-1 (A_tau u + alpha u0 - beta v0)
Pins: tests/test_oracle_time.py (closed forms for dG(0..2), cGP(1..2); backward
Euler and Crank-Nicolson special cases; constant preservation; positivity of
the dG symmetric part; convergence orders of the slab marching).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import fe1d

DG, CGP = "dg", "cgp"
HEAT, WAVE = "heat", "wave"


@dataclass
class TimeWeights:
    scheme: str
    k: int
    nodes: np.ndarray      # free time nodes in [0, 1] (N_t of them)
    Mhat: np.ndarray
    Ahat: np.ndarray
    alpha: np.ndarray
    betahat: np.ndarray    # zeros for dG

    @property
    def nt(self) -> int:
        return len(self.nodes)


def dg_weights(k: int) -> TimeWeights:
    nodes, _ = fe1d.gauss_radau_right(k + 1)
    tq, wq = fe1d.gauss_legendre(k + 3)
    V, D = fe1d.basis_table(nodes, tq)          # (q, j)
    V0, _ = fe1d.basis_table(nodes, np.array([0.0]))
    n = k + 1
    Mhat = np.zeros((n, n))
    Ahat = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            Mhat[i, j] = np.sum(wq * V[:, j] * V[:, i])
            Ahat[i, j] = np.sum(wq * D[:, j] * V[:, i]) + V0[0, j] * V0[0, i]
    alpha = V0[0, :].copy()
    return TimeWeights(DG, k, nodes, Mhat, Ahat, alpha, np.zeros(n))


def cgp_weights(k: int) -> TimeWeights:
    assert k >= 1
    gl, _ = fe1d.gauss_lobatto(k + 1)
    test_nodes = gl[1:]
    tq, wq = fe1d.gauss_legendre(k + 3)
    Xi, dXi = fe1d.basis_table(gl, tq)            # trial, (q, k+1)
    if k == 1:
        Psi = np.ones((len(tq), 1))
    else:
        Psi, _ = fe1d.basis_table(test_nodes, tq)  # test, (q, k)
    Mhat = np.zeros((k, k))
    Ahat = np.zeros((k, k))
    beta = np.zeros(k)
    alpha = np.zeros(k)
    for i in range(k):
        for j in range(1, k + 1):
            Mhat[i, j - 1] = np.sum(wq * Xi[:, j] * Psi[:, i])
            Ahat[i, j - 1] = np.sum(wq * dXi[:, j] * Psi[:, i])
        beta[i] = np.sum(wq * Xi[:, 0] * Psi[:, i])
        alpha[i] = np.sum(wq * dXi[:, 0] * Psi[:, i])
    return TimeWeights(CGP, k, test_nodes, Mhat, Ahat, alpha, beta)


def weights(scheme: str, k: int) -> TimeWeights:
    return dg_weights(k) if scheme == DG else cgp_weights(k)


@dataclass
class SlabSystem:
    """S = T_A (x) A_h + T_M (x) M_h and the coefficient matrices of the right-hand side.

    rhs = sum over known data d of  RA[d] (x) A_h d + RM[d] (x) M_h d   with d in
    {"f": (N_t blocks), "f0", "u0", "v0"}; RA/RM entries are (N_t,) or (N_t, N_t).
    """
    pde: str
    tw: TimeWeights
    tau: float
    TA: np.ndarray
    TM: np.ndarray
    RM_f: np.ndarray
    RM_f0: np.ndarray
    RA_u0: np.ndarray
    RM_u0: np.ndarray
    RM_v0: np.ndarray
    # velocity update v = VU u + Vu0 u0 + Vv0 v0  (wave only)
    VU: np.ndarray | None = None
    Vu0: np.ndarray | None = None
    Vv0: np.ndarray | None = None


def slab_system(pde: str, scheme: str, k: int, tau: float) -> SlabSystem:
    tw = weights(scheme, k)
    n = tw.nt
    Mt = tau * tw.Mhat
    At = tw.Ahat.copy()
    beta = tau * tw.betahat
    alpha = tw.alpha
    z = np.zeros(n)
    if pde == HEAT:
        if scheme == DG:
            return SlabSystem(pde, tw, tau, Mt, At, Mt, z, z, alpha.copy(), z)
        return SlabSystem(pde, tw, tau, Mt, At, Mt, beta.copy(), -beta, -alpha, z)
    Minv = np.linalg.inv(Mt)
    AMA = At @ Minv @ At
    if scheme == DG:
        # eq. wave-cg-dg: v = M^-1 A u - M^-1 alpha u_prev
        return SlabSystem(pde, tw, tau, Mt, AMA, Mt, z, z, At @ Minv @ alpha, alpha.copy(),
                          VU=Minv @ At, Vu0=-(Minv @ alpha), Vv0=z.copy())
    # cGP wave, derived from the variational form (see module docstring)
    return SlabSystem(pde, tw, tau, Mt, AMA, Mt, beta.copy(), -beta, -(At @ Minv @ alpha),
                      -(alpha - At @ Minv @ beta),
                      VU=Minv @ At, Vu0=Minv @ alpha, Vv0=-(Minv @ beta))
