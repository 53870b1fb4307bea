"""Shared set-up of the GPU parity tests: seeded cases, library loading, oracle hierarchies."""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@dataclass(frozen=True)
class Case:
    name: str
    dim: int
    N: int
    p: int
    k: int
    pde: str
    scheme: str
    tau: float
    jitter: bool
    coeff: str  # "one", "blocks", "layers"

    def vertices(self):
        return synth.jittered_vertices(self.N, self.dim) if self.jitter else synth.cartesian_vertices(self.N, self.dim)

    def rho_cell(self):
        if self.coeff == "blocks":
            b = 2 if self.N % 2 == 0 else 1
            return synth.block_coefficient(self.N, self.dim, blocks=b)
        if self.coeff == "layers":
            return synth.layer_coefficient(self.N, self.dim, 1.0, 16.0)
        return np.ones(self.N ** self.dim)


CASES = [
    Case("heat2d_q2_dg1", 2, 4, 2, 1, "heat", "dg", 1 / 16, False, "one"),
    Case("heat3d_q2_dg2_jit", 3, 4, 2, 2, "heat", "dg", 1 / 32, True, "blocks"),
    Case("wave3d_q3_cgp2_jit", 3, 3, 3, 2, "wave", "cgp", 1 / 64, True, "layers"),
    Case("heat2d_q4_dg3_jit", 2, 3, 4, 3, "heat", "dg", 0.05, True, "blocks"),
    Case("heat3d_q1_dg0", 3, 2, 1, 0, "heat", "dg", 0.1, False, "one"),
    Case("heat3d_q2_cgp1_jit", 3, 4, 2, 1, "heat", "cgp", 1 / 16, True, "blocks"),
    Case("wave2d_q2_dg1", 2, 4, 2, 1, "wave", "dg", 1 / 32, True, "layers"),
    # 3D Cartesian grids with a constant coefficient: the library picks fast diagonalisation (exact here)
    Case("heat3d_q3_dg1_cart_fd", 3, 4, 3, 1, "heat", "dg", 1 / 16, False, "one"),
    Case("wave3d_q2_cgp2_cart_fd", 3, 4, 2, 2, "wave", "cgp", 1 / 32, False, "one"),
    Case("heat3d_q4_dg3_cart_fd", 3, 2, 4, 3, "heat", "dg", 1 / 8, False, "one"),
]

_HIER = {}


def oracle_hierarchy(case: Case):
    from oracle import mg
    if case.name not in _HIER:
        _HIER[case.name] = mg.Hierarchy(case.dim, case.N, case.p, case.k, case.pde, case.scheme, case.tau,
                                        case.vertices(), rho_cell=case.rho_cell())
    return _HIER[case.name]


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_04372_gb300 as stmg
    if not os.path.exists(stmg.LIB_PATH):
        from paper_2408_04372_gb300 import build
        build.build()
    stmg.load()
    return torch, stmg


def make_context(stmg, case: Case, H, **kw):
    pde = stmg.HEAT if case.pde == "heat" else stmg.WAVE
    scheme = stmg.DG if case.scheme == "dg" else stmg.CGP
    kw.setdefault("omega", H.omegas())
    return stmg.Context(case.dim, case.N, case.p, case.k, case.tau, pde=pde, scheme=scheme,
                        vertices=case.vertices(), coeff=case.rho_cell(), **kw)


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
