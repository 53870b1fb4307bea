"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds no arithmetic of the space-time multigrid method: it only draws
meshes, coefficients, sources and random vectors.  Everything here is input data.

Conventions shared with the library (all arrays FP64, lexicographic, x fastest):
  vertices  : ((N+1)^dim, dim)  structured hexahedral / quadrilateral grid
  cell data : (N^dim,)          cell (ix, iy, iz) -> ix + N*(iy + N*iz)
  vectors   : (N_t, n_nodes)    time-major blocks of nodal values

Seeds follow the workload recipes: mesh jitter 11, coefficients 12, Gaussian
paths 13, random test vectors 14.
"""
from __future__ import annotations

import math
import numpy as np

SEED_JITTER = 11
SEED_COEFF = 12
SEED_PATHS = 13
SEED_VECTORS = 14

_MASK64 = (1 << 64) - 1


def splitmix64(i: int) -> int:
    """SplitMix64 (Steele, Lea, Flood 2014): 64-bit counter-based generator."""
    z = (i + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def splitmix_uniform(n: int, key: int = 0) -> np.ndarray:
    """n values in [-1, 1): u_i = 2*(splitmix64(key*2^32 + i) >> 11) * 2^-53 - 1."""
    out = np.empty(n, dtype=np.float64)
    base = (key << 32) & _MASK64
    for i in range(n):
        out[i] = 2.0 * ((splitmix64(base + i) >> 11) * 2.0 ** -53) - 1.0
    return out


def cartesian_vertices(N, dim, lo=0.0, hi=1.0) -> np.ndarray:
    """Vertices of a uniform grid of N^dim cells on [lo, hi]^dim."""
    t = np.linspace(lo, hi, N + 1)
    grids = np.meshgrid(*([t] * dim), indexing="ij")
    # lexicographic with x fastest -> reverse the axis order of an ij meshgrid
    cols = [g.transpose(tuple(range(dim))[::-1]).reshape(-1) for g in grids]
    return np.stack(cols, axis=1)


def jittered_vertices(N, dim, frac=0.15, seed=SEED_JITTER, lo=0.0, hi=1.0) -> np.ndarray:
    """Cartesian vertices with every interior vertex coordinate moved by U[-frac*h, frac*h].

    Boundary vertices stay fixed so the domain remains [lo, hi]^dim.
    """
    v = cartesian_vertices(N, dim, lo, hi)
    h = (hi - lo) / N
    rng = np.random.default_rng(seed)
    shift = rng.uniform(-frac * h, frac * h, size=v.shape)
    idx = np.indices((N + 1,) * dim).reshape(dim, -1)[::-1].T  # (nv, dim), x index first
    interior = np.all((idx > 0) & (idx < N), axis=1)
    v[interior] += shift[interior]
    return v


def cell_index_grid(N, dim) -> np.ndarray:
    """(N^dim, dim) integer cell indices, x index first, lexicographic x fastest."""
    return np.indices((N,) * dim).reshape(dim, -1)[::-1].T.copy()


def block_coefficient(N, dim, blocks=4, seed=SEED_COEFF, log10_range=(-2.0, 2.0)) -> np.ndarray:
    """Per-cell coefficient, constant on a blocks^dim grid of equal blocks, log-uniform values."""
    assert N % blocks == 0
    rng = np.random.default_rng(seed)
    vals = 10.0 ** rng.uniform(log10_range[0], log10_range[1], size=(blocks,) * dim)
    c = cell_index_grid(N, dim) // (N // blocks)
    return np.array([vals[tuple(ci)] for ci in c], dtype=np.float64)


def layer_coefficient(N, dim, below=1.0, above=16.0, z_split=0.5) -> np.ndarray:
    """Per-cell coefficient: `below` for cells whose logical centre has z < z_split, else `above`."""
    c = cell_index_grid(N, dim)
    zc = (c[:, dim - 1] + 0.5) / N
    return np.where(zc < z_split, below, above).astype(np.float64)


def smooth_coefficient_params(dim, seed=SEED_COEFF):
    """Frequencies a_d in {1..4} and phases phi_d in U[0, 2pi) for rho = 1 + 0.5 prod sin(a pi x + phi)."""
    rng = np.random.default_rng(seed)
    a = rng.integers(1, 5, size=dim).astype(np.float64)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=dim)
    return a, phi


def smooth_coefficient_at(points: np.ndarray, a, phi) -> np.ndarray:
    """rho(x) = 1 + 0.5 * prod_d sin(a_d pi x_d + phi_d) at the given (..., dim) points."""
    s = np.ones(points.shape[:-1])
    for d in range(points.shape[-1]):
        s = s * np.sin(a[d] * math.pi * points[..., d] + phi[d])
    return 1.0 + 0.5 * s


def random_vector(shape, seed=SEED_VECTORS) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal(shape)


# ---- analytic problem data (evaluated at points the caller supplies) ----

def heat_sine_solution(x: np.ndarray, t: float) -> np.ndarray:
    """u = prod_d sin(pi x_d) * sin(pi t)."""
    s = np.full(x.shape[:-1], math.sin(math.pi * t))
    for d in range(x.shape[-1]):
        s = s * np.sin(math.pi * x[..., d])
    return s


def heat_sine_source(x: np.ndarray, t: float) -> np.ndarray:
    """f = u_t - Laplace(u) for u = prod sin(pi x_d) sin(pi t), unit diffusivity."""
    dim = x.shape[-1]
    s = np.ones(x.shape[:-1])
    for d in range(dim):
        s = s * np.sin(math.pi * x[..., d])
    return s * (math.pi * math.cos(math.pi * t) + dim * math.pi ** 2 * math.sin(math.pi * t))


def wave_pulse(x: np.ndarray, x0=(0.5, 0.5, 0.25), sigma=0.05) -> np.ndarray:
    """Gaussian pulse exp(-|x - x0|^2 / (2 sigma^2))."""
    r2 = np.zeros(x.shape[:-1])
    for d in range(x.shape[-1]):
        r2 = r2 + (x[..., d] - x0[d]) ** 2
    return np.exp(-r2 / (2.0 * sigma ** 2))


# ---- structural-health-monitoring-like wave problem (Section 4.3 of the paper, reduced) ----

SHM_POINTS = ((0.75, 0.0, 0.0), (0.0, 0.0, 0.75), (0.75, 0.1, 0.75))  # goal-quantity points


def shm_coefficient(N, rough=False, seed=SEED_COEFF, coarse=5) -> np.ndarray:
    """Per-cell coefficient on [-1, 1]^3 with N cells per direction (N a multiple of `coarse`):
    1 for y < 0.2, 9 for y >= 0.2 and z < 0.2, 16 for y >= 0.2 and z >= 0.2 (at the cell centre);
    rough: times c ~ U[0.4, 1.6] drawn per cell of the coarse^3 grid (seeded)."""
    assert N % coarse == 0
    c = cell_index_grid(N, 3)
    ctr = -1.0 + (c + 0.5) * (2.0 / N)
    y, z = ctr[:, 1], ctr[:, 2]
    rho = np.where(y < 0.2, 1.0, np.where(z < 0.2, 9.0, 16.0))
    if rough:
        fac = np.random.default_rng(seed).uniform(0.4, 1.6, size=coarse ** 3)
        cc = c // (N // coarse)
        rho = rho * fac[cc[:, 0] + coarse * (cc[:, 1] + coarse * cc[:, 2])]
    return rho.astype(np.float64)


def shm_initial(x: np.ndarray, s=0.01) -> np.ndarray:
    """u0 = exp(-|x/s|^2) (1 - |x/s|^2) for |x| < s, else 0."""
    r2 = np.zeros(x.shape[:-1])
    for d in range(x.shape[-1]):
        r2 = r2 + (x[..., d] / s) ** 2
    return np.where(r2 < 1.0, np.exp(-r2) * (1.0 - r2), 0.0)


class MovingGaussians:
    """Source f(x, t) = sum_g A_g exp(-|x - c_g(t)|^2 / (2 w^2)), c_g(t) = 0.5 + 0.3 sin(2 pi om t + phi)."""

    def __init__(self, n=8, dim=3, width=0.06, seed=SEED_PATHS):
        rng = np.random.default_rng(seed)
        self.amp = rng.uniform(0.5, 2.0, size=n)
        self.om = rng.uniform(0.5, 2.0, size=(n, dim))
        self.phi = rng.uniform(0.0, 2.0 * math.pi, size=(n, dim))
        self.width = width

    def __call__(self, x: np.ndarray, t: float) -> np.ndarray:
        f = np.zeros(x.shape[:-1])
        for g in range(len(self.amp)):
            c = 0.5 + 0.3 * np.sin(2.0 * math.pi * self.om[g] * t + self.phi[g])
            r2 = np.zeros(x.shape[:-1])
            for d in range(x.shape[-1]):
                r2 = r2 + (x[..., d] - c[d]) ** 2
            f = f + self.amp[g] * np.exp(-r2 / (2.0 * self.width ** 2))
        return f


def conv_net_init(channels=(4, 60, 60, 60, 2), seed=15, last_scale=0.1):
    """He-normal weights (Co, Ci, 27) and zero biases for a chain of 3x3x3 convolutions."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for l in range(len(channels) - 1):
        ci, co = channels[l], channels[l + 1]
        std = math.sqrt(2.0 / (27 * ci))
        w = rng.standard_normal((co, ci, 27)) * std
        if l == len(channels) - 2:
            w *= last_scale
        W.append(w)
        b.append(np.zeros(co))
    return W, b
