"""Pins of the oracle's point evaluation (goal quantities, Section 4.3) and of the reduced SHM inputs."""
import numpy as np
import pytest

import synth
from oracle import points, space


@pytest.mark.parametrize("p", [1, 2, 3])
def test_qp_polynomials_are_reproduced_at_arbitrary_points_of_a_cartesian_grid(p):
    N = 5
    g = space.Grid(N, 3, p, synth.cartesian_vertices(N, 3, lo=-1.0, hi=1.0))
    X = g.node_coords()
    q = lambda x: (x[..., 0] ** p + 0.5) * (x[..., 1] - 0.3) ** min(p, 2) * (1.0 + x[..., 2] ** p)
    pts = np.random.default_rng(3).uniform(-0.99, 0.99, size=(6, 3))
    vals = points.point_values(g, q(X), pts)
    assert np.allclose(vals, q(pts), rtol=1e-12, atol=1e-12)


def test_linear_functions_are_reproduced_on_a_jittered_grid():
    N = 4
    g = space.Grid(N, 3, 2, synth.jittered_vertices(N, 3))
    X = g.node_coords()
    lin = lambda x: 0.3 + x @ np.array([1.0, -2.0, 0.5])
    pts = np.random.default_rng(4).uniform(0.02, 0.98, size=(6, 3))
    assert np.allclose(points.point_values(g, lin(X), pts), lin(pts), atol=1e-12)
    # a node returns its nodal value; the located reference point maps back to the point
    u = synth.random_vector(g.n_nodes, seed=5)
    k = 123
    assert np.isclose(points.point_values(g, u, [X[k]])[0], u[k], atol=1e-12)
    c, xi = points.locate(g, pts[0])
    val, _ = g.q1_shape(xi[None, :])
    assert np.allclose(val[0] @ g.cell_vertices()[c], pts[0], atol=1e-13)


def test_shm_coefficient_layers_and_rough_factor():
    N = 10
    rho = synth.shm_coefficient(N)
    c = synth.cell_index_grid(N, 3)
    ctr = -1.0 + (c + 0.5) * (2.0 / N)
    assert np.all(rho[ctr[:, 1] < 0.2] == 1.0)
    assert np.all(rho[(ctr[:, 1] > 0.2) & (ctr[:, 2] < 0.2)] == 9.0)
    assert np.all(rho[(ctr[:, 1] > 0.2) & (ctr[:, 2] > 0.2)] == 16.0)
    rough = synth.shm_coefficient(N, rough=True)
    f = rough / rho
    assert f.min() >= 0.4 and f.max() <= 1.6
    # one factor per cell of the 5^3 coarse grid: constant on the 2^3 fine cells inside it
    cc = c // 2
    key = cc[:, 0] + 5 * (cc[:, 1] + 5 * cc[:, 2])
    for k in range(125):
        assert np.ptp(f[key == k]) < 1e-15
    assert len(np.unique(np.round(f, 12))) == 125
    # initial bump: 1 at the origin, 0 outside radius s, value exp(-r^2)(1 - r^2) inside
    x = np.array([[0.0, 0.0, 0.0], [0.005, 0.0, 0.0], [0.02, 0.0, 0.0]])
    assert np.allclose(synth.shm_initial(x), [1.0, np.exp(-0.25) * 0.75, 0.0])
