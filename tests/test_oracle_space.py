"""Pins of the oracle's spatial operators (eq. space-matrices) and the Kronecker slab structure."""
import numpy as np
import scipy.sparse as sp

import synth
from oracle import fe1d, space, timeint


def _grid(N, dim, p, jitter=False):
    V = synth.jittered_vertices(N, dim) if jitter else synth.cartesian_vertices(N, dim)
    return space.Grid(N, dim, p, V)


def test_cartesian_matrices_are_kronecker_sums():
    N, p = 3, 2
    g1 = space.Grid(N, 1, p, synth.cartesian_vertices(N, 1))
    A1, M1 = g1.assemble(np.ones((N, p + 1)))
    for dim in (2, 3):
        g = _grid(N, dim, p)
        A, M = g.assemble(space.rho_qp_from_cells(g, np.ones(g.n_cells)))
        if dim == 2:
            Ak = sp.kron(M1, A1) + sp.kron(A1, M1)
            Mk = sp.kron(M1, M1)
        else:
            Ak = sp.kron(sp.kron(M1, M1), A1) + sp.kron(sp.kron(M1, A1), M1) + sp.kron(sp.kron(A1, M1), M1)
            Mk = sp.kron(sp.kron(M1, M1), M1)
        assert abs(A - Ak).max() < 1e-12 and abs(M - Mk).max() < 1e-14


def test_mass_constants_and_linear_energy_on_perturbed_meshes():
    for dim, p in ((2, 1), (2, 3), (3, 2)):
        g = _grid(4, dim, p, jitter=True)
        A, M = g.assemble(space.rho_qp_from_cells(g, np.ones(g.n_cells)))
        one = np.ones(g.n_nodes)
        assert np.isclose(one @ M @ one, 1.0, atol=1e-13)          # |Omega| = 1
        assert np.abs(A @ one).max() < 1e-11                        # constants have no energy
        a = np.array([0.3, -1.2, 0.7][:dim])
        u = g.node_coords() @ a                                     # linear functions lie in the space
        assert np.isclose(u @ A @ u, a @ a, rtol=1e-12)             # int |a|^2 = |a|^2 |Omega|


def test_coefficient_scales_stiffness():
    g = _grid(2, 3, 2, jitter=True)
    A1, _ = g.assemble(space.rho_qp_from_cells(g, np.ones(g.n_cells)))
    A7, _ = g.assemble(space.rho_qp_from_cells(g, 7.0 * np.ones(g.n_cells)))
    assert abs(A7 - 7.0 * A1).max() < 1e-12


def test_direct_space_time_assembly_equals_kronecker_form():
    """Assemble S by space-time quadrature on K x I_n and compare with M_tau(x)A_h + A_tau(x)M_h."""
    dim, N, p, k, tau = 2, 3, 2, 2, 0.3
    g = _grid(N, dim, p, jitter=True)
    rng = np.random.default_rng(5)
    rho_qp = rng.uniform(0.5, 2.0, size=(g.n_cells, (p + 1) ** dim))
    A, M = g.assemble(rho_qp)
    tw = timeint.dg_weights(k)
    S_kron = sp.kron(tau * tw.Mhat, A) + sp.kron(tw.Ahat, M)

    phi, dphi = g.ref_basis()
    J = g.jacobians(g.quad_points_ref())
    jw = np.abs(np.linalg.det(J)) * g.quad_weights()[None, :]
    grad = np.einsum("cqed,qbe->cqbd", np.linalg.inv(J), dphi)
    ts, ws = fe1d.gauss_legendre(k + 3)
    Xi, dXi = fe1d.basis_table(tw.nodes, ts)
    Xi0, _ = fe1d.basis_table(tw.nodes, np.array([0.0]))
    nt, nb, nn = k + 1, phi.shape[1], g.n_nodes
    S = np.zeros((nt * nn, nt * nn))
    dofs = g.cell_dofs()
    for c in range(g.n_cells):
        for i in range(nt):
            for j in range(nt):
                blk = np.zeros((nb, nb))
                for s in range(len(ts)):
                    # d/dt of xi_j on I_n is xi_j'/tau; dt = tau dt^
                    wt = tau * ws[s]
                    blk += wt * (dXi[s, j] / tau) * Xi[s, i] * np.einsum("q,qa,qb->ab", jw[c], phi, phi)
                    blk += wt * Xi[s, j] * Xi[s, i] * np.einsum("q,qad,qbd->ab", jw[c] * rho_qp[c], grad[c], grad[c])
                blk += Xi0[0, j] * Xi0[0, i] * np.einsum("q,qa,qb->ab", jw[c], phi, phi)
                r = i * nn + dofs[c]
                cidx = j * nn + dofs[c]
                S[np.ix_(r, cidx)] += blk
    assert np.abs(S - S_kron.toarray()).max() < 1e-12 * np.abs(S).max()
