// Host-side FP64 tables: quadrature rules, Lagrange bases, time weights,
// slab-system coefficients and small dense linear algebra.
#pragma once

#include <complex>
#include <vector>

namespace stmg {

using cplx = std::complex<double>;

// Quadrature rules on [0, 1].
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);
void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w);
void gauss_radau_right(int n, std::vector<double>& x, std::vector<double>& w);

double lagrange(const std::vector<double>& nodes, int j, double t);
double lagrange_deriv(const std::vector<double>& nodes, int j, double t);

// Nodes of the 1D Q_p basis (Gauss-Lobatto points).
std::vector<double> space_nodes(int p);

// Time weights (Section 2, eqs. dg-time-weights and cg-time-weights).
struct TimeWeights {
  int scheme;  // 0 dG, 1 cGP
  int k;
  int nt;
  std::vector<double> nodes;   // free nodes in [0,1]
  std::vector<double> Mhat, Ahat, alpha, betahat;  // nt x nt row-major, nt
};
TimeWeights time_weights(int scheme, int k);

// Slab system S = TA (x) A_h + TM (x) M_h and the right-hand-side coefficients:
// rhs = RM_f (x) M_h f + RM_f0 (x) M_h f0 + RA_u0 (x) A_h u0 + RM_u0 (x) M_h u0 + RM_v0 (x) M_h v0
// velocity (wave): v = VU u + Vu0 u0 + Vv0 v0.
struct SlabCoeffs {
  int nt;
  std::vector<double> TA, TM, RM_f;         // nt x nt
  std::vector<double> RM_f0, RA_u0, RM_u0, RM_v0, Vu0, Vv0;  // nt
  std::vector<double> VU;                   // nt x nt
};
SlabCoeffs slab_coeffs(int pde, int scheme, int k, double tau);

// Dense helpers (row-major).
bool invert(int n, std::vector<double>& a);                 // in place, partial pivoting
std::vector<cplx> eigenvalues(int n, const std::vector<double>& a);   // real matrix
// Eigen-decomposition of a real matrix with simple eigenvalues: V (n x n complex, columns
// eigenvectors), lambda.  Returns false if the eigenvector matrix is singular.
bool eigen_decompose(int n, const std::vector<double>& a, std::vector<cplx>& lambda, std::vector<cplx>& V);
bool invert_complex(int n, std::vector<cplx>& a);

// 1D prolongation in reference coordinates: for each fine 1D node, the first coarse
// node of its window and the (pc+1) weights.
void prolongation_1d(int pf, int Nf, int pc, int Nc, std::vector<int>& start, std::vector<double>& w);
// Time prolongation P_tau (nt_f x nt_c, row-major).
std::vector<double> time_prolongation(int scheme, int kf, int kc);
// dG(k) prolongation from one slab of length 2 tau to its two halves of length tau:
// (2 (k+1)) x (k+1) row-major, row h (k+1) + t = coarse basis functions at fine Radau node t of half h.
std::vector<double> tau_prolongation(int k);

// Fast diagonalisation tables of one direction of a uniform Cartesian grid (N cells of size h):
// for cell type t (0: first cell, left node constrained; 1: interior; 2: last cell, right node
// constrained) the global 1D mass M and stiffness A restricted to the cell's p+1 nodes (neighbour
// halves included), and the generalized eigenpairs A s = lambda M s on the unconstrained nodes with
// s^T M s = 1.  S[t][a][i] = component a of eigenvector i (0 on constrained nodes and unused i).
void fd_tables_1d(int p, int N, std::vector<double>& S, std::vector<double>& lam);
// Symmetric eigen-decomposition (cyclic Jacobi): a (n x n, symmetric) -> eigenvalues w, vectors V (columns).
void jacobi_eigen(int n, std::vector<double> a, std::vector<double>& w, std::vector<double>& V);

}  // namespace stmg
