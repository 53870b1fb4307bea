// Host-side FP64 tables for the STMG library.  See tables.h.
#include "tables.h"

#include <algorithm>
#include <cmath>

namespace stmg {

namespace {

// Legendre P_n(x) and P_n'(x) by the three-term recurrence and
// P'_{m+1} = P'_{m-1} + (2m+1) P_m.
void legendre(int n, double x, double& P, double& dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { P = 1.0; dP = 0.0; return; }
  for (int m = 1; m < n; ++m) {
    double p2 = ((2 * m + 1) * x * p1 - m * p0) / (m + 1);
    double d2 = d0 + (2 * m + 1) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  P = p1; dP = d1;
}

void to_unit_interval(std::vector<double>& x, std::vector<double>& w) {
  for (size_t i = 0; i < x.size(); ++i) { x[i] = 0.5 * (x[i] + 1.0); if (!w.empty()) w[i] *= 0.5; }
}

// w_j = int_0^1 l_j(t) dt (interpolatory weights)
std::vector<double> interpolatory_weights(const std::vector<double>& t) {
  std::vector<double> xq, wq;
  gauss_legendre((int)t.size() + 2, xq, wq);
  std::vector<double> w(t.size(), 0.0);
  for (size_t j = 0; j < t.size(); ++j)
    for (size_t q = 0; q < xq.size(); ++q) w[j] += wq[q] * lagrange(t, (int)j, xq[q]);
  return w;
}

}  // namespace

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0); w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP; legendre(n, z, P, dP);
      double dz = P / dP; z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P, dP; legendre(n, z, P, dP);
    x[i] = z; w[i] = 2.0 / ((1.0 - z * z) * dP * dP);
  }
  // ascending order
  std::reverse(x.begin(), x.end()); std::reverse(w.begin(), w.end());
  to_unit_interval(x, w);
}

void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  x[0] = -1.0; x[n - 1] = 1.0;
  int m = n - 1;
  for (int j = 1; j < n - 1; ++j) {
    double z = -std::cos(M_PI * j / m);
    for (int it = 0; it < 100; ++it) {
      double P, dP; legendre(m, z, P, dP);
      double d2P = (2.0 * z * dP - m * (m + 1) * P) / (1.0 - z * z);
      double dz = dP / d2P; z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[j] = z;
  }
  std::vector<double> none;
  to_unit_interval(x, none);
  w = interpolatory_weights(x);
}

void gauss_radau_right(int n, std::vector<double>& x, std::vector<double>& w) {
  if (n == 1) { x = {1.0}; w = {1.0}; return; }
  x.assign(n, 1.0);
  // interior nodes: roots of h(x) = (P_{n-1}(x) - P_n(x)) / (1 - x)
  for (int j = 1; j < n; ++j) {
    double z = std::cos(2.0 * M_PI * j / (2 * n - 1));
    for (int it = 0; it < 200; ++it) {
      double Pa, dPa, Pb, dPb; legendre(n - 1, z, Pa, dPa); legendre(n, z, Pb, dPb);
      double g = Pa - Pb, dg = dPa - dPb;
      double dz = g * (1.0 - z) / (dg * (1.0 - z) + g);
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[j - 1] = z;
  }
  x[n - 1] = 1.0;
  std::sort(x.begin(), x.end());
  std::vector<double> none;
  to_unit_interval(x, none);
  x[n - 1] = 1.0;
  w = interpolatory_weights(x);
}

double lagrange(const std::vector<double>& nodes, int j, double t) {
  double v = 1.0;
  for (size_t m = 0; m < nodes.size(); ++m)
    if ((int)m != j) v *= (t - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

double lagrange_deriv(const std::vector<double>& nodes, int j, double t) {
  double s = 0.0;
  for (size_t m = 0; m < nodes.size(); ++m) {
    if ((int)m == j) continue;
    double term = 1.0 / (nodes[j] - nodes[m]);
    for (size_t l = 0; l < nodes.size(); ++l)
      if ((int)l != j && l != m) term *= (t - nodes[l]) / (nodes[j] - nodes[l]);
    s += term;
  }
  return s;
}

std::vector<double> space_nodes(int p) {
  std::vector<double> x, w;
  gauss_lobatto(p + 1, x, w);
  return x;
}

TimeWeights time_weights(int scheme, int k) {
  TimeWeights tw;
  tw.scheme = scheme; tw.k = k;
  std::vector<double> tq, wq;
  gauss_legendre(k + 3, tq, wq);
  if (scheme == 0) {
    int n = k + 1;
    tw.nt = n;
    std::vector<double> w;
    gauss_radau_right(n, tw.nodes, w);
    tw.Mhat.assign(n * n, 0.0); tw.Ahat.assign(n * n, 0.0);
    tw.alpha.assign(n, 0.0); tw.betahat.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
      for (int j = 0; j < n; ++j) {
        double m = 0.0, a = 0.0;
        for (size_t q = 0; q < tq.size(); ++q) {
          double xi = lagrange(tw.nodes, i, tq[q]);
          m += wq[q] * lagrange(tw.nodes, j, tq[q]) * xi;
          a += wq[q] * lagrange_deriv(tw.nodes, j, tq[q]) * xi;
        }
        a += lagrange(tw.nodes, j, 0.0) * lagrange(tw.nodes, i, 0.0);  // upwind jump term
        tw.Mhat[i * n + j] = m; tw.Ahat[i * n + j] = a;
      }
      tw.alpha[i] = lagrange(tw.nodes, i, 0.0);
    }
  } else {
    int n = k;
    tw.nt = n;
    std::vector<double> gl, w;
    gauss_lobatto(k + 1, gl, w);
    tw.nodes.assign(gl.begin() + 1, gl.end());
    tw.Mhat.assign(n * n, 0.0); tw.Ahat.assign(n * n, 0.0);
    tw.alpha.assign(n, 0.0); tw.betahat.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
      for (size_t q = 0; q < tq.size(); ++q) {
        double psi = (k == 1) ? 1.0 : lagrange(tw.nodes, i, tq[q]);
        for (int j = 1; j <= k; ++j) {
          tw.Mhat[i * n + j - 1] += wq[q] * lagrange(gl, j, tq[q]) * psi;
          tw.Ahat[i * n + j - 1] += wq[q] * lagrange_deriv(gl, j, tq[q]) * psi;
        }
        tw.betahat[i] += wq[q] * lagrange(gl, 0, tq[q]) * psi;
        tw.alpha[i] += wq[q] * lagrange_deriv(gl, 0, tq[q]) * psi;
      }
    }
  }
  return tw;
}

namespace {
std::vector<double> matmul(int n, const std::vector<double>& a, const std::vector<double>& b) {
  std::vector<double> c(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < n; ++l)
      for (int j = 0; j < n; ++j) c[i * n + j] += a[i * n + l] * b[l * n + j];
  return c;
}
std::vector<double> matvec(int n, const std::vector<double>& a, const std::vector<double>& x) {
  std::vector<double> y(n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) y[i] += a[i * n + j] * x[j];
  return y;
}
}  // namespace

SlabCoeffs slab_coeffs(int pde, int scheme, int k, double tau) {
  TimeWeights tw = time_weights(scheme, k);
  int n = tw.nt;
  SlabCoeffs c;
  c.nt = n;
  std::vector<double> Mt(n * n), beta(n);
  for (int i = 0; i < n * n; ++i) Mt[i] = tau * tw.Mhat[i];
  for (int i = 0; i < n; ++i) beta[i] = tau * tw.betahat[i];
  const std::vector<double>& At = tw.Ahat;
  const std::vector<double>& alpha = tw.alpha;
  std::vector<double> z(n, 0.0);
  c.TA = Mt;
  c.RM_f = Mt;
  c.VU.assign(n * n, 0.0); c.Vu0 = z; c.Vv0 = z;
  if (pde == 0) {  // heat
    c.TM = At;
    if (scheme == 0) {  // eq. heat-cg-dg
      c.RM_f0 = z; c.RA_u0 = z; c.RM_u0 = alpha; c.RM_v0 = z;
    } else {            // eq. heat-cg-cg, signs from the variational form
      c.RM_f0 = beta;
      c.RA_u0.resize(n); c.RM_u0.resize(n);
      for (int i = 0; i < n; ++i) { c.RA_u0[i] = -beta[i]; c.RM_u0[i] = -alpha[i]; }
      c.RM_v0 = z;
    }
    return c;
  }
  std::vector<double> Minv = Mt;
  invert(n, Minv);
  std::vector<double> MinvA = matmul(n, Minv, At);
  c.TM = matmul(n, At, MinvA);
  std::vector<double> AMa = matvec(n, At, matvec(n, Minv, alpha));
  c.VU = MinvA;
  if (scheme == 0) {  // eq. wave-cg-dg
    c.RM_f0 = z; c.RA_u0 = z; c.RM_u0 = AMa; c.RM_v0 = alpha;
    std::vector<double> ma = matvec(n, Minv, alpha);
    for (int i = 0; i < n; ++i) c.Vu0[i] = -ma[i];
  } else {            // eq. wave-cg-cg, signs from the variational form
    std::vector<double> AMb = matvec(n, At, matvec(n, Minv, beta));
    std::vector<double> ma = matvec(n, Minv, alpha), mb = matvec(n, Minv, beta);
    c.RM_f0 = beta;
    c.RA_u0.resize(n); c.RM_u0.resize(n); c.RM_v0.resize(n);
    for (int i = 0; i < n; ++i) {
      c.RA_u0[i] = -beta[i];
      c.RM_u0[i] = -AMa[i];
      c.RM_v0[i] = -(alpha[i] - AMb[i]);
      c.Vu0[i] = ma[i];
      c.Vv0[i] = -mb[i];
    }
  }
  return c;
}

bool invert(int n, std::vector<double>& a) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i) if (std::fabs(a[i * n + k]) > std::fabs(a[p * n + k])) p = i;
    if (a[p * n + k] == 0.0) return false;
    piv[k] = p;
    if (p != k) for (int j = 0; j < n; ++j) std::swap(a[k * n + j], a[p * n + j]);
    double d = 1.0 / a[k * n + k];
    a[k * n + k] = 1.0;
    for (int j = 0; j < n; ++j) a[k * n + j] *= d;
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      double f = a[i * n + k];
      if (f == 0.0) continue;
      a[i * n + k] = 0.0;
      for (int j = 0; j < n; ++j) a[i * n + j] -= f * a[k * n + j];
    }
  }
  for (int k = n - 1; k >= 0; --k)
    if (piv[k] != k) for (int i = 0; i < n; ++i) std::swap(a[i * n + k], a[i * n + piv[k]]);
  return true;
}

bool invert_complex(int n, std::vector<cplx>& a) {
  std::vector<int> piv(n);
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i) if (std::abs(a[i * n + k]) > std::abs(a[p * n + k])) p = i;
    if (std::abs(a[p * n + k]) == 0.0) return false;
    piv[k] = p;
    if (p != k) for (int j = 0; j < n; ++j) std::swap(a[k * n + j], a[p * n + j]);
    cplx d = 1.0 / a[k * n + k];
    a[k * n + k] = 1.0;
    for (int j = 0; j < n; ++j) a[k * n + j] *= d;
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      cplx f = a[i * n + k];
      a[i * n + k] = 0.0;
      for (int j = 0; j < n; ++j) a[i * n + j] -= f * a[k * n + j];
    }
  }
  for (int k = n - 1; k >= 0; --k)
    if (piv[k] != k) for (int i = 0; i < n; ++i) std::swap(a[i * n + k], a[i * n + piv[k]]);
  return true;
}

// Eigenvalues by Householder reduction to Hessenberg form followed by the
// single-shift complex QR iteration with Wilkinson shifts (Givens rotations),
// deflation at the bottom of the active block and a closed form for the last 2x2 block.
std::vector<cplx> eigenvalues(int n, const std::vector<double>& ar) {
  std::vector<cplx> a(ar.begin(), ar.end());
  auto A = [&](int i, int j) -> cplx& { return a[i * n + j]; };
  for (int k = 0; k + 2 < n; ++k) {  // Householder on column k below the subdiagonal
    double nrm = 0.0;
    for (int i = k + 1; i < n; ++i) nrm += std::norm(A(i, k));
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    std::vector<cplx> v(n, 0.0);
    cplx x0 = A(k + 1, k);
    cplx ph = std::abs(x0) > 0 ? x0 / std::abs(x0) : cplx(1.0, 0.0);
    for (int i = k + 1; i < n; ++i) v[i] = A(i, k);
    v[k + 1] += ph * nrm;
    double vn = 0.0;
    for (int i = k + 1; i < n; ++i) vn += std::norm(v[i]);
    if (vn == 0.0) continue;
    // A <- H A H, H = I - 2 v v^H / (v^H v)
    for (int j = 0; j < n; ++j) {
      cplx s = 0.0;
      for (int i = k + 1; i < n; ++i) s += std::conj(v[i]) * A(i, j);
      s *= 2.0 / vn;
      for (int i = k + 1; i < n; ++i) A(i, j) -= v[i] * s;
    }
    for (int i = 0; i < n; ++i) {
      cplx s = 0.0;
      for (int j = k + 1; j < n; ++j) s += A(i, j) * v[j];
      s *= 2.0 / vn;
      for (int j = k + 1; j < n; ++j) A(i, j) -= s * std::conj(v[j]);
    }
  }
  std::vector<cplx> ev;
  double anorm = 0.0;
  for (auto& x : a) anorm = std::max(anorm, std::abs(x));
  int m = n;
  int its = 0;
  while (m > 0) {
    if (m == 1) { ev.push_back(A(0, 0)); break; }
    if (m == 2) {  // closed form for the last 2x2 block
      cplx a11 = A(0, 0), a12 = A(0, 1), a21 = A(1, 0), a22 = A(1, 1);
      cplx h = 0.5 * (a11 - a22);
      cplx disc = std::sqrt(h * h + a12 * a21);
      ev.push_back(0.5 * (a11 + a22) + disc);
      ev.push_back(0.5 * (a11 + a22) - disc);
      break;
    }
    double scale = std::abs(A(m - 1, m - 1)) + std::abs(A(m - 2, m - 2));
    if (scale == 0.0) scale = anorm;
    if (std::abs(A(m - 1, m - 2)) <= 1e-15 * scale || its > 300) {  // deflate (forced after 300 sweeps)
      ev.push_back(A(m - 1, m - 1));
      --m;
      its = 0;
      continue;
    }
    ++its;
    // Wilkinson shift from the trailing 2x2 block
    cplx a11 = A(m - 2, m - 2), a12 = A(m - 2, m - 1), a21 = A(m - 1, m - 2), a22 = A(m - 1, m - 1);
    cplx h = 0.5 * (a11 - a22);
    cplx disc = std::sqrt(h * h + a12 * a21);
    cplx l1 = 0.5 * (a11 + a22) + disc, l2 = 0.5 * (a11 + a22) - disc;
    cplx mu = (std::abs(l1 - a22) < std::abs(l2 - a22)) ? l1 : l2;
    if (its % 11 == 0) mu += cplx(std::abs(a21), 0.0);  // exceptional shift
    for (int i = 0; i < m; ++i) A(i, i) -= mu;
    std::vector<cplx> cs(m), sn(m);
    for (int k = 0; k + 1 < m; ++k) {  // QR by Givens
      cplx x = A(k, k), y = A(k + 1, k);
      double r = std::sqrt(std::norm(x) + std::norm(y));
      cplx c = r > 0 ? x / r : cplx(1.0, 0.0), s = r > 0 ? y / r : cplx(0.0, 0.0);
      cs[k] = c; sn[k] = s;
      for (int j = k; j < m; ++j) {
        cplx t1 = A(k, j), t2 = A(k + 1, j);
        A(k, j) = std::conj(c) * t1 + std::conj(s) * t2;
        A(k + 1, j) = -s * t1 + c * t2;
      }
    }
    for (int k = 0; k + 1 < m; ++k) {  // R Q
      cplx c = cs[k], s = sn[k];
      for (int i = 0; i <= std::min(k + 2, m - 1); ++i) {
        cplx t1 = A(i, k), t2 = A(i, k + 1);
        A(i, k) = t1 * c + t2 * s;
        A(i, k + 1) = -t1 * std::conj(s) + t2 * std::conj(c);
      }
    }
    for (int i = 0; i < m; ++i) A(i, i) += mu;
  }
  return ev;
}

bool eigen_decompose(int n, const std::vector<double>& a, std::vector<cplx>& lambda, std::vector<cplx>& V) {
  lambda = eigenvalues(n, a);
  if ((int)lambda.size() != n) return false;
  // snap nearly real eigenvalues; order: real ones first (ascending), then by imaginary part
  for (auto& l : lambda) if (std::fabs(l.imag()) <= 1e-12 * std::abs(l)) l = cplx(l.real(), 0.0);
  std::sort(lambda.begin(), lambda.end(), [](const cplx& x, const cplx& y) {
    bool rx = x.imag() == 0.0, ry = y.imag() == 0.0;
    if (rx != ry) return rx;
    if (x.real() != y.real()) return x.real() < y.real();
    return x.imag() < y.imag();
  });
  V.assign(n * n, 0.0);
  for (int e = 0; e < n; ++e) {
    // inverse iteration with a slightly perturbed shift
    cplx mu = lambda[e] * (1.0 + 1e-11) + cplx(1e-13, 0.0);
    std::vector<cplx> M(n * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) M[i * n + j] = a[i * n + j] - (i == j ? mu : cplx(0.0, 0.0));
    if (!invert_complex(n, M)) return false;
    std::vector<cplx> v(n, 1.0);
    for (int i = 0; i < n; ++i) v[i] = cplx(1.0 + 0.1 * i, 0.05 * i);
    for (int it = 0; it < 4; ++it) {
      std::vector<cplx> w(n, 0.0);
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) w[i] += M[i * n + j] * v[j];
      double nr = 0.0;
      int imax = 0;
      for (int i = 0; i < n; ++i) { nr += std::norm(w[i]); if (std::abs(w[i]) > std::abs(w[imax])) imax = i; }
      cplx ph = w[imax] / std::abs(w[imax]);
      for (int i = 0; i < n; ++i) v[i] = w[i] / (std::sqrt(nr) * ph);
    }
    if (lambda[e].imag() == 0.0) for (auto& x : v) x = cplx(x.real(), 0.0);
    for (int i = 0; i < n; ++i) V[i * n + e] = v[i];
  }
  std::vector<cplx> W = V;
  return invert_complex(n, W);
}

void prolongation_1d(int pf, int Nf, int pc, int Nc, std::vector<int>& start, std::vector<double>& w) {
  std::vector<double> xf = space_nodes(pf), xc = space_nodes(pc);
  int nf = pf * Nf + 1;
  start.assign(nf, 0);
  w.assign((size_t)nf * (pc + 1), 0.0);
  for (int cf = 0; cf < Nf; ++cf)
    for (int a = 0; a <= pf; ++a) {
      int gf = cf * pf + a;
      double s = (cf + xf[a]) / Nf;
      int cc = std::min((int)std::floor(s * Nc), Nc - 1);
      double xi = s * Nc - cc;
      start[gf] = cc * pc;
      for (int b = 0; b <= pc; ++b) {
        double v = lagrange(xc, b, xi);
        w[(size_t)gf * (pc + 1) + b] = std::fabs(v) < 1e-15 ? 0.0 : v;
      }
    }
}

std::vector<double> time_prolongation(int scheme, int kf, int kc) {
  std::vector<double> P;
  if (scheme == 0) {
    std::vector<double> tf, tc, w;
    gauss_radau_right(kf + 1, tf, w);
    gauss_radau_right(kc + 1, tc, w);
    P.assign((kf + 1) * (kc + 1), 0.0);
    for (int i = 0; i <= kf; ++i)
      for (int j = 0; j <= kc; ++j) P[i * (kc + 1) + j] = lagrange(tc, j, tf[i]);
  } else {
    std::vector<double> tf, tc, w;
    gauss_lobatto(kf + 1, tf, w);
    gauss_lobatto(kc + 1, tc, w);
    P.assign(kf * kc, 0.0);
    for (int i = 1; i <= kf; ++i)
      for (int j = 1; j <= kc; ++j) P[(i - 1) * kc + (j - 1)] = lagrange(tc, j, tf[i]);
  }
  return P;
}

std::vector<double> tau_prolongation(int k) {
  std::vector<double> t, w;
  gauss_radau_right(k + 1, t, w);
  const int n = k + 1;
  std::vector<double> P(2 * n * n, 0.0);
  for (int h = 0; h < 2; ++h)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) P[(h * n + i) * n + j] = lagrange(t, j, 0.5 * (h + t[i]));
  return P;
}

void jacobi_eigen(int n, std::vector<double> a, std::vector<double>& w, std::vector<double>& V) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) (i == j ? diag : off) += a[i * n + j] * a[i * n + j];
    if (off <= 1e-30 * diag) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // a <- a J (columns p, q)
          const double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // a <- J^T a (rows p, q)
          const double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a[i * n + i];
}

void fd_tables_1d(int p, int N, std::vector<double>& S, std::vector<double>& lam) {
  const int n = p + 1;
  const double h = 1.0 / N;
  std::vector<double> xn = space_nodes(p), xq, wq;
  gauss_legendre(n, xq, wq);
  std::vector<double> Me(n * n, 0.0), Ae(n * n, 0.0);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int q = 0; q < n; ++q) {
        Me[a * n + b] += h * wq[q] * lagrange(xn, a, xq[q]) * lagrange(xn, b, xq[q]);
        Ae[a * n + b] += wq[q] * lagrange_deriv(xn, a, xq[q]) * lagrange_deriv(xn, b, xq[q]) / h;
      }
  S.assign(3 * n * n, 0.0);
  lam.assign(3 * n, 1.0);
  for (int t = 0; t < 3; ++t) {
    std::vector<double> M = Me, A = Ae;
    const bool has_left = t != 0 || N == 1 ? (t != 0) : false;
    const bool has_right = t != 2;
    if (has_left) { M[0] += Me[p * n + p]; A[0] += Ae[p * n + p]; }      // node 0 shared with the left cell
    if (has_right) { M[p * n + p] += Me[0]; A[p * n + p] += Ae[0]; }     // node p shared with the right cell
    std::vector<int> free_nodes;
    for (int a = 0; a < n; ++a)
      if (!((t == 0 && a == 0) || (t == 2 && a == p))) free_nodes.push_back(a);
    const int m = (int)free_nodes.size();
    std::vector<double> Mf(m * m), Af(m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        Mf[i * m + j] = M[free_nodes[i] * n + free_nodes[j]];
        Af[i * m + j] = A[free_nodes[i] * n + free_nodes[j]];
      }
    // Cholesky M = L L^T, C = L^-1 A L^-T, C Q = Q w, S = L^-T Q
    std::vector<double> L(m * m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j <= i; ++j) {
        double sum = Mf[i * m + j];
        for (int k = 0; k < j; ++k) sum -= L[i * m + k] * L[j * m + k];
        L[i * m + j] = (i == j) ? std::sqrt(sum) : sum / L[j * m + j];
      }
    std::vector<double> Li(m * m, 0.0);  // L^-1 by forward substitution
    for (int c = 0; c < m; ++c)
      for (int i = 0; i < m; ++i) {
        double sum = (i == c) ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) sum -= L[i * m + k] * Li[k * m + c];
        Li[i * m + c] = sum / L[i * m + i];
      }
    std::vector<double> C(m * m, 0.0), T(m * m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        for (int k = 0; k < m; ++k) T[i * m + j] += Li[i * m + k] * Af[k * m + j];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        for (int k = 0; k < m; ++k) C[i * m + j] += T[i * m + k] * Li[j * m + k];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < i; ++j) { const double v = 0.5 * (C[i * m + j] + C[j * m + i]); C[i * m + j] = C[j * m + i] = v; }
    std::vector<double> w, Q;
    jacobi_eigen(m, C, w, Q);
    for (int i = 0; i < m; ++i) {
      lam[t * n + i] = w[i];
      for (int a = 0; a < m; ++a) {
        double sv = 0.0;  // (L^-T Q)[a][i] = sum_k Li[k][a] Q[k][i]
        for (int k = 0; k < m; ++k) sv += Li[k * m + a] * Q[k * m + i];
        S[(t * n + free_nodes[a]) * n + i] = sv;
      }
    }
  }
}

}  // namespace stmg
