// Geometry of the Q1-mapped cells at the Gauss points (setup, FP64).
//
// For every cell and Gauss point q of the (p+1)^dim tensor rule:
//   G_q = rho_q w_q |det J_q| J_q^-1 J_q^-T   (so that (rho grad u, grad v) = sum_q grad^ v . G_q grad^ u)
//   m_q = w_q |det J_q|                        (mass weight)
// with J the Jacobian of the multilinear map from the cell's 2^dim vertices
// (eq. space-matrices evaluated by quadrature, Section 3.1).
#include "common.cuh"
#include "kernels.h"

namespace stmg {

namespace {

__global__ void geometry_kernel(GridDesc g, const double* __restrict__ vert, const double* __restrict__ rho_qp,
                                const double* __restrict__ xq, const double* __restrict__ wq, int nq,
                                double* __restrict__ geo64, float* __restrict__ geo32, df64* __restrict__ geodf) {
  const int dim = g.dim;
  const int nqd = dim == 3 ? nq * nq * nq : nq * nq;
  const int ncomp = dim == 3 ? 7 : 4;
  const int64_t total = g.n_cells * nqd;
  const int nv1 = g.N + 1;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = idx / nqd;
    const int q = (int)(idx % nqd);
    const int qx = q % nq, qy = (q / nq) % nq, qz = q / (nq * nq);
    const int cx = (int)(cell % g.N);
    const int cy = (int)((cell / g.N) % g.N);
    const int cz = dim == 3 ? (int)(cell / ((int64_t)g.N * g.N)) : 0;
    const double xi[3] = {xq[qx], xq[qy], dim == 3 ? xq[qz] : 0.0};
    const double w = wq[qx] * wq[qy] * (dim == 3 ? wq[qz] : 1.0);
    const double rho = rho_qp[idx];
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const int nvert = dim == 3 ? 8 : 4;
    for (int b = 0; b < nvert; ++b) {
      const int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
      const int64_t vid = (cx + bx) + (int64_t)nv1 * ((cy + by) + (int64_t)nv1 * (cz + bz));
      double f[3], df[3];
      const int bits[3] = {bx, by, bz};
      for (int d = 0; d < dim; ++d) {
        f[d] = bits[d] ? xi[d] : 1.0 - xi[d];
        df[d] = bits[d] ? 1.0 : -1.0;
      }
      for (int e = 0; e < dim; ++e) {
        double gr = 1.0;
        for (int d = 0; d < dim; ++d) gr *= (d == e) ? df[d] : f[d];
        for (int d = 0; d < dim; ++d) J[d][e] += vert[vid * dim + d] * gr;
      }
    }
    double out[7];
    if (dim == 3) {
      const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
      const double c01 = J[0][2] * J[2][1] - J[0][1] * J[2][2];
      const double c02 = J[0][1] * J[1][2] - J[0][2] * J[1][1];
      const double c10 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
      const double c11 = J[0][0] * J[2][2] - J[0][2] * J[2][0];
      const double c12 = J[0][2] * J[1][0] - J[0][0] * J[1][2];
      const double c20 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
      const double c21 = J[0][1] * J[2][0] - J[0][0] * J[2][1];
      const double c22 = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      const double det = J[0][0] * c00 + J[0][1] * c10 + J[0][2] * c20;
      const double Ji[3][3] = {{c00 / det, c01 / det, c02 / det},
                               {c10 / det, c11 / det, c12 / det},
                               {c20 / det, c21 / det, c22 / det}};
      const double jw = w * fabs(det);
      double G[3][3];
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[a][b] = (Ji[a][0] * Ji[b][0] + Ji[a][1] * Ji[b][1] + Ji[a][2] * Ji[b][2]) * jw * rho;
      out[0] = G[0][0]; out[1] = G[0][1]; out[2] = G[0][2];
      out[3] = G[1][1]; out[4] = G[1][2]; out[5] = G[2][2];
      out[6] = jw;
    } else {
      const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
      const double Ji[2][2] = {{J[1][1] / det, -J[0][1] / det}, {-J[1][0] / det, J[0][0] / det}};
      const double jw = w * fabs(det);
      out[0] = (Ji[0][0] * Ji[0][0] + Ji[0][1] * Ji[0][1]) * jw * rho;
      out[1] = (Ji[0][0] * Ji[1][0] + Ji[0][1] * Ji[1][1]) * jw * rho;
      out[2] = (Ji[1][0] * Ji[1][0] + Ji[1][1] * Ji[1][1]) * jw * rho;
      out[3] = jw;
    }
    const bool chunked = geo_chunked(dim, nq);
    for (int c = 0; c < ncomp; ++c) {
      const int64_t o = (cell * ncomp + c) * nqd + q;
      const int64_t oc =
          chunked ? (((cell / kGeoChunk * nqd + q) * 2 + c / 4) * kGeoChunk + cell % kGeoChunk) * 4 + c % 4 : o;
      geo64[o] = out[c];
      geo32[oc] = (float)out[c];
      if (geodf) {
        const float h = (float)out[c];
        geodf[o] = df64(h, (float)(out[c] - (double)h));
      }
    }
    if (chunked) geo32[(((cell / kGeoChunk * nqd + q) * 2 + 1) * kGeoChunk + cell % kGeoChunk) * 4 + 3] = 0.0f;
  }
}

}  // namespace

cudaError_t launch_geometry(const GridDesc& g, const double* vertices, const double* rho_qp, const double* xq,
                            const double* wq, double* geo64, float* geo32, df64* geodf, cudaStream_t s) {
  const int nq = g.p + 1;
  const int64_t total = g.n_cells * (g.dim == 3 ? nq * nq * nq : nq * nq);
  int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 64);
  geometry_kernel<<<blocks < 1 ? 1 : blocks, 256, 0, s>>>(g, vertices, rho_qp, xq, wq, nq, geo64, geo32, geodf);
  return cudaGetLastError();
}

}  // namespace stmg
