// Local matrices of the cell-wise additive Schwarz smoother (eqs. vanka0, vanka): the global
// stiffness and mass matrices A_h, M_h restricted to the nodes of one cell, i.e. the cell's own
// element matrices plus the contributions of the neighbour cells on shared faces, edges and
// vertices, by Gauss quadrature on every cell of the 3^dim patch.  FP64, one CTA per cell.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace stmg {

// Aloc, Mloc: NB x NB row-major in shared memory (NB = (p+1)^dim); every thread of the CTA takes part.
template <int DIM, int N>
__device__ void assemble_local(const GridDesc& g, const double* __restrict__ geo, const LocalTab& lt, int cx, int cy,
                               int cz, double* Aloc, double* Mloc) {
  constexpr int NB = DIM == 3 ? N * N * N : N * N;
  constexpr int NQ = NB;
  constexpr int NG = DIM == 3 ? 7 : 4;
  const int tid = threadIdx.x;
  const int p = g.p;
  for (int pr = tid; pr < NB * NB; pr += (int)blockDim.x) { Aloc[pr] = 0.0; Mloc[pr] = 0.0; }
  __syncthreads();
  // global matrices restricted to this cell's nodes: sum over the cells of the 3^dim patch
  const int noff = DIM == 3 ? 27 : 9;
  for (int o = 0; o < noff; ++o) {
    const int ox = o % 3 - 1, oy = (o / 3) % 3 - 1, oz = DIM == 3 ? o / 9 - 1 : 0;
    const int nx = cx + ox, ny = cy + oy, nz = cz + oz;
    if (nx < 0 || nx >= g.N || ny < 0 || ny >= g.N || nz < 0 || nz >= (DIM == 3 ? g.N : 1)) continue;
    const int64_t nc = nx + (int64_t)g.N * (ny + (int64_t)g.N * nz);
    const double* gc = geo + nc * NG * NQ;
    for (int pr = tid; pr < NB * NB; pr += (int)blockDim.x) {
      const int a = pr / NB, b = pr % NB;
      const int ax = a % N - ox * p, ay = (a / N) % N - oy * p, az = DIM == 3 ? a / (N * N) - oz * p : 0;
      const int bx = b % N - ox * p, by = (b / N) % N - oy * p, bz = DIM == 3 ? b / (N * N) - oz * p : 0;
      if (ax < 0 || ax > p || ay < 0 || ay > p || az < 0 || az > p) continue;
      if (bx < 0 || bx > p || by < 0 || by > p || bz < 0 || bz > p) continue;
      double sa = 0.0, sm = 0.0;
      for (int q = 0; q < NQ; ++q) {
        const int qx = q % N, qy = (q / N) % N, qz = DIM == 3 ? q / (N * N) : 0;
        if (DIM == 3) {
          const double va = lt.B[qx][ax] * lt.B[qy][ay] * lt.B[qz][az];
          const double vb = lt.B[qx][bx] * lt.B[qy][by] * lt.B[qz][bz];
          const double da0 = lt.Dn[qx][ax] * lt.B[qy][ay] * lt.B[qz][az];
          const double da1 = lt.B[qx][ax] * lt.Dn[qy][ay] * lt.B[qz][az];
          const double da2 = lt.B[qx][ax] * lt.B[qy][ay] * lt.Dn[qz][az];
          const double db0 = lt.Dn[qx][bx] * lt.B[qy][by] * lt.B[qz][bz];
          const double db1 = lt.B[qx][bx] * lt.Dn[qy][by] * lt.B[qz][bz];
          const double db2 = lt.B[qx][bx] * lt.B[qy][by] * lt.Dn[qz][bz];
          const double G00 = gc[0 * NQ + q], G01 = gc[1 * NQ + q], G02 = gc[2 * NQ + q];
          const double G11 = gc[3 * NQ + q], G12 = gc[4 * NQ + q], G22 = gc[5 * NQ + q];
          sa += da0 * (G00 * db0 + G01 * db1 + G02 * db2) + da1 * (G01 * db0 + G11 * db1 + G12 * db2) +
                da2 * (G02 * db0 + G12 * db1 + G22 * db2);
          sm += gc[6 * NQ + q] * va * vb;
        } else {
          const double va = lt.B[qx][ax] * lt.B[qy][ay];
          const double vb = lt.B[qx][bx] * lt.B[qy][by];
          const double da0 = lt.Dn[qx][ax] * lt.B[qy][ay], da1 = lt.B[qx][ax] * lt.Dn[qy][ay];
          const double db0 = lt.Dn[qx][bx] * lt.B[qy][by], db1 = lt.B[qx][bx] * lt.Dn[qy][by];
          const double G00 = gc[0 * NQ + q], G01 = gc[1 * NQ + q], G11 = gc[2 * NQ + q];
          sa += da0 * (G00 * db0 + G01 * db1) + da1 * (G01 * db0 + G11 * db1);
          sm += gc[3 * NQ + q] * va * vb;
        }
      }
      Aloc[pr] += sa;
      Mloc[pr] += sm;
    }
    __syncthreads();
  }
}

}  // namespace stmg
