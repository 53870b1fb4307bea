// Additive Schwarz local solves by fast diagonalisation (Cartesian cells, 3D).
//
// On a uniform Cartesian grid with a coefficient that is constant (rho_K) on the cells that
// share nodes with K, the global A_h, M_h restricted to K's nodes are Kronecker products of
// the restricted 1D matrices: A_K = rho_K (A1 x M1 x M1 + M1 x A1 x M1 + M1 x M1 x A1),
// M_K = M1 x M1 x M1.  With A1 s = lambda M1 s, S^T M1 S = I per direction,
//   (A_K + lambda_m M_K)^-1 = (Sz x Sy x Sx) diag(1 / (rho_K (lx + ly + lz) + lambda_m)) (Sz x Sy x Sx)^T,
// combined with the same time diagonalisation as the dense path (asm.cu).  Exact in that case;
// with a coefficient that varies inside the patch, rho_K = the cell mean gives an approximate
// local solver.  Cost: 6 one-dimensional sweeps per time plane, no stored inverses.
#include "common.cuh"
#include "kernels.h"

namespace stmg {

namespace {

template <int N> constexpr int fd_cells_per_block() { return N == 2 ? 32 : N == 3 ? 14 : N == 4 ? 8 : N == 5 ? 5 : 3; }

template <int N, int NT, typename T, int CPB>
__global__ void __launch_bounds__(CPB * N * N)
fd_apply_kernel(const T* __restrict__ r, T* __restrict__ u, const T* __restrict__ rho_cell, GridDesc g, FDTab<T> fd,
                ModeTab<T> mt, const T* __restrict__ copy_src, T* __restrict__ copy_dst) {
  pdl_wait();
  pdl_trigger();
  constexpr int N2 = N * N, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int slot = threadIdx.x / N2;
  const int lid = threadIdx.x - slot * N2;
  const int i = lid % N, j = lid / N;
  const int64_t cell = (int64_t)blockIdx.x * CPB + slot;
  const bool active = cell < g.n_cells;
  T* s0 = smem + (size_t)slot * 2 * NT * N3;
  T* s1 = s0 + NT * N3;
  auto I4 = [](int t, int c, int b, int a) { return ((t * N + c) * N + b) * N + a; };
  const int64_t cc = active ? cell : 0;
  int cx, cy, cz;
  cell_xyz(cc, g, cx, cy, cz);
  const int tx = cx == 0 ? 0 : (cx == g.N - 1 ? 2 : 1);
  const int ty = cy == 0 ? 0 : (cy == g.N - 1 ? 2 : 1);
  const int tz = cz == 0 ? 0 : (cz == g.N - 1 ? 2 : 1);
  const int gx = cx * g.p + i, gy = cy * g.p + j;
  const bool bxy = on_boundary(gx, g.nn1) || on_boundary(gy, g.nn1);
  const T rho = rho_cell[cc];
  // residual column, time transform into NT planes (real modes, then re/im of complex modes)
  T pl[NT][N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int gz = cz * g.p + k;
    const bool live = active && !bxy && !on_boundary(gz, g.nn1);
    const int64_t node = gx + (int64_t)g.nn1 * (gy + (int64_t)g.nn1 * gz);
    T rr[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) rr[t] = live ? r[t * g.n_nodes + node] : T(0);
    if (copy_dst && active) {  // side job for the V-cycle: copy_dst := copy_src on this cell's nodes
#pragma unroll
      for (int t = 0; t < NT; ++t) copy_dst[t * g.n_nodes + node] = copy_src[t * g.n_nodes + node];
    }
#pragma unroll
    for (int m = 0; m < NT; ++m) {
      const bool is_real = m < mt.nreal;
      const int mode = is_real ? m : mt.nreal + (m - mt.nreal) / 2;
      const bool im_part = !is_real && ((m - mt.nreal) & 1);
      T v = 0;
#pragma unroll
      for (int t = 0; t < NT; ++t) v += (im_part ? mt.Wi[mode][t] : mt.Wr[mode][t]) * rr[t];
      pl[m][k] = v;
    }
  }
  // forward spatial transform: z in registers
#pragma unroll
  for (int m = 0; m < NT; ++m)
#pragma unroll
    for (int q = 0; q < N; ++q) {
      T v = 0;
#pragma unroll
      for (int k = 0; k < N; ++k) v += fd.S[tz][k][q] * pl[m][k];
      s0[I4(m, q, j, i)] = v;
    }
  __syncthreads();
  // y: thread (i, qy = j)
#pragma unroll
  for (int m = 0; m < NT; ++m)
#pragma unroll
    for (int qz = 0; qz < N; ++qz) {
      T v = 0;
#pragma unroll
      for (int b = 0; b < N; ++b) v += fd.S[ty][b][j] * s0[I4(m, qz, b, i)];
      s1[I4(m, qz, j, i)] = v;
    }
  __syncthreads();
  // x: thread (qx = i, qy = j); then scale by the inverse eigenvalues
  T hat[NT][N];
#pragma unroll
  for (int m = 0; m < NT; ++m)
#pragma unroll
    for (int qz = 0; qz < N; ++qz) {
      T v = 0;
#pragma unroll
      for (int a = 0; a < N; ++a) v += fd.S[tx][a][i] * s1[I4(m, qz, j, a)];
      hat[m][qz] = v;
    }
#pragma unroll
  for (int qz = 0; qz < N; ++qz) {
    const T sp = rho * (fd.lam[tx][i] + fd.lam[ty][j] + fd.lam[tz][qz]);
#pragma unroll
    for (int m = 0; m < NT; ++m) {
      if (m < mt.nreal) {
        hat[m][qz] = hat[m][qz] / (sp + mt.lre[m]);
      } else if (m + 1 < NT && ((m - mt.nreal) & 1) == 0) {
        const int mode = mt.nreal + (m - mt.nreal) / 2;
        const T a = sp + mt.lre[mode], b = mt.lim[mode];
        const T inv = T(1) / (a * a + b * b);
        const T xr = hat[m][qz], xi = hat[m + 1][qz];
        hat[m][qz] = (xr * a + xi * b) * inv;
        hat[m + 1][qz] = (xi * a - xr * b) * inv;
      }
    }
  }
  __syncthreads();  // s0 was last read before the previous barrier; s1 is read below only after this one
#pragma unroll
  for (int m = 0; m < NT; ++m)
#pragma unroll
    for (int qz = 0; qz < N; ++qz) s0[I4(m, qz, j, i)] = hat[m][qz];
  __syncthreads();
  // back transform x: thread (node a = i, qy = j)
#pragma unroll
  for (int m = 0; m < NT; ++m)
#pragma unroll
    for (int qz = 0; qz < N; ++qz) {
      T v = 0;
#pragma unroll
      for (int q = 0; q < N; ++q) v += fd.S[tx][i][q] * s0[I4(m, qz, j, q)];
      s1[I4(m, qz, j, i)] = v;
    }
  __syncthreads();
  // y and z back transforms, inverse time transform, scatter
  T w[NT][N];
#pragma unroll
  for (int m = 0; m < NT; ++m)
#pragma unroll
    for (int qz = 0; qz < N; ++qz) {
      T v = 0;
#pragma unroll
      for (int q = 0; q < N; ++q) v += fd.S[ty][j][q] * s1[I4(m, qz, q, i)];
      w[m][qz] = v;
    }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T z[NT];
#pragma unroll
    for (int m = 0; m < NT; ++m) {
      T v = 0;
#pragma unroll
      for (int q = 0; q < N; ++q) v += fd.S[tz][k][q] * w[m][q];
      z[m] = v;
    }
    const int gz = cz * g.p + k;
    if (!active || bxy || on_boundary(gz, g.nn1)) continue;
    const int64_t node = gx + (int64_t)g.nn1 * (gy + (int64_t)g.nn1 * gz);
    const T wsc = mt.weighted ? mt.omega * node_weight<T>(gx, gy, gz, 3, g.p) : mt.omega;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      T o = 0;
#pragma unroll
      for (int m = 0; m < NT; ++m) {
        if (m < mt.nreal) {
          o += mt.Vr[t][m] * z[m];
        } else if (m + 1 < NT && ((m - mt.nreal) & 1) == 0) {
          const int mode = mt.nreal + (m - mt.nreal) / 2;
          o += T(2) * (mt.Vr[t][mode] * z[m] - mt.Vi[t][mode] * z[m + 1]);
        }
      }
      atomicAdd(u + t * g.n_nodes + node, wsc * o);
    }
  }
}

template <int N, int NT, typename T>
cudaError_t fd_t(const T* r, T* u, const T* rho, const GridDesc& g, const FDTab<T>& fd, const ModeTab<T>& mt,
                 const T* cs, T* cd, cudaStream_t s) {
  constexpr int CPB = fd_cells_per_block<N>();
  const size_t smem = (size_t)CPB * 2 * NT * N * N * N * sizeof(T);
  auto k = fd_apply_kernel<N, NT, T, CPB>;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t blocks = (g.n_cells + CPB - 1) / CPB;
  { const cudaError_t e_ = launch_k(k, dim3((unsigned)blocks), dim3(CPB * N * N), smem, s, r, u, rho, g, fd, mt, cs, cd); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

}  // namespace

#define STMG_FD_CASE(N, NT) \
  if (n == N && nt == NT) return fd_t<N, NT, T>(r, u, rho, g, fd, mt, cs, cd, s);

template <typename T>
cudaError_t launch_fd_apply(int n, int nt, const T* r, T* u, const T* rho, const GridDesc& g, const FDTab<T>& fd,
                            const ModeTab<T>& mt, const T* cs, T* cd, cudaStream_t s) {
  STMG_FD_CASE(2, 1) STMG_FD_CASE(2, 2) STMG_FD_CASE(2, 3) STMG_FD_CASE(2, 4)
  STMG_FD_CASE(3, 1) STMG_FD_CASE(3, 2) STMG_FD_CASE(3, 3) STMG_FD_CASE(3, 4)
  STMG_FD_CASE(4, 1) STMG_FD_CASE(4, 2) STMG_FD_CASE(4, 3) STMG_FD_CASE(4, 4)
  STMG_FD_CASE(5, 1) STMG_FD_CASE(5, 2) STMG_FD_CASE(5, 3) STMG_FD_CASE(5, 4)
  STMG_FD_CASE(2, 5) STMG_FD_CASE(3, 5) STMG_FD_CASE(4, 5) STMG_FD_CASE(5, 5) STMG_FD_CASE(6, 5)
  return cudaErrorInvalidValue;
}

template cudaError_t launch_fd_apply<float>(int, int, const float*, float*, const float*, const GridDesc&,
                                            const FDTab<float>&, const ModeTab<float>&, const float*, float*,
                                            cudaStream_t);
template cudaError_t launch_fd_apply<double>(int, int, const double*, double*, const double*, const GridDesc&,
                                             const FDTab<double>&, const ModeTab<double>&, const double*, double*,
                                             cudaStream_t);

}  // namespace stmg
