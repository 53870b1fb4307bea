// Kernel templates of the matrix-free space-time operator y (+)= sign * (TA (x) A_h + TM (x) M_h) x   (Section 3.1).
// TA must be diagonal: it is M_tau, diagonal for the Lagrange time bases at quadrature
// nodes of dG(k) and cGP(k) (the host checks this at set-up).
//
// Two kernels.  3D with n = p + 1 <= 3 nodes per direction in FP32 arithmetic:
// apply3d_reg_kernel, one thread per cell and time DoF, everything in registers (described below).
// Otherwise (FP64 arithmetic, higher degrees, 2D): one group of n^(dim-1) threads per cell ("pencil"
// threads, one per (x,y) node column in 3D, one per x node line in 2D), several cells per CTA.  Per cell and
// time DoF the pencil threads do the sum-factorised interpolation to the Gauss
// points (B), collocation derivatives there (D), the space-time mixing with the
// two N_t x N_t time matrices and the metric (rho w |J| J^-1 J^-T) at each point,
// then the transposed sweeps (D^T, B^T).  The last direction runs in registers,
// the others through shared memory.  Results go to global memory with atomic
// adds on unconstrained rows; the caller initialises the output (identity on
// constrained rows, 0 or the right-hand side elsewhere).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "df64.cuh"
#include "kernels.h"
#include "apply_reg.cuh"

namespace stmg {
namespace apply_detail {

template <int N> constexpr int cells_per_block(int dim) {
  return dim == 3 ? (N == 2 ? 32 : N == 3 ? 14 : N == 4 ? 8 : N == 5 ? 5 : 3)
                  : (N == 2 ? 64 : N == 3 ? 42 : N == 4 ? 32 : 25);
}

// Output accumulation: the result of every cell is added to its nodes' rows.  Float and double-float
// results enter FP64 rows through exact bit-field conversions (f2d_exact, df64.cuh), a double-float one
// as two additions (hi, then lo): no FP64 instruction in the kernel, whose FP64 pipe is slow.
__device__ __forceinline__ void add_out(float* p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void add_out(double* p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void add_out(double* p, float v) { atomicAdd(p, f2d_exact(v)); }
__device__ __forceinline__ void add_out(double* p, df64 v) {
  atomicAdd(p, f2d_exact(v.hi));
  if (v.lo != 0.0f) atomicAdd(p, f2d_exact(v.lo));
}

// Gathered input in the arithmetic's terms: an FP64 input entering double-float arithmetic is split
// into two floats (x = hi + lo to 48 bits, below the arithmetic's own 44; bit-field split, df64.cuh);
// other inputs keep their type.
template <typename T, typename TI> struct gather_of { using type = TI; };
template <> struct gather_of<df64, double> { using type = df64; };
template <typename G, typename TI> __device__ __forceinline__ G to_gather(TI v) { return (G)v; }
template <> __device__ __forceinline__ df64 to_gather<df64, double>(double v) { return df_split_fast(v); }

// T: arithmetic (float, double or double-float), TI: input vector type, TO: output vector type.
// MASS: mass part only, y (+)= sign * (TM (x) M_h) x (no derivative sweeps, TA ignored).
template <int N, int NT, typename T, int CPB, typename TI, typename TO, bool MASS = false>
__global__ void __launch_bounds__(CPB * N * N)
apply3d_kernel(const TI* __restrict__ x, TO* __restrict__ y, const T* __restrict__ geo, GridDesc g,
               OpTab<T> tab, int mask_input) {
  pdl_wait();
  pdl_trigger();
  using Acc = typename acc_of<T>::type;
  constexpr int N2 = N * N, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int slot = threadIdx.x / N2;
  const int lid = threadIdx.x - slot * N2;
  const int i = lid % N, j = lid / N;
  const int64_t cell = (int64_t)blockIdx.x * CPB + slot;
  const bool active = cell < g.n_cells;
  T* s0 = smem + (size_t)slot * 3 * NT * N3;
  T* s1 = s0 + NT * N3;
  T* s2 = s1 + NT * N3;
  // the 1D tables, for the reads indexed by this thread's node (i, j): from shared memory every
  // thread reads its own entry in one pass (the parameter bank would serialise differing addresses);
  // the first read follows the barrier after the z sweep
  __shared__ T sB[N][N], sD[N][N];
  if (threadIdx.x < N2) {
    sB[threadIdx.x / N][threadIdx.x % N] = tab.B[threadIdx.x / N][threadIdx.x % N];
    sD[threadIdx.x / N][threadIdx.x % N] = tab.D[threadIdx.x / N][threadIdx.x % N];
  }
  auto I4 = [](int t, int c, int b, int a) { return ((t * N + c) * N + b) * N + a; };

  const int64_t cc = active ? cell : 0;
  int cx, cy, cz;
  cell_xyz(cc, g, cx, cy, cz);
  const int gx = cx * g.p + i, gy = cy * g.p + j;
  const bool bxy = on_boundary(gx, g.nn1) || on_boundary(gy, g.nn1);
  // FP32: the metric of this thread's column of Gauss points is loaded first, so that its latency
  // overlaps the gather and the interpolation sweeps (wider types keep their registers for arithmetic)
  constexpr bool kPre = sizeof(T) == 4 && !MASS;
  T gpre[kPre ? 7 : 1][kPre ? N : 1];
  if constexpr (kPre) {
    const T* gc0 = geo + cc * 7 * N3;
#pragma unroll
    for (int c = 0; c < 7; ++c)
#pragma unroll
      for (int qz = 0; qz < N; ++qz) gpre[c][qz] = gc0[c * N3 + i + N * (j + N * qz)];
  }

  // gather + interpolation in z (registers)
  {
    using GI = typename gather_of<T, TI>::type;
    GI xcol[NT][N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int gz = cz * g.p + k;
      const bool bnd = bxy || on_boundary(gz, g.nn1);
      const int64_t node = gx + (int64_t)g.nn1 * (gy + (int64_t)g.nn1 * gz);
#pragma unroll
      for (int t = 0; t < NT; ++t)
        xcol[t][k] = (active && !(mask_input && bnd)) ? to_gather<GI>(x[t * g.n_nodes + node]) : GI(0);
    }
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int q = 0; q < N; ++q) {
        Acc v = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) v += tab.B[q][k] * xcol[t][k];
        s0[I4(t, q, j, i)] = v;
      }
  }
  __syncthreads();
  // interpolation in y: thread (i, qy = j)
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int qz = 0; qz < N; ++qz) {
      Acc v = 0;
#pragma unroll
      for (int b = 0; b < N; ++b) v += sB[j][b] * s0[I4(t, qz, b, i)];
      s1[I4(t, qz, j, i)] = v;
    }
  __syncthreads();
  // interpolation in x: thread (qx = i, qy = j); values at the column of Gauss points in registers
  T u[NT][N];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int qz = 0; qz < N; ++qz) {
      Acc v = 0;
#pragma unroll
      for (int a = 0; a < N; ++a) v += sB[i][a] * s1[I4(t, qz, j, a)];
      const T vt = v;
      u[t][qz] = vt;
      if constexpr (!MASS) s0[I4(t, qz, j, i)] = vt;
    }
  if constexpr (MASS) {
    // time mixing and mass weight at each Gauss point of the column; s0 is free (nobody reads it)
    const T* gm = geo + cc * 7 * N3 + 6 * N3;
#pragma unroll
    for (int qz = 0; qz < N; ++qz) {
      const T m = gm[i + N * (j + N * qz)];
      T w[NT];
#pragma unroll
      for (int it = 0; it < NT; ++it) {
        Acc v = 0;
#pragma unroll
        for (int jt = 0; jt < NT; ++jt) v += tab.TM[it][jt] * u[jt][qz];
        w[it] = m * v;
      }
#pragma unroll
      for (int it = 0; it < NT; ++it) s0[I4(it, qz, j, i)] = w[it];
    }
    __syncthreads();
  } else {
  __syncthreads();
  // derivatives, time mixing and metric at each Gauss point of the column
  T fz[NT][N], val[NT][N];
  const T* gc = geo + cc * 7 * N3;
#pragma unroll
  for (int qz = 0; qz < N; ++qz) {
    T ux[NT], uy[NT], uz[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      Acc a0 = 0, a1 = 0, a2 = 0;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        a0 += sD[i][a] * s0[I4(t, qz, j, a)];
        a1 += sD[j][a] * s0[I4(t, qz, a, i)];
        a2 += tab.D[qz][a] * u[t][a];
      }
      ux[t] = a0; uy[t] = a1; uz[t] = a2;
    }
    const int q = i + N * (j + N * qz);
    T G00, G01, G02, G11, G12, G22, m;
    if constexpr (kPre) {
      G00 = gpre[0][qz]; G01 = gpre[1][qz]; G02 = gpre[2][qz];
      G11 = gpre[3][qz]; G12 = gpre[4][qz]; G22 = gpre[5][qz]; m = gpre[6][qz];
    } else {
      G00 = gc[0 * N3 + q]; G01 = gc[1 * N3 + q]; G02 = gc[2 * N3 + q];
      G11 = gc[3 * N3 + q]; G12 = gc[4 * N3 + q]; G22 = gc[5 * N3 + q]; m = gc[6 * N3 + q];
    }
#pragma unroll
    for (int it = 0; it < NT; ++it) {
      // TA = M_tau is diagonal (Lagrange time basis at the quadrature nodes): no mixing of gradients
      const T ta = tab.TA[it][it];
      const T gx_ = ta * ux[it], gy_ = ta * uy[it], gz_ = ta * uz[it];
      Acc v = 0;
#pragma unroll
      for (int jt = 0; jt < NT; ++jt) v += tab.TM[it][jt] * u[jt][qz];
      s1[I4(it, qz, j, i)] = G00 * gx_ + G01 * gy_ + G02 * gz_;
      s2[I4(it, qz, j, i)] = G01 * gx_ + G11 * gy_ + G12 * gz_;
      fz[it][qz] = G02 * gx_ + G12 * gy_ + G22 * gz_;
      val[it][qz] = m * v;
    }
  }
  __syncthreads();
  // transposed derivatives: test-function contributions at each Gauss point
#pragma unroll
  for (int it = 0; it < NT; ++it)
#pragma unroll
    for (int qz = 0; qz < N; ++qz) {
      Acc v = val[it][qz];
#pragma unroll
      for (int a = 0; a < N; ++a) {
        v += sD[a][i] * s1[I4(it, qz, j, a)];
        v += sD[a][j] * s2[I4(it, qz, a, i)];
        v += tab.D[a][qz] * fz[it][a];
      }
      u[it][qz] = v;
    }
  // s0 was last read before the previous barrier
#pragma unroll
  for (int it = 0; it < NT; ++it)
#pragma unroll
    for (int qz = 0; qz < N; ++qz) s0[I4(it, qz, j, i)] = u[it][qz];
  __syncthreads();
  }
  // B^T in x: thread (node i, qy = j)
#pragma unroll
  for (int it = 0; it < NT; ++it)
#pragma unroll
    for (int qz = 0; qz < N; ++qz) {
      Acc v = 0;
#pragma unroll
      for (int a = 0; a < N; ++a) v += sB[a][i] * s0[I4(it, qz, j, a)];
      s1[I4(it, qz, j, i)] = v;
    }
  __syncthreads();
  // B^T in y and z, scatter
#pragma unroll
  for (int it = 0; it < NT; ++it) {
    T r[N];
#pragma unroll
    for (int qz = 0; qz < N; ++qz) {
      Acc v = 0;
#pragma unroll
      for (int b = 0; b < N; ++b) v += sB[b][j] * s1[I4(it, qz, b, i)];
      r[qz] = v;
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
      Acc v = 0;
#pragma unroll
      for (int qz = 0; qz < N; ++qz) v += tab.B[qz][k] * r[qz];
      const int gz = cz * g.p + k;
      if (active && !bxy && !on_boundary(gz, g.nn1)) {
        const int64_t node = gx + (int64_t)g.nn1 * (gy + (int64_t)g.nn1 * gz);
        add_out(y + it * g.n_nodes + node, tab.sign * v);
      }
    }
  }
}

template <int N, int NT, typename T, int CPB, typename TI, typename TO, bool MASS = false>
__global__ void __launch_bounds__(CPB * N)
apply2d_kernel(const TI* __restrict__ x, TO* __restrict__ y, const T* __restrict__ geo, GridDesc g,
               OpTab<T> tab, int mask_input) {
  pdl_wait();
  pdl_trigger();
  using Acc = typename acc_of<T>::type;
  constexpr int N2 = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* smem = reinterpret_cast<T*>(smem_raw);
  const int slot = threadIdx.x / N;
  const int i = threadIdx.x - slot * N;
  const int64_t cell = (int64_t)blockIdx.x * CPB + slot;
  const bool active = cell < g.n_cells;
  T* s0 = smem + (size_t)slot * 2 * NT * N2;
  T* s1 = s0 + NT * N2;
  __shared__ T sB[N][N], sD[N][N];  // as in the 3D kernel
  if (threadIdx.x < N2) {
    sB[threadIdx.x / N][threadIdx.x % N] = tab.B[threadIdx.x / N][threadIdx.x % N];
    sD[threadIdx.x / N][threadIdx.x % N] = tab.D[threadIdx.x / N][threadIdx.x % N];
  }
  auto I3 = [](int t, int b, int a) { return (t * N + b) * N + a; };
  const int64_t cc = active ? cell : 0;
  int cx, cy, cz_unused;
  cell_xyz(cc, g, cx, cy, cz_unused);
  const int gx = cx * g.p + i;
  const bool bx = on_boundary(gx, g.nn1);
  {
    using GI = typename gather_of<T, TI>::type;
    GI xcol[NT][N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const int gy = cy * g.p + k;
      const bool bnd = bx || on_boundary(gy, g.nn1);
      const int64_t node = gx + (int64_t)g.nn1 * gy;
#pragma unroll
      for (int t = 0; t < NT; ++t)
        xcol[t][k] = (active && !(mask_input && bnd)) ? to_gather<GI>(x[t * g.n_nodes + node]) : GI(0);
    }
#pragma unroll
    for (int t = 0; t < NT; ++t)
#pragma unroll
      for (int q = 0; q < N; ++q) {
        Acc v = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) v += tab.B[q][k] * xcol[t][k];
        s0[I3(t, q, i)] = v;
      }
  }
  __syncthreads();
  T u[NT][N];
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int qy = 0; qy < N; ++qy) {
      Acc v = 0;
#pragma unroll
      for (int a = 0; a < N; ++a) v += sB[i][a] * s0[I3(t, qy, a)];
      const T vt = v;
      u[t][qy] = vt;
      if constexpr (!MASS) s1[I3(t, qy, i)] = vt;
    }
  if constexpr (MASS) {
    const T* gm = geo + cc * 4 * N2 + 3 * N2;
#pragma unroll
    for (int qy = 0; qy < N; ++qy) {
      const T m = gm[i + N * qy];
      T w[NT];
#pragma unroll
      for (int it = 0; it < NT; ++it) {
        Acc v = 0;
#pragma unroll
        for (int jt = 0; jt < NT; ++jt) v += tab.TM[it][jt] * u[jt][qy];
        w[it] = m * v;
      }
#pragma unroll
      for (int it = 0; it < NT; ++it) s1[I3(it, qy, i)] = w[it];
    }
    __syncthreads();
  } else {
  __syncthreads();
  T fy[NT][N], val[NT][N];
  const T* gc = geo + cc * 4 * N2;
#pragma unroll
  for (int qy = 0; qy < N; ++qy) {
    T ux[NT], uy[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      Acc a0 = 0, a1 = 0;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        a0 += sD[i][a] * s1[I3(t, qy, a)];
        a1 += tab.D[qy][a] * u[t][a];
      }
      ux[t] = a0; uy[t] = a1;
    }
    const int q = i + N * qy;
    const T G00 = gc[0 * N2 + q], G01 = gc[1 * N2 + q], G11 = gc[2 * N2 + q], m = gc[3 * N2 + q];
#pragma unroll
    for (int it = 0; it < NT; ++it) {
      const T ta = tab.TA[it][it];
      const T gx_ = ta * ux[it], gy_ = ta * uy[it];
      Acc v = 0;
#pragma unroll
      for (int jt = 0; jt < NT; ++jt) v += tab.TM[it][jt] * u[jt][qy];
      s0[I3(it, qy, i)] = G00 * gx_ + G01 * gy_;
      fy[it][qy] = G01 * gx_ + G11 * gy_;
      val[it][qy] = m * v;
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < NT; ++it)
#pragma unroll
    for (int qy = 0; qy < N; ++qy) {
      Acc v = val[it][qy];
#pragma unroll
      for (int a = 0; a < N; ++a) {
        v += sD[a][i] * s0[I3(it, qy, a)];
        v += tab.D[a][qy] * fy[it][a];
      }
      u[it][qy] = v;
    }
#pragma unroll
  for (int it = 0; it < NT; ++it)
#pragma unroll
    for (int qy = 0; qy < N; ++qy) s1[I3(it, qy, i)] = u[it][qy];
  __syncthreads();
  }
#pragma unroll
  for (int it = 0; it < NT; ++it) {
    T r[N];
#pragma unroll
    for (int qy = 0; qy < N; ++qy) {
      Acc v = 0;
#pragma unroll
      for (int a = 0; a < N; ++a) v += sB[a][i] * s1[I3(it, qy, a)];
      r[qy] = v;
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
      Acc v = 0;
#pragma unroll
      for (int qy = 0; qy < N; ++qy) v += tab.B[qy][k] * r[qy];
      const int gy = cy * g.p + k;
      if (active && !bx && !on_boundary(gy, g.nn1))
        add_out(y + it * g.n_nodes + gx + (int64_t)g.nn1 * gy, tab.sign * v);
    }
  }
}

template <int DIM, int N, int NT, typename T, typename TI, typename TO, bool MASS = false>
cudaError_t launch_apply_t(const TI* x, TO* y, const T* geo, const GridDesc& g, const OpTab<T>& tab,
                           int mask_input, cudaStream_t s) {
  if constexpr (DIM == 3 && geo_chunked(3, N) && std::is_same<T, float>::value) {
    return launch_apply_reg<N, NT, TI, TO, MASS>(x, y, geo, g, tab, mask_input, s);
  } else {
  constexpr int CPB = cells_per_block<N>(DIM);
  const int64_t blocks = (g.n_cells + CPB - 1) / CPB;
  if constexpr (DIM == 3) {
    const size_t smem = (size_t)CPB * 3 * NT * N * N * N * sizeof(T);
    auto k = apply3d_kernel<N, NT, T, CPB, TI, TO, MASS>;
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = true;
    }
    { const cudaError_t e_ = launch_k(k, dim3((unsigned)blocks), dim3(CPB * N * N), smem, s, x, y, geo, g, tab, mask_input); if (e_ != cudaSuccess) return e_; }
  } else {
    const size_t smem = (size_t)CPB * 2 * NT * N * N * sizeof(T);
    auto k = apply2d_kernel<N, NT, T, CPB, TI, TO, MASS>;
    { const cudaError_t e_ = launch_k(k, dim3((unsigned)blocks), dim3(CPB * N), smem, s, x, y, geo, g, tab, mask_input); if (e_ != cudaSuccess) return e_; }
  }
  }
  return cudaGetLastError();
}

}  // namespace apply_detail
}  // namespace stmg
