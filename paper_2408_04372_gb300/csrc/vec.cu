// Vector kernels of the FP64 outer FGMRES and small helpers: conversions, the fused
// classical Gram-Schmidt passes (deterministic single-launch reductions), multi-AXPY,
// time-only mixing of nodal blocks, the dense coarsest-level solve.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace stmg {

namespace {

constexpr int kMaxVec = 72;
constexpr int kCgsThreads = 256;
constexpr int kCgsBlocks = 152 * 4;

inline int grid_blocks(int64_t total) {
  int64_t b = (total + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin* __restrict__ x, Tout* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (Tout)x[i];
}

__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

__global__ void scale_by_device_kernel(double* __restrict__ x, const double* __restrict__ sc, int64_t n) {
  const double s = sc[0];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= s;
}

// One pass of classical Gram-Schmidt against V_0..V_{nv-1} (V_j = V0 + j * stride):
//   sub : w -= sum_j c[j] V_j             (c on the device)
//   dot : s_j = V_j . w, j < nv            (after the subtraction)
//   norm: s_nv = w . w                     (after the subtraction)
// Every block reduces a fixed contiguous slice; the last block to arrive sums the per-block
// partials in block order, so the results do not depend on scheduling.  It then writes
//   fin 0: out[j] = s_j (j < nv) and out[nv] = s_nv when norm is set;
//   fin 1: the Arnoldi column out[j] = h_prev[j] + c[j], out[nv] = sqrt(s_nv), out[nv+1] = 1/out[nv].
// One thread keeps the K values V_j[i] of its element in registers between the subtraction and
// the dot products, so every basis vector is read once per pass.
template <int K>
__global__ void __launch_bounds__(kCgsThreads)
cgs_pass_kernel(const double* __restrict__ V0, int64_t stride, int nv, double* __restrict__ w, int64_t n,
                const double* __restrict__ c, int sub, int dot, int norm, const double* __restrict__ h_prev, int fin,
                double* __restrict__ partial, unsigned int* __restrict__ counter, double* __restrict__ out) {
  __shared__ double red[kCgsThreads / 32][K + 1];
  __shared__ double cs[K];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < K; j += blockDim.x) cs[j] = (sub && j < nv) ? c[j] : 0.0;
  __syncthreads();
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < n ? lo + per : n;
  double acc[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) acc[j] = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kCgsThreads) {
    double v[K];
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = j < nv ? __ldg(V0 + j * stride + i) : 0.0;
    double wi = w[i];
    if (sub) {
      double sv = 0.0;
#pragma unroll
      for (int j = 0; j < K; ++j) sv += cs[j] * v[j];
      wi -= sv;
      w[i] = wi;
    }
    if (dot) {
#pragma unroll
      for (int j = 0; j < K; ++j) acc[j] += v[j] * wi;
    }
    acc[K] += wi * wi;
  }
  // block partials: slot j < nv (dot), slot K (norm)
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    if ((j < K && dot && j < nv) || (j == K && norm)) {
      double x = acc[j];
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      if (lane == 0) red[warp][j] = x;
    }
  }
  __syncthreads();
  const int nb = gridDim.x;
  for (int j = threadIdx.x; j <= K; j += blockDim.x) {
    if ((j < K && dot && j < nv) || (j == K && norm)) {
      double x = 0.0;
      for (int wv = 0; wv < kCgsThreads / 32; ++wv) x += red[wv][j];
      partial[(int64_t)j * nb + blockIdx.x] = x;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned)nb - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  // fixed-order sums over blocks: warp w takes slots w, w + 8, ...
  __shared__ double tot[K + 1];
  for (int j = warp; j <= K; j += kCgsThreads / 32) {
    if ((j < K && dot && j < nv) || (j == K && norm)) {
      double x = 0.0;
      for (int b = lane; b < nb; b += 32) x += __ldcg(partial + (int64_t)j * nb + b);
      for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      if (lane == 0) tot[j] = x;
    }
  }
  __syncthreads();
  if (fin == 0) {
    for (int j = threadIdx.x; j < nv; j += blockDim.x)
      if (dot) out[j] = tot[j];
    if (norm && threadIdx.x == 0) out[nv] = tot[K];
  } else {
    for (int j = threadIdx.x; j < nv; j += blockDim.x) out[j] = h_prev[j] + cs[j];
    if (threadIdx.x == 0) {
      const double hn = sqrt(fmax(tot[K], 0.0));
      out[nv] = hn;
      out[nv + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
}

__global__ void multi_axpy_kernel(double* __restrict__ w, const double* __restrict__ V0, int64_t stride,
                                  const double* __restrict__ h, int nv, double sign, int64_t n) {
  __shared__ double sh[kMaxVec];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) sh[j] = h[j];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < nv; ++j) s += sh[j] * __ldg(V0 + j * stride + i);
    w[i] += sign * s;
  }
}

__global__ void broadcast_time_kernel(const double* __restrict__ u0, double* __restrict__ u, int nt, int64_t nn) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = u0[i];
    for (int t = 0; t < nt; ++t) u[t * nn + i] = v;
  }
}

struct MixTab { const double* x[8]; double C[kMaxNT][8]; };

__global__ void time_mix_kernel(MixTab m, int nin, int nout, double* __restrict__ y, int64_t nn, int accumulate) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
    double xv[8];
    for (int j = 0; j < nin; ++j) xv[j] = m.x[j][i];
    for (int t = 0; t < nout; ++t) {
      double s = accumulate ? y[t * nn + i] : 0.0;
      for (int j = 0; j < nin; ++j) s += m.C[t][j] * xv[j];
      y[t * nn + i] = s;
    }
  }
}

template <typename T>
__global__ void coarse_solve_kernel(const T* __restrict__ f, T* __restrict__ u, const T* __restrict__ inv,
                                    const int64_t* __restrict__ map, int n) {
  // inv stored column-major: inv[j * n + i]
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T s = 0;
    for (int j = 0; j < n; ++j) s += inv[(int64_t)j * n + i] * f[map[j]];
    u[map[i]] = s;
  }
}

__global__ void zero_constrained_kernel(double* __restrict__ y, GridDesc g, int nt) {
  for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n_nodes;
       node += (int64_t)gridDim.x * blockDim.x) {
    const int gx = (int)(node % g.nn1);
    const int64_t rest = node / g.nn1;
    bool bnd = on_boundary(gx, g.nn1);
    if (g.dim == 3) bnd = bnd || on_boundary((int)(rest % g.nn1), g.nn1) || on_boundary((int)(rest / g.nn1), g.nn1);
    else bnd = bnd || on_boundary((int)rest, g.nn1);
    if (bnd)
      for (int t = 0; t < nt; ++t) y[t * g.n_nodes + node] = 0.0;
  }
}

}  // namespace


template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin* x, Tout* y, int64_t n, cudaStream_t s) {
  convert_kernel<Tin, Tout><<<grid_blocks(n), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);

cudaError_t launch_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t s) {
  axpby_kernel<<<grid_blocks(n), 256, 0, s>>>(a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t launch_scale_by_device(double* x, const double* sc, int64_t n, cudaStream_t s) {
  scale_by_device_kernel<<<grid_blocks(n), 256, 0, s>>>(x, sc, n);
  return cudaGetLastError();
}

int cgs_blocks() { return kCgsBlocks; }

cudaError_t launch_cgs_pass(const double* V0, int64_t stride, int nv, double* w, int64_t n, const double* c, int sub,
                            int dot, int norm, const double* h_prev, int fin, double* partial, unsigned int* counter,
                            double* out, cudaStream_t s) {
  if (nv < 0 || nv > 64) return cudaErrorInvalidValue;
  // one wave: blocks per SM as the register use of each width allows (4, 4, 2, 1, 1)
#define STMG_CGS(KK, BPS) \
  cgs_pass_kernel<KK><<<152 * (BPS), kCgsThreads, 0, s>>>(V0, stride, nv, w, n, c, sub, dot, norm, h_prev, fin, partial, counter, out)
  if (nv <= 4) STMG_CGS(4, 4);
  else if (nv <= 8) STMG_CGS(8, 4);
  else if (nv <= 16) STMG_CGS(16, 2);
  else if (nv <= 32) STMG_CGS(32, 1);
  else STMG_CGS(64, 1);
#undef STMG_CGS
  return cudaGetLastError();
}

cudaError_t launch_multi_axpy(double* w, const double* V0, int64_t stride, const double* h, int nv, double sign,
                              int64_t n, cudaStream_t s) {
  if (nv > kMaxVec) return cudaErrorInvalidValue;
  multi_axpy_kernel<<<grid_blocks(n), 256, 0, s>>>(w, V0, stride, h, nv, sign, n);
  return cudaGetLastError();
}

cudaError_t launch_broadcast_time(const double* u0, double* u, int nt, int64_t nn, cudaStream_t s) {
  broadcast_time_kernel<<<grid_blocks(nn), 256, 0, s>>>(u0, u, nt, nn);
  return cudaGetLastError();
}

cudaError_t launch_time_mix(const double* const* xs, int nin, const double* C, int nout, double* y, int64_t nn,
                            int accumulate, cudaStream_t s) {
  if (nin > 8 || nout > kMaxNT) return cudaErrorInvalidValue;
  MixTab m{};
  for (int j = 0; j < nin; ++j) m.x[j] = xs[j];
  for (int t = 0; t < nout; ++t)
    for (int j = 0; j < nin; ++j) m.C[t][j] = C[t * nin + j];
  time_mix_kernel<<<grid_blocks(nn), 256, 0, s>>>(m, nin, nout, y, nn, accumulate);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve(const T* f, T* u, const T* inv, const int64_t* map, int n, int64_t total,
                                cudaStream_t s) {
  (void)total;
  coarse_solve_kernel<T><<<(n + 127) / 128, 128, 0, s>>>(f, u, inv, map, n);
  return cudaGetLastError();
}
template cudaError_t launch_coarse_solve<float>(const float*, float*, const float*, const int64_t*, int, int64_t,
                                                cudaStream_t);
template cudaError_t launch_coarse_solve<double>(const double*, double*, const double*, const int64_t*, int, int64_t,
                                                 cudaStream_t);

cudaError_t launch_zero_constrained(double* y, const GridDesc& g, int nt, cudaStream_t s) {
  zero_constrained_kernel<<<grid_blocks(g.n_nodes), 256, 0, s>>>(y, g, nt);
  return cudaGetLastError();
}

}  // namespace stmg
