// Vector kernels of the FP64 outer FGMRES and small helpers: conversions,
// deterministic multi-dot products (two-stage reduction in a fixed order: per-block
// partial sums in a scratch buffer, then one block per product),
// multi-AXPY, time-only mixing of nodal blocks, the dense coarsest-level solve.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace stmg {

namespace {

constexpr int kMaxVec = 72;
constexpr int kDotBlocks = 152 * 4;
constexpr int kDotThreads = 256;
constexpr int kChunk = 8;

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

__device__ inline double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;  // valid in thread 0
}

// stage 1: partial[j * nblocks + b] = sum over block b's fixed slice of V_j . w ; j = nv holds w . w
__global__ void __launch_bounds__(kDotThreads)
multidot_stage1(const double* __restrict__ V0, int64_t stride, int nv, const double* __restrict__ w, int64_t n,
                int with_norm, double* __restrict__ partial) {
  __shared__ double red[kDotThreads / 32][kChunk];
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * per, hi = std::min<int64_t>(n, lo + per);
  const int ntot = nv + (with_norm ? 1 : 0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j0 = 0; j0 < ntot; j0 += kChunk) {
    double acc[kChunk];
#pragma unroll
    for (int c = 0; c < kChunk; ++c) acc[c] = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
      const double wi = w[i];
#pragma unroll
      for (int c = 0; c < kChunk; ++c) {
        const int j = j0 + c;
        if (j < nv) acc[c] += __ldg(V0 + j * stride + i) * wi;
        else if (j == nv && with_norm) acc[c] += wi * wi;
      }
    }
#pragma unroll
    for (int c = 0; c < kChunk; ++c) {
      double v = acc[c];
      for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
      if (lane == 0) red[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < kChunk && j0 + (int)threadIdx.x < ntot) {
      double s = 0.0;
      for (int wv = 0; wv < kDotThreads / 32; ++wv) s += red[wv][threadIdx.x];
      partial[(int64_t)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

// stage 2: block j sums partial[j][0..nblocks) by a fixed-order tree
__global__ void __launch_bounds__(kDotThreads)
multidot_stage2(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  __shared__ double red[kDotThreads / 32];
  const double* p = partial + (int64_t)blockIdx.x * nblocks;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += p[b];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
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

int multidot_blocks() { return kDotBlocks; }

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

cudaError_t launch_multidot(const double* V0, int64_t stride, int nv, const double* w, int64_t n, int with_norm,
                            double* partial, int nblocks, double* out, cudaStream_t s) {
  if (nv > kMaxVec || nblocks < 1) return cudaErrorInvalidValue;
  const int ntot = nv + (with_norm ? 1 : 0);
  multidot_stage1<<<nblocks, kDotThreads, 0, s>>>(V0, stride, nv, w, n, with_norm, partial);
  multidot_stage2<<<ntot, kDotThreads, 0, s>>>(partial, nblocks, out);
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
