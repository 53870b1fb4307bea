// Grid transfers between multigrid levels (Section 3.2).
//
// Prolongation = embedding of the coarse space in the fine one, taken in the
// reference coordinates of the structured grid: a Kronecker product of one 1D
// matrix per direction (space levels, p- or h-coarsening) or the N_t x N_t
// matrix P_tau on the time blocks (k-levels).  Restriction = transpose.
// Both are written in gather form -- every output node sums its own inputs by
// index arithmetic on the structured grid -- so no colouring and no atomics are
// needed and results are deterministic.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace stmg {

namespace {

inline int grid_blocks(int64_t total) {
  int64_t b = (total + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

template <typename T>
__global__ void prolong_space_add_kernel(T* __restrict__ uf, const T* __restrict__ ec, GridDesc gf, GridDesc gc,
                                         int nt, Transfer1D tr) {
  const int64_t total = gf.n_nodes * nt;
  const int W = tr.width_p;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx / gf.n_nodes);
    const int64_t node = idx - (int64_t)t * gf.n_nodes;
    const int gx = (int)(node % gf.nn1);
    const int64_t rest = node / gf.nn1;
    const int gy = gf.dim == 3 ? (int)(rest % gf.nn1) : (int)rest;
    const int gz = gf.dim == 3 ? (int)(rest / gf.nn1) : 0;
    if (on_boundary(gx, gf.nn1) || on_boundary(gy, gf.nn1) || (gf.dim == 3 && on_boundary(gz, gf.nn1))) continue;
    const int sx = tr.p_start[gx], sy = tr.p_start[gy], sz = gf.dim == 3 ? tr.p_start[gz] : 0;
    const T* e = ec + (int64_t)t * gc.n_nodes;
    T acc = 0;
    const int wz_n = gf.dim == 3 ? W : 1;
    for (int bz = 0; bz < wz_n; ++bz) {
      const T wz = gf.dim == 3 ? (T)tr.p_w[gz * W + bz] : T(1);
      if (wz == T(0)) continue;
      for (int by = 0; by < W; ++by) {
        const T wy = (T)tr.p_w[gy * W + by];
        if (wy == T(0)) continue;
        const int64_t row = (int64_t)gc.nn1 * ((sy + by) + (int64_t)gc.nn1 * (sz + bz));
        T s = 0;
        for (int bx = 0; bx < W; ++bx) s += (T)tr.p_w[gx * W + bx] * e[row + sx + bx];
        acc += wz * wy * s;
      }
    }
    uf[idx] += acc;
  }
}

template <typename T>
__global__ void restrict_space_kernel(T* __restrict__ rc, const T* __restrict__ rf, GridDesc gf, GridDesc gc, int nt,
                                      Transfer1D tr) {
  const int64_t total = gc.n_nodes * nt;
  const int R = tr.width_r;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(idx / gc.n_nodes);
    const int64_t node = idx - (int64_t)t * gc.n_nodes;
    const int Gx = (int)(node % gc.nn1);
    const int64_t rest = node / gc.nn1;
    const int Gy = gc.dim == 3 ? (int)(rest % gc.nn1) : (int)rest;
    const int Gz = gc.dim == 3 ? (int)(rest / gc.nn1) : 0;
    if (on_boundary(Gx, gc.nn1) || on_boundary(Gy, gc.nn1) || (gc.dim == 3 && on_boundary(Gz, gc.nn1))) {
      rc[idx] = T(0);
      continue;
    }
    const T* r = rf + (int64_t)t * gf.n_nodes;
    T acc = 0;
    const int rz_n = gc.dim == 3 ? R : 1;
    for (int cz = 0; cz < rz_n; ++cz) {
      const int fz = gc.dim == 3 ? tr.r_idx[Gz * R + cz] : 0;
      if (fz < 0) continue;
      const T wz = gc.dim == 3 ? (T)tr.r_w[Gz * R + cz] : T(1);
      for (int cy = 0; cy < R; ++cy) {
        const int fy = tr.r_idx[Gy * R + cy];
        if (fy < 0) continue;
        const T wy = (T)tr.r_w[Gy * R + cy];
        const int64_t row = (int64_t)gf.nn1 * (fy + (int64_t)gf.nn1 * fz);
        T s = 0;
        for (int cx = 0; cx < R; ++cx) {
          const int fx = tr.r_idx[Gx * R + cx];
          if (fx < 0) continue;
          s += (T)tr.r_w[Gx * R + cx] * r[row + fx];
        }
        acc += wz * wy * s;
      }
    }
    rc[idx] = acc;
  }
}

__device__ inline bool node_on_boundary(int64_t node, const GridDesc& g) {
  const int gx = (int)(node % g.nn1);
  const int64_t rest = node / g.nn1;
  if (on_boundary(gx, g.nn1)) return true;
  if (g.dim == 3) return on_boundary((int)(rest % g.nn1), g.nn1) || on_boundary((int)(rest / g.nn1), g.nn1);
  return on_boundary((int)rest, g.nn1);
}

template <typename T>
__global__ void prolong_time_add_kernel(T* __restrict__ uf, const T* __restrict__ ec, GridDesc g, TimeTransfer tt) {
  for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n_nodes;
       node += (int64_t)gridDim.x * blockDim.x) {
    if (node_on_boundary(node, g)) continue;
    T ev[kMaxNT];
    for (int j = 0; j < tt.ntc; ++j) ev[j] = ec[j * g.n_nodes + node];
    for (int i = 0; i < tt.ntf; ++i) {
      T s = 0;
      for (int j = 0; j < tt.ntc; ++j) s += (T)tt.P[i][j] * ev[j];
      uf[i * g.n_nodes + node] += s;
    }
  }
}

template <typename T>
__global__ void restrict_time_kernel(T* __restrict__ rc, const T* __restrict__ rf, GridDesc g, TimeTransfer tt) {
  for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n_nodes;
       node += (int64_t)gridDim.x * blockDim.x) {
    const bool bnd = node_on_boundary(node, g);
    T rv[kMaxNT];
    for (int i = 0; i < tt.ntf; ++i) rv[i] = bnd ? T(0) : rf[i * g.n_nodes + node];
    for (int j = 0; j < tt.ntc; ++j) {
      T s = 0;
      for (int i = 0; i < tt.ntf; ++i) s += (T)tt.P[i][j] * rv[i];
      rc[j * g.n_nodes + node] = s;
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_prolong_space_add(T* uf, const T* ec, const GridDesc& gf, const GridDesc& gc, int nt,
                                     const Transfer1D& t, cudaStream_t s) {
  prolong_space_add_kernel<T><<<grid_blocks(gf.n_nodes * nt), 256, 0, s>>>(uf, ec, gf, gc, nt, t);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_restrict_space(T* rc, const T* rf, const GridDesc& gf, const GridDesc& gc, int nt,
                                  const Transfer1D& t, cudaStream_t s) {
  restrict_space_kernel<T><<<grid_blocks(gc.n_nodes * nt), 256, 0, s>>>(rc, rf, gf, gc, nt, t);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_prolong_time_add(T* uf, const T* ec, const GridDesc& g, const TimeTransfer& t, cudaStream_t s) {
  prolong_time_add_kernel<T><<<grid_blocks(g.n_nodes), 256, 0, s>>>(uf, ec, g, t);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_restrict_time(T* rc, const T* rf, const GridDesc& g, const TimeTransfer& t, cudaStream_t s) {
  restrict_time_kernel<T><<<grid_blocks(g.n_nodes), 256, 0, s>>>(rc, rf, g, t);
  return cudaGetLastError();
}

#define STMG_TR_INST(T)                                                                                        \
  template cudaError_t launch_prolong_space_add<T>(T*, const T*, const GridDesc&, const GridDesc&, int,          \
                                                   const Transfer1D&, cudaStream_t);                             \
  template cudaError_t launch_restrict_space<T>(T*, const T*, const GridDesc&, const GridDesc&, int,             \
                                                const Transfer1D&, cudaStream_t);                                \
  template cudaError_t launch_prolong_time_add<T>(T*, const T*, const GridDesc&, const TimeTransfer&, cudaStream_t); \
  template cudaError_t launch_restrict_time<T>(T*, const T*, const GridDesc&, const TimeTransfer&, cudaStream_t);
STMG_TR_INST(float)
STMG_TR_INST(double)

}  // namespace stmg
