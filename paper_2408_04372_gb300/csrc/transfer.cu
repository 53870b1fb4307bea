// Grid transfers between multigrid levels (Section 3.2).
//
// Prolongation = embedding of the coarse space in the fine one, taken in the
// reference coordinates of the structured grid: a Kronecker product of one 1D
// matrix per direction (space levels, p- or h-coarsening) or the N_t x N_t
// matrix P_tau on the time blocks (k-levels), or, between slabs of length tau and 2 tau
// (tau-levels), the coarse dG(k) basis evaluated at the Radau nodes of the two fine halves.
// Restriction = transpose.
// Space transfers run as separable 1D passes (x, y, z), each in gather form -- every
// output entry sums its own inputs by index arithmetic on the structured grid -- so no
// colouring and no atomics are needed, results are deterministic, and a coarse node
// costs 3 (2p_f+1) instead of (2p_f+1)^3 terms.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace stmg {

namespace {

inline int grid_blocks(int64_t total) {
  int64_t b = (total + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

// Optional side job of a transfer's final pass over output entries e (V-cycle fusion):
// copy_dst[e] = copy_src[e] and/or zero_dst[e] = 0.
template <typename T>
struct SideJob {
  const T* copy_src = nullptr;
  T* copy_dst = nullptr;
  T* zero_dst = nullptr;
  __device__ void run(int64_t e) const {
    if (copy_dst) copy_dst[e] = copy_src[e];
    if (zero_dst) zero_dst[e] = T(0);
  }
};

// One 1D pass of a separable transfer along `axis` of a [nt][d2][d1][d0] array (d0 fastest):
// out[..., i, ...] (+)= sum_r w[i][r] in[..., idx[i][r], ...], the axis length changing from
// in_dims[axis] to n_out.
template <typename T>
__global__ void gather_axis_kernel(const T* __restrict__ in, T* __restrict__ out, int d0, int d1, int d2, int nt,
                                   int axis, int n_out, const int* __restrict__ idx, const T* __restrict__ w,
                                   int R, int accumulate, SideJob<T> side) {
  pdl_wait();
  pdl_trigger();
  const int o0 = axis == 0 ? n_out : d0, o1 = axis == 1 ? n_out : d1, o2 = axis == 2 ? n_out : d2;
  const int64_t total = (int64_t)nt * o2 * o1 * o0;
  const int64_t sin_ = axis == 0 ? 1 : (axis == 1 ? d0 : (int64_t)d0 * d1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t r = (uint32_t)e;  // every index of a level is below 2^31
    const int x0 = (int)(r % (uint32_t)o0); r /= (uint32_t)o0;
    const int x1 = (int)(r % (uint32_t)o1); r /= (uint32_t)o1;
    const int x2 = (int)(r % (uint32_t)o2);
    const int t = (int)(r / (uint32_t)o2);
    const int i = axis == 0 ? x0 : (axis == 1 ? x1 : x2);
    const int64_t base = (((int64_t)t * d2 + (axis == 2 ? 0 : x2)) * d1 + (axis == 1 ? 0 : x1)) * d0 + (axis == 0 ? 0 : x0);
    T acc = 0;
    for (int k = 0; k < R; ++k) {
      const int j = idx[i * R + k];
      if (j < 0) break;
      acc += w[i * R + k] * in[base + (int64_t)j * sin_];
    }
    if (accumulate) out[e] += acc;
    else out[e] = acc;
    side.run(e);
  }
}

// Fused single launch when the stencil is narrow or the level small (launch latency dominates),
// separable passes otherwise.
__host__ __device__ inline bool transfer_fused(int terms, int64_t n_out) {
  return terms <= 8 || (terms <= 27 && n_out < (int64_t)4 << 20);
}

// Fused form for narrow 1D stencils: every output node sums the tensor product of its 1D
// lists directly (R^DIM terms), one launch instead of DIM.  The list width R is a template
// parameter: each thread reads its three lists first (padding entries become weight 0 on
// index 0) and then issues all R^DIM input loads at once.
template <typename T, int R, int DIM>
__global__ void gather_fused_kernel(const T* __restrict__ in, T* __restrict__ out, int nt, int nin, int nout,
                                    const int* __restrict__ idx, const T* __restrict__ w, int accumulate,
                                    SideJob<T> side) {
  pdl_wait();
  pdl_trigger();
  const int64_t per = DIM == 3 ? (int64_t)nout * nout * nout : (int64_t)nout * nout;
  const int64_t per_in = DIM == 3 ? (int64_t)nin * nin * nin : (int64_t)nin * nin;
  const int64_t total = per * nt;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    // 32-bit index arithmetic (every index of a level is below 2^31)
    const uint32_t e32 = (uint32_t)e, per32 = (uint32_t)per, no = (uint32_t)nout;
    const int t = (int)(e32 / per32);
    uint32_t r = e32 - (uint32_t)t * per32;
    const uint32_t ry = r / no;
    const int x = (int)(r - ry * no);
    const int y = DIM == 3 ? (int)(ry % no) : (int)ry;
    const int z = DIM == 3 ? (int)(ry / no) : 0;
    int jx[R], jy[R], jz[R];
    T wx[R], wy[R], wz[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int ix = __ldg(idx + x * R + k), iy = __ldg(idx + y * R + k);
      jx[k] = ix < 0 ? 0 : ix;
      wx[k] = ix < 0 ? T(0) : __ldg(w + x * R + k);
      jy[k] = iy < 0 ? 0 : iy;
      wy[k] = iy < 0 ? T(0) : __ldg(w + y * R + k);
      if (DIM == 3) {
        const int iz = __ldg(idx + z * R + k);
        jz[k] = iz < 0 ? 0 : iz;
        wz[k] = iz < 0 ? T(0) : __ldg(w + z * R + k);
      } else {
        jz[k] = 0;
        wz[k] = k == 0 ? T(1) : T(0);
      }
    }
    const T* src = in + (int64_t)t * per_in;
    T acc = 0;
#pragma unroll
    for (int kz = 0; kz < (DIM == 3 ? R : 1); ++kz) {
      T sy = 0;
#pragma unroll
      for (int ky = 0; ky < R; ++ky) {
        const T* row = src + ((int64_t)jz[kz] * nin + jy[ky]) * nin;
        T sx = 0;
#pragma unroll
        for (int kx = 0; kx < R; ++kx) sx += wx[kx] * row[jx[kx]];
        sy += wy[ky] * sx;
      }
      acc += wz[kz] * sy;
    }
    if (accumulate) out[e] += acc;
    else out[e] = acc;
    side.run(e);
  }
}

// The transfer weights in the arithmetic's own type (FP64 table or its FP32 copy).
template <typename T> const T* weights(const double* w64, const float* w32);
template <> const double* weights<double>(const double* w64, const float*) { return w64; }
template <> const float* weights<float>(const double*, const float* w32) { return w32; }

template <typename T>
cudaError_t separable(const T* in, T* out, int dim, int nt, int nin, int nout, const int* idx, const T* w, int R,
                      T* t1, T* t2, int accumulate, SideJob<T> side, cudaStream_t s) {
  const SideJob<T> none{};
  // passes x, y(, z): dims go from nin^dim to nout^dim
  auto blocks = [](int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32)); };
  const int terms = dim == 3 ? R * R * R : R * R;
  const int64_t nout_total = (int64_t)nt * (dim == 3 ? (int64_t)nout * nout * nout : (int64_t)nout * nout);
  if (transfer_fused(terms, nout_total)) {  // R <= 3 in 3D, R <= 5 in 2D
    const int nb = blocks(nout_total);
#define STMG_FUSED(RR, DD) \
  return launch_k(gather_fused_kernel<T, RR, DD>, dim3(nb), dim3(256), 0, s, in, out, nt, nin, nout, idx, w, accumulate, side)
    if (dim == 3) {
      if (R == 1) STMG_FUSED(1, 3); else if (R == 2) STMG_FUSED(2, 3); else STMG_FUSED(3, 3);
    } else {
      if (R == 1) STMG_FUSED(1, 2); else if (R == 2) STMG_FUSED(2, 2); else if (R == 3) STMG_FUSED(3, 2);
      else if (R == 4) STMG_FUSED(4, 2); else STMG_FUSED(5, 2);
    }
#undef STMG_FUSED
    return cudaGetLastError();
  }
  if (dim == 2) {
    const int64_t n1 = (int64_t)nt * nin * nout;
    { const cudaError_t e_ = launch_k(gather_axis_kernel<T>, dim3(blocks(n1)), dim3(256), 0, s, in, t1, nin, nin, 1, nt, 0, nout, idx, w, R, 0, none); if (e_ != cudaSuccess) return e_; }
    const int64_t n2 = (int64_t)nt * nout * nout;
    { const cudaError_t e_ = launch_k(gather_axis_kernel<T>, dim3(blocks(n2)), dim3(256), 0, s, t1, out, nout, nin, 1, nt, 1, nout, idx, w, R, accumulate, side); if (e_ != cudaSuccess) return e_; }
  } else {
    const int64_t n1 = (int64_t)nt * nin * nin * nout;
    { const cudaError_t e_ = launch_k(gather_axis_kernel<T>, dim3(blocks(n1)), dim3(256), 0, s, in, t1, nin, nin, nin, nt, 0, nout, idx, w, R, 0, none); if (e_ != cudaSuccess) return e_; }
    const int64_t n2 = (int64_t)nt * nin * nout * nout;
    { const cudaError_t e_ = launch_k(gather_axis_kernel<T>, dim3(blocks(n2)), dim3(256), 0, s, t1, t2, nout, nin, nin, nt, 1, nout, idx, w, R, 0, none); if (e_ != cudaSuccess) return e_; }
    const int64_t n3 = (int64_t)nt * nout * nout * nout;
    { const cudaError_t e_ = launch_k(gather_axis_kernel<T>, dim3(blocks(n3)), dim3(256), 0, s, t2, out, nout, nout, nin, nt, 2, nout, idx, w, R, accumulate, side); if (e_ != cudaSuccess) return e_; }
  }
  return cudaGetLastError();
}

__device__ inline bool node_on_boundary(int64_t node, const GridDesc& g) {
  int gx, gy, gz;
  node_xyz(node, g.nn1, gx, gy, gz);
  return on_boundary(gx, g.nn1) || on_boundary(gy, g.nn1) || (g.dim == 3 && on_boundary(gz, g.nn1));
}

template <typename T>
__global__ void prolong_time_add_kernel(T* __restrict__ uf, const T* __restrict__ ec, GridDesc g, TimeTransfer tt,
                                       SideJob<T> side) {
  pdl_wait();
  pdl_trigger();
  const int64_t nn = g.n_nodes;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn * tt.nb; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = (uint32_t)e / (uint32_t)nn, node = e - b * nn;
    T* ub = uf + b * tt.ntf * nn;
    const T* eb = ec + b * tt.ntc * nn;
    for (int i = 0; i < tt.ntf; ++i) side.run(b * tt.ntf * nn + i * nn + node);
    if (node_on_boundary(node, g)) continue;
    T ev[kMaxNT];
    for (int j = 0; j < tt.ntc; ++j) ev[j] = eb[j * nn + node];
    for (int i = 0; i < tt.ntf; ++i) {
      T s = 0;
      for (int j = 0; j < tt.ntc; ++j) s += (T)tt.P[i][j] * ev[j];
      ub[i * nn + node] += s;
    }
  }
}

template <typename T>
__global__ void restrict_time_kernel(T* __restrict__ rc, const T* __restrict__ rf, GridDesc g, TimeTransfer tt,
                                     SideJob<T> side) {
  pdl_wait();
  pdl_trigger();
  const int64_t nn = g.n_nodes;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn * tt.nb; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = (uint32_t)e / (uint32_t)nn, node = e - b * nn;
    T* cb = rc + b * tt.ntc * nn;
    const T* fb = rf + b * tt.ntf * nn;
    for (int j = 0; j < tt.ntc; ++j) side.run(b * tt.ntc * nn + j * nn + node);
    const bool bnd = node_on_boundary(node, g);
    T rv[2 * kMaxNT];
    for (int i = 0; i < tt.ntf; ++i) rv[i] = bnd ? T(0) : fb[i * nn + node];
    for (int j = 0; j < tt.ntc; ++j) {
      T s = 0;
      for (int i = 0; i < tt.ntf; ++i) s += (T)tt.P[i][j] * rv[i];
      cb[j * nn + node] = s;
    }
  }
}

}  // namespace

template <typename T>
cudaError_t launch_prolong_space_add(T* uf, const T* ec, const GridDesc& gf, const GridDesc& gc, int nt,
                                     const Transfer1D& t, const T* copy_src, T* copy_dst, cudaStream_t s) {
  SideJob<T> side;
  side.copy_src = copy_src;
  side.copy_dst = copy_dst;
  return separable<T>(ec, uf, gf.dim, nt, gc.nn1, gf.nn1, t.p_idx, weights<T>(t.p_w, t.p_w32), t.width_p,
                      reinterpret_cast<T*>(t.tmp1),
                      reinterpret_cast<T*>(t.tmp2), 1, side, s);
}
template <typename T>
cudaError_t launch_restrict_space(T* rc, const T* rf, const GridDesc& gf, const GridDesc& gc, int nt,
                                  const Transfer1D& t, T* zero_dst, cudaStream_t s) {
  SideJob<T> side;
  side.zero_dst = zero_dst;
  return separable<T>(rf, rc, gf.dim, nt, gf.nn1, gc.nn1, t.r_idx, weights<T>(t.r_w, t.r_w32), t.width_r,
                      reinterpret_cast<T*>(t.tmp1),
                      reinterpret_cast<T*>(t.tmp2), 0, side, s);
}
template <typename T>
cudaError_t launch_prolong_time_add(T* uf, const T* ec, const GridDesc& g, const TimeTransfer& t, const T* copy_src,
                                    T* copy_dst, cudaStream_t s) {
  SideJob<T> side;
  side.copy_src = copy_src;
  side.copy_dst = copy_dst;
  { const cudaError_t e_ = launch_k(prolong_time_add_kernel<T>, dim3(grid_blocks(g.n_nodes * t.nb)), dim3(256), 0, s, uf, ec, g, t, side); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_restrict_time(T* rc, const T* rf, const GridDesc& g, const TimeTransfer& t, T* zero_dst,
                                 cudaStream_t s) {
  SideJob<T> side;
  side.zero_dst = zero_dst;
  { const cudaError_t e_ = launch_k(restrict_time_kernel<T>, dim3(grid_blocks(g.n_nodes * t.nb)), dim3(256), 0, s, rc, rf, g, t, side); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

#define STMG_TR_INST(T)                                                                                        \
  template cudaError_t launch_prolong_space_add<T>(T*, const T*, const GridDesc&, const GridDesc&, int,          \
                                                   const Transfer1D&, const T*, T*, cudaStream_t);               \
  template cudaError_t launch_restrict_space<T>(T*, const T*, const GridDesc&, const GridDesc&, int,             \
                                                const Transfer1D&, T*, cudaStream_t);                            \
  template cudaError_t launch_prolong_time_add<T>(T*, const T*, const GridDesc&, const TimeTransfer&, const T*, T*, \
                                                  cudaStream_t);                                                 \
  template cudaError_t launch_restrict_time<T>(T*, const T*, const GridDesc&, const TimeTransfer&, T*, cudaStream_t);
STMG_TR_INST(float)
STMG_TR_INST(double)

}  // namespace stmg
