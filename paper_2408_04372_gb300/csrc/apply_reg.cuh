// Register-resident 3D operator kernel y (+)= sign * (TA (x) A_h + TM (x) M_h) x in FP32 arithmetic
// (Section 3.1) for n = p + 1 <= 3 nodes per direction; the general kernels are in apply_kernels.cuh.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "df64.cuh"
#include "kernels.h"

namespace stmg {
namespace apply_detail {

// ---- register-resident variant: one thread per (cell, time DoF) ----
//
// For n = p + 1 <= 3 nodes per direction the whole sum factorisation of one cell and time DoF fits
// in a thread's registers (n^3 values at the Gauss points, n^3 accumulators), so no shared memory is
// touched: the interpolation sweeps run in place; at each Gauss point the thread forms the three
// collocation derivatives, applies the metric and adds the transposed derivatives straight into the
// accumulators; the time mixing of the mass term, sum_j TM[t][j] u_j, takes the other time DoFs' values
// at the point from the lanes that hold them (warp shuffles); the transposed interpolation runs in
// place and the result is added to the output rows.  A warp holds CW = 32 / NT cells, lane t * CW + c
// being cell c at time DoF t; the lanes above NT * CW only take part in the shuffles.  The geometry is
// in the chunked layout; each warp first stages its cells' geometry in shared memory with
// asynchronous 16-byte copies (cp.async), issued before the gather, so that their latency overlaps the
// gather and the interpolation sweeps (the kernel is latency-bound: 16 warps per SM at 128 registers).
// Double-float arithmetic is not taken here: its n^3 values and accumulators need twice the
// registers (255 with spills for n = 3, two CTAs per SM), which measured 2x slower than the
// shared-memory kernel.
constexpr int kRegWarps = 4;

__device__ __forceinline__ float shfl_from(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }

template <int N, int NT, typename TI, typename TO, bool MASS>
__global__ void __launch_bounds__(32 * kRegWarps, 4)
apply3d_reg_kernel(const TI* __restrict__ x, TO* __restrict__ y, const float* __restrict__ geo, GridDesc g,
                   OpTab<float> tab, int mask_input) {
  using T = float;
  pdl_wait();
  pdl_trigger();
  constexpr int N3 = N * N * N;
  constexpr int CW = 32 / NT;
  const int lane = threadIdx.x & 31;
  const int tl = lane / CW;
  const int cs = lane - tl * CW;
  const int t = tl < NT ? tl : NT - 1;
  const int64_t cell0 = ((int64_t)blockIdx.x * kRegWarps + (threadIdx.x >> 5)) * CW;  // the warp's first cell
  const int64_t cell = cell0 + cs;
  const bool active = tl < NT && cell < g.n_cells;
  const int64_t cc = cell < g.n_cells ? cell : 0;

  // stage the warp's geometry: piece i = (point q, part h, cell slot c) -> sg[(q * 2 + h) * CW + c]
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* sg = reinterpret_cast<float4*>(smem_raw) + (threadIdx.x >> 5) * (2 * N3 * CW);
  {
    const float4* g4 = reinterpret_cast<const float4*>(geo);
    for (int i = lane; i < 2 * N3 * CW; i += 32) {
      const int c = i % CW, qh = i / CW;
      const int64_t ci = cell0 + c < g.n_cells ? cell0 + c : 0;
      const float4* src = g4 + ((ci / kGeoChunk) * (2 * N3) + qh) * kGeoChunk + ci % kGeoChunk;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sg + i)),
                   "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }

  // this thread's time row: TA[t][t] and TM[t][(t + d) % NT] with the operator's sign folded in
  T ta = tab.TA[0][0];
  T tmr[NT];
#pragma unroll
  for (int d = 0; d < NT; ++d) tmr[d] = tab.TM[0][d];
#pragma unroll
  for (int s = 1; s < NT; ++s)
    if (t == s) {
      ta = tab.TA[s][s];
#pragma unroll
      for (int d = 0; d < NT; ++d) tmr[d] = tab.TM[s][(s + d) % NT];
    }
  ta = ta * tab.sign;
#pragma unroll
  for (int d = 0; d < NT; ++d) tmr[d] = tmr[d] * tab.sign;

  int cx, cy, cz;
  cell_xyz(cc, g, cx, cy, cz);
  const int gx0 = cx * g.p, gy0 = cy * g.p, gz0 = cz * g.p;
  const int64_t nn1 = g.nn1, nn2 = nn1 * nn1;
  const int64_t base = (int64_t)t * g.n_nodes + gx0 + nn1 * (gy0 + nn1 * gz0);
  bool bx[N], by[N], bz[N];
#pragma unroll
  for (int a = 0; a < N; ++a) {
    bx[a] = on_boundary(gx0 + a, g.nn1);
    by[a] = on_boundary(gy0 + a, g.nn1);
    bz[a] = on_boundary(gz0 + a, g.nn1);
  }
  // this cell's staged geometry: point q, part h at gp[(q * 2 + h) * CW]
  const float4* gp = sg + cs;

  // gather [z][y][x] and interpolate to the Gauss points in place
  T u[N][N][N];
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int b = 0; b < N; ++b) {
      const TI* xr = x + base + nn1 * b + nn2 * k;
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const bool ld = active && !(mask_input && (bx[a] || by[b] || bz[k]));
        u[k][b][a] = ld ? T(xr[a]) : T(0.0f);
      }
    }
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int b = 0; b < N; ++b) {
      T w[N];
#pragma unroll
      for (int q = 0; q < N; ++q) {
        T v = 0;
#pragma unroll
        for (int a = 0; a < N; ++a) v += tab.B[q][a] * u[k][b][a];
        w[q] = v;
      }
#pragma unroll
      for (int q = 0; q < N; ++q) u[k][b][q] = w[q];
    }
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int a = 0; a < N; ++a) {
      T w[N];
#pragma unroll
      for (int q = 0; q < N; ++q) {
        T v = 0;
#pragma unroll
        for (int b = 0; b < N; ++b) v += tab.B[q][b] * u[k][b][a];
        w[q] = v;
      }
#pragma unroll
      for (int q = 0; q < N; ++q) u[k][q][a] = w[q];
    }
#pragma unroll
  for (int b = 0; b < N; ++b)
#pragma unroll
    for (int a = 0; a < N; ++a) {
      T w[N];
#pragma unroll
      for (int q = 0; q < N; ++q) {
        T v = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) v += tab.B[q][k] * u[k][b][a];
        w[q] = v;
      }
#pragma unroll
      for (int q = 0; q < N; ++q) u[q][b][a] = w[q];
    }

  // the staged geometry is complete and visible to the whole warp
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();

  // stiffness part at the Gauss points: acc = sum over points of D^T (G grad u)
  T acc[N][N][N];
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int a = 0; a < N; ++a) acc[k][b][a] = 0;
  if constexpr (!MASS) {
#pragma unroll
    for (int qz = 0; qz < N; ++qz)
#pragma unroll
      for (int qy = 0; qy < N; ++qy)
#pragma unroll
        for (int qx = 0; qx < N; ++qx) {
          T sx = 0, sy = 0, sz = 0;
#pragma unroll
          for (int a = 0; a < N; ++a) {
            sx += tab.D[qx][a] * u[qz][qy][a];
            sy += tab.D[qy][a] * u[qz][a][qx];
            sz += tab.D[qz][a] * u[a][qy][qx];
          }
          const T gx = sx, gy = sy, gz = sz;
          const int q = qx + N * (qy + N * qz);
          const float4 g0 = gp[(q * 2) * CW];
          const float2 g1 = *reinterpret_cast<const float2*>(gp + (q * 2 + 1) * CW);
          const T G00 = g0.x, G01 = g0.y, G02 = g0.z, G11 = g0.w, G12 = g1.x, G22 = g1.y;
          T fxa = G00 * gx, fya = G01 * gx, fza = G02 * gx;
          fxa += G01 * gy; fya += G11 * gy; fza += G12 * gy;
          fxa += G02 * gz; fya += G12 * gz; fza += G22 * gz;
          const T fx = fxa, fy = fya, fz = fza;
#pragma unroll
          for (int a = 0; a < N; ++a) {
            acc[qz][qy][a] += tab.D[qx][a] * fx;
            acc[qz][a][qx] += tab.D[qy][a] * fy;
            acc[a][qy][qx] += tab.D[qz][a] * fz;
          }
        }
  }

  // mass part with the time mixing; out = TA[t][t] acc + m sum_d TM[t][t+d] u_{t+d}
  int src[NT];
#pragma unroll
  for (int d = 0; d < NT; ++d) src[d] = cs + ((t + d) % NT) * CW;
  T o[N][N][N];
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const T m = reinterpret_cast<const float*>(gp + ((a + N * (b + N * k)) * 2 + 1) * CW)[2];
        T mix = tmr[0] * u[k][b][a];
#pragma unroll
        for (int d = 1; d < NT; ++d) mix += tmr[d] * shfl_from(u[k][b][a], src[d]);
        const T mv = mix;
        T r = m * mv;
        if constexpr (!MASS) r += ta * acc[k][b][a];
        o[k][b][a] = r;
      }

  // transposed interpolation in place, then the output rows
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int b = 0; b < N; ++b) {
      T w[N];
#pragma unroll
      for (int a = 0; a < N; ++a) {
        T v = 0;
#pragma unroll
        for (int q = 0; q < N; ++q) v += tab.B[q][a] * o[k][b][q];
        w[a] = v;
      }
#pragma unroll
      for (int a = 0; a < N; ++a) o[k][b][a] = w[a];
    }
#pragma unroll
  for (int k = 0; k < N; ++k)
#pragma unroll
    for (int a = 0; a < N; ++a) {
      T w[N];
#pragma unroll
      for (int b = 0; b < N; ++b) {
        T v = 0;
#pragma unroll
        for (int q = 0; q < N; ++q) v += tab.B[q][b] * o[k][q][a];
        w[b] = v;
      }
#pragma unroll
      for (int b = 0; b < N; ++b) o[k][b][a] = w[b];
    }
#pragma unroll
  for (int b = 0; b < N; ++b)
#pragma unroll
    for (int a = 0; a < N; ++a) {
      T w[N];
#pragma unroll
      for (int k = 0; k < N; ++k) {
        T v = 0;
#pragma unroll
        for (int q = 0; q < N; ++q) v += tab.B[q][k] * o[q][b][a];
        w[k] = v;
      }
#pragma unroll
      for (int k = 0; k < N; ++k) o[k][b][a] = w[k];
    }
  if (active) {
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
      for (int b = 0; b < N; ++b) {
        TO* yr = y + base + nn1 * b + nn2 * k;
#pragma unroll
        for (int a = 0; a < N; ++a)
          if (!(bx[a] || by[b] || bz[k])) {
            if constexpr (std::is_same<TO, double>::value) atomicAdd(yr + a, f2d_exact(o[k][b][a]));
            else atomicAdd(yr + a, o[k][b][a]);
          }
      }
  }
}

template <int N, int NT, typename TI, typename TO, bool MASS>
cudaError_t launch_apply_reg(const TI* x, TO* y, const float* geo, const GridDesc& g, const OpTab<float>& tab,
                             int mask_input, cudaStream_t s) {
  constexpr int cells_per_cta = kRegWarps * (32 / NT);
  const int64_t blocks = (g.n_cells + cells_per_cta - 1) / cells_per_cta;
  const size_t smem = (size_t)kRegWarps * 2 * N * N * N * (32 / NT) * sizeof(float4);
  auto k = apply3d_reg_kernel<N, NT, TI, TO, MASS>;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  { const cudaError_t e_ = launch_k(k, dim3((unsigned)blocks), dim3(32 * kRegWarps), smem, s, x, y, geo, g, tab, mask_input); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

}  // namespace apply_detail
}  // namespace stmg
