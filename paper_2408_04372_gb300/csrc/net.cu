// Learned initial guess: a chain of 3x3x3 convolutions on the node grid, BF16 activations and
// weights, FP32 accumulation on the tensor cores, trained by Adam on FP32 master weights.
//
// Layouts: activations [V][CP] (channels last, CP = channels padded to a multiple of 16),
// voxel v = x + nx (y + ny z) = the library's node numbering; weights Wt[tap][co][ci] (forward)
// and WtT[tap][ci][co] (backward data), tap = (dx+1) + 3 (dy+1) + 9 (dz+1).
//
// conv_kernel: implicit GEMM.  A CTA computes 64 voxels x CO_P outputs; per tap it stages the
// tap's weight matrix and the 64 shifted input rows in shared memory and runs
// mma.m16n8k16 (BF16 in, FP32 accumulate) over the input channels.
//   forward:        out[v][co] = sum_tap sum_ci in[v + off(tap)][ci] Wt[tap][co][ci] (+ bias, ReLU)
//   backward data:  din[v][ci] = sum_tap sum_co dout[v - off(tap)][co] WtT[tap][ci][co] (x ReLU mask)
// wgrad_kernel: dW[tap][co][ci] = sum_v dout[v][co] in[v + off(tap)][ci], split over voxel chunks,
//   FP32 atomics into the gradient.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "net.h"

namespace stmg {

namespace {

__device__ inline void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ inline uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ inline int tap_dx(int t) { return t % 3 - 1; }
__device__ inline int tap_dy(int t) { return (t / 3) % 3 - 1; }
__device__ inline int tap_dz(int t) { return t / 9 - 1; }

struct VGrid { int nx, ny, nz; int64_t V; };

// neighbour voxel of v shifted by s*(dx,dy,dz); -1 outside the grid
__device__ inline int64_t neighbour(int64_t v, int s, int tap, const VGrid& g) {
  const int x = (int)(v % g.nx);
  const int64_t r = v / g.nx;
  const int y = (int)(r % g.ny), z = (int)(r / g.ny);
  const int xx = x + s * tap_dx(tap), yy = y + s * tap_dy(tap), zz = z + s * tap_dz(tap);
  if (xx < 0 || xx >= g.nx || yy < 0 || yy >= g.ny || zz < 0 || zz >= g.nz) return -1;
  return xx + (int64_t)g.nx * (yy + (int64_t)g.ny * zz);
}

constexpr int kTileV = 64;
constexpr int kThreads = 128;

// mode: 0 forward hidden (bias + ReLU -> bf16), 1 forward last (bias -> f32), 2 backward data (x mask -> bf16)
template <int CI_P, int CO_P>
__global__ void __launch_bounds__(kThreads)
conv_kernel(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ w, const float* __restrict__ bias,
            __nv_bfloat16* __restrict__ out16, float* __restrict__ out32, const __nv_bfloat16* __restrict__ mask,
            VGrid g, int sgn, int mode) {
  constexpr int AS = CI_P + 8;   // padded row strides (16-byte aligned, fewer bank conflicts)
  constexpr int WS = CI_P + 8;
  __shared__ __align__(16) __nv_bfloat16 As[kTileV * AS];
  __shared__ __align__(16) __nv_bfloat16 Ws[CO_P * WS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gq = lane >> 2, tq = lane & 3;
  const int64_t v0 = (int64_t)blockIdx.x * kTileV;
  float acc[CO_P / 8][4];
#pragma unroll
  for (int j = 0; j < CO_P / 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;

  for (int tap = 0; tap < 27; ++tap) {
    // weights of this tap: CO_P rows of CI_P
    const uint4* wsrc = reinterpret_cast<const uint4*>(w + (int64_t)tap * CO_P * CI_P);
    for (int i = tid; i < CO_P * CI_P / 8; i += kThreads) {
      const int row = i / (CI_P / 8), c8 = i % (CI_P / 8);
      *reinterpret_cast<uint4*>(&Ws[row * WS + c8 * 8]) = __ldg(wsrc + i);
    }
    // shifted input rows
    for (int i = tid; i < kTileV * CI_P / 8; i += kThreads) {
      const int row = i / (CI_P / 8), c8 = i % (CI_P / 8);
      const int64_t v = v0 + row;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (v < g.V) {
        const int64_t nb = neighbour(v, sgn, tap, g);
        if (nb >= 0) val = __ldg(reinterpret_cast<const uint4*>(in + nb * CI_P) + c8);
      }
      *reinterpret_cast<uint4*>(&As[row * AS + c8 * 8]) = val;
    }
    __syncthreads();
    const int r0 = warp * 16;
#pragma unroll
    for (int kk = 0; kk < CI_P; kk += 16) {
      const uint32_t a0 = *reinterpret_cast<const uint32_t*>(&As[(r0 + gq) * AS + kk + 2 * tq]);
      const uint32_t a1 = *reinterpret_cast<const uint32_t*>(&As[(r0 + gq + 8) * AS + kk + 2 * tq]);
      const uint32_t a2 = *reinterpret_cast<const uint32_t*>(&As[(r0 + gq) * AS + kk + 8 + 2 * tq]);
      const uint32_t a3 = *reinterpret_cast<const uint32_t*>(&As[(r0 + gq + 8) * AS + kk + 8 + 2 * tq]);
#pragma unroll
      for (int j = 0; j < CO_P / 8; ++j) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&Ws[(j * 8 + gq) * WS + kk + 2 * tq]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&Ws[(j * 8 + gq) * WS + kk + 8 + 2 * tq]);
        mma_bf16(acc[j], a0, a1, a2, a3, b0, b1);
      }
    }
    __syncthreads();
  }
  // epilogue
#pragma unroll
  for (int j = 0; j < CO_P / 8; ++j)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int row = warp * 16 + gq + (e >= 2 ? 8 : 0);
      const int col = j * 8 + 2 * tq + (e & 1);
      const int64_t v = v0 + row;
      if (v >= g.V) continue;
      float x = acc[j][e];
      if (mode == 0) {
        x += bias[col];
        out16[v * CO_P + col] = __float2bfloat16(fmaxf(x, 0.f));
      } else if (mode == 1) {
        out32[v * CO_P + col] = x + bias[col];
      } else {
        const float m = __bfloat162float(mask[v * CO_P + col]);
        out16[v * CO_P + col] = __float2bfloat16(m > 0.f ? x : 0.f);
      }
    }
}

// dW[tap][co][ci] += sum over a voxel chunk of dout[v][co] * in[v + off(tap)][ci]
template <int CI_P, int CO_P>
__global__ void __launch_bounds__(kThreads)
wgrad_kernel(const __nv_bfloat16* __restrict__ in, const __nv_bfloat16* __restrict__ dout, float* __restrict__ dW,
             VGrid g, int64_t chunk) {
  constexpr int SD = CO_P + 8, SA = CI_P + 8;
  constexpr int MT = CO_P / 16, NT8 = CI_P / 8, TILES = MT * NT8;
  constexpr int TPW = (TILES + 3) / 4;  // tiles per warp
  __shared__ __align__(16) __nv_bfloat16 Sd[kTileV * SD];
  __shared__ __align__(16) __nv_bfloat16 Sa[kTileV * SA];
  const int tap = blockIdx.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gq = lane >> 2, tq = lane & 3;
  float acc[TPW][4];
#pragma unroll
  for (int i = 0; i < TPW; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[i][e] = 0.f;
  const int64_t lo = (int64_t)blockIdx.x * chunk, hi = std::min<int64_t>(g.V, lo + chunk);
  for (int64_t v0 = lo; v0 < hi; v0 += kTileV) {
    for (int i = tid; i < kTileV * CO_P / 8; i += kThreads) {
      const int row = i / (CO_P / 8), c8 = i % (CO_P / 8);
      const int64_t v = v0 + row;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (v < hi) val = __ldg(reinterpret_cast<const uint4*>(dout + v * CO_P) + c8);
      *reinterpret_cast<uint4*>(&Sd[row * SD + c8 * 8]) = val;
    }
    for (int i = tid; i < kTileV * CI_P / 8; i += kThreads) {
      const int row = i / (CI_P / 8), c8 = i % (CI_P / 8);
      const int64_t v = v0 + row;
      uint4 val = make_uint4(0u, 0u, 0u, 0u);
      if (v < hi) {
        const int64_t nb = neighbour(v, 1, tap, g);
        if (nb >= 0) val = __ldg(reinterpret_cast<const uint4*>(in + nb * CI_P) + c8);
      }
      *reinterpret_cast<uint4*>(&Sa[row * SA + c8 * 8]) = val;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTileV; kk += 16) {
#pragma unroll
      for (int i = 0; i < TPW; ++i) {
        const int tile = warp + 4 * i;
        if (tile >= TILES) break;
        const int m0 = (tile / NT8) * 16, n0 = (tile % NT8) * 8;
        // A = dout^T (rows co, columns v), B = shifted input (rows v, columns ci)
        const int k0 = kk + 2 * tq;
        const uint32_t a0 = pack2(Sd[k0 * SD + m0 + gq], Sd[(k0 + 1) * SD + m0 + gq]);
        const uint32_t a1 = pack2(Sd[k0 * SD + m0 + gq + 8], Sd[(k0 + 1) * SD + m0 + gq + 8]);
        const uint32_t a2 = pack2(Sd[(k0 + 8) * SD + m0 + gq], Sd[(k0 + 9) * SD + m0 + gq]);
        const uint32_t a3 = pack2(Sd[(k0 + 8) * SD + m0 + gq + 8], Sd[(k0 + 9) * SD + m0 + gq + 8]);
        const uint32_t b0 = pack2(Sa[k0 * SA + n0 + gq], Sa[(k0 + 1) * SA + n0 + gq]);
        const uint32_t b1 = pack2(Sa[(k0 + 8) * SA + n0 + gq], Sa[(k0 + 9) * SA + n0 + gq]);
        mma_bf16(acc[i], a0, a1, a2, a3, b0, b1);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TPW; ++i) {
    const int tile = warp + 4 * i;
    if (tile >= TILES) break;
    const int m0 = (tile / NT8) * 16, n0 = (tile % NT8) * 8;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int co = m0 + gq + (e >= 2 ? 8 : 0);
      const int ci = n0 + 2 * tq + (e & 1);
      atomicAdd(dW + ((int64_t)tap * CO_P + co) * CI_P + ci, acc[i][e]);
    }
  }
}

__global__ void bias_grad_kernel(const __nv_bfloat16* __restrict__ dout, float* __restrict__ db, int64_t V, int CP) {
  extern __shared__ float sdb[];
  for (int c = threadIdx.x; c < CP; c += blockDim.x) sdb[c] = 0.f;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V * CP; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&sdb[i % CP], __bfloat162float(dout[i]));
  __syncthreads();
  for (int c = threadIdx.x; c < CP; c += blockDim.x) atomicAdd(&db[c], sdb[c]);
}

// x0[v][c]: c < nt: u_prev[c][v] * su ; nt <= c < 2 nt: f[c - nt][v] * sf ; else 0
__global__ void features_kernel(const double* __restrict__ u_prev, const double* __restrict__ f, int nt, int64_t V,
                                float su, float sf, __nv_bfloat16* __restrict__ x0, int CP) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < V * CP; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / CP;
    const int c = (int)(i % CP);
    float x = 0.f;
    if (c < nt) x = (float)u_prev[(int64_t)c * V + v] * su;
    else if (c < 2 * nt) x = (float)f[(int64_t)(c - nt) * V + v] * sf;
    x0[i] = __float2bfloat16(x);
  }
}

__device__ inline bool grid_boundary(int64_t v, const VGrid& g) {
  const int x = (int)(v % g.nx);
  const int64_t r = v / g.nx;
  const int y = (int)(r % g.ny), z = (int)(r / g.ny);
  return x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1 || z == 0 || z == g.nz - 1;
}

// target t = (u[c] - u_prev_end) * so ; d_out = 2 (out - t) / count on interior voxels ; loss += sum (out-t)^2 / count
__global__ void loss_grad_kernel(const float* __restrict__ out, const double* __restrict__ u,
                                 const double* __restrict__ u_prev, int nt, VGrid g, float so, double inv_count,
                                 __nv_bfloat16* __restrict__ dout, int CP, double* __restrict__ loss) {
  double local = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.V * CP; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / CP;
    const int c = (int)(i % CP);
    float d = 0.f;
    if (c < nt && !grid_boundary(v, g)) {
      const double base = u_prev[(int64_t)(nt - 1) * g.V + v];
      const double t = (u[(int64_t)c * g.V + v] - base) * so;
      const double diff = (double)out[v * CP + c] - t;
      local += diff * diff;
      d = (float)(2.0 * diff * inv_count);
    }
    dout[i] = __float2bfloat16(d);
  }
  for (int off = 16; off > 0; off >>= 1) local += __shfl_down_sync(0xffffffffu, local, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, local * inv_count);
}

// guess[c][v] = u_prev_end[v] + out[v][c] / so on interior voxels, 0 on the boundary
__global__ void guess_kernel(const float* __restrict__ out, const double* __restrict__ u_prev, int nt, VGrid g,
                             float inv_so, double* __restrict__ guess, int CP) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.V * nt; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / g.V);
    const int64_t v = i - (int64_t)c * g.V;
    guess[i] = grid_boundary(v, g) ? 0.0 : u_prev[(int64_t)(nt - 1) * g.V + v] + (double)out[v * CP + c] * inv_so;
  }
}

// Adam (Kingma & Ba) on FP32 masters, then BF16 copies in forward (Wt) and transposed (WtT) layouts
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m,
                            float* __restrict__ vv, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * vv[i] + (1.f - b2) * g * g;
    m[i] = mi;
    vv[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void weights_to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wt,
                                       __nv_bfloat16* __restrict__ wtT, int CO_P, int CI_P) {
  const int64_t n = (int64_t)27 * CO_P * CI_P;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int tap = (int)(i / ((int64_t)CO_P * CI_P));
    const int rem = (int)(i % ((int64_t)CO_P * CI_P));
    const int co = rem / CI_P, ci = rem % CI_P;
    const __nv_bfloat16 b = __float2bfloat16(w[i]);
    wt[i] = b;
    wtT[((int64_t)tap * CI_P + ci) * CO_P + co] = b;
  }
}

inline int blocks_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

template <int CI_P, int CO_P>
cudaError_t conv_t(const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias, __nv_bfloat16* o16, float* o32,
                   const __nv_bfloat16* mask, const VGrid& g, int sgn, int mode, cudaStream_t s) {
  const int64_t blocks = (g.V + kTileV - 1) / kTileV;
  conv_kernel<CI_P, CO_P><<<(unsigned)blocks, kThreads, 0, s>>>(in, w, bias, o16, o32, mask, g, sgn, mode);
  return cudaGetLastError();
}

cudaError_t conv_dispatch(int ci, int co, const __nv_bfloat16* in, const __nv_bfloat16* w, const float* bias,
                          __nv_bfloat16* o16, float* o32, const __nv_bfloat16* mask, const VGrid& g, int sgn, int mode,
                          cudaStream_t s) {
  if (ci == 16 && co == 64) return conv_t<16, 64>(in, w, bias, o16, o32, mask, g, sgn, mode, s);
  if (ci == 64 && co == 64) return conv_t<64, 64>(in, w, bias, o16, o32, mask, g, sgn, mode, s);
  if (ci == 64 && co == 16) return conv_t<64, 16>(in, w, bias, o16, o32, mask, g, sgn, mode, s);
  if (ci == 16 && co == 16) return conv_t<16, 16>(in, w, bias, o16, o32, mask, g, sgn, mode, s);
  return cudaErrorInvalidValue;
}

template <int CI_P, int CO_P>
cudaError_t wgrad_t(const __nv_bfloat16* in, const __nv_bfloat16* dout, float* dW, const VGrid& g, cudaStream_t s) {
  const int64_t chunk = 4096;
  dim3 grid((unsigned)((g.V + chunk - 1) / chunk), 27);
  wgrad_kernel<CI_P, CO_P><<<grid, kThreads, 0, s>>>(in, dout, dW, g, chunk);
  return cudaGetLastError();
}

cudaError_t wgrad_dispatch(int ci, int co, const __nv_bfloat16* in, const __nv_bfloat16* dout, float* dW,
                           const VGrid& g, cudaStream_t s) {
  if (ci == 16 && co == 64) return wgrad_t<16, 64>(in, dout, dW, g, s);
  if (ci == 64 && co == 64) return wgrad_t<64, 64>(in, dout, dW, g, s);
  if (ci == 64 && co == 16) return wgrad_t<64, 16>(in, dout, dW, g, s);
  if (ci == 16 && co == 16) return wgrad_t<16, 16>(in, dout, dW, g, s);
  return cudaErrorInvalidValue;
}

}  // namespace

int net_pad(int c) { return c <= 16 ? 16 : 64; }

cudaError_t net_forward(const NetDev& n, const double* u_prev, const double* f, cudaStream_t s) {
  const VGrid g{n.nx, n.ny, n.nz, n.V};
  features_kernel<<<blocks_for(n.V * n.cp[0]), 256, 0, s>>>(u_prev, f, n.nt, n.V, n.su, n.sf, n.act[0], n.cp[0]);
  for (int l = 0; l < n.L; ++l) {
    const bool last = l == n.L - 1;
    cudaError_t e = conv_dispatch(n.cp[l], n.cp[l + 1], n.act[l], n.wt[l], n.bias[l], last ? nullptr : n.act[l + 1],
                                  last ? n.out : nullptr, nullptr, g, 1, last ? 1 : 0, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t net_guess(const NetDev& n, const double* u_prev, double* guess, cudaStream_t s) {
  const VGrid g{n.nx, n.ny, n.nz, n.V};
  guess_kernel<<<blocks_for(n.V * n.nt), 256, 0, s>>>(n.out, u_prev, n.nt, g, 1.0f / n.so, guess, n.cp[n.L]);
  return cudaGetLastError();
}

cudaError_t net_backward(NetDev& n, const double* u_prev, const double* u_target, double* loss, cudaStream_t s) {
  const VGrid g{n.nx, n.ny, n.nz, n.V};
  cudaMemsetAsync(loss, 0, sizeof(double), s);
  const int cpL = n.cp[n.L];
  int64_t interior = (int64_t)(n.nx - 2) * (n.ny - 2) * (n.nz - 2);
  const double inv_count = 1.0 / (double)(interior * n.nt);
  loss_grad_kernel<<<blocks_for(n.V * cpL), 256, 0, s>>>(n.out, u_target, u_prev, n.nt, g, n.so, inv_count,
                                                           n.grad[n.L], cpL, loss);
  for (int l = n.L - 1; l >= 0; --l) {
    // gradients of layer l from grad[l+1] (= dL/dy_l) and act[l]
    cudaMemsetAsync(n.gw[l], 0, sizeof(float) * 27 * n.cp[l + 1] * n.cp[l], s);
    cudaMemsetAsync(n.gb[l], 0, sizeof(float) * n.cp[l + 1], s);
    cudaError_t e = wgrad_dispatch(n.cp[l], n.cp[l + 1], n.act[l], n.grad[l + 1], n.gw[l], g, s);
    if (e != cudaSuccess) return e;
    bias_grad_kernel<<<blocks_for(n.V * n.cp[l + 1]), 256, n.cp[l + 1] * sizeof(float), s>>>(n.grad[l + 1], n.gb[l],
                                                                                               n.V, n.cp[l + 1]);
    if (l > 0) {  // dL/dy_{l-1} = conv^T(grad[l+1]) masked by relu'(y_{l-1}) (act[l] > 0)
      e = conv_dispatch(n.cp[l + 1], n.cp[l], n.grad[l + 1], n.wtT[l], nullptr, n.grad[l], nullptr, n.act[l], g, -1, 2, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaGetLastError();
}

cudaError_t net_adam(NetDev& n, float lr, cudaStream_t s) {
  n.step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)n.step), c2 = 1.f - powf(b2, (float)n.step);
  for (int l = 0; l < n.L; ++l) {
    const int64_t nw = (int64_t)27 * n.cp[l + 1] * n.cp[l];
    adam_kernel<<<blocks_for(nw), 256, 0, s>>>(n.w32[l], n.gw[l], n.mw[l], n.vw[l], nw, lr, b1, b2, eps, c1, c2);
    adam_kernel<<<1, 256, 0, s>>>(n.bias[l], n.gb[l], n.mb[l], n.vb[l], n.cp[l + 1], lr, b1, b2, eps, c1, c2);
  }
  return net_refresh_bf16(n, s);
}

cudaError_t net_refresh_bf16(NetDev& n, cudaStream_t s) {
  for (int l = 0; l < n.L; ++l) {
    const int64_t nw = (int64_t)27 * n.cp[l + 1] * n.cp[l];
    weights_to_bf16_kernel<<<blocks_for(nw), 256, 0, s>>>(n.w32[l], n.wt[l], n.wtT[l], n.cp[l + 1], n.cp[l]);
  }
  return cudaGetLastError();
}

}  // namespace stmg
