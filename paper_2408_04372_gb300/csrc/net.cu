// Learned initial guess: a chain of 3x3x3 convolutions on the node grid, BF16 activations and
// weights, FP32 accumulation on the tensor cores, trained by Adam on FP32 master weights.
//
// Layouts: activations [Vp][CP] (channels last, CP = channels padded to 16 or 64) on the node grid
// padded by one zero layer on each side, row r = (x+1) + nxp ((y+1) + nyp (z+1)); the halo rows are
// zero at allocation and never written, so the neighbour of a grid node at tap offset
// off = dx + nxp (dy + nyp dz) is always row r + off.  Weights Wt[tap][co][ci] (forward) and
// WtT[tap][ci][co] (backward data), tap = (dx+1) + 3 (dy+1) + 9 (dz+1).
//
// conv_tc_kernel: implicit GEMM on the fifth-generation tensor cores.  A CTA computes 128 rows x CO_P
// outputs: for each of the 27 taps a TMA load brings the 128 shifted input rows (one contiguous block
// of the activation matrix) and the tap's weight matrix into a ring of shared-memory stages, one
// thread issues tcgen05.mma (M = 128, N = CO_P, K = 16 per instruction, BF16 in, FP32 accumulator in
// tensor memory) and commits each stage back to the loader; four epilogue warps read the
// accumulator rows from tensor memory.
//   forward:        out[r][co] = sum_tap sum_ci in[r + off(tap)][ci] Wt[tap][co][ci] (+ bias, ReLU)
//   backward data:  din[r][ci] = sum_tap sum_co dout[r - off(tap)][co] WtT[tap][ci][co] (x ReLU mask)
// wgrad_tc_kernel: dW[tap][co][ci] = sum_r dout[r][co] in[r + off(tap)][ci] on the same tensor cores,
//   taps stacked along M so that every MMA shares the output-gradient tile, FP32 atomics at the end.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "net.h"
#include "tc05.cuh"

namespace stmg {

namespace {

// ---- tensor-core convolution ----
template <int CI_P, int CO_P>
struct ConvCfg {
  static constexpr int BM = 128;                        // output rows per CTA (TMEM lanes)
  static constexpr int A_BYTES = BM * CI_P * 2;
  static constexpr int B_BYTES = CO_P * CI_P * 2;
  static constexpr int STAGE = (A_BYTES + B_BYTES + 1023) / 1024 * 1024;
  static constexpr int S = CI_P == 64 ? 4 : 6;          // ring of stages
  static constexpr size_t SMEM = (size_t)S * STAGE + 1024;  // + slack to align the ring to 1024 bytes
  static constexpr tc::Swizzle SW = CI_P == 64 ? tc::kSw128 : tc::kSw32;
  static constexpr uint32_t SBO = CI_P == 64 ? 1024 : 256;  // 8 rows of CI_P * 2 bytes
  static constexpr uint32_t TMEM_COLS = CO_P < 32 ? 32 : CO_P;
  static constexpr int THREADS = 192;                   // warp 0 loads, warp 1 issues MMAs, warps 2-5 epilogue
};

struct PGrid { int nxp, nyp, nzp; int64_t Vp; };

__device__ __forceinline__ bool halo_row(int64_t r, const PGrid& g) {
  if (r >= g.Vp) return true;
  const int x = (int)(r % g.nxp);
  const int64_t q = r / g.nxp;
  const int y = (int)(q % g.nyp), z = (int)(q / g.nyp);
  return x == 0 || x == g.nxp - 1 || y == 0 || y == g.nyp - 1 || z == 0 || z == g.nzp - 1;
}

// mode: 0 forward hidden (bias + ReLU -> bf16), 1 forward last (bias -> f32), 2 backward data (x mask -> bf16)
template <int CI_P, int CO_P>
__global__ void __launch_bounds__(ConvCfg<CI_P, CO_P>::THREADS)
conv_tc_kernel(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_w,
               const float* __restrict__ bias, __nv_bfloat16* __restrict__ out16, float* __restrict__ out32,
               const __nv_bfloat16* __restrict__ mask, PGrid g, int sgn, int mode, int* status) {
  using C = ConvCfg<CI_P, CO_P>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[C::S], empty[C::S], acc_full;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail, s_issued, s_consumed;
  unsigned char* ring = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t)blockIdx.x * C::BM;
  if (threadIdx.x == 0) {
    s_fail = *reinterpret_cast<const volatile int*>(status);
    s_issued = 0;
    s_consumed = 0;
    for (int s = 0; s < C::S; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    tc::mbar_init(&acc_full, 1);
    tc::mbar_fence_init();
  }
  if (warp == 1) tc::tmem_alloc(&tmem_base, C::TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const bool skip = s_fail != 0;  // an earlier wait of this context gave up: issue nothing

  if (warp == 0 && lane == 0 && !skip) {
    // loader: tap t -> stage t % S; the stage is free once the MMAs of tap t - S completed
    tc::prefetch_tmap(&tm_in);
    tc::prefetch_tmap(&tm_w);
    for (int t = 0; t < 27; ++t) {
      const int s = t % C::S;
      if (t >= C::S && !tc::mbar_wait_bounded(&empty[s], (uint32_t)(((t / C::S) - 1) & 1), status)) {
        atomicExch(status, STMG_DEVICE_TIMEOUT);
        break;
      }
      const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
      const int64_t off = dx + (int64_t)g.nxp * (dy + (int64_t)g.nyp * dz);
      unsigned char* st = ring + (size_t)s * C::STAGE;
      tc::mbar_expect_tx(&full[s], (uint32_t)(C::A_BYTES + C::B_BYTES));
      tc::tma_load_2d(st, &tm_in, 0, (int)(r0 + sgn * off), &full[s]);
      tc::tma_load_2d(st + C::A_BYTES, &tm_w, 0, t * CO_P, &full[s]);
      s_issued = t + 1;
    }
  } else if (warp == 1 && lane == 0 && !skip) {
    // MMA issuer
    constexpr uint32_t idesc = tc::idesc_bf16_f32(C::BM, CO_P);
    bool ok = true;
    for (int t = 0; t < 27 && ok; ++t) {
      const int s = t % C::S;
      if (!tc::mbar_wait_bounded(&full[s], (uint32_t)((t / C::S) & 1), status)) {
        atomicExch(status, STMG_DEVICE_TIMEOUT);
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t a = tc::smem_addr(ring + (size_t)s * C::STAGE);
      const uint32_t b = a + C::A_BYTES;
#pragma unroll
      for (int k = 0; k < CI_P / 16; ++k) {
        const uint64_t ad = tc::smem_desc(a + 32 * k, 16, C::SBO, C::SW);
        const uint64_t bd = tc::smem_desc(b + 32 * k, 16, C::SBO, C::SW);
        tc::mma_bf16(tmem, ad, bd, idesc, (t > 0 || k > 0) ? 1u : 0u);
      }
      tc::mma_commit(&empty[s]);
      s_consumed = t + 1;
    }
    if (ok) tc::mma_commit(&acc_full);
  } else if (warp >= 2) {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) ..; one output row per thread
    const int q = warp & 3;
    const int row = 32 * q + lane;
    const int64_t r = r0 + row;
    bool ok = !skip && tc::mbar_wait_bounded(&acc_full, 0u, status);
    if (!skip && !ok && lane == 0) atomicExch(status, STMG_DEVICE_TIMEOUT);
    __syncwarp();  // the tensor-memory loads below are warp-collective
    tc::fence_after_sync();
    const bool store = ok && !halo_row(r, g);
#pragma unroll
    for (int c0 = 0; c0 < CO_P; c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);  // every lane of the warp takes part
      if (!store) continue;
      if (mode == 1) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(out32 + r * CO_P + c0 + j) =
              make_float4(v[j] + bias[c0 + j], v[j + 1] + bias[c0 + j + 1], v[j + 2] + bias[c0 + j + 2],
                          v[j + 3] + bias[c0 + j + 3]);
      } else {
        uint32_t pk[8];
        if (mode == 0) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float a0 = fmaxf(v[2 * j] + bias[c0 + 2 * j], 0.f), a1 = fmaxf(v[2 * j + 1] + bias[c0 + 2 * j + 1], 0.f);
            pk[j] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(a0)) |
                    ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(a1)) << 16);
          }
        } else {
          const uint4* mp = reinterpret_cast<const uint4*>(mask + r * CO_P + c0);
          const uint4 m0 = __ldg(mp), m1 = __ldg(mp + 1);
          const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const bool k0 = __uint_as_float(mw[j] << 16) > 0.f, k1 = __uint_as_float(mw[j] & 0xffff0000u) > 0.f;
            pk[j] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16(k0 ? v[2 * j] : 0.f)) |
                    ((uint32_t)__bfloat16_as_ushort(__float2bfloat16(k1 ? v[2 * j + 1] : 0.f)) << 16);
          }
        }
        uint4* op = reinterpret_cast<uint4*>(out16 + r * CO_P + c0);
        op[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        op[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (!skip && *reinterpret_cast<const volatile int*>(status) != 0) {
    // a wait gave up: before leaving, wait (bounded) for the loads still in flight and for the MMAs
    // already issued, so that nothing lands in shared or tensor memory after the CTA is gone
    if (threadIdx.x == 0)
      for (int t = s_consumed; t < s_issued; ++t)
        tc::mbar_wait_bounded(&full[t % C::S], (uint32_t)((t / C::S) & 1), nullptr);
    if (threadIdx.x == 32 && s_consumed > 0) {
      const int t = s_consumed - 1;
      tc::mbar_wait_bounded(&empty[t % C::S], (uint32_t)((t / C::S) & 1), nullptr);
    }
    __syncthreads();
  }
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

struct VGrid { int nx, ny, nz; int64_t V; };

// ---- tensor-core weight gradient ----
// dW[tap][co][ci] = sum_r in[r + off(tap)][ci] dout[r][co], as D[(tap, ci)][co] = A B with the K dimension
// running over activation rows r: A = the shifted input tiles of G = 128 / CI_P taps stacked along M
// (each tile one 128-byte or 32-byte swizzle column of the M dimension, M-major), B = the output-gradient
// tile (N = co contiguous, N-major) shared by every tap.  A CTA owns a range of 128-row blocks and a set
// of tap groups; its accumulators (one 128 x CO_P block per group) stay in tensor memory over the whole
// range and are added to dW with FP32 atomics at the end (one atomic per element and CTA).
template <int CI_P, int CO_P>
struct WgCfg {
  static constexpr int BK = 128;                          // rows per block (K of 8 MMAs)
  static constexpr int G = 128 / CI_P;                    // taps per group (M = G * CI_P = 128)
  static constexpr int NGROUPS = (27 + G - 1) / G;
  static constexpr int GPS_MAX = 512 / CO_P;              // groups whose accumulators fit in TMEM
  static constexpr int GPS = NGROUPS < GPS_MAX ? NGROUPS : (NGROUPS + 1) / 2;  // groups per CTA (tap set)
  static constexpr int TAPSETS = (NGROUPS + GPS - 1) / GPS;
  static constexpr int TILE_A = BK * CI_P * 2;            // one tap's rows
  static constexpr int A_BYTES = G * TILE_A;               // 32 KB
  static constexpr int B_BYTES = BK * CO_P * 2;
  static constexpr int STAGE = (A_BYTES + B_BYTES + 1023) / 1024 * 1024;
  static constexpr int S = 3;
  static constexpr size_t SMEM = (size_t)S * STAGE + 1024;
  static constexpr tc::Swizzle SWA = CI_P == 64 ? tc::kSw128 : tc::kSw32;
  static constexpr tc::Swizzle SWB = CO_P == 64 ? tc::kSw128 : tc::kSw32;
  static constexpr uint32_t ATOM_A = CI_P == 64 ? 1024 : 256;  // 8 rows of one tile
  static constexpr uint32_t ATOM_B = CO_P == 64 ? 1024 : 256;
  static constexpr uint32_t TMEM_COLS = GPS * CO_P <= 32 ? 32 : GPS * CO_P <= 64 ? 64 : GPS * CO_P <= 128 ? 128
                                        : GPS * CO_P <= 256 ? 256 : 512;
  static constexpr int THREADS = 192;
};

// Instruction descriptor of kind::f16 with both operands M/N-major (transpose bits set).
__host__ __device__ constexpr uint32_t idesc_bf16_f32_mn(int M, int N) {
  return tc::idesc_bf16_f32(M, N) | (1u << 15) | (1u << 16);
}

template <int CI_P, int CO_P>
__global__ void __launch_bounds__(WgCfg<CI_P, CO_P>::THREADS)
wgrad_tc_kernel(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_dout,
                float* __restrict__ dW, PGrid g, int64_t blocks_per_cta, int* status) {
  using C = WgCfg<CI_P, CO_P>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[C::S], empty[C::S], acc_full;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail, s_issued, s_consumed;
  unsigned char* ring = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nblocks = (g.Vp + C::BK - 1) / C::BK;
  const int64_t rb0 = (int64_t)blockIdx.x * blocks_per_cta;
  const int64_t rb1 = rb0 + blocks_per_cta < nblocks ? rb0 + blocks_per_cta : nblocks;
  const int g0 = blockIdx.y * C::GPS;
  const int ng = C::NGROUPS - g0 < C::GPS ? C::NGROUPS - g0 : C::GPS;
  const int steps = rb1 > rb0 ? (int)((rb1 - rb0) * ng) : 0;
  if (threadIdx.x == 0) {
    s_fail = *reinterpret_cast<const volatile int*>(status);
    s_issued = 0;
    s_consumed = 0;
    for (int s = 0; s < C::S; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    tc::mbar_init(&acc_full, 1);
    tc::mbar_fence_init();
  }
  if (warp == 1) tc::tmem_alloc(&tmem_base, C::TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const bool skip = s_fail != 0 || steps == 0;

  if (warp == 0 && lane == 0 && !skip) {
    tc::prefetch_tmap(&tm_in);
    tc::prefetch_tmap(&tm_dout);
    for (int i = 0; i < steps; ++i) {
      const int s = i % C::S;
      if (i >= C::S && !tc::mbar_wait_bounded(&empty[s], (uint32_t)(((i / C::S) - 1) & 1), status)) {
        atomicExch(status, STMG_DEVICE_TIMEOUT);
        break;
      }
      const int64_t r0 = (rb0 + i / ng) * C::BK;
      const int grp = g0 + i % ng;
      unsigned char* st = ring + (size_t)s * C::STAGE;
      tc::mbar_expect_tx(&full[s], (uint32_t)(C::A_BYTES + C::B_BYTES));
#pragma unroll 1
      for (int h = 0; h < C::G; ++h) {
        const int t = grp * C::G + h < 27 ? grp * C::G + h : 26;  // a short last group repeats a tap
        const int dx = t % 3 - 1, dy = (t / 3) % 3 - 1, dz = t / 9 - 1;
        const int64_t off = dx + (int64_t)g.nxp * (dy + (int64_t)g.nyp * dz);
        tc::tma_load_2d(st + h * C::TILE_A, &tm_in, 0, (int)(r0 + off), &full[s]);
      }
      tc::tma_load_2d(st + C::A_BYTES, &tm_dout, 0, (int)r0, &full[s]);
      s_issued = i + 1;
    }
  } else if (warp == 1 && lane == 0 && !skip) {
    constexpr uint32_t idesc = idesc_bf16_f32_mn(128, CO_P);
    bool ok = true;
    for (int i = 0; i < steps; ++i) {
      const int s = i % C::S;
      if (!tc::mbar_wait_bounded(&full[s], (uint32_t)((i / C::S) & 1), status)) {
        atomicExch(status, STMG_DEVICE_TIMEOUT);
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const int grp_local = i % ng;
      const bool first_block = i < ng;
      const uint32_t a = tc::smem_addr(ring + (size_t)s * C::STAGE);
      const uint32_t b = a + C::A_BYTES;
      const uint32_t d = tmem + (uint32_t)(grp_local * CO_P);
#pragma unroll
      for (int ks = 0; ks < C::BK / 16; ++ks) {
        // 16 rows = two 8-row swizzle atoms along K; M-atoms (taps) C::TILE_A apart
        const uint64_t ad = tc::smem_desc(a + ks * 2 * C::ATOM_A, C::TILE_A, C::ATOM_A, C::SWA);
        const uint64_t bd = tc::smem_desc(b + ks * 2 * C::ATOM_B, C::B_BYTES, C::ATOM_B, C::SWB);
        tc::mma_bf16(d, ad, bd, idesc, (first_block && ks == 0) ? 0u : 1u);
      }
      tc::mma_commit(&empty[s]);
      s_consumed = i + 1;
    }
    if (ok) tc::mma_commit(&acc_full);
  } else if (warp >= 2) {
    const int q = warp & 3;
    const int m = 32 * q + lane;             // accumulator row = (tap h, ci)
    const int h = m / CI_P, ci = m % CI_P;
    bool ok = !skip && tc::mbar_wait_bounded(&acc_full, 0u, status);
    if (!skip && !ok && lane == 0) atomicExch(status, STMG_DEVICE_TIMEOUT);
    __syncwarp();
    tc::fence_after_sync();
    for (int gl = 0; gl < ng; ++gl) {
      const int t = (g0 + gl) * C::G + h;
#pragma unroll
      for (int c0 = 0; c0 < CO_P; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(gl * CO_P + c0), v);
        if (!ok || t >= 27) continue;
#pragma unroll
        for (int j = 0; j < 16; ++j) atomicAdd(dW + ((int64_t)t * CO_P + c0 + j) * CI_P + ci, v[j]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (!skip && *reinterpret_cast<const volatile int*>(status) != 0) {
    if (threadIdx.x == 0)
      for (int i = s_consumed; i < s_issued; ++i)
        tc::mbar_wait_bounded(&full[i % C::S], (uint32_t)((i / C::S) & 1), nullptr);
    if (threadIdx.x == 32 && s_consumed > 0) {
      const int i = s_consumed - 1;
      tc::mbar_wait_bounded(&empty[i % C::S], (uint32_t)((i / C::S) & 1), nullptr);
    }
    __syncthreads();
  }
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, C::TMEM_COLS);
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

// padded row of node v of the nx x ny x nz grid
__device__ __forceinline__ int64_t prow(int64_t v, const VGrid& g, const PGrid& pg) {
  const int64_t x = v % g.nx, q = v / g.nx;
  const int64_t y = q % g.ny, z = q / g.ny;
  return (x + 1) + (int64_t)pg.nxp * ((y + 1) + (int64_t)pg.nyp * (z + 1));
}

// x0[row(v)][c]: c < nt: u_prev[c][v] * su ; nt <= c < 2 nt: f[c - nt][v] * sf ; else 0
__global__ void features_kernel(const double* __restrict__ u_prev, const double* __restrict__ f, int nt, VGrid g,
                                PGrid pg, float su, float sf, __nv_bfloat16* __restrict__ x0, int CP) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.V * CP; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / CP;
    const int c = (int)(i % CP);
    float x = 0.f;
    if (c < nt) x = (float)u_prev[(int64_t)c * g.V + v] * su;
    else if (c < 2 * nt) x = (float)f[(int64_t)(c - nt) * g.V + v] * sf;
    x0[prow(v, g, pg) * CP + c] = __float2bfloat16(x);
  }
}

__device__ inline bool grid_boundary(int64_t v, const VGrid& g) {
  const int x = (int)(v % g.nx);
  const int64_t r = v / g.nx;
  const int y = (int)(r % g.ny), z = (int)(r / g.ny);
  return x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1 || z == 0 || z == g.nz - 1;
}

// target t = (u[c] - u_prev_end) * so ; d_out = 2 (out - t) / count on interior nodes ; loss += sum (out-t)^2 / count
__global__ void loss_grad_kernel(const float* __restrict__ out, const double* __restrict__ u,
                                 const double* __restrict__ u_prev, int nt, VGrid g, PGrid pg, float so,
                                 double inv_count, __nv_bfloat16* __restrict__ dout, int CP, double* __restrict__ loss) {
  double local = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.V * CP; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / CP;
    const int c = (int)(i % CP);
    const int64_t row = prow(v, g, pg);
    float d = 0.f;
    if (c < nt && !grid_boundary(v, g)) {
      const double base = u_prev[(int64_t)(nt - 1) * g.V + v];
      const double t = (u[(int64_t)c * g.V + v] - base) * so;
      const double diff = (double)out[row * CP + c] - t;
      local += diff * diff;
      d = (float)(2.0 * diff * inv_count);
    }
    dout[row * CP + c] = __float2bfloat16(d);
  }
  for (int off = 16; off > 0; off >>= 1) local += __shfl_down_sync(0xffffffffu, local, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, local * inv_count);
}

// guess[c][v] = u_prev_end[v] + out[row(v)][c] / so on interior nodes, 0 on the boundary
__global__ void guess_kernel(const float* __restrict__ out, const double* __restrict__ u_prev, int nt, VGrid g,
                             PGrid pg, float inv_so, double* __restrict__ guess, int CP) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.V * nt; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i / g.V);
    const int64_t v = i - (int64_t)c * g.V;
    guess[i] = grid_boundary(v, g) ? 0.0
                                   : u_prev[(int64_t)(nt - 1) * g.V + v] + (double)out[prow(v, g, pg) * CP + c] * inv_so;
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
cudaError_t conv_t(const CUtensorMap& tin, const CUtensorMap& tw, const float* bias, __nv_bfloat16* o16, float* o32,
                   const __nv_bfloat16* mask, const PGrid& g, int sgn, int mode, int* status, cudaStream_t s) {
  using C = ConvCfg<CI_P, CO_P>;
  auto k = conv_tc_kernel<CI_P, CO_P>;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t blocks = (g.Vp + C::BM - 1) / C::BM;
  k<<<(unsigned)blocks, C::THREADS, C::SMEM, s>>>(tin, tw, bias, o16, o32, mask, g, sgn, mode, status);
  return cudaGetLastError();
}

cudaError_t conv_dispatch(int ci, int co, const CUtensorMap& tin, const CUtensorMap& tw, const float* bias,
                          __nv_bfloat16* o16, float* o32, const __nv_bfloat16* mask, const PGrid& g, int sgn, int mode,
                          int* status, cudaStream_t s) {
  if (ci == 16 && co == 64) return conv_t<16, 64>(tin, tw, bias, o16, o32, mask, g, sgn, mode, status, s);
  if (ci == 64 && co == 64) return conv_t<64, 64>(tin, tw, bias, o16, o32, mask, g, sgn, mode, status, s);
  if (ci == 64 && co == 16) return conv_t<64, 16>(tin, tw, bias, o16, o32, mask, g, sgn, mode, status, s);
  if (ci == 16 && co == 16) return conv_t<16, 16>(tin, tw, bias, o16, o32, mask, g, sgn, mode, status, s);
  return cudaErrorInvalidValue;
}

template <int CI_P, int CO_P>
cudaError_t wgrad_t(const CUtensorMap& tin, const CUtensorMap& tdout, float* dW, const PGrid& g, int* status,
                    cudaStream_t s) {
  using C = WgCfg<CI_P, CO_P>;
  auto k = wgrad_tc_kernel<CI_P, CO_P>;
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t nblocks = (g.Vp + C::BK - 1) / C::BK;
  const int64_t ctas_x = std::max<int64_t>(1, std::min<int64_t>(nblocks, 152 / C::TAPSETS));
  const int64_t per = (nblocks + ctas_x - 1) / ctas_x;
  const dim3 grid((unsigned)((nblocks + per - 1) / per), (unsigned)C::TAPSETS);
  k<<<grid, C::THREADS, C::SMEM, s>>>(tin, tdout, dW, g, per, status);
  return cudaGetLastError();
}

cudaError_t wgrad_dispatch(int ci, int co, const CUtensorMap& tin, const CUtensorMap& tdout, float* dW, const PGrid& g,
                           int* status, cudaStream_t s) {
  if (ci == 16 && co == 64) return wgrad_t<16, 64>(tin, tdout, dW, g, status, s);
  if (ci == 64 && co == 64) return wgrad_t<64, 64>(tin, tdout, dW, g, status, s);
  if (ci == 64 && co == 16) return wgrad_t<64, 16>(tin, tdout, dW, g, status, s);
  if (ci == 16 && co == 16) return wgrad_t<16, 16>(tin, tdout, dW, g, status, s);
  return cudaErrorInvalidValue;
}

}  // namespace

int net_pad(int c) { return c <= 16 ? 16 : 64; }

cudaError_t make_tmap_bf16_2d(CUtensorMap* map, const void* base, uint64_t rows, uint32_t cols, uint32_t box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw = cols * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : cols * 2 == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t net_make_tmaps(NetDev& n) {
  for (int l = 0; l < n.L; ++l) {
    const uint32_t ci = (uint32_t)n.cp[l], co = (uint32_t)n.cp[l + 1];
    cudaError_t e = make_tmap_bf16_2d(&n.tm_in_f[l], n.act[l], (uint64_t)n.Vp, ci, 128);
    if (e == cudaSuccess) e = make_tmap_bf16_2d(&n.tm_w_f[l], n.wt[l], (uint64_t)27 * co, ci, co);
    if (e == cudaSuccess) e = make_tmap_bf16_2d(&n.tm_in_b[l], n.grad[l + 1], (uint64_t)n.Vp, co, 128);
    if (e == cudaSuccess) e = make_tmap_bf16_2d(&n.tm_w_b[l], n.wtT[l], (uint64_t)27 * ci, co, ci);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t net_forward(const NetDev& n, const double* u_prev, const double* f, cudaStream_t s) {
  const VGrid g{n.nx, n.ny, n.nz, n.V};
  const PGrid pg{n.nxp, n.nyp, n.nzp, n.Vp};
  features_kernel<<<blocks_for(n.V * n.cp[0]), 256, 0, s>>>(u_prev, f, n.nt, g, pg, n.su, n.sf, n.act[0], n.cp[0]);
  for (int l = 0; l < n.L; ++l) {
    const bool last = l == n.L - 1;
    cudaError_t e = conv_dispatch(n.cp[l], n.cp[l + 1], n.tm_in_f[l], n.tm_w_f[l], n.bias[l],
                                  last ? nullptr : n.act[l + 1], last ? n.out : nullptr, nullptr, pg, 1, last ? 1 : 0,
                                  n.status, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

cudaError_t net_guess(const NetDev& n, const double* u_prev, double* guess, cudaStream_t s) {
  const VGrid g{n.nx, n.ny, n.nz, n.V};
  const PGrid pg{n.nxp, n.nyp, n.nzp, n.Vp};
  guess_kernel<<<blocks_for(n.V * n.nt), 256, 0, s>>>(n.out, u_prev, n.nt, g, pg, 1.0f / n.so, guess, n.cp[n.L]);
  return cudaGetLastError();
}

cudaError_t net_backward(NetDev& n, const double* u_prev, const double* u_target, double* loss, cudaStream_t s) {
  const VGrid g{n.nx, n.ny, n.nz, n.V};
  const PGrid pg{n.nxp, n.nyp, n.nzp, n.Vp};
  cudaMemsetAsync(loss, 0, sizeof(double), s);
  const int cpL = n.cp[n.L];
  int64_t interior = (int64_t)(n.nx - 2) * (n.ny - 2) * (n.nz - 2);
  const double inv_count = 1.0 / (double)(interior * n.nt);
  loss_grad_kernel<<<blocks_for(n.V * cpL), 256, 0, s>>>(n.out, u_target, u_prev, n.nt, g, pg, n.so, inv_count,
                                                           n.grad[n.L], cpL, loss);
  for (int l = n.L - 1; l >= 0; --l) {
    // gradients of layer l from grad[l+1] (= dL/dy_l) and act[l]; halo rows of both are zero
    cudaMemsetAsync(n.gw[l], 0, sizeof(float) * 27 * n.cp[l + 1] * n.cp[l], s);
    cudaMemsetAsync(n.gb[l], 0, sizeof(float) * n.cp[l + 1], s);
    cudaError_t e = wgrad_dispatch(n.cp[l], n.cp[l + 1], n.tm_in_f[l], n.tm_in_b[l], n.gw[l], pg, n.status, s);
    if (e != cudaSuccess) return e;
    bias_grad_kernel<<<blocks_for(n.Vp * n.cp[l + 1]), 256, n.cp[l + 1] * sizeof(float), s>>>(n.grad[l + 1], n.gb[l],
                                                                                                n.Vp, n.cp[l + 1]);
    if (l > 0) {  // dL/dy_{l-1} = conv^T(grad[l+1]) masked by relu'(y_{l-1}) (act[l] > 0)
      e = conv_dispatch(n.cp[l + 1], n.cp[l], n.tm_in_b[l], n.tm_w_b[l], nullptr, n.grad[l], nullptr, n.act[l], pg, -1,
                        2, n.status, s);
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
