// Vector kernels of the FP64 outer FGMRES and small helpers: conversions, the fused
// classical Gram-Schmidt passes (deterministic single-launch reductions), multi-AXPY,
// time-only mixing of nodal blocks, the dense coarsest-level solve.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "df64.cuh"
#include "kernels.h"

namespace stmg {

namespace {

constexpr int kMaxVec = 72;
constexpr int kCgsThreads = 256;

// Nearest double-float to an FP64 value (hi = x rounded to float, lo = the rounded remainder), formed
// without the FP64 pipe where the exponent allows (df64.cuh).
__device__ __forceinline__ df64 df_from_double(double x) { return df_split_fast(x); }
// Renormalised pair (Fast2Sum): hi becomes the float nearest to hi + lo.
__device__ __forceinline__ df64 df_renorm(df64 a) {
  const float h = __fadd_rn(a.hi, a.lo);
  return df64(h, __fsub_rn(a.lo, __fsub_rn(h, a.hi)));
}
constexpr int kCgsBlocks = 152 * 4;

inline int grid_blocks(int64_t total) {
  int64_t b = (total + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin* __restrict__ x, Tout* __restrict__ y, int64_t n) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (Tout)x[i];
}

__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, double* __restrict__ y, int64_t n) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + b * y[i];
}

// x (FP64) * scale written over x as double-float pairs, and its FP32 copy (the first Krylov vector
// of a double-float basis and the first V-cycle input, from the restart residual)
__global__ void scale_to_df_kernel(double* __restrict__ x, double scale, int64_t n, float* __restrict__ y32) {
  pdl_wait();
  pdl_trigger();
  float2* xd = reinterpret_cast<float2*>(x);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const df64 v = df_from_double(x[i] * scale);
    xd[i] = make_float2(v.hi, v.lo);
    if (y32) y32[i] = v.hi;
  }
}

// One pass of classical Gram-Schmidt against V_0..V_{nv-1} (V_j = V0 + j * stride):
//   sub : w -= sum_j c[j] V_j             (c on the device)
//   dot : s_j = V_j . w, j < nv            (after the subtraction)
//   norm: s_nv = w . w                     (after the subtraction)
// Every block reduces a fixed contiguous slice; the last block to arrive sums the per-block
// partials in a fixed order (final_sums), so the results do not depend on scheduling.  It then writes
//   fin 0: out[j] = s_j (j < nv) and out[nv] = s_nv when norm is set;
//   fin 1: the Arnoldi column out[j] = h_prev[j] + c[j], out[nv] = sqrt(s_nv), out[nv+1] = 1/out[nv].
// nrm2 (fin 1 only, norm unset): the pass also normalises.  nrm2[0] is |w|^2 before this pass's
// subtraction (from the previous pass); with an orthonormal basis the subtracted vector has
// |w - V c|^2 = nrm2[0] - |c|^2, so every block knows the norm hn before it starts, scales its
// elements by 1 / hn and, with copy32, writes their FP32 copy; out[nv] = hn.  One pass over w and
// one launch fewer than a separate normalisation.
// One thread keeps the K values V_j[i] of its element in registers between the subtraction and
// the dot products, so every basis vector is read once per pass.
// Final fixed-order sums over the nb per-block partials of every needed slot j (j < nv with dot, slot K
// with norm), by all THREADS threads of the last block: thread t adds blocks t, t + THREADS, ... for
// eight slots at a time (all those loads issued together), then a fixed warp-shuffle tree and a fixed
// sum over the warps.  The order does not depend on scheduling, so the result is bit-reproducible.
template <int K, int THREADS>
__device__ __forceinline__ void final_sums(const double* __restrict__ partial, int nb, int nv, int dot, int norm,
                                           double (*red)[K + 1], double* tot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int JC = 8;
#pragma unroll 1
  for (int j0 = 0; j0 <= K; j0 += JC) {
    double x[JC];
#pragma unroll
    for (int i = 0; i < JC; ++i) x[i] = 0.0;
    for (int b = tid; b < nb; b += THREADS) {
#pragma unroll
      for (int i = 0; i < JC; ++i) {
        const int j = j0 + i;
        if (j <= K && ((j < K && dot && j < nv) || (j == K && norm))) x[i] += __ldcg(partial + (int64_t)j * nb + b);
      }
    }
#pragma unroll
    for (int i = 0; i < JC; ++i) {
      const int j = j0 + i;
      if (j <= K && ((j < K && dot && j < nv) || (j == K && norm))) {
        double v = x[i];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][j] = v;
      }
    }
  }
  __syncthreads();
  for (int j = tid; j <= K; j += THREADS) {
    if ((j < K && dot && j < nv) || (j == K && norm)) {
      double v = 0.0;
      for (int w = 0; w < THREADS / 32; ++w) v += red[w][j];
      tot[j] = v;
    }
  }
}

// sqrt(|w|^2 - |c|^2) (0 when the difference is not positive: w lies in the span of the basis)
__device__ __forceinline__ double fused_norm(double w2, const double* cs, int nv) {
  double c2 = 0.0;
  for (int j = 0; j < nv; ++j) c2 += cs[j] * cs[j];
  const double d = w2 - c2;
  return d > 0.0 ? sqrt(d) : 0.0;
}

// The norm h = sqrt(nrm2[0] - |c|^2) of the subtracted vector and 1 / h, formed once per block by thread 0
// (FP64 square root and division are slow on this GPU's FP64 pipe, and every thread needs the same values).
__device__ __forceinline__ void block_fused_norm(const double* nrm2, const double* cs, int nv, double* s_hn,
                                                 double* s_inv) {
  if (threadIdx.x == 0) {
    const double h = nrm2 ? fused_norm(nrm2[0], cs, nv) : 0.0;
    *s_hn = h;
    *s_inv = h > 0.0 ? 1.0 / h : 0.0;
  }
  __syncthreads();
}

// Sum of a double-float value over the warp in double-float arithmetic (FP32 pipe), valid in lane 0.
__device__ __forceinline__ df64 warp_sum_df(df_acc a) {
  df64 v = a;
  df_acc s(v);
  for (int off = 16; off > 0; off >>= 1) {
    const df64 cur = s;
    const df64 o(__shfl_down_sync(0xffffffffu, cur.hi, off), __shfl_down_sync(0xffffffffu, cur.lo, off));
    s += o;
  }
  return s;
}

// The final sums in double-float: per-block partials as (hi, lo) pairs, sums in double-float, one
// conversion to FP64 per slot at the end (the FP64 pipe of this GPU is slow, conversions included).
template <int K, int THREADS>
__device__ __forceinline__ void final_sums_df(const float2* __restrict__ partial, int nb, int nv, int dot, int norm,
                                              float2 (*red)[K + 1], double* tot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int JC = 8;
#pragma unroll 1
  for (int j0 = 0; j0 <= K; j0 += JC) {
    df_acc x[JC];
#pragma unroll
    for (int i = 0; i < JC; ++i) x[i] = df_acc(0.0f);
    for (int b = tid; b < nb; b += THREADS) {
#pragma unroll
      for (int i = 0; i < JC; ++i) {
        const int j = j0 + i;
        if (j <= K && ((j < K && dot && j < nv) || (j == K && norm))) {
          const float2 v = __ldcg(partial + (int64_t)j * nb + b);
          x[i] += df64(v.x, v.y);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < JC; ++i) {
      const int j = j0 + i;
      if (j <= K && ((j < K && dot && j < nv) || (j == K && norm))) {
        const df64 v = warp_sum_df(x[i]);
        if (lane == 0) red[warp][j] = make_float2(v.hi, v.lo);
      }
    }
  }
  __syncthreads();
  for (int j = tid; j <= K; j += THREADS) {
    if ((j < K && dot && j < nv) || (j == K && norm)) {
      df_acc v(0.0f);
      for (int w = 0; w < THREADS / 32; ++w) v += df64(red[w][j].x, red[w][j].y);
      const df64 t = v;
      tot[j] = f2d_exact(t.hi) + f2d_exact(t.lo);
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kCgsThreads)
cgs_pass_kernel(const double* __restrict__ V0, int64_t stride, int nv, double* __restrict__ w, int64_t n,
                const double* __restrict__ c, int sub, int dot, int norm, const double* __restrict__ h_prev, int fin,
                double* __restrict__ partial, unsigned int* __restrict__ counter, double* __restrict__ out,
                const double* __restrict__ nrm2, float* __restrict__ copy32) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[kCgsThreads / 32][K + 1];
  __shared__ double cs[K];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ double s_hn, s_inv;
  for (int j = threadIdx.x; j < K; j += blockDim.x) cs[j] = (sub && j < nv) ? c[j] : 0.0;
  __syncthreads();
  block_fused_norm(nrm2, cs, nv, &s_hn, &s_inv);
  const double hn_fused = s_hn, inv = s_inv;
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
      if (nrm2) {
        wi *= inv;
        if (copy32) copy32[i] = (float)wi;
      }
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
  __shared__ double tot[K + 1];
  final_sums<K, kCgsThreads>(partial, nb, nv, dot, norm, red, tot);
  __syncthreads();
  if (fin == 0) {
    for (int j = threadIdx.x; j < nv; j += blockDim.x)
      if (dot) out[j] = tot[j];
    if (norm && threadIdx.x == 0) out[nv] = tot[K];
  } else {
    for (int j = threadIdx.x; j < nv; j += blockDim.x) out[j] = h_prev[j] + cs[j];
    if (threadIdx.x == 0) {
      const double hn = nrm2 ? hn_fused : sqrt(fmax(tot[K], 0.0));
      out[nv] = hn;
      out[nv + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// ---- double-float pass with direct loads (basis widths up to 16) ----
// The basis and w hold double-float pairs (w in FP64 when w64: converted and written back when w64 = 1,
// read only when w64 = 2, e.g. for a norm); each thread
// takes two consecutive elements of every vector with one 16-byte load, all nv + 1 loads of a pair issued
// before they are used, so that every SM keeps well over 100 KB in flight; the last element of an odd
// n is taken by one thread.  Results, reduction order and side outputs as in the FP64 passes.
constexpr int kCgsDfThreads = 256;
template <int K> struct CgsDf;
template <> struct CgsDf<4> { static constexpr int BPS = 4; };
template <> struct CgsDf<8> { static constexpr int BPS = 3; };
template <> struct CgsDf<16> { static constexpr int BPS = 2; };

template <int K>
__global__ void __launch_bounds__(kCgsDfThreads, CgsDf<K>::BPS)
cgs_pass_df_kernel(const double* __restrict__ V0, int64_t stride, int nv, double* __restrict__ w, int64_t n,
                   const double* __restrict__ c, int sub, int dot, int norm, const double* __restrict__ h_prev,
                   int fin, double* __restrict__ partial, unsigned int* __restrict__ counter,
                   double* __restrict__ out, const double* __restrict__ nrm2, float* __restrict__ copy32, int w64) {
  pdl_wait();
  pdl_trigger();
  __shared__ float2 redd[kCgsDfThreads / 32][K + 1];
  __shared__ double cs[K];
  __shared__ df64 csd[K];
  __shared__ bool last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ double s_hn, s_inv;
  __shared__ df64 s_invd;
  for (int j = tid; j < K; j += blockDim.x) {
    cs[j] = (sub && j < nv) ? c[j] : 0.0;
    csd[j] = df_from_double(cs[j]);
  }
  __syncthreads();
  block_fused_norm(nrm2, cs, nv, &s_hn, &s_inv);
  if (tid == 0) s_invd = df_from_double(s_inv);
  __syncthreads();
  const double hn_fused = s_hn;
  const df64 invd = s_invd;
  df_acc acc[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) acc[j] = df_acc(0.0f);
  // one or two elements: e = 2p (+1); the pair's entries arrive together
  auto step = [&](int64_t e, bool pair) {
    df64 wv[2];
    df64 vr[K][2];
    if (pair) {
      if (w64) {
        const double2 d = *reinterpret_cast<const double2*>(w + e);
        wv[0] = df_from_double(d.x);
        wv[1] = df_from_double(d.y);
      } else {
        const float4 f = *reinterpret_cast<const float4*>(w + e);
        wv[0] = df64(f.x, f.y);
        wv[1] = df64(f.z, f.w);
      }
#pragma unroll
      for (int j = 0; j < K; ++j) {
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < nv) f = __ldg(reinterpret_cast<const float4*>(V0 + j * stride + e));
        vr[j][0] = df64(f.x, f.y);
        vr[j][1] = df64(f.z, f.w);
      }
    } else {
      if (w64) {
        wv[0] = df_from_double(w[e]);
      } else {
        const float2 f = *reinterpret_cast<const float2*>(w + e);
        wv[0] = df64(f.x, f.y);
      }
      wv[1] = df64(0.0f);
#pragma unroll
      for (int j = 0; j < K; ++j) {
        float2 f = make_float2(0.f, 0.f);
        if (j < nv) f = *reinterpret_cast<const float2*>(V0 + j * stride + e);
        vr[j][0] = df64(f.x, f.y);
        vr[j][1] = df64(0.0f);
      }
    }
    if (sub) {
      df_acc sv[2] = {df_acc(0.0f), df_acc(0.0f)};
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j < nv) {
          sv[0] += csd[j] * vr[j][0];
          sv[1] += csd[j] * vr[j][1];
        }
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const df64 sm = sv[i];
        wv[i] = df_add(wv[i], df64(-sm.hi, -sm.lo));
        if (nrm2) wv[i] = df_renorm(wv[i] * invd);
      }
      if (!pair) wv[1] = df64(0.0f);
    }
    if (sub || w64 == 1) {
      if (pair) *reinterpret_cast<float4*>(w + e) = make_float4(wv[0].hi, wv[0].lo, wv[1].hi, wv[1].lo);
      else *reinterpret_cast<float2*>(w + e) = make_float2(wv[0].hi, wv[0].lo);
    }
    if (sub && nrm2 && copy32) {
      if (pair) *reinterpret_cast<float2*>(copy32 + e) = make_float2(wv[0].hi, wv[1].hi);
      else copy32[e] = wv[0].hi;
    }
    if (dot) {
#pragma unroll
      for (int j = 0; j < K; ++j)
        if (j < nv) {
          acc[j] += vr[j][0] * wv[0];
          acc[j] += vr[j][1] * wv[1];
        }
    }
    if (norm) {
      acc[K] += wv[0] * wv[0];
      acc[K] += wv[1] * wv[1];
    }
  };
  const int64_t npairs = n / 2;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + tid; p < npairs; p += (int64_t)gridDim.x * blockDim.x)
    step(2 * p, true);
  if ((n & 1) && blockIdx.x == 0 && tid == 0) step(n - 1, false);
  // block partials as double-float pairs (warp and block sums in double-float), then the last block sums
  // them in a fixed order (final_sums_df) and converts once per slot
  float2* partd = reinterpret_cast<float2*>(partial);
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    if ((j < K && dot && j < nv) || (j == K && norm)) {
      const df64 x = warp_sum_df(acc[j]);
      if (lane == 0) redd[warp][j] = make_float2(x.hi, x.lo);
    }
  }
  __syncthreads();
  const int nb = gridDim.x;
  for (int j = tid; j <= K; j += blockDim.x) {
    if ((j < K && dot && j < nv) || (j == K && norm)) {
      df_acc x(0.0f);
      for (int wv = 0; wv < kCgsDfThreads / 32; ++wv) x += df64(redd[wv][j].x, redd[wv][j].y);
      const df64 t = x;
      partd[(int64_t)j * nb + blockIdx.x] = make_float2(t.hi, t.lo);
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(counter, 1u) == (unsigned)nb - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double tot[K + 1];
  final_sums_df<K, kCgsDfThreads>(partd, nb, nv, dot, norm, redd, tot);
  __syncthreads();
  if (fin == 0) {
    for (int j = tid; j < nv; j += blockDim.x)
      if (dot) out[j] = tot[j];
    if (norm && tid == 0) out[nv] = tot[K];
  } else {
    for (int j = tid; j < nv; j += blockDim.x) out[j] = h_prev[j] + cs[j];
    if (tid == 0) {
      const double hn = nrm2 ? hn_fused : sqrt(fmax(tot[K], 0.0));
      out[nv] = hn;
      out[nv + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    }
  }
  if (tid == 0) *counter = 0u;
}

// ---- the same pass fed by bulk copies (TMA) ----
// Each CTA walks chunks of E elements (chunk c, c + gridDim.x, ...); per chunk one bulk copy per
// basis vector and one for w land in a shared-memory stage (S stages in flight, mbarrier
// completion).  Only whole 16-byte units are copied; an odd last element is read directly, so no
// copy runs past the end of a vector.  Waits are bounded: after kCgsWaitNs, or at once when
// *status is already set, the CTA records STMG_DEVICE_TIMEOUT, drains its copies and leaves the
// pass (the results are then invalid and the caller reports the status).
constexpr uint64_t kCgsWaitNs = 1000000000ull;
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, const int* status) {
  const uint64_t t0 = now_ns();
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(smem_addr(bar)), "r"(parity) : "memory");
    if (done) return true;
    if ((it & 63) == 63) {
      if (now_ns() - t0 > kCgsWaitNs) return false;
      if (status && *reinterpret_cast<const volatile int*>(status) != 0) return false;
    }
  }
}

// Chunk elements E, stages S and CTAs per SM of the bulk-copy pass.  FP64 passes are bound by the FP64
// pipe: few large chunks.  Double-float passes run on the FP32 pipe, where the per-element chains need
// more warps: smaller chunks, more CTAs per SM.
template <int K, bool DFV> struct CgsTma;
template <> struct CgsTma<4, false> { static constexpr int E = 1024, S = 2, BPS = 2; };
template <> struct CgsTma<8, false> { static constexpr int E = 768, S = 2, BPS = 2; };
template <> struct CgsTma<16, false> { static constexpr int E = 512, S = 2, BPS = 1; };
template <> struct CgsTma<32, false> { static constexpr int E = 128, S = 3, BPS = 1; };
template <> struct CgsTma<64, false> { static constexpr int E = 64, S = 3, BPS = 1; };
template <> struct CgsTma<4, true> { static constexpr int E = 512, S = 2, BPS = 4; };
template <> struct CgsTma<8, true> { static constexpr int E = 512, S = 2, BPS = 3; };
template <> struct CgsTma<16, true> { static constexpr int E = 256, S = 2, BPS = 2; };
template <> struct CgsTma<32, true> { static constexpr int E = 128, S = 3, BPS = 1; };
template <> struct CgsTma<64, true> { static constexpr int E = 64, S = 3, BPS = 1; };
template <int K, bool DFV> constexpr size_t cgs_tma_smem() {
  return (size_t)CgsTma<K, DFV>::S * (K + 1) * CgsTma<K, DFV>::E * sizeof(double);
}

// DFV: the basis and w hold double-float pairs (hi, lo) in their 8 bytes per entry and the pass
// computes in double-float arithmetic on the FP32 pipe (GB300 issues FP64 at 1/64 of the FP32 rate,
// and the FP64 pass is bound by the FP64 pipe); w64: w arrives in FP64 (the operator's output) and
// is written back as a pair.  Dot products and norms are summed per thread in double-float and
// reduced across threads and blocks in FP64 as in the FP64 pass.
template <int K, bool DFV>
__global__ void __launch_bounds__(kCgsThreads, CgsTma<K, DFV>::BPS)
cgs_pass_tma_kernel(const double* __restrict__ V0, int64_t stride, int nv, double* __restrict__ w, int64_t n,
                    const double* __restrict__ c, int sub, int dot, int norm, const double* __restrict__ h_prev,
                    int fin, double* __restrict__ partial, unsigned int* __restrict__ counter,
                    double* __restrict__ out, int* status, const double* __restrict__ nrm2,
                    float* __restrict__ copy32, int w64) {
  pdl_wait();
  pdl_trigger();
  constexpr int E = CgsTma<K, DFV>::E, S = CgsTma<K, DFV>::S;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[S];
  __shared__ double red[kCgsThreads / 32][K + 1];
  __shared__ double cs[K];
  __shared__ bool last;
  __shared__ int fail;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t stage_bytes = (size_t)(K + 1) * E * sizeof(double);
  const int64_t nch = (n + E - 1) / E;
  for (int j = tid; j < K; j += blockDim.x) cs[j] = (sub && j < nv) ? c[j] : 0.0;
  if (tid == 0) {
    fail = *reinterpret_cast<const volatile int*>(status) != 0;
    for (int st = 0; st < S; ++st)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar[st])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  __shared__ double s_hn, s_inv;
  block_fused_norm(nrm2, cs, nv, &s_hn, &s_inv);
  const double hn_fused = s_hn, inv = s_inv;
  auto main_bytes = [&](int64_t ch) -> uint32_t {
    const int64_t ne = n - ch * E < E ? n - ch * E : E;
    return (uint32_t)((ne * (int64_t)sizeof(double)) / 16 * 16);
  };
  auto issue = [&](int64_t ch, int st) {  // thread 0
    const uint32_t bytes = main_bytes(ch);
    unsigned char* dst = smem_raw + (size_t)st * stage_bytes;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(&bar[st])), "r"(bytes * (uint32_t)(nv + 1)) : "memory");
    if (bytes == 0) return;
    for (int j = 0; j <= nv; ++j) {
      const double* src = (j < nv ? V0 + j * stride : w) + ch * E;
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                   ::"r"(smem_addr(dst + (size_t)j * E * sizeof(double))), "l"(src), "r"(bytes),
                   "r"(smem_addr(&bar[st])) : "memory");
    }
  };
  double acc[K + 1];
#pragma unroll
  for (int j = 0; j <= K; ++j) acc[j] = 0.0;
  df_acc accd[DFV ? K + 1 : 1];
#pragma unroll
  for (int j = 0; j < (DFV ? K + 1 : 1); ++j) accd[j] = df_acc(0.0f);
  __shared__ df64 csd[DFV ? K : 1];
  df64 invd(0.0f);
  __shared__ df64 s_invd;
  if constexpr (DFV) {
    for (int j = tid; j < K; j += blockDim.x) csd[j] = df_from_double(cs[j]);
    if (tid == 0) s_invd = df_from_double(inv);
    __syncthreads();
    invd = s_invd;
  }
  int64_t issued = 0, k = 0;
  if (!fail) {
    if (tid == 0)
      for (int st = 0; st < S; ++st) {
        const int64_t ch = blockIdx.x + (int64_t)st * gridDim.x;
        if (ch < nch) issue(ch, st);
      }
    for (int st = 0; st < S; ++st)
      if (blockIdx.x + (int64_t)st * gridDim.x < nch) ++issued;
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x, ++k) {
      const int st = (int)(k % S);
      if (!bar_wait(&bar[st], (uint32_t)((k / S) & 1), status)) {
        atomicExch(status, STMG_DEVICE_TIMEOUT);
        fail = 1;
      }
      __syncthreads();
      if (fail) break;
      const double* buf = reinterpret_cast<const double*>(smem_raw + (size_t)st * stage_bytes);
      const int64_t e0 = ch * E;
      const int ne = (int)(n - e0 < E ? n - e0 : E);
      const int nin = (int)(main_bytes(ch) / sizeof(double));  // elements that came by bulk copy
      if constexpr (DFV) {
        // the thread's EPT elements of the chunk together (independent double-float chains), each
        // basis entry read from the stage once for both the subtraction and the dot products
        constexpr int EPT = (E + kCgsThreads - 1) / kCgsThreads;
        const float2* bufd = reinterpret_cast<const float2*>(buf);
        const float2* V0d = reinterpret_cast<const float2*>(V0);
        float2* wd = reinterpret_cast<float2*>(w);
        bool ok[EPT], in[EPT];
        df64 wv[EPT];
        df64 vr[K][EPT];
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
          const int e = tid + i * kCgsThreads;
          ok[i] = e < ne;
          in[i] = e < nin;
          if (!ok[i]) {
            wv[i] = df64(0.0f);
          } else if (w64) {
            wv[i] = df_from_double(in[i] ? buf[nv * E + e] : w[e0 + e]);
          } else {
            const float2 v = in[i] ? bufd[nv * E + e] : wd[e0 + e];
            wv[i] = df64(v.x, v.y);
          }
#pragma unroll
          for (int j = 0; j < K; ++j) {
            vr[j][i] = df64(0.0f);
            if (j < nv && ok[i]) {
              const float2 v = in[i] ? bufd[j * E + e] : V0d[j * stride + e0 + e];
              vr[j][i] = df64(v.x, v.y);
            }
          }
        }
        if (sub) {
          df_acc sv[EPT];
#pragma unroll
          for (int i = 0; i < EPT; ++i) sv[i] = df_acc(0.0f);
#pragma unroll
          for (int j = 0; j < K; ++j)
            if (j < nv) {
#pragma unroll
              for (int i = 0; i < EPT; ++i) sv[i] += csd[j] * vr[j][i];
            }
#pragma unroll
          for (int i = 0; i < EPT; ++i) {
            const df64 sm = sv[i];
            df64 wi = df_add(wv[i], df64(-sm.hi, -sm.lo));
            if (nrm2) wi = df_renorm(wi * invd);
            wv[i] = ok[i] ? wi : df64(0.0f);
          }
        }
#pragma unroll
        for (int i = 0; i < EPT; ++i) {
          const int e = tid + i * kCgsThreads;
          if (ok[i] && (sub || w64)) wd[e0 + e] = make_float2(wv[i].hi, wv[i].lo);
          if (ok[i] && sub && nrm2 && copy32) copy32[e0 + e] = wv[i].hi;
        }
        if (dot) {
#pragma unroll
          for (int j = 0; j < K; ++j)
            if (j < nv) {
#pragma unroll
              for (int i = 0; i < EPT; ++i) accd[j] += vr[j][i] * wv[i];
            }
        }
        if (norm) {
#pragma unroll
          for (int i = 0; i < EPT; ++i) accd[K] += wv[i] * wv[i];
        }
      } else
      for (int e = tid; e < ne; e += kCgsThreads) {
        const bool in = e < nin;
        // basis entries straight from the stage (read twice rather than kept in registers)
        auto vj = [&](int j) { return in ? buf[j * E + e] : V0[j * stride + e0 + e]; };
        double wi = in ? buf[nv * E + e] : w[e0 + e];
        if (sub) {
          double sv = 0.0;
#pragma unroll
          for (int j = 0; j < K; ++j)
            if (j < nv) sv += cs[j] * vj(j);
          wi -= sv;
          if (nrm2) {
            wi *= inv;
            if (copy32) copy32[e0 + e] = (float)wi;
          }
          w[e0 + e] = wi;
        }
        if (dot) {
#pragma unroll
          for (int j = 0; j < K; ++j)
            if (j < nv) acc[j] += vj(j) * wi;
        }
        if (norm) acc[K] += wi * wi;
      }
      __syncthreads();  // stage free again
      const int64_t nx = ch + (int64_t)S * gridDim.x;
      if (nx < nch) {
        if (tid == 0) issue(nx, st);
        ++issued;
      }
    }
    if (fail) {  // drain the copies still in flight, then leave without a result
      for (int64_t q = k; q < issued; ++q) bar_wait(&bar[q % S], (uint32_t)((q / S) & 1), nullptr);
      return;
    }
  } else {
    return;
  }
  // block partials, then the last block sums them in a fixed order (final_sums); double-float sums are
  // reduced over the warp in double-float and converted once per warp
#pragma unroll
  for (int j = 0; j <= K; ++j) {
    if ((j < K && dot && j < nv) || (j == K && norm)) {
      double x;
      if constexpr (DFV) {
        const df64 v = warp_sum_df(accd[j]);
        x = f2d_exact(v.hi) + f2d_exact(v.lo);
      } else {
        x = acc[j];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
      }
      if (lane == 0) red[warp][j] = x;
    }
  }
  __syncthreads();
  const int nb = gridDim.x;
  for (int j = tid; j <= K; j += blockDim.x) {
    if ((j < K && dot && j < nv) || (j == K && norm)) {
      double x = 0.0;
      for (int wv = 0; wv < kCgsThreads / 32; ++wv) x += red[wv][j];
      partial[(int64_t)j * nb + blockIdx.x] = x;
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(counter, 1u) == (unsigned)nb - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double tot[K + 1];
  final_sums<K, kCgsThreads>(partial, nb, nv, dot, norm, red, tot);
  __syncthreads();
  if (fin == 0) {
    for (int j = tid; j < nv; j += blockDim.x)
      if (dot) out[j] = tot[j];
    if (norm && tid == 0) out[nv] = tot[K];
  } else {
    for (int j = tid; j < nv; j += blockDim.x) out[j] = h_prev[j] + cs[j];
    if (tid == 0) {
      const double hn = nrm2 ? hn_fused : sqrt(fmax(tot[K], 0.0));
      out[nv] = hn;
      out[nv + 1] = hn > 0.0 ? 1.0 / hn : 0.0;
    }
  }
  if (tid == 0) *counter = 0u;
}

// w += sign * sum_j h_j V_j.  FP32 vectors (the FGMRES update from the FP32 preconditioned vectors): the
// sum in double-float on the FP32 pipe, then one conversion and one FP64 addition per entry, so that w
// keeps its FP64 value.
template <typename TV>
__global__ void multi_axpy_kernel(double* __restrict__ w, const TV* __restrict__ V0, int64_t stride,
                                  const double* __restrict__ h, int nv, double sign, int64_t n) {
  pdl_wait();
  pdl_trigger();
  __shared__ double sh[kMaxVec];
  __shared__ df64 shd[kMaxVec];
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    sh[j] = h[j];
    if constexpr (std::is_same<TV, float>::value) shd[j] = df_from_double(sign * h[j]);
  }
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (std::is_same<TV, float>::value) {
      df_acc s(0.0f);
      for (int j = 0; j < nv; ++j) s += shd[j] * __ldg(V0 + j * stride + i);
      const df64 t = s;
      w[i] += f2d_exact(t.hi) + f2d_exact(t.lo);
    } else {
      double s = 0.0;
      for (int j = 0; j < nv; ++j) s += sh[j] * (double)__ldg(V0 + j * stride + i);
      w[i] += sign * s;
    }
  }
}

// out[pt][c] = sum_a w[pt][a] u[c][nodes[pt][a]]: one block per point, threads over components
__global__ void point_values_kernel(const double* __restrict__ u, int64_t nn, int ncomp,
                                    const int64_t* __restrict__ nodes, const double* __restrict__ w, int nb,
                                    double* __restrict__ out) {
  pdl_wait();
  pdl_trigger();
  const int pt = blockIdx.x;
  for (int c = threadIdx.x; c < ncomp; c += blockDim.x) {
    double s = 0.0;
    for (int a = 0; a < nb; ++a) s += w[(int64_t)pt * nb + a] * u[(int64_t)c * nn + nodes[(int64_t)pt * nb + a]];
    out[(int64_t)pt * ncomp + c] = s;
  }
}

__global__ void broadcast_time_kernel(const double* __restrict__ u0, double* __restrict__ u, int nt, int64_t nn) {
  pdl_wait();
  pdl_trigger();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = u0[i];
    for (int t = 0; t < nt; ++t) u[t * nn + i] = v;
  }
}

struct MixTab { const double* x[8]; double C[kMaxNT][8]; };

__global__ void time_mix_kernel(MixTab m, int nin, int nout, double* __restrict__ y, int64_t nn, int accumulate) {
  pdl_wait();
  pdl_trigger();
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

// Coarsest-level solve u[map[i]] = sum_j inv[i][j] f[map[j]] with the inverse stored row-major, rows
// of ld entries (ld a multiple of 4, zero padding, 16-byte aligned rows): each block gathers the
// right-hand side into shared memory, each warp takes one row in 16-byte loads with four independent
// accumulators (a few memory round trips per row instead of one per 32 entries) and reduces it with
// shuffles in a fixed order (deterministic).
template <typename T> struct CoarseVec;
template <> struct CoarseVec<float> {
  using V = float4;
  static constexpr int W = 4;
  static __device__ __forceinline__ float dot(const float4 a, const float4 b) {
    return (a.x * b.x + a.y * b.y) + (a.z * b.z + a.w * b.w);
  }
};
template <> struct CoarseVec<double> {
  using V = double2;
  static constexpr int W = 2;
  static __device__ __forceinline__ double dot(const double2 a, const double2 b) { return a.x * b.x + a.y * b.y; }
};
template <typename T>
__global__ void coarse_solve_kernel(const T* __restrict__ f, T* __restrict__ u, const T* __restrict__ inv,
                                    const int64_t* __restrict__ map, int n, int ld) {
  pdl_wait();
  pdl_trigger();
  using CV = CoarseVec<T>;
  using V = typename CV::V;
  extern __shared__ __align__(16) unsigned char cs_raw[];
  T* fc = reinterpret_cast<T*>(cs_raw);
  for (int j = threadIdx.x; j < ld; j += blockDim.x) fc[j] = j < n ? f[map[j]] : T(0);
  __syncthreads();
  const int lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  const int nc = ld / CV::W;
  const V* fv = reinterpret_cast<const V*>(fc);
  for (int i = blockIdx.x * warps + (threadIdx.x >> 5); i < n; i += gridDim.x * warps) {
    const V* row = reinterpret_cast<const V*>(inv + (int64_t)i * ld);
    T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    int c = lane;
    for (; c + 96 < nc; c += 128) {
      const V r0 = __ldg(row + c), r1 = __ldg(row + c + 32), r2 = __ldg(row + c + 64), r3 = __ldg(row + c + 96);
      a0 += CV::dot(r0, fv[c]);
      a1 += CV::dot(r1, fv[c + 32]);
      a2 += CV::dot(r2, fv[c + 64]);
      a3 += CV::dot(r3, fv[c + 96]);
    }
    for (; c < nc; c += 32) a0 += CV::dot(__ldg(row + c), fv[c]);
    T s = (a0 + a1) + (a2 + a3);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if (lane == 0) u[map[i]] = s;
  }
}

__global__ void zero_constrained_kernel(double* __restrict__ y, GridDesc g, int nt) {
  pdl_wait();
  pdl_trigger();
  for (int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; node < g.n_nodes;
       node += (int64_t)gridDim.x * blockDim.x) {
    int gx, gy, gz;
    node_xyz(node, g.nn1, gx, gy, gz);
    bool bnd = on_boundary(gx, g.nn1) || on_boundary(gy, g.nn1);
    if (g.dim == 3) bnd = bnd || on_boundary(gz, g.nn1);
    if (bnd)
      for (int t = 0; t < nt; ++t) y[t * g.n_nodes + node] = 0.0;
  }
}

}  // namespace


template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin* x, Tout* y, int64_t n, cudaStream_t s) {
  { const cudaError_t e_ = launch_k(convert_kernel<Tin, Tout>, dim3(grid_blocks(n)), dim3(256), 0, s, x, y, n); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);

cudaError_t launch_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t s) {
  { const cudaError_t e_ = launch_k(axpby_kernel, dim3(grid_blocks(n)), dim3(256), 0, s, a, x, b, y, n); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_scale_to_df(double* x, double scale, int64_t n, float* copy32, cudaStream_t s) {
  { const cudaError_t e_ = launch_k(scale_to_df_kernel, dim3(grid_blocks(n)), dim3(256), 0, s, x, scale, n, copy32); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

int cgs_blocks() { return kCgsBlocks; }

template <int K, bool DFV>
cudaError_t launch_cgs_tma(const double* V0, int64_t stride, int nv, double* w, int64_t n, const double* c, int sub,
                           int dot, int norm, const double* h_prev, int fin, double* partial, unsigned int* counter,
                           double* out, int* status, cudaStream_t s, const double* nrm2, float* copy32, int w64) {
  static bool attr = false;
  auto k = cgs_pass_tma_kernel<K, DFV>;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cgs_tma_smem<K, DFV>());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  { const cudaError_t e_ = launch_k(k, dim3(152 * CgsTma<K, DFV>::BPS), dim3(kCgsThreads), cgs_tma_smem<K, DFV>(), s, V0, stride, nv, w, n, c, sub, dot, norm, h_prev, fin,
                                                                 partial, counter, out, status, nrm2, copy32, w64); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_cgs_pass(const double* V0, int64_t stride, int nv, double* w, int64_t n, const double* c, int sub,
                            int dot, int norm, const double* h_prev, int fin, double* partial, unsigned int* counter,
                            double* out, cudaStream_t s, int* status, const double* nrm2, float* copy32,
                            int vfmt) {
  if (nv < 0 || nv > 64) return cudaErrorInvalidValue;
  if (nrm2 && (!fin || norm || !sub)) return cudaErrorInvalidValue;
  // bulk copies need 16-byte aligned sources: w, V0 and the stride between basis vectors
  const bool aligned = ((uintptr_t)w % 16 == 0) && (nv == 0 || (((uintptr_t)V0 % 16 == 0) && stride % 2 == 0));
  if (vfmt == 3 && !(status && aligned)) vfmt = 0;  // a norm of an FP64 vector: the FP64 pass serves as well
  if (vfmt != 0 && !(status && aligned)) return cudaErrorInvalidValue;  // double-float: aligned vectors only
  if (vfmt != 0 && nv <= 16) {
#define STMG_CGS_DF(KK)                                                                                        \
  return launch_k(cgs_pass_df_kernel<KK>, dim3(152 * CgsDf<KK>::BPS), dim3(kCgsDfThreads), 0, s, V0, stride, nv, w, n, \
                  c, sub, dot, norm, h_prev, fin, partial, counter, out, nrm2, copy32, vfmt == 2 ? 1 : vfmt == 3 ? 2 : 0)
    if (nv <= 4) STMG_CGS_DF(4);
    if (nv <= 8) STMG_CGS_DF(8);
    STMG_CGS_DF(16);
#undef STMG_CGS_DF
  }
  if (status && aligned) {
#define STMG_CGS_TMA(KK)                                                                                              \
  return vfmt == 0 ? launch_cgs_tma<KK, false>(V0, stride, nv, w, n, c, sub, dot, norm, h_prev, fin, partial, counter,  \
                                               out, status, s, nrm2, copy32, 0)                                       \
                   : launch_cgs_tma<KK, true>(V0, stride, nv, w, n, c, sub, dot, norm, h_prev, fin, partial, counter,   \
                                              out, status, s, nrm2, copy32, vfmt == 2)
    if (nv <= 4) STMG_CGS_TMA(4);
    if (nv <= 8) STMG_CGS_TMA(8);
    if (nv <= 16) STMG_CGS_TMA(16);
    if (nv <= 32) STMG_CGS_TMA(32);
    STMG_CGS_TMA(64);
#undef STMG_CGS_TMA
  }
  // one wave: blocks per SM as the register use of each width allows (4, 4, 2, 1, 1)
#define STMG_CGS(KK, BPS) \
  return launch_k(cgs_pass_kernel<KK>, dim3(152 * (BPS)), dim3(kCgsThreads), 0, s, V0, stride, nv, w, n, c, sub, dot, \
                  norm, h_prev, fin, partial, counter, out, nrm2, copy32)
  if (nv <= 4) STMG_CGS(4, 4);
  else if (nv <= 8) STMG_CGS(8, 4);
  else if (nv <= 16) STMG_CGS(16, 2);
  else if (nv <= 32) STMG_CGS(32, 1);
  else STMG_CGS(64, 1);
#undef STMG_CGS
  return cudaGetLastError();
}

template <typename TV>
cudaError_t launch_multi_axpy(double* w, const TV* V0, int64_t stride, const double* h, int nv, double sign,
                              int64_t n, cudaStream_t s) {
  if (nv > kMaxVec) return cudaErrorInvalidValue;
  { const cudaError_t e_ = launch_k(multi_axpy_kernel<TV>, dim3(grid_blocks(n)), dim3(256), 0, s, w, V0, stride, h, nv, sign, n); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}
template cudaError_t launch_multi_axpy<double>(double*, const double*, int64_t, const double*, int, double, int64_t,
                                               cudaStream_t);
template cudaError_t launch_multi_axpy<float>(double*, const float*, int64_t, const double*, int, double, int64_t,
                                              cudaStream_t);

cudaError_t launch_point_values(const double* u, int64_t nn, int ncomp, const int64_t* nodes, const double* w, int nb,
                                int npts, double* out, cudaStream_t s) {
  { const cudaError_t e_ = launch_k(point_values_kernel, dim3((unsigned)npts), dim3(64), 0, s, u, nn, ncomp, nodes, w, nb, out); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_broadcast_time(const double* u0, double* u, int nt, int64_t nn, cudaStream_t s) {
  { const cudaError_t e_ = launch_k(broadcast_time_kernel, dim3(grid_blocks(nn)), dim3(256), 0, s, u0, u, nt, nn); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_time_mix(const double* const* xs, int nin, const double* C, int nout, double* y, int64_t nn,
                            int accumulate, cudaStream_t s) {
  if (nin > 8 || nout > kMaxNT) return cudaErrorInvalidValue;
  MixTab m{};
  for (int j = 0; j < nin; ++j) m.x[j] = xs[j];
  for (int t = 0; t < nout; ++t)
    for (int j = 0; j < nin; ++j) m.C[t][j] = C[t * nin + j];
  { const cudaError_t e_ = launch_k(time_mix_kernel, dim3(grid_blocks(nn)), dim3(256), 0, s, m, nin, nout, y, nn, accumulate); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarse_solve(const T* f, T* u, const T* inv, const int64_t* map, int n, int64_t total,
                                cudaStream_t s) {
  (void)total;
  const int ld = coarse_ld(n);
  const size_t smem = (size_t)ld * sizeof(T);  // n <= 4096 unknowns: at most 32 KB
  const int blocks = std::max(1, std::min((n + 7) / 8, 152 * 4));
  { const cudaError_t e_ = launch_k(coarse_solve_kernel<T>, dim3(blocks), dim3(256), smem, s, f, u, inv, map, n, ld); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}
template cudaError_t launch_coarse_solve<float>(const float*, float*, const float*, const int64_t*, int, int64_t,
                                                cudaStream_t);
template cudaError_t launch_coarse_solve<double>(const double*, double*, const double*, const int64_t*, int, int64_t,
                                                 cudaStream_t);

cudaError_t launch_zero_constrained(double* y, const GridDesc& g, int nt, cudaStream_t s) {
  { const cudaError_t e_ = launch_k(zero_constrained_kernel, dim3(grid_blocks(g.n_nodes)), dim3(256), 0, s, y, g, nt); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

}  // namespace stmg
