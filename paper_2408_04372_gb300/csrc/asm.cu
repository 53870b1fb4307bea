// Space-time cell-wise additive Schwarz smoother (eqs. vanka0, vanka).
//
// The block of space-time cell T = K x I_n holds all unconstrained nodes of the
// spatial cell K for all N_t time DoFs of the slab.  Its matrix is the global
// S = TA (x) A_h + TM (x) M_h restricted to those DoFs,
//     L_T = TA (x) A_K + TM (x) M_K ,
// A_K, M_K = global A_h, M_h restricted to the nodes of K (neighbour cells
// contribute on shared faces, edges and vertices).  With TA^-1 TM = V diag(lambda) V^-1
//     L_T^-1 = (V (x) I) diag_m (A_K + lambda_m M_K)^-1 (V^-1 TA^-1 (x) I),
// so each cell stores N_t real planes of (p+1)^dim x (p+1)^dim numbers: one
// plane per real lambda, two (re, im) per conjugate pair.  This is exact (up to
// rounding) and takes N_t times less memory than the dense (N_t (p+1)^dim)^2 block.
// Constrained (Dirichlet) nodes get identity rows/columns and zero residual.
//
// asm_apply: u += omega * sum_T R_T^T D_T L_T^-1 R_T r (D_T = I, or the inverse number of
// cells containing each node for the weighted sum; the set-up folds D_T into the stored rows):
// time transform of the residual, the planes' matrix-vector products, inverse transform; the
// additive sum over overlapping cells uses atomic adds.  The bulk-copy kernel streams groups of
// cells' planes (FP64, FP32, BF16, or FP8 with per-plane scales) into shared memory -- the kernel is
// bound by this stream, N_t (p+1)^(2 dim) numbers per cell -- and, with several slabs in one
// system, applies each landed group to every slab; the row-streaming kernel serves the cases
// whose stages would not fit in shared memory.
#include <algorithm>
#include <type_traits>

#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.h"
#include "local_mats.cuh"

namespace stmg {

namespace {

template <int DIM, int N>
struct Shape {
  static constexpr int NB = DIM == 3 ? N * N * N : N * N;
};

// Inverse store: per cell N_t planes of NB rows x NBP columns, row-major, NBP = NB rounded up to a
// multiple of 4 (zero padding), so that a row starts on a 4-entry boundary and is read four entries
// at a time; cell blocks padded to 16-byte boundaries.  FP8 (e4m3) planes carry one FP32 scale each
// (entry = stored value x scale, the plane's largest magnitude mapped to 448), stored after the
// cell's planes, so that one bulk copy brings a cell's planes and scales together.
__host__ __device__ constexpr int nb_pad(int nb) { return (nb + 3) / 4 * 4; }
__host__ __device__ constexpr int64_t cell_stride(int nb, int nt, int esz = 2) {
  return esz == 1 ? ((int64_t)nt * nb * nb_pad(nb) + 4 * nt + 15) / 16 * 16
                  : ((int64_t)nt * nb * nb_pad(nb) + 7) / 8 * 8;
}
template <typename TI> constexpr bool is_fp8() { return std::is_same<TI, __nv_fp8_e4m3>::value; }
// FP8 planes: the scale of plane m, stored after the cell's planes (other types: 1)
template <typename TI, int NB, int NT>
__device__ __forceinline__ float plane_scale(const TI* cell, int m) {
  if constexpr (is_fp8<TI>()) return reinterpret_cast<const float*>(cell + (int64_t)NT * NB * nb_pad(NB))[m];
  else return 1.0f;
}

__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline double2 cinv(double2 a) {
  const double d = a.x * a.x + a.y * a.y;
  return make_double2(a.x / d, -a.y / d);
}

template <int DIM, int N>
__global__ void __launch_bounds__(256)
asm_setup_kernel(GridDesc g, const double* __restrict__ geo, LocalTab lt, const double* __restrict__ lam_re,
                 const double* __restrict__ lam_im, int nreal, int ncplx, void* __restrict__ inv_out, int inv_prec,
                 int weighted) {
  constexpr int NB = Shape<DIM, N>::NB;
  constexpr int NQ = NB;
  constexpr int NG = DIM == 3 ? 7 : 4;
  const int nt = nreal + 2 * ncplx;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Aloc = reinterpret_cast<double*>(smem_raw);
  double* Mloc = Aloc + NB * NB;
  double2* C = reinterpret_cast<double2*>(Mloc + NB * NB);
  double2* fcol = C + NB * NB;
  int* ipiv = reinterpret_cast<int*>(fcol + NB);
  __shared__ int s_piv;
  __shared__ double s_scale;
  const int64_t cell = blockIdx.x;
  const int tid = threadIdx.x;
  const int p = g.p;
  const int cx = (int)(cell % g.N), cy = (int)((cell / g.N) % g.N);
  const int cz = DIM == 3 ? (int)(cell / ((int64_t)g.N * g.N)) : 0;

  assemble_local<DIM, N>(g, geo, lt, cx, cy, cz, Aloc, Mloc);
  // constrained local nodes
  auto constrained = [&](int a) {
    const int gx = cx * p + a % N, gy = cy * p + (a / N) % N;
    bool bnd = on_boundary(gx, g.nn1) || on_boundary(gy, g.nn1);
    if (DIM == 3) bnd = bnd || on_boundary(cz * p + a / (N * N), g.nn1);
    return bnd;
  };
  int plane = 0;
  for (int m = 0; m < nreal + ncplx; ++m) {
    const double lr = lam_re[m], li = m < nreal ? 0.0 : lam_im[m];
    for (int pr = tid; pr < NB * NB; pr += blockDim.x) {
      const int a = pr / NB, b = pr % NB;
      double2 v = make_double2(Aloc[pr] + lr * Mloc[pr], li * Mloc[pr]);
      if (constrained(a) || constrained(b)) v = make_double2(a == b ? 1.0 : 0.0, 0.0);
      C[pr] = v;
    }
    __syncthreads();
    // Gauss-Jordan inversion in place with partial pivoting
    for (int k = 0; k < NB; ++k) {
      if (tid < 32) {
        double best = -1.0;
        int bi = k;
        for (int r = k + tid; r < NB; r += 32) {
          const double2 c = C[r * NB + k];
          const double mag = c.x * c.x + c.y * c.y;
          if (mag > best) { best = mag; bi = r; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          const double ob = __shfl_down_sync(0xffffffffu, best, off);
          const int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (tid == 0) { s_piv = bi; ipiv[k] = bi; }
      }
      __syncthreads();
      const int pv = s_piv;
      if (pv != k)
        for (int jj = tid; jj < NB; jj += blockDim.x) {
          const double2 t = C[k * NB + jj];
          C[k * NB + jj] = C[pv * NB + jj];
          C[pv * NB + jj] = t;
        }
      __syncthreads();
      const double2 d = cinv(C[k * NB + k]);
      for (int ii = tid; ii < NB; ii += blockDim.x) fcol[ii] = ii == k ? make_double2(0.0, 0.0) : C[ii * NB + k];
      __syncthreads();
      for (int jj = tid; jj < NB; jj += blockDim.x) C[k * NB + jj] = jj == k ? d : cmul(C[k * NB + jj], d);
      __syncthreads();
      for (int pr = tid; pr < NB * NB; pr += blockDim.x) {
        const int ii = pr / NB, jj = pr % NB;
        if (ii == k) continue;
        const double2 base = jj == k ? make_double2(0.0, 0.0) : C[pr];
        const double2 f = cmul(fcol[ii], C[k * NB + jj]);
        C[pr] = make_double2(base.x - f.x, base.y - f.y);
      }
      __syncthreads();
    }
    for (int k = NB - 1; k >= 0; --k) {
      const int pv = ipiv[k];
      if (pv != k)
        for (int ii = tid; ii < NB; ii += blockDim.x) {
          const double2 t = C[ii * NB + k];
          C[ii * NB + k] = C[ii * NB + pv];
          C[ii * NB + pv] = t;
        }
      __syncthreads();
    }
    // store row-major planes: element (a, b) at a * NBP + b, zero padding columns
    constexpr int NBP = nb_pad(NB);
    const int nplanes = m < nreal ? 1 : 2;
    for (int pl = 0; pl < nplanes; ++pl) {
      const int64_t cbase = (int64_t)cell * cell_stride(NB, nt, inv_prec == 3 ? 1 : 2);
      const int64_t base = cbase + (int64_t)(plane + pl) * NB * NBP;
      double fp8_inv_scale = 1.0;
      if (inv_prec == 3) {
        // the plane's largest weighted magnitude maps to 448, the largest finite e4m3 value
        if (tid == 0) {
          double mx = 0.0;
          for (int a = 0; a < NB; ++a) {
            double wa = 1.0;
            if (weighted) wa = node_weight<double>(cx * p + a % N, cy * p + (a / N) % N, cz * p + a / (N * N), DIM, p);
            for (int b = 0; b < NB; ++b) {
              const double2 v = C[a * NB + b];
              mx = fmax(mx, fabs((pl == 0 ? v.x : v.y) * wa));
            }
          }
          reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(inv_out) + cbase + (int64_t)nt * NB * NBP)[plane + pl] =
              mx > 0.0 ? (float)(mx / 448.0) : 1.0f;
          s_scale = mx > 0.0 ? 448.0 / mx : 1.0;
        }
        __syncthreads();
        fp8_inv_scale = s_scale;
      }
      for (int pr = tid; pr < NB * NBP; pr += blockDim.x) {
        const int a = pr / NBP, b = pr % NBP;
        const double2 v = b < NB ? C[a * NB + b] : make_double2(0.0, 0.0);
        double x = pl == 0 ? v.x : v.y;
        // weighted sum: row a (the cell's node a) divided by the number of cells containing the node;
        // the factor is a power of two, exact in every storage type, and commutes with the time modes
        if (weighted) x *= node_weight<double>(cx * p + a % N, cy * p + (a / N) % N, cz * p + a / (N * N), DIM, p);
        if (inv_prec == 0) reinterpret_cast<double*>(inv_out)[base + pr] = x;
        else if (inv_prec == 1) reinterpret_cast<float*>(inv_out)[base + pr] = (float)x;
        else if (inv_prec == 2) reinterpret_cast<__nv_bfloat16*>(inv_out)[base + pr] = __float2bfloat16((float)x);
        else reinterpret_cast<__nv_fp8_e4m3*>(inv_out)[base + pr] = __nv_fp8_e4m3((float)(x * fp8_inv_scale));
      }
      __syncthreads();  // s_scale is rewritten by the next plane
    }
    plane += nplanes;
    __syncthreads();
  }
}

template <typename TI> __device__ inline float to_f(TI v);
template <typename TI> __device__ inline TI ldg_inv(const TI* p) { return __ldg(p); }
template <> __device__ inline __nv_bfloat16 ldg_inv<__nv_bfloat16>(const __nv_bfloat16* p) {
  const unsigned short v = __ldg(reinterpret_cast<const unsigned short*>(p));
  return __ushort_as_bfloat16(v);
}
template <> __device__ inline float to_f<float>(float v) { return v; }
template <> __device__ inline float to_f<__nv_fp8_e4m3>(__nv_fp8_e4m3 v) { return (float)v; }
template <> __device__ inline float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <typename T, typename TI> __device__ inline T inv_val(TI v) { return (T)to_f<TI>(v); }
template <> __device__ inline double inv_val<double, double>(double v) { return v; }
template <> __device__ inline float inv_val<float, double>(double v) { return (float)v; }

template <int DIM, int N, int NT, typename TI>
struct AsmCfg {
  static constexpr int NB = Shape<DIM, N>::NB;
  static constexpr int TPC = (NB + 31) / 32 * 32;
  static constexpr int64_t CS = cell_stride(NB, NT, (int)sizeof(TI));
  static constexpr int CPB = TPC >= 128 ? 1 : 128 / TPC;
};

// One warp-multiple per cell, thread a = local row.  Each thread streams its row of
// every plane straight from HBM; the column loop is fully unrolled so that all NB
// loads of a plane are in flight together (the kernel is bound by this stream).
template <int DIM, int N, int NT, typename T, typename TI>
__global__ void __launch_bounds__(AsmCfg<DIM, N, NT, TI>::CPB * AsmCfg<DIM, N, NT, TI>::TPC)
asm_apply_kernel(const T* __restrict__ r, T* __restrict__ u, const TI* __restrict__ inv, GridDesc g, ModeTab<T> mt,
                 const T* __restrict__ copy_src, T* __restrict__ copy_dst) {
  pdl_wait();
  pdl_trigger();
  using C = AsmCfg<DIM, N, NT, TI>;
  constexpr int NB = C::NB, TPC = C::TPC, CPB = C::CPB, NBP = nb_pad(NB);
  constexpr int64_t CS = C::CS;
  __shared__ T s_r[CPB][NT][NB];
  const int slot = threadIdx.x / TPC;
  const int a = threadIdx.x - slot * TPC;
  const int64_t cell = (int64_t)blockIdx.x * CPB + slot;
  const bool active = cell < g.n_cells && a < NB;
  const int64_t cc = cell < g.n_cells ? cell : 0;
  int cx, cy, cz;
  cell_xyz(cc, g, cx, cy, cz);
  const int aa = a < NB ? a : 0;
  const int gx = cx * g.p + aa % N, gy = cy * g.p + (aa / N) % N;
  const int gz = DIM == 3 ? cz * g.p + aa / (N * N) : 0;
  bool bnd = on_boundary(gx, g.nn1) || on_boundary(gy, g.nn1);
  if (DIM == 3) bnd = bnd || on_boundary(gz, g.nn1);
  const int64_t node = gx + (int64_t)g.nn1 * (gy + (int64_t)g.nn1 * gz);
  const bool live = active && !bnd;
  T rr[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) rr[t] = live ? r[t * g.n_nodes + node] : T(0);
  if (copy_dst && active) {  // side job for the V-cycle: copy_dst := copy_src on this cell's nodes
#pragma unroll
    for (int t = 0; t < NT; ++t) copy_dst[t * g.n_nodes + node] = copy_src[t * g.n_nodes + node];
  }
  if (a < NB) {
#pragma unroll
    for (int m = 0; m < NT; ++m) {
      // plane m: real mode m (m < nreal) or re/im part of complex mode nreal + (m - nreal) / 2
      const bool is_real = m < mt.nreal;
      const int mode = is_real ? m : mt.nreal + (m - mt.nreal) / 2;
      const bool im_part = !is_real && ((m - mt.nreal) & 1);
      T v = 0;
#pragma unroll
      for (int t = 0; t < NT; ++t) v += (im_part ? mt.Wi[mode][t] : mt.Wr[mode][t]) * rr[t];
      s_r[slot][m][a] = v;
    }
  }
  __syncthreads();
  if (!live) return;
  const TI* ic = inv + cell * CS;
  T z[NT];
#pragma unroll
  for (int m = 0; m < NT; ++m) z[m] = 0;
#pragma unroll
  for (int m = 0; m < NT; ++m) {
    if (m < mt.nreal) {
      const TI* pl = ic + (m * NB + a) * NBP;
      T acc = 0;
#pragma unroll
      for (int b = 0; b < NB; ++b) acc += inv_val<T, TI>(ldg_inv(pl + b)) * s_r[slot][m][b];
      z[m] = acc;
    } else if (m + 1 < NT && ((m - mt.nreal) & 1) == 0) {
      const TI* pr_ = ic + (m * NB + a) * NBP;
      const TI* pi_ = pr_ + NB * NBP;
      T zr = 0, zi = 0;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const T ir = inv_val<T, TI>(ldg_inv(pr_ + b)), ii = inv_val<T, TI>(ldg_inv(pi_ + b));
        const T sre = s_r[slot][m][b], sim = s_r[slot][m + 1][b];
        zr += ir * sre - ii * sim;
        zi += ir * sim + ii * sre;
      }
      z[m] = zr;
      z[m + 1] = zi;
    }
  }
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
    atomicAdd(u + t * g.n_nodes + node, mt.omega * o);
  }
}

// ---- TMA-fed variant: bulk copies of whole cell groups into a ring of shared-memory stages ----
//
// The inverse store is contiguous over cells, so the planes of CPG consecutive cells are one
// bulk copy (cp.async.bulk, completion counted on an mbarrier).  Each CTA walks its groups with
// S stages in flight; while a group's copy lands, its threads form the modal residual of the
// group's cells.  With several slabs in one system (nslab > 1, vectors nslab blocks of
// slab_stride entries) every slab has the same local inverses, so a landed group serves all
// slabs before its stage is reused: the inverse stream, which bounds the kernel, is read once
// per sweep instead of once per slab.  Every wait is bounded: on timeout the kernel records
// STMG_DEVICE_TIMEOUT in *status, drains the copies it issued (bounded as well) and returns.
template <int DIM, int N, int NT, typename TI>
struct TmaCfg {
  static constexpr int NB = Shape<DIM, N>::NB;
  static constexpr int64_t CS = cell_stride(NB, NT, (int)sizeof(TI));
  static constexpr int CELL_BYTES = (int)(CS * sizeof(TI));
  static constexpr int CPG0 = 128 / NB;
  static constexpr int CPG_MEM = 20480 / CELL_BYTES;
  static constexpr int CPG = CPG0 < CPG_MEM ? (CPG0 > 0 ? CPG0 : 1) : (CPG_MEM > 0 ? CPG_MEM : 1);
  static constexpr int THREADS = (CPG * NB + 31) / 32 * 32;
  static constexpr int STAGE_BYTES = CPG * CELL_BYTES;
  static constexpr int S = 2;  // measured on GB300: two stages (more CTAs per SM) beat three or four
  static constexpr size_t SMEM = (size_t)S * STAGE_BYTES;
};



__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Four consecutive entries of an inverse row in shared memory (8-byte aligned for BF16, 16 for FP32/FP64).
__device__ __forceinline__ float4 inv4(const __nv_bfloat16* p) {
  const uint2 w = *reinterpret_cast<const uint2*>(p);  // bf16 -> f32 places the 16 bits high
  return make_float4(__uint_as_float(w.x << 16), __uint_as_float(w.x & 0xffff0000u), __uint_as_float(w.y << 16),
                     __uint_as_float(w.y & 0xffff0000u));
}
__device__ __forceinline__ float4 inv4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 inv4(const __nv_fp8_e4m3* p) {  // 4-byte aligned
  const unsigned int w = *reinterpret_cast<const unsigned int*>(p);
  const __half2 lo = __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3));
  const __half2 hi = __half2(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3));
  const float2 a = __half22float2(lo), b = __half22float2(hi);
  return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float4 inv4(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  return make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

// sum_b row[b] s[b] over NBP entries (padding zero in both), two independent FP32x2 accumulators
template <int NBP, typename TI>
__device__ __forceinline__ float dot_row(const TI* row, const float* s) {
  float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
  for (int c = 0; c < NBP; c += 4) {
    const float4 w = inv4(row + c);
    const float4 v = *reinterpret_cast<const float4*>(s + c);
    a0 = __ffma2_rn(make_float2(w.x, w.y), make_float2(v.x, v.y), a0);
    a1 = __ffma2_rn(make_float2(w.z, w.w), make_float2(v.z, v.w), a1);
  }
  return (a0.x + a0.y) + (a1.x + a1.y);
}

__device__ __forceinline__ void tma_bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

// The same for the stored inverses, read once per sweep: marked evict-first in L2, so that the stream
// does not push out the residual and correction vectors, which every cell's threads gather and update.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void tma_bulk_load_stream(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                                     uint64_t pol) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol) : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait on phase `parity` of an mbarrier: false after kWaitNs nanoseconds, or as soon as
// *status (if given) is nonzero because another CTA already gave up.
constexpr uint64_t kWaitNs = 1000000000ull;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const int* status) {
  const uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    if (done) return true;
    if ((it & 63) == 63) {
      if (global_ns() - t0 > kWaitNs) return false;
      if (status && *reinterpret_cast<const volatile int*>(status) != 0) return false;
    }
  }
}

// Test hook for the timeout path: one thread waits on an mbarrier that nothing will complete (no
// copy is issued), gives up after the bounded wait and records the timeout.  Nothing faults.
__global__ void wait_selftest_kernel(int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
  if (!mbar_wait(&bar, 0u, nullptr)) atomicExch(status, STMG_DEVICE_TIMEOUT);
}

// MULTI: several slabs (the slab loop and its offsets exist only in this instance, so that the
// one-slab kernel keeps its registers and occupancy)
template <int DIM, int N, int NT, typename T, typename TI, bool MULTI>
__global__ void __launch_bounds__(TmaCfg<DIM, N, NT, TI>::THREADS)
asm_apply_tma_kernel(const T* __restrict__ r, T* __restrict__ u, const TI* __restrict__ inv, GridDesc g,
                     ModeTab<T> mt, const T* __restrict__ copy_src, T* __restrict__ copy_dst, int* status,
                     int nslab_arg, int64_t slab_stride) {
  const int nslab = MULTI ? nslab_arg : 1;
  pdl_wait();
  pdl_trigger();
  using C = TmaCfg<DIM, N, NT, TI>;
  constexpr int NB = C::NB, CPG = C::CPG, S = C::S;
  constexpr int64_t CS = C::CS;
  constexpr int NBP = nb_pad(NB);
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[S];
  __shared__ __align__(16) T s_r[CPG][NT][NBP];  // modal residual of the group's cells, zero padding
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  const int64_t ngroups = (g.n_cells + CPG - 1) / CPG;
  auto group_bytes = [&](int64_t grp) -> uint32_t {
    const int64_t c0 = grp * CPG;
    const int64_t nc = g.n_cells - c0 < CPG ? g.n_cells - c0 : CPG;
    return (uint32_t)(nc * C::CELL_BYTES);
  };
  if (tid == 0) s_fail = *reinterpret_cast<const volatile int*>(status);
  for (int i = tid; i < CPG * NT * NBP; i += blockDim.x) (&s_r[0][0][0])[i] = T(0);
  __syncthreads();
  if (s_fail) return;  // an earlier wait gave up: issue nothing
  if (tid == 0) {
    for (int s = 0; s < S; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  // prologue: the first S groups of this CTA
  int64_t issued = 0;  // groups issued by this CTA (thread 0's count; all threads track it alike)
  const uint64_t pol = l2_evict_first_policy();
  if (tid == 0)
    for (int s = 0; s < S; ++s) {
      const int64_t grp = blockIdx.x + (int64_t)s * gridDim.x;
      if (grp < ngroups)
        tma_bulk_load_stream(smem_raw + (size_t)s * C::STAGE_BYTES, inv + grp * CPG * CS, group_bytes(grp), &bar[s], pol);
    }
  for (int s = 0; s < S; ++s)
    if (blockIdx.x + (int64_t)s * gridDim.x < ngroups) ++issued;
  int64_t k = 0;
  // residual (and side-job source) of a group's node for this thread, loaded one group ahead so
  // that their latency overlaps the previous group's work
  const int slot = tid / NB, a = tid - slot * NB;
  struct Pre { int64_t node; bool active, live; T rr[NT], cp[NT]; };
  // work item (group grp, slab sl): the node of this thread and slab sl's residual there
  auto prefetch = [&](int64_t grp, int sl, Pre& P) {
    const int64_t cell = grp * CPG + slot;
    P.active = grp < ngroups && slot < CPG && cell < g.n_cells;
    P.live = false;
    P.node = 0;
    if (!P.active) return;
    const int64_t so = MULTI ? (int64_t)sl * slab_stride : 0;
    int cx, cy, cz;
    cell_xyz(cell, g, cx, cy, cz);
    const int gx = cx * g.p + a % N, gy = cy * g.p + (a / N) % N;
    const int gz = DIM == 3 ? cz * g.p + a / (N * N) : 0;
    bool bnd = on_boundary(gx, g.nn1) || on_boundary(gy, g.nn1);
    if (DIM == 3) bnd = bnd || on_boundary(gz, g.nn1);
    P.node = gx + (int64_t)g.nn1 * (gy + (int64_t)g.nn1 * gz);
    P.live = !bnd;
#pragma unroll
    for (int t = 0; t < NT; ++t) P.rr[t] = P.live ? r[so + t * g.n_nodes + P.node] : T(0);
    if (copy_dst) {
#pragma unroll
      for (int t = 0; t < NT; ++t) P.cp[t] = copy_src[so + t * g.n_nodes + P.node];
    }
  };
  Pre cur, nxt;
  prefetch(blockIdx.x, 0, cur);
  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++k) {
    const int stage = (int)(k % S);
    const uint32_t parity = (uint32_t)((k / S) & 1);
   for (int sl = 0; sl < nslab; ++sl) {
    const int64_t so = MULTI ? (int64_t)sl * slab_stride : 0;
    if (sl + 1 < nslab) prefetch(grp, sl + 1, nxt);
    else prefetch(grp + gridDim.x, 0, nxt);
    const bool active = cur.active, live = cur.live;
    const int64_t node = so + cur.node;
    // modal residual of this group's cells (independent of the copy in flight)
    if (active) {
      if (copy_dst) {
#pragma unroll
        for (int t = 0; t < NT; ++t) copy_dst[t * g.n_nodes + node] = cur.cp[t];
      }
#pragma unroll
      for (int m = 0; m < NT; ++m) {
        const bool is_real = m < mt.nreal;
        const int mode = is_real ? m : mt.nreal + (m - mt.nreal) / 2;
        const bool im_part = !is_real && ((m - mt.nreal) & 1);
        T v = 0;
#pragma unroll
        for (int t = 0; t < NT; ++t) v += (im_part ? mt.Wi[mode][t] : mt.Wr[mode][t]) * cur.rr[t];
        s_r[slot][m][a] = v;
      }
    }
    if (sl == 0 && !mbar_wait(&bar[stage], parity, status)) {
      atomicExch(status, STMG_DEVICE_TIMEOUT);
      s_fail = 1;
    }
    __syncthreads();
    if (s_fail) break;
    if (active && live) {
      const TI* ic = reinterpret_cast<const TI*>(smem_raw + (size_t)stage * C::STAGE_BYTES) + slot * CS;
      T z[NT];
#pragma unroll
      for (int m = 0; m < NT; ++m) z[m] = 0;
#pragma unroll
      for (int m = 0; m < NT; ++m) {
        const TI* rr = ic + (m * NB + a) * NBP;  // row a of plane m
        if (m < mt.nreal) {
          const T sc = (T)plane_scale<TI, NB, NT>(ic, m);
          if constexpr (std::is_same<T, float>::value) {
            z[m] = sc * dot_row<NBP>(rr, s_r[slot][m]);
          } else {
            T acc = 0;
#pragma unroll
            for (int b = 0; b < NB; ++b) acc += inv_val<T, TI>(rr[b]) * s_r[slot][m][b];
            z[m] = sc * acc;
          }
        } else if (m + 1 < NT && ((m - mt.nreal) & 1) == 0) {
          const TI* ri = rr + NB * NBP;  // imaginary part: the next plane
          const T sr = (T)plane_scale<TI, NB, NT>(ic, m), si = (T)plane_scale<TI, NB, NT>(ic, m + 1);
          if constexpr (std::is_same<T, float>::value) {
            z[m] = sr * dot_row<NBP>(rr, s_r[slot][m]) - si * dot_row<NBP>(ri, s_r[slot][m + 1]);
            z[m + 1] = sr * dot_row<NBP>(rr, s_r[slot][m + 1]) + si * dot_row<NBP>(ri, s_r[slot][m]);
          } else {
            T zr = 0, zi = 0;
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              const T ir = sr * inv_val<T, TI>(rr[b]), ii = si * inv_val<T, TI>(ri[b]);
              const T sre = s_r[slot][m][b], sim = s_r[slot][m + 1][b];
              zr += ir * sre - ii * sim;
              zi += ir * sim + ii * sre;
            }
            z[m] = zr;
            z[m + 1] = zi;
          }
        }
      }
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
        atomicAdd(u + t * g.n_nodes + node, mt.omega * o);
      }
    }
    __syncthreads();  // s_r free again (and, after the last slab, the stage)
    if (sl + 1 < nslab) cur = nxt;
   }
    if (s_fail) break;
    const int64_t next = grp + (int64_t)S * gridDim.x;
    if (next < ngroups) {
      if (tid == 0)
        tma_bulk_load_stream(smem_raw + (size_t)stage * C::STAGE_BYTES, inv + next * CPG * CS, group_bytes(next), &bar[stage], pol);
      ++issued;
    }
    cur = nxt;  // the next group's first slab
  }
  // after a timeout: wait (bounded) for the copies still in flight before the CTA exits
  if (s_fail) {
    for (int64_t q = k; q < issued; ++q) mbar_wait(&bar[q % S], (uint32_t)((q / S) & 1), nullptr);
  }
}

// Several slabs in one system, FP32 vectors, BF16 inverses (cells of at most 27 nodes): after a group's
// planes land, each thread keeps its NT rows (packed BF16, NT * NBP / 2 registers) and the stage is
// released at once, so the next group's copy starts before this group's work; the slabs then run in
// batches of up to SB: every thread loads the batch's residuals at its node together, forms the modal
// residuals, and after one barrier multiplies each slab's modal residual by its rows from registers.
// Two barriers per batch instead of two per slab, and the stored rows are read from shared memory once
// per group.
// SB slabs per batch (8).  For one slab the early release of the stage does not pay: the rows held in
// registers cost 4 CTAs per SM instead of 6, and the sweep measured 34.9 us against 29.6 us for
// asm_apply_tma_kernel (bench workload, GB300).
constexpr int kMultiSB = 8;
template <int DIM, int N, int NT, int SB>
struct MultiCfg {
  using C = TmaCfg<DIM, N, NT, __nv_bfloat16>;
  static constexpr int NBP = nb_pad(C::NB);
  static constexpr size_t SR_BYTES = (size_t)C::CPG * SB * NT * NBP * sizeof(float);
  static constexpr size_t SMEM = C::SMEM + SR_BYTES;
};

__device__ __forceinline__ float2 bf16x2_lo_hi(uint32_t w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

template <int DIM, int N, int NT, int SB>
__global__ void __launch_bounds__(TmaCfg<DIM, N, NT, __nv_bfloat16>::THREADS, 4)
asm_multi_rows_kernel(const float* __restrict__ r, float* __restrict__ u, const __nv_bfloat16* __restrict__ inv,
                      GridDesc g, ModeTab<float> mt, const float* __restrict__ copy_src, float* __restrict__ copy_dst,
                      int* status, int nslab, int64_t slab_stride) {
  pdl_wait();
  pdl_trigger();
  using C = TmaCfg<DIM, N, NT, __nv_bfloat16>;
  constexpr int NB = C::NB, CPG = C::CPG, S = C::S;
  constexpr int64_t CS = C::CS;
  constexpr int NBP = nb_pad(NB), NW = NBP / 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float (*s_r)[SB][NT][NBP] = reinterpret_cast<float (*)[SB][NT][NBP]>(smem_raw + C::SMEM);
  __shared__ __align__(8) uint64_t bar[S];
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  const int64_t ngroups = (g.n_cells + CPG - 1) / CPG;
  auto group_bytes = [&](int64_t grp) -> uint32_t {
    const int64_t c0 = grp * CPG;
    const int64_t nc = g.n_cells - c0 < CPG ? g.n_cells - c0 : CPG;
    return (uint32_t)(nc * C::CELL_BYTES);
  };
  if (tid == 0) s_fail = *reinterpret_cast<const volatile int*>(status);
  for (int i = tid; i < CPG * SB * NT * NBP; i += blockDim.x) (&s_r[0][0][0][0])[i] = 0.0f;
  __syncthreads();
  if (s_fail) return;
  if (tid == 0) {
    for (int st = 0; st < S; ++st)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[st])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  int64_t issued = 0;
  const uint64_t pol = l2_evict_first_policy();
  if (tid == 0)
    for (int st = 0; st < S; ++st) {
      const int64_t grp = blockIdx.x + (int64_t)st * gridDim.x;
      if (grp < ngroups)
        tma_bulk_load_stream(smem_raw + (size_t)st * C::STAGE_BYTES, inv + grp * CPG * CS, group_bytes(grp), &bar[st], pol);
    }
  for (int st = 0; st < S; ++st)
    if (blockIdx.x + (int64_t)st * gridDim.x < ngroups) ++issued;
  const int slot = tid / NB, a = tid - slot * NB;
  int64_t k = 0;
  for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x, ++k) {
    const int stage = (int)(k % S);
    const uint32_t parity = (uint32_t)((k / S) & 1);
    const int64_t cell = grp * CPG + slot;
    const bool active = slot < CPG && cell < g.n_cells;
    int64_t node = 0;
    bool live = false;
    if (active) {
      int cx, cy, cz;
      cell_xyz(cell, g, cx, cy, cz);
      const int gx = cx * g.p + a % N, gy = cy * g.p + (a / N) % N;
      const int gz = DIM == 3 ? cz * g.p + a / (N * N) : 0;
      bool bnd = on_boundary(gx, g.nn1) || on_boundary(gy, g.nn1);
      if (DIM == 3) bnd = bnd || on_boundary(gz, g.nn1);
      node = gx + (int64_t)g.nn1 * (gy + (int64_t)g.nn1 * gz);
      live = !bnd;
    }
    if (!mbar_wait(&bar[stage], parity, status)) {
      atomicExch(status, STMG_DEVICE_TIMEOUT);
      s_fail = 1;
    }
    // this thread's rows (planes 0..NT-1, row a) from the landed stage, kept packed
    uint32_t rw[NT][NW];
    if (active && live && !s_fail) {
      const __nv_bfloat16* ic =
          reinterpret_cast<const __nv_bfloat16*>(smem_raw + (size_t)stage * C::STAGE_BYTES) + slot * CS;
#pragma unroll
      for (int m = 0; m < NT; ++m) {
        const uint2* src = reinterpret_cast<const uint2*>(ic + (m * NB + a) * NBP);
#pragma unroll
        for (int c = 0; c < NW / 2; ++c) {
          const uint2 v = src[c];
          rw[m][2 * c] = v.x;
          rw[m][2 * c + 1] = v.y;
        }
      }
    }
    __syncthreads();  // every thread holds its rows: the stage is free
    if (s_fail) break;
    const int64_t next = grp + (int64_t)S * gridDim.x;
    if (next < ngroups) {
      if (tid == 0)
        tma_bulk_load_stream(smem_raw + (size_t)stage * C::STAGE_BYTES, inv + next * CPG * CS, group_bytes(next), &bar[stage], pol);
      ++issued;
    }
    for (int b0 = 0; b0 < nslab; b0 += SB) {
      // modal residuals of the batch's slabs at this thread's node
      if (active) {
        float rr[SB][NT];
#pragma unroll
        for (int sb = 0; sb < SB; ++sb)
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            const int64_t o = (int64_t)(b0 + sb) * slab_stride + t * g.n_nodes + node;
            rr[sb][t] = (b0 + sb < nslab && live) ? r[o] : 0.0f;
            if (copy_dst && b0 + sb < nslab) copy_dst[o] = copy_src[o];
          }
#pragma unroll
        for (int sb = 0; sb < SB; ++sb)
#pragma unroll
          for (int m = 0; m < NT; ++m) {
            const bool is_real = m < mt.nreal;
            const int mode = is_real ? m : mt.nreal + (m - mt.nreal) / 2;
            const bool im_part = !is_real && ((m - mt.nreal) & 1);
            float v = 0.0f;
#pragma unroll
            for (int t = 0; t < NT; ++t) v += (im_part ? mt.Wi[mode][t] : mt.Wr[mode][t]) * rr[sb][t];
            s_r[slot][sb][m][a] = v;
          }
      }
      __syncthreads();
      if (active && live) {
#pragma unroll 1
        for (int sb = 0; sb < SB; ++sb) {
          if (b0 + sb >= nslab) break;
          const float* sr = &s_r[slot][sb][0][0];
          // row m against modal residual q: the dot products each mode needs
          auto dot = [&](int m, int q) {
            float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int c = 0; c < NBP / 4; ++c) {
              const float4 v = *reinterpret_cast<const float4*>(sr + q * NBP + 4 * c);
              a0 = __ffma2_rn(bf16x2_lo_hi(rw[m][2 * c]), make_float2(v.x, v.y), a0);
              a1 = __ffma2_rn(bf16x2_lo_hi(rw[m][2 * c + 1]), make_float2(v.z, v.w), a1);
            }
            return (a0.x + a0.y) + (a1.x + a1.y);
          };
          float z[NT];
#pragma unroll
          for (int m = 0; m < NT; ++m) {
            if (m < mt.nreal) {
              z[m] = dot(m, m);
            } else if (m + 1 < NT && ((m - mt.nreal) & 1) == 0) {
              z[m] = dot(m, m) - dot(m + 1, m + 1);
              z[m + 1] = dot(m, m + 1) + dot(m + 1, m);
            }
          }
          const int64_t so = (int64_t)(b0 + sb) * slab_stride;
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            float o = 0.0f;
#pragma unroll
            for (int m = 0; m < NT; ++m) {
              if (m < mt.nreal) {
                o += mt.Vr[t][m] * z[m];
              } else if (m + 1 < NT && ((m - mt.nreal) & 1) == 0) {
                const int mode = mt.nreal + (m - mt.nreal) / 2;
                o += 2.0f * (mt.Vr[t][mode] * z[m] - mt.Vi[t][mode] * z[m + 1]);
              }
            }
            atomicAdd(u + so + t * g.n_nodes + node, mt.omega * o);
          }
        }
      }
      __syncthreads();  // s_r free again
    }
  }
  if (s_fail) {
    for (int64_t q = k; q < issued; ++q) mbar_wait(&bar[q % S], (uint32_t)((q / S) & 1), nullptr);
  }
}

template <int DIM, int N, int NT, int SB>
cudaError_t launch_multi_rows(const float* r, float* u, const void* inv, const GridDesc& g, const ModeTab<float>& mt,
                              const float* cs, float* cd, int* status, int nslab, int64_t ss, cudaStream_t s) {
  using C = TmaCfg<DIM, N, NT, __nv_bfloat16>;
  using M = MultiCfg<DIM, N, NT, SB>;
  auto k = asm_multi_rows_kernel<DIM, N, NT, SB>;
  static int per_sm = 0, sms = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)M::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::THREADS, M::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  const int64_t groups = (g.n_cells + C::CPG - 1) / C::CPG;
  const int64_t grid = std::min<int64_t>(groups, (int64_t)sms * per_sm);
  { const cudaError_t e_ = launch_k(k, dim3((unsigned)grid), dim3(C::THREADS), M::SMEM, s, r, u, reinterpret_cast<const __nv_bfloat16*>(inv), g, mt, cs, cd, status, nslab, ss); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

template <int DIM, int N>
cudaError_t setup_t(const GridDesc& g, const double* geo64, const LocalTab& lt, const double* lr, const double* li,
                    int nreal, int ncplx, void* inv, int inv_prec, int weighted, cudaStream_t s) {
  constexpr int NB = Shape<DIM, N>::NB;
  const size_t smem = (size_t)2 * NB * NB * sizeof(double) + (size_t)NB * NB * sizeof(double2) +
                      NB * sizeof(double2) + NB * sizeof(int);
  auto k = asm_setup_kernel<DIM, N>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)g.n_cells, 256, smem, s>>>(g, geo64, lt, lr, li, nreal, ncplx, inv, inv_prec, weighted);
  return cudaGetLastError();
}

template <int DIM, int N, int NT, typename T, typename TI, bool MULTI>
cudaError_t launch_tma(const T* r, T* u, const void* inv, const GridDesc& g, const ModeTab<T>& mt, const T* cs, T* cd,
                       int* status, int nslab, int64_t ss, cudaStream_t s) {
  using C = TmaCfg<DIM, N, NT, TI>;
  auto k = asm_apply_tma_kernel<DIM, N, NT, T, TI, MULTI>;
  static int per_sm = 0, sms = 0;  // one value per instantiation (same device for all contexts)
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, C::THREADS, C::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  const int64_t groups = (g.n_cells + C::CPG - 1) / C::CPG;
  const int64_t grid = std::min<int64_t>(groups, (int64_t)sms * per_sm);
  { const cudaError_t e_ = launch_k(k, dim3((unsigned)grid), dim3(C::THREADS), C::SMEM, s, r, u, reinterpret_cast<const TI*>(inv), g, mt, cs, cd, status, nslab, ss); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

template <int DIM, int N, int NT, typename T, typename TI>
cudaError_t apply_t(const T* r, T* u, const void* inv, const GridDesc& g, const ModeTab<T>& mt, const T* cs, T* cd,
                    int* status, int nslab, int64_t ss, cudaStream_t s) {
  // row-streaming kernel (one launch per slab) when there is no device status word to report a
  // timeout to, or when S stages of one cell's planes exceed the shared memory of an SM (p = 3,
  // N_t = 4, FP64)
  if (!status || TmaCfg<DIM, N, NT, TI>::SMEM > (size_t)200 * 1024) {
    if constexpr (is_fp8<TI>()) {
      return cudaErrorInvalidValue;  // FP8 planes carry scales that only the bulk-copy kernel reads
    } else {
    using C = AsmCfg<DIM, N, NT, TI>;
    const int64_t blocks = (g.n_cells + C::CPB - 1) / C::CPB;
    for (int sl = 0; sl < nslab; ++sl) {
      const int64_t o = sl * ss;
      const cudaError_t e_ = launch_k(asm_apply_kernel<DIM, N, NT, T, TI>, dim3((unsigned)blocks), dim3(C::CPB * C::TPC),
                                      0, s, r + o, u + o, reinterpret_cast<const TI*>(inv), g, mt, cs ? cs + o : nullptr,
                                      cd ? cd + o : nullptr);
      if (e_ != cudaSuccess) return e_;
    }
    return cudaGetLastError();
    }
  }
  if constexpr (std::is_same<T, float>::value && std::is_same<TI, __nv_bfloat16>::value &&
                Shape<DIM, N>::NB <= 27) {
    if (nslab > 1) return launch_multi_rows<DIM, N, NT, kMultiSB>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s);
  }
  return nslab > 1 ? launch_tma<DIM, N, NT, T, TI, true>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s)
                   : launch_tma<DIM, N, NT, T, TI, false>(r, u, inv, g, mt, cs, cd, status, 1, ss, s);
}

}  // namespace

cudaError_t launch_wait_selftest(int* status, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(status);
  return cudaGetLastError();
}

int64_t asm_cell_stride(int dim, int n, int nt, int esz) { return cell_stride(dim == 3 ? n * n * n : n * n, nt, esz); }

cudaError_t launch_asm_setup(int dim, int n, int nt, const GridDesc& g, const double* geo64, const LocalTab& lt,
                             const double* lam_re, const double* lam_im, int nreal, int ncplx, void* inv,
                             int inv_prec, int weighted, cudaStream_t s) {
  (void)nt;
  if (dim == 3) {
    if (n == 2) return setup_t<3, 2>(g, geo64, lt, lam_re, lam_im, nreal, ncplx, inv, inv_prec, weighted, s);
    if (n == 3) return setup_t<3, 3>(g, geo64, lt, lam_re, lam_im, nreal, ncplx, inv, inv_prec, weighted, s);
    if (n == 4) return setup_t<3, 4>(g, geo64, lt, lam_re, lam_im, nreal, ncplx, inv, inv_prec, weighted, s);
  } else {
    if (n == 2) return setup_t<2, 2>(g, geo64, lt, lam_re, lam_im, nreal, ncplx, inv, inv_prec, weighted, s);
    if (n == 3) return setup_t<2, 3>(g, geo64, lt, lam_re, lam_im, nreal, ncplx, inv, inv_prec, weighted, s);
    if (n == 4) return setup_t<2, 4>(g, geo64, lt, lam_re, lam_im, nreal, ncplx, inv, inv_prec, weighted, s);
    if (n == 5) return setup_t<2, 5>(g, geo64, lt, lam_re, lam_im, nreal, ncplx, inv, inv_prec, weighted, s);
  }
  return cudaErrorInvalidValue;
}

#define STMG_ASM_CASE(DIM, N, NT)                                                                  \
  if (dim == DIM && n == N && nt == NT) {                                                          \
    if (inv_prec == 0) return apply_t<DIM, N, NT, T, double>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s); \
    if (inv_prec == 1) return apply_t<DIM, N, NT, T, float>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s);  \
    if (inv_prec == 2) return apply_t<DIM, N, NT, T, __nv_bfloat16>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s); \
    return apply_t<DIM, N, NT, T, __nv_fp8_e4m3>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s);            \
  }

template <typename T>
cudaError_t launch_asm_apply(int dim, int n, int nt, const T* r, T* u, const void* inv, int inv_prec,
                             const GridDesc& g, const ModeTab<T>& mt, const T* cs, T* cd, int* status,
                             int nslab, int64_t ss, cudaStream_t s) {
  STMG_ASM_CASE(3, 2, 1) STMG_ASM_CASE(3, 2, 2) STMG_ASM_CASE(3, 2, 3) STMG_ASM_CASE(3, 2, 4)
  STMG_ASM_CASE(3, 3, 1) STMG_ASM_CASE(3, 3, 2) STMG_ASM_CASE(3, 3, 3) STMG_ASM_CASE(3, 3, 4)
  STMG_ASM_CASE(3, 4, 1) STMG_ASM_CASE(3, 4, 2) STMG_ASM_CASE(3, 4, 3) STMG_ASM_CASE(3, 4, 4)
  STMG_ASM_CASE(2, 2, 1) STMG_ASM_CASE(2, 2, 2) STMG_ASM_CASE(2, 2, 3) STMG_ASM_CASE(2, 2, 4)
  STMG_ASM_CASE(2, 3, 1) STMG_ASM_CASE(2, 3, 2) STMG_ASM_CASE(2, 3, 3) STMG_ASM_CASE(2, 3, 4)
  STMG_ASM_CASE(2, 4, 1) STMG_ASM_CASE(2, 4, 2) STMG_ASM_CASE(2, 4, 3) STMG_ASM_CASE(2, 4, 4)
  STMG_ASM_CASE(2, 5, 1) STMG_ASM_CASE(2, 5, 2) STMG_ASM_CASE(2, 5, 3) STMG_ASM_CASE(2, 5, 4)
  return cudaErrorInvalidValue;
}

template cudaError_t launch_asm_apply<float>(int, int, int, const float*, float*, const void*, int, const GridDesc&,
                                             const ModeTab<float>&, const float*, float*, int*, int, int64_t,
                                             cudaStream_t);
template cudaError_t launch_asm_apply<double>(int, int, int, const double*, double*, const void*, int,
                                              const GridDesc&, const ModeTab<double>&, const double*, double*, int*,
                                              int, int64_t, cudaStream_t);

}  // namespace stmg
