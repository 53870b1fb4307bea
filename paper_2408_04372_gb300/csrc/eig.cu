// Space-time additive Schwarz local solves (eqs. vanka0, vanka) through a generalized eigen-
// decomposition in space, per cell.
//
// The block of space-time cell T is L_T = TA (x) A_K + TM (x) M_K, with A_K, M_K the global
// stiffness and mass matrices restricted to the unconstrained nodes of spatial cell K.  With the
// M_K-orthonormal eigenvectors of the symmetric pencil, A_K Q = M_K Q diag(mu), Q^T M_K Q = I, and
// the time diagonalisation TA^-1 TM = V diag(lambda) V^-1,
//     L_T^-1 = (V (x) Q) diag_{m,j} 1 / (lambda_m + mu_j) (V^-1 TA^-1 (x) Q^T),
// exact up to rounding: (A_K + lambda M_K)^-1 = Q diag(1 / (mu + lambda)) Q^T for every time mode.
// A cell therefore stores one (p+1)^dim x (p+1)^dim matrix Q and (p+1)^dim eigenvalues mu instead of
// N_t inverse planes: N_t times fewer bytes for the HBM-bound sweep, at twice the multiply-adds
// (Q^T on the way in, Q on the way out), which the CUDA cores have to spare.
//
// eig_setup_kernel (FP64, one CTA per cell): local matrices, Cholesky M_K = L L^T,
// C = L^-1 A_K L^-T, cyclic Jacobi on C (parallel round-robin ordering, rotations by Golub and
// Van Loan's symmetric Schur decomposition) until the off-diagonal part is below 1e-15 of C,
// Q = L^-T U.  Store per cell: Q[a][j] row-major over the local nodes a (rows and columns of
// constrained nodes zero) with row stride NBP (NB rounded up to whole 4-entry chunks, an odd number
// of them), then NBP eigenvalues (FP64 next to an FP64 Q, else FP32; 1 in the padding), the block
// padded to 16 bytes.
//
// eig_apply_kernel: TMA-fed like the plane smoother -- each persistent CTA walks groups of
// consecutive cells whose blocks arrive by one bulk copy into a ring of two shared-memory stages
// (bounded mbarrier waits); per cell and slab: modal residual (V^-1 TA^-1 in time), y = Q^T s (a
// thread per eigenvector), z_hat = y / (lambda + mu) (complex for conjugate time modes), z = Q z_hat
// (a thread per node), back to the time basis (V), weighted by the node's inverse cell count when the
// weighted sum is selected, and added with atomics.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.h"
#include "local_mats.cuh"
#include "tc05.cuh"

namespace stmg {

namespace {

// Row stride of Q: NB rounded up to a multiple of 4 entries with an odd number of 4-entry chunks, so
// that the threads of a warp, each reading its own row four entries at a time, hit distinct banks.
__host__ __device__ constexpr int eig_nbp(int nb) { return ((nb + 3) / 4) % 2 == 1 ? (nb + 3) / 4 * 4 : (nb + 3) / 4 * 4 + 4; }
// eigenvalues in FP64 next to an FP64 Q, in FP32 otherwise
__host__ __device__ constexpr int eig_mu_bytes(int esz) { return esz == 8 ? 8 : 4; }
__host__ __device__ constexpr int64_t eig_cell_bytes_c(int nb, int esz) {
  return ((int64_t)nb * eig_nbp(nb) * esz + (int64_t)eig_nbp(nb) * eig_mu_bytes(esz) + 15) / 16 * 16;
}

// tensor-core variant: Q padded to NQ x NQ (16, 32 or 64 rows of 32, 64 or 128 bytes)
__host__ __device__ constexpr int eig_tc_nq(int nb) { return nb <= 16 ? 16 : nb <= 32 ? 32 : 64; }

constexpr int kEigThreads = 256;
constexpr int kMaxSweeps = 24;

__device__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
  return t;
}

template <int DIM, int N>
__global__ void __launch_bounds__(kEigThreads)
eig_setup_kernel(GridDesc g, const double* __restrict__ geo, LocalTab lt, unsigned char* __restrict__ out, int prec) {
  constexpr int NB = DIM == 3 ? N * N * N : N * N;
  constexpr int NBP = eig_nbp(NB);
  constexpr int NPAIR = (NB + 1) / 2;
  extern __shared__ __align__(16) double sm[];
  double* A = sm;            // local stiffness -> C -> diagonalised C
  double* M = A + NB * NB;   // local mass -> Cholesky factor L (lower)
  double* U = M + NB * NB;   // scratch -> eigenvectors -> Q
  __shared__ int s_free[NB], s_loc[NB], s_m;
  __shared__ int s_p[NPAIR], s_q[NPAIR];
  __shared__ double s_c[NPAIR], s_s[NPAIR];
  __shared__ double s_red[kEigThreads / 32];
  __shared__ int s_done;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int64_t cell = blockIdx.x;
  const int cx = (int)(cell % g.N), cy = (int)((cell / g.N) % g.N);
  const int cz = DIM == 3 ? (int)(cell / ((int64_t)g.N * g.N)) : 0;
  assemble_local<DIM, N>(g, geo, lt, cx, cy, cz, A, M);
  if (tid == 0) {
    int m = 0;
    for (int a = 0; a < NB; ++a) {
      const int gx = cx * g.p + a % N, gy = cy * g.p + (a / N) % N;
      bool bnd = on_boundary(gx, g.nn1) || on_boundary(gy, g.nn1);
      if (DIM == 3) bnd = bnd || on_boundary(cz * g.p + a / (N * N), g.nn1);
      s_loc[a] = bnd ? -1 : m;
      if (!bnd) s_free[m++] = a;
    }
    s_m = m;
  }
  __syncthreads();
  const int m = s_m;
  // compress A and M to the unconstrained nodes (row stride m)
  for (int i = tid; i < m * m; i += nth) U[i] = A[s_free[i / m] * NB + s_free[i % m]];
  __syncthreads();
  for (int i = tid; i < m * m; i += nth) A[i] = U[i];
  __syncthreads();
  for (int i = tid; i < m * m; i += nth) U[i] = M[s_free[i / m] * NB + s_free[i % m]];
  __syncthreads();
  for (int i = tid; i < m * m; i += nth) M[i] = U[i];
  __syncthreads();
  // Cholesky M = L L^T (right-looking, lower triangle)
  for (int k = 0; k < m; ++k) {
    if (tid == 0) M[k * m + k] = sqrt(M[k * m + k]);
    __syncthreads();
    for (int i = k + 1 + tid; i < m; i += nth) M[i * m + k] /= M[k * m + k];
    __syncthreads();
    const int rem = m - k - 1;
    for (int idx = tid; idx < rem * rem; idx += nth) {
      const int i = k + 1 + idx / rem, j = k + 1 + idx % rem;
      if (j <= i) M[i * m + j] -= M[i * m + k] * M[j * m + k];
    }
    __syncthreads();
  }
  // X = L^-1 A (columns in place), then C = L^-1 X^T
  for (int c = tid; c < m; c += nth)
    for (int i = 0; i < m; ++i) {
      double x = A[i * m + c];
      for (int l = 0; l < i; ++l) x -= M[i * m + l] * A[l * m + c];
      A[i * m + c] = x / M[i * m + i];
    }
  __syncthreads();
  for (int i = tid; i < m * m; i += nth) U[i] = A[(i % m) * m + i / m];
  __syncthreads();
  for (int c = tid; c < m; c += nth)
    for (int i = 0; i < m; ++i) {
      double x = U[i * m + c];
      for (int l = 0; l < i; ++l) x -= M[i * m + l] * U[l * m + c];
      U[i * m + c] = x / M[i * m + i];
    }
  __syncthreads();
  for (int i = tid; i < m * m; i += nth) A[i] = 0.5 * (U[i] + U[(i % m) * m + i / m]);
  __syncthreads();
  for (int i = tid; i < m * m; i += nth) U[i] = (i / m == i % m) ? 1.0 : 0.0;
  __syncthreads();
  // cyclic Jacobi, round-robin pairs: position 0 fixed, the others rotate; an odd m adds a dummy
  const int me = m + (m & 1), npairs = me / 2;
  for (int sweep = 0; sweep < kMaxSweeps && m > 1; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = tid; i < m * m; i += nth) {
      const double v = A[i] * A[i];
      tot += v;
      if (i / m != i % m) off += v;
    }
    off = block_sum(off, s_red);
    tot = block_sum(tot, s_red);
    if (tid == 0) s_done = off <= 1e-30 * tot;
    __syncthreads();
    if (s_done) break;
    for (int r = 0; r < me - 1; ++r) {
      if (tid < npairs) {
        auto pos = [&](int k) { return k == 0 ? 0 : 1 + (k - 1 + r) % (me - 1); };
        int p = pos(tid), q = pos(me - 1 - tid);
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < m) {
          const double app = A[p * m + p], aqq = A[q * m + q], apq = A[p * m + q];
          if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        } else {
          p = -1;
        }
        s_p[tid] = p; s_q[tid] = q; s_c[tid] = c; s_s[tid] = s;
      }
      __syncthreads();
      for (int idx = tid; idx < npairs * m; idx += nth) {  // rows p, q
        const int pr = idx / m, k = idx % m, p = s_p[pr];
        if (p < 0) continue;
        const int q = s_q[pr];
        const double c = s_c[pr], s = s_s[pr], ap = A[p * m + k], aq = A[q * m + k];
        A[p * m + k] = c * ap - s * aq;
        A[q * m + k] = s * ap + c * aq;
      }
      __syncthreads();
      for (int idx = tid; idx < npairs * m; idx += nth) {  // columns p, q of A and of U
        const int pr = idx / m, k = idx % m, p = s_p[pr];
        if (p < 0) continue;
        const int q = s_q[pr];
        const double c = s_c[pr], s = s_s[pr];
        const double ap = A[k * m + p], aq = A[k * m + q];
        A[k * m + p] = c * ap - s * aq;
        A[k * m + q] = s * ap + c * aq;
        const double up = U[k * m + p], uq = U[k * m + q];
        U[k * m + p] = c * up - s * uq;
        U[k * m + q] = s * up + c * uq;
      }
      __syncthreads();
    }
  }
  // Q = L^-T U (back substitution, columns in place)
  for (int c = tid; c < m; c += nth)
    for (int i = m - 1; i >= 0; --i) {
      double x = U[i * m + c];
      for (int l = i + 1; l < m; ++l) x -= M[l * m + i] * U[l * m + c];
      U[i * m + c] = x / M[i * m + i];
    }
  __syncthreads();
  if (prec == 3) {
    // tensor-core operand image: Q padded to NQ x NQ, rows of NQ BF16, the 16-byte chunks of each row
    // permuted by the swizzle of the row width (the pattern TMA and the tensor core use), eigenvalues apart
    constexpr int NQ = eig_tc_nq(NB);
    constexpr uint32_t mask = NQ == 16 ? 1u : NQ == 32 ? 3u : 7u;
    unsigned char* img = out + cell * (int64_t)NQ * NQ * 2;
    for (int idx = tid; idx < NQ * NQ; idx += nth) {
      const int a = idx / NQ, j = idx % NQ;
      const int ia = a < NB ? s_loc[a] : -1;
      const double v = (ia >= 0 && j < m) ? U[ia * m + j] : 0.0;
      const uint32_t o = (uint32_t)(a * NQ * 2 + 2 * j);
      const uint32_t sw = o ^ (((o >> 7) & mask) << 4);
      *reinterpret_cast<__nv_bfloat16*>(img + sw) = __float2bfloat16((float)v);
    }
    float* mu = reinterpret_cast<float*>(out + (int64_t)g.n_cells * NQ * NQ * 2) + cell * NQ;
    for (int j = tid; j < NQ; j += nth) mu[j] = j < m ? (float)A[j * m + j] : 1.0f;
    return;
  }
  const int esz = prec == 0 ? 8 : prec == 1 ? 4 : 2;
  unsigned char* blk = out + cell * eig_cell_bytes_c(NB, esz);
  for (int idx = tid; idx < NB * NBP; idx += nth) {
    const int a = idx / NBP, j = idx % NBP, ia = s_loc[a];
    const double v = (ia >= 0 && j < m) ? U[ia * m + j] : 0.0;
    if (prec == 0) reinterpret_cast<double*>(blk)[idx] = v;
    else if (prec == 1) reinterpret_cast<float*>(blk)[idx] = (float)v;
    else reinterpret_cast<__nv_bfloat16*>(blk)[idx] = __float2bfloat16((float)v);
  }
  unsigned char* mu = blk + (int64_t)NB * NBP * esz;
  for (int j = tid; j < NBP; j += nth) {
    const double v = j < m ? A[j * m + j] : 1.0;
    if (prec == 0) reinterpret_cast<double*>(mu)[j] = v;
    else reinterpret_cast<float*>(mu)[j] = (float)v;
  }
}

// ---- apply ----
template <typename TI> __device__ __forceinline__ float ld_f(const TI* p);
template <> __device__ __forceinline__ float ld_f<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ld_f<double>(const double* p) { return (float)*p; }
template <> __device__ __forceinline__ float ld_f<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(*p); }
template <typename T, typename TI> __device__ __forceinline__ T ld_t(const TI* p) { return (T)ld_f<TI>(p); }
template <> __device__ __forceinline__ double ld_t<double, double>(const double* p) { return *p; }

// four consecutive entries of a row (8-byte aligned for BF16, 16 for FP32, 32 for FP64)
__device__ __forceinline__ float4 row4(const __nv_bfloat16* p) {
  const uint2 w = *reinterpret_cast<const uint2*>(p);
  return make_float4(__uint_as_float(w.x << 16), __uint_as_float(w.x & 0xffff0000u), __uint_as_float(w.y << 16),
                     __uint_as_float(w.y & 0xffff0000u));
}
__device__ __forceinline__ float4 row4(const float* p) { return *reinterpret_cast<const float4*>(p); }

template <int DIM, int N, int NT, typename TI>
struct EigCfg {
  static constexpr int NB = DIM == 3 ? N * N * N : N * N;
  static constexpr int NBP = eig_nbp(NB);
  static constexpr int CELL_BYTES = (int)eig_cell_bytes_c(NB, (int)sizeof(TI));
  static constexpr int CPG0 = 128 / NB;
  static constexpr int CPG_MEM = 24576 / CELL_BYTES;
  static constexpr int CPG = CPG0 < CPG_MEM ? (CPG0 > 0 ? CPG0 : 1) : (CPG_MEM > 0 ? CPG_MEM : 1);
  static constexpr int THREADS = (CPG * NB + 31) / 32 * 32;
  static constexpr int STAGE_BYTES = CPG * CELL_BYTES;
  static constexpr int S = 2;
  static constexpr size_t SMEM = (size_t)S * STAGE_BYTES;
};

template <int DIM, int N, int NT, typename T, typename TI, bool MULTI>
__global__ void __launch_bounds__(EigCfg<DIM, N, NT, TI>::THREADS)
eig_apply_kernel(const T* __restrict__ r, T* __restrict__ u, const unsigned char* __restrict__ inv, GridDesc g,
                 ModeTab<T> mt, const T* __restrict__ copy_src, T* __restrict__ copy_dst, int* status, int nslab_arg,
                 int64_t slab_stride) {
  const int nslab = MULTI ? nslab_arg : 1;
  pdl_wait();
  pdl_trigger();
  using C = EigCfg<DIM, N, NT, TI>;
  constexpr int NB = C::NB, NBP = C::NBP, CPG = C::CPG, S = C::S;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[S];
  __shared__ __align__(16) T s_r[CPG][NT][NBP];  // modal residual (rows: time modes, columns: nodes)
  __shared__ __align__(16) T s_z[CPG][NT][NBP];  // eigen-coefficients scaled by 1 / (lambda + mu)
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  const int64_t ngroups = (g.n_cells + CPG - 1) / CPG;
  auto group_bytes = [&](int64_t grp) -> uint32_t {
    const int64_t c0 = grp * CPG;
    const int64_t nc = g.n_cells - c0 < CPG ? g.n_cells - c0 : CPG;
    return (uint32_t)(nc * C::CELL_BYTES);
  };
  if (tid == 0) s_fail = *reinterpret_cast<const volatile int*>(status);
  for (int i = tid; i < CPG * NT * NBP; i += blockDim.x) {
    (&s_r[0][0][0])[i] = T(0);
    (&s_z[0][0][0])[i] = T(0);
  }
  __syncthreads();
  if (s_fail) return;
  if (tid == 0) {
    for (int s = 0; s < S; ++s) tc::mbar_init(&bar[s], 1);
    tc::mbar_fence_init();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  int64_t issued = 0;
  if (tid == 0)
    for (int s = 0; s < S; ++s) {
      const int64_t grp = blockIdx.x + (int64_t)s * gridDim.x;
      if (grp < ngroups)
        tc::bulk_load(smem_raw + (size_t)s * C::STAGE_BYTES, inv + grp * CPG * (int64_t)C::CELL_BYTES, group_bytes(grp),
                      &bar[s]);
    }
  for (int s = 0; s < S; ++s)
    if (blockIdx.x + (int64_t)s * gridDim.x < ngroups) ++issued;
  int64_t k = 0;
  const int slot = tid / NB, a = tid - slot * NB;
  struct Pre { int64_t node; bool active, live; T w; T rr[NT], cp[NT]; };
  auto prefetch = [&](int64_t grp, int sl, Pre& P) {
    const int64_t cell = grp * CPG + slot;
    P.active = grp < ngroups && slot < CPG && cell < g.n_cells;
    P.live = false;
    P.node = 0;
    P.w = T(1);
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
    if (mt.weighted) P.w = node_weight<T>(gx, gy, gz, DIM, g.p);
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
      if (sl == 0 && !tc::mbar_wait_bounded(&bar[stage], parity, status)) {
        atomicExch(status, STMG_DEVICE_TIMEOUT);
        s_fail = 1;
      }
      __syncthreads();
      if (s_fail) break;
      const unsigned char* blk = smem_raw + (size_t)stage * C::STAGE_BYTES + (size_t)slot * C::CELL_BYTES;
      const TI* Q = reinterpret_cast<const TI*>(blk);
      using MuT = typename std::conditional<sizeof(TI) == 8, double, float>::type;
      const MuT* mu = reinterpret_cast<const MuT*>(blk + (size_t)NB * NBP * sizeof(TI));
      if (active) {
        // y = Q^T s for eigenvector j = a, all time modes at once; then z_hat = y / (lambda + mu_j)
        T y[NT];
#pragma unroll
        for (int m = 0; m < NT; ++m) y[m] = 0;
#pragma unroll 9
        for (int b = 0; b < NB; ++b) {
          const T q = ld_t<T, TI>(Q + b * NBP + a);
#pragma unroll
          for (int m = 0; m < NT; ++m) y[m] += q * s_r[slot][m][b];
        }
        const T muj = (T)mu[a];
#pragma unroll
        for (int m = 0; m < NT; ++m) {
          if (m < mt.nreal) {
            s_z[slot][m][a] = y[m] / (mt.lre[m] + muj);
          } else if (m + 1 < NT && ((m - mt.nreal) & 1) == 0) {
            const int mode = mt.nreal + (m - mt.nreal) / 2;
            const T dr = mt.lre[mode] + muj, di = mt.lim[mode];
            const T inv_den = T(1) / (dr * dr + di * di);
            s_z[slot][m][a] = (y[m] * dr + y[m + 1] * di) * inv_den;
            s_z[slot][m + 1][a] = (y[m + 1] * dr - y[m] * di) * inv_den;
          }
        }
      }
      __syncthreads();
      if (active && live) {
        // z = Q z_hat for node a (row a of Q), all modes at once
        T z[NT];
#pragma unroll
        for (int m = 0; m < NT; ++m) z[m] = 0;
        if constexpr (std::is_same<T, float>::value && !std::is_same<TI, double>::value) {
          // row a four entries at a time (padding entries of Q and of s_z are zero)
#pragma unroll 4
          for (int j = 0; j < NBP; j += 4) {
            const float4 q = row4(Q + a * NBP + j);
#pragma unroll
            for (int m = 0; m < NT; ++m) {
              const float4 v = *reinterpret_cast<const float4*>(&s_z[slot][m][j]);
              z[m] += q.x * v.x + q.y * v.y + q.z * v.z + q.w * v.w;
            }
          }
        } else {
#pragma unroll 9
          for (int j = 0; j < NB; ++j) {
            const T q = ld_t<T, TI>(Q + a * NBP + j);
#pragma unroll
            for (int m = 0; m < NT; ++m) z[m] += q * s_z[slot][m][j];
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
          atomicAdd(u + t * g.n_nodes + node, mt.omega * cur.w * o);
        }
      }
      __syncthreads();  // s_r, s_z free again (and, after the last slab, the stage)
      if (sl + 1 < nslab) cur = nxt;
    }
    if (s_fail) break;
    const int64_t next = grp + (int64_t)S * gridDim.x;
    if (next < ngroups) {
      if (tid == 0)
        tc::bulk_load(smem_raw + (size_t)stage * C::STAGE_BYTES, inv + next * CPG * (int64_t)C::CELL_BYTES,
                      group_bytes(next), &bar[stage]);
      ++issued;
    }
    cur = nxt;
  }
  if (s_fail) {
    for (int64_t q = k; q < issued; ++q) tc::mbar_wait_bounded(&bar[q % S], (uint32_t)((q / S) & 1), nullptr);
  }
}

// ---- tensor-core sweep ----
// A CTA of 128 threads owns tiles of CPT = 128 / NQ consecutive cells; thread t is accumulator row t =
// (cell c = t / NQ, local node or eigenvector index a = t % NQ).  Per tile the Q images of its cells arrive
// by one bulk copy (two stages); per round (all slabs of the system at once when they fit, NSL <= 8):
//   1. threads write the modal residual of their node, split into BF16 high and low parts, into the
//      right-hand-side operand B_c of their cell (rows = (part, slab, time mode), K = node);
//   2. one thread issues, per cell c, D_c = Q_stack^T B_c^T on the tensor cores: A = the tile's Q images
//      read M-major (M = (cell, eigenvector index), each cell one swizzle column), so the rows of cell c
//      hold Q_c^T s_c (the other cells' rows are not read);
//   3. threads read their row of D_c from tensor memory, add the two parts, divide by lambda_m + mu_j and
//      write z_hat (again as two BF16 parts) into B_c;
//   4. per cell, D_c = Q_stack B_c^T with A read K-major (rows (cell, node), K = eigenvector index);
//   5. threads read their row (node a of cell c), add the parts, transform back to the time basis and
//      add omega w_a times it to u with atomics.
template <int DIM, int N, int NT, int NSL>
struct EigTcCfg {
  static constexpr int NB = DIM == 3 ? N * N * N : N * N;
  static constexpr int NQ = eig_tc_nq(NB);
  static constexpr int CPT = 128 / NQ;
  static constexpr int RB = NQ * 2;
  static constexpr uint32_t ATOM = 8 * RB;
  static constexpr tc::Swizzle SW = NQ == 16 ? tc::kSw32 : NQ == 32 ? tc::kSw64 : tc::kSw128;
  static constexpr uint32_t SWMASK = NQ == 16 ? 1u : NQ == 32 ? 3u : 7u;
  static constexpr int CELL_Q = NQ * NQ * 2;
  static constexpr int TILE_Q = CPT * CELL_Q;
  // right-hand sides of one cell: slabs x time modes, each as a high and a low BF16 part for one slab
  // (16 rows either way), the high part alone for several slabs (precision of Q itself, 8 bits)
  static constexpr int PARTS = NSL == 1 ? 2 : 1;
  static constexpr int NR = PARTS * NT * NSL;
  // N of the MMAs and the column stride of the cells' accumulators in tensor memory: a power of two
  // (16, 32 or 64), so that every accumulator starts on a multiple of its own width
  static constexpr int NP = NR <= 16 ? 16 : NR <= 32 ? 32 : 64;
  static constexpr int B_CELL = NP * RB;
  static constexpr int B_BYTES = CPT * B_CELL;
  static constexpr int S = 2;
  static constexpr size_t SMEM = (size_t)S * TILE_Q + B_BYTES + 1024;
  static constexpr uint32_t TMEM_COLS = CPT * NP <= 32 ? 32 : CPT * NP <= 64 ? 64 : CPT * NP <= 128 ? 128
                                        : CPT * NP <= 256 ? 256 : 512;
  static_assert(NR <= 64, "at most 64 right-hand-side rows per cell");
};

// This thread's accumulator row (TMEM lane = thread index) in the column block of its cell c.  The load
// is warp-collective: a warp that spans several cells (NQ = 16) loads every cell's block and keeps its own.
template <int NP, int NQ>
__device__ __forceinline__ void load_row(uint32_t tmem, int warp, int c, float (&v)[NP]) {
  constexpr int CPW = NQ >= 32 ? 1 : 32 / NQ;
#pragma unroll
  for (int i = 0; i < CPW; ++i) {
    const int cw = (32 * warp) / NQ + i;
#pragma unroll
    for (int c0 = 0; c0 < NP; c0 += 16) {
      float t16[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(cw * NP + c0), t16);
      if (cw == c) {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[c0 + j] = t16[j];
      }
    }
  }
}

__device__ __forceinline__ void store_bf16_swz(unsigned char* base, uint32_t o, uint32_t mask, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + (o ^ (((o >> 7) & mask) << 4))) = __float2bfloat16(v);
}

template <int DIM, int N, int NT, int NSL>
__global__ void __launch_bounds__(128)
eig_tc_kernel(const float* __restrict__ r, float* __restrict__ u, const unsigned char* __restrict__ qimg,
              const float* __restrict__ mu_all, GridDesc g, ModeTab<float> mt, const float* __restrict__ copy_src,
              float* __restrict__ copy_dst, int* status, int nslab, int64_t slab_stride) {
  pdl_wait();
  pdl_trigger();
  using C = EigTcCfg<DIM, N, NT, NSL>;
  constexpr int NB = C::NB, NQ = C::NQ, CPT = C::CPT, S = C::S;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[S], mma_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail, s_ok;
  unsigned char* ring = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* bops = ring + (size_t)S * C::TILE_Q;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int c = tid / NQ, a = tid % NQ;
  const int64_t ntiles = (g.n_cells + CPT - 1) / CPT;
  auto tile_bytes = [&](int64_t tl) -> uint32_t {
    const int64_t c0 = tl * CPT;
    const int64_t nc = g.n_cells - c0 < CPT ? g.n_cells - c0 : CPT;
    return (uint32_t)(nc * C::CELL_Q);
  };
  if (tid == 0) {
    s_fail = *reinterpret_cast<const volatile int*>(status);
    for (int s = 0; s < S; ++s) tc::mbar_init(&bar[s], 1);
    tc::mbar_init(&mma_bar, 1);
    tc::mbar_fence_init();
  }
  for (int i = tid; i < C::B_BYTES / 16; i += 128) reinterpret_cast<uint4*>(bops)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) tc::tmem_alloc(&tmem_base, C::TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  const bool skip = s_fail != 0;
  int64_t issued = 0, k = 0;
  uint32_t mma_phase = 0;
  int pending = -1;  // parity of an MMA round whose completion a wait gave up on
  if (!skip) {
    if (tid == 0)
      for (int s = 0; s < S; ++s) {
        const int64_t tl = blockIdx.x + (int64_t)s * gridDim.x;
        if (tl < ntiles) tc::bulk_load(ring + (size_t)s * C::TILE_Q, qimg + tl * (int64_t)C::TILE_Q, tile_bytes(tl), &bar[s]);
      }
    for (int s = 0; s < S; ++s)
      if (blockIdx.x + (int64_t)s * gridDim.x < ntiles) ++issued;
  }
  unsigned char* Bc = bops + (size_t)c * C::B_CELL;
  constexpr uint32_t idesc_t = tc::idesc_bf16_f32(128, C::NP) | (1u << 15);  // A read M-major (Q^T)
  constexpr uint32_t idesc_n = tc::idesc_bf16_f32(128, C::NP);               // A read K-major (Q)
  const int nsl = NSL > 1 ? nslab : 1;
  for (int64_t tl = blockIdx.x; tl < ntiles && !skip; tl += gridDim.x, ++k) {
    const int stage = (int)(k % S);
    const uint32_t parity = (uint32_t)((k / S) & 1);
    const int64_t cell = tl * CPT + c;
    const int ncells = (int)(g.n_cells - tl * CPT < CPT ? g.n_cells - tl * CPT : CPT);
    const bool active = cell < g.n_cells && a < NB;
    bool live = false;
    int64_t node = 0;
    float w = 1.f, muj = 1.f;
    if (active) {
      int cx, cy, cz;
      cell_xyz(cell, g, cx, cy, cz);
      const int gx = cx * g.p + a % N, gy = cy * g.p + (a / N) % N;
      const int gz = DIM == 3 ? cz * g.p + a / (N * N) : 0;
      bool bnd = on_boundary(gx, g.nn1) || on_boundary(gy, g.nn1);
      if (DIM == 3) bnd = bnd || on_boundary(gz, g.nn1);
      node = gx + (int64_t)g.nn1 * (gy + (int64_t)g.nn1 * gz);
      live = !bnd;
      if (mt.weighted) w = node_weight<float>(gx, gy, gz, DIM, g.p);
    }
    if (cell < g.n_cells) muj = __ldg(mu_all + cell * NQ + a);
    // 1. modal residual of every slab into B_c (all slabs' loads issued before the first use); side job
    float rr[NSL][NT];
#pragma unroll
    for (int sl = 0; sl < NSL; ++sl)
#pragma unroll
      for (int t = 0; t < NT; ++t)
        rr[sl][t] = (sl < nsl && live) ? r[(int64_t)sl * slab_stride + t * g.n_nodes + node] : 0.f;
    if (copy_dst && active) {
#pragma unroll 1
      for (int sl = 0; sl < nsl; ++sl)
#pragma unroll
        for (int t = 0; t < NT; ++t)
          copy_dst[(int64_t)sl * slab_stride + t * g.n_nodes + node] = copy_src[(int64_t)sl * slab_stride + t * g.n_nodes + node];
    }
#pragma unroll
    for (int sl = 0; sl < NSL; ++sl) {
      if (sl >= nsl) break;
#pragma unroll
      for (int m = 0; m < NT; ++m) {
        const bool is_real = m < mt.nreal;
        const int mode = is_real ? m : mt.nreal + (m - mt.nreal) / 2;
        const bool im_part = !is_real && ((m - mt.nreal) & 1);
        float v = 0.f;
#pragma unroll
        for (int t = 0; t < NT; ++t) v += (im_part ? mt.Wi[mode][t] : mt.Wr[mode][t]) * rr[sl][t];
        const float hi = __bfloat162float(__float2bfloat16(v));
        store_bf16_swz(Bc, (uint32_t)((sl * NT + m) * C::RB + 2 * a), C::SWMASK, hi);
        if (C::PARTS == 2) store_bf16_swz(Bc, (uint32_t)((NT * NSL + sl * NT + m) * C::RB + 2 * a), C::SWMASK, v - hi);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0 && !tc::mbar_wait_bounded(&bar[stage], parity, status)) {
      atomicExch(status, STMG_DEVICE_TIMEOUT);
      s_fail = 1;
    }
    __syncthreads();
    if (s_fail) break;
    const uint32_t qa = tc::smem_addr(ring + (size_t)stage * C::TILE_Q);
    const uint32_t ba = tc::smem_addr(bops);
    // 2. y = Q^T s per cell
    if (tid == 0) {
      tc::fence_after_sync();
      for (int cc = 0; cc < ncells; ++cc)
#pragma unroll
        for (int ks = 0; ks < NQ / 16; ++ks) {
          const uint64_t ad = tc::smem_desc(qa + ks * 2 * C::ATOM, C::CELL_Q, C::ATOM, C::SW);
          const uint64_t bd = tc::smem_desc(ba + cc * C::B_CELL + ks * 32, 16, C::ATOM, C::SW);
          tc::mma_bf16(tmem + (uint32_t)(cc * C::NP), ad, bd, idesc_t, ks > 0 ? 1u : 0u);
        }
      tc::mma_commit(&mma_bar);
    }
    // one thread waits for the MMA round (the others sleep at the barrier instead of polling)
    if (tid == 0) s_ok = tc::mbar_wait_bounded(&mma_bar, mma_phase, status) ? 1 : 0;
    __syncthreads();
    bool ok = s_ok != 0;
    if (!ok) pending = (int)mma_phase;
    mma_phase ^= 1u;
    tc::fence_after_sync();
    // 3. z_hat = y / (lambda + mu_a) into B_c
    {
      float v[C::NP];
      load_row<C::NP, NQ>(tmem, warp, c, v);
#pragma unroll
      for (int sl = 0; sl < NSL; ++sl) {
        if (sl >= nsl) break;
        float y[NT];
#pragma unroll
        for (int m = 0; m < NT; ++m) y[m] = v[sl * NT + m] + (C::PARTS == 2 ? v[NT * NSL + sl * NT + m] : 0.f);
        float zh[NT];
#pragma unroll
        for (int m = 0; m < NT; ++m) {
          if (m < mt.nreal) {
            zh[m] = y[m] / (mt.lre[m] + muj);
          } else if (m + 1 < NT && ((m - mt.nreal) & 1) == 0) {
            const int mode = mt.nreal + (m - mt.nreal) / 2;
            const float dr = mt.lre[mode] + muj, di = mt.lim[mode];
            const float inv_den = 1.f / (dr * dr + di * di);
            zh[m] = (y[m] * dr + y[m + 1] * di) * inv_den;
            zh[m + 1] = (y[m + 1] * dr - y[m] * di) * inv_den;
          }
        }
#pragma unroll
        for (int m = 0; m < NT; ++m) {
          const float hi = __bfloat162float(__float2bfloat16(zh[m]));
          store_bf16_swz(Bc, (uint32_t)((sl * NT + m) * C::RB + 2 * a), C::SWMASK, hi);
          if (C::PARTS == 2)
            store_bf16_swz(Bc, (uint32_t)((NT * NSL + sl * NT + m) * C::RB + 2 * a), C::SWMASK, zh[m] - hi);
        }
      }
    }
    tc::fence_before_sync();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // 4. z = Q z_hat per cell
    if (tid == 0 && ok) {
      tc::fence_after_sync();
      for (int cc = 0; cc < ncells; ++cc)
#pragma unroll
        for (int ks = 0; ks < NQ / 16; ++ks) {
          const uint64_t ad = tc::smem_desc(qa + ks * 32, 16, C::ATOM, C::SW);
          const uint64_t bd = tc::smem_desc(ba + cc * C::B_CELL + ks * 32, 16, C::ATOM, C::SW);
          tc::mma_bf16(tmem + (uint32_t)(cc * C::NP), ad, bd, idesc_n, ks > 0 ? 1u : 0u);
        }
      tc::mma_commit(&mma_bar);
    }
    if (ok) {
      if (tid == 0) s_ok = tc::mbar_wait_bounded(&mma_bar, mma_phase, status) ? 1 : 0;
      __syncthreads();
      ok = s_ok != 0;
      if (!ok) pending = (int)mma_phase;
      mma_phase ^= 1u;
    }
    tc::fence_after_sync();
    // 5. back to the time basis, weighted atomics
    {
      float v[C::NP];
      load_row<C::NP, NQ>(tmem, warp, c, v);
      if (ok && active && live) {
#pragma unroll
        for (int sl = 0; sl < NSL; ++sl) {
          if (sl >= nsl) break;
          float z[NT];
#pragma unroll
          for (int m = 0; m < NT; ++m) z[m] = v[sl * NT + m] + (C::PARTS == 2 ? v[NT * NSL + sl * NT + m] : 0.f);
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            float o = 0.f;
#pragma unroll
            for (int m = 0; m < NT; ++m) {
              if (m < mt.nreal) {
                o += mt.Vr[t][m] * z[m];
              } else if (m + 1 < NT && ((m - mt.nreal) & 1) == 0) {
                const int mode = mt.nreal + (m - mt.nreal) / 2;
                o += 2.f * (mt.Vr[t][mode] * z[m] - mt.Vi[t][mode] * z[m + 1]);
              }
            }
            atomicAdd(u + (int64_t)sl * slab_stride + t * g.n_nodes + node, mt.omega * w * o);
          }
        }
      }
    }
    if (!ok && tid == 0) {
      atomicExch(status, STMG_DEVICE_TIMEOUT);
      s_fail = 1;
    }
    tc::fence_before_sync();
    __syncthreads();  // B operands, tensor memory and the stage are free again
    if (s_fail) break;
    const int64_t next = tl + (int64_t)S * gridDim.x;
    if (next < ntiles) {
      if (tid == 0)
        tc::bulk_load(ring + (size_t)stage * C::TILE_Q, qimg + next * (int64_t)C::TILE_Q, tile_bytes(next), &bar[stage]);
      ++issued;
    }
  }
  if (s_fail) {
    // drain: copies still in flight, then any MMA round still running
    if (tid == 0) {
      for (int64_t q = k; q < issued; ++q) tc::mbar_wait_bounded(&bar[q % S], (uint32_t)((q / S) & 1), nullptr);
      if (pending >= 0) tc::mbar_wait_bounded(&mma_bar, (uint32_t)pending, nullptr);
    }
    __syncthreads();
  }
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

template <int DIM, int N, int NT, int NSL>
cudaError_t eig_tc_launch(const float* r, float* u, const void* inv, const GridDesc& g, const ModeTab<float>& mt,
                          const float* cs, float* cd, int* status, int nslab, int64_t ss, cudaStream_t s) {
  using C = EigTcCfg<DIM, N, NT, NSL>;
  auto k = eig_tc_kernel<DIM, N, NT, NSL>;
  static int per_sm = 0, sms = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // resident CTAs per SM from shared memory and tensor memory (every CTA holds TMEM_COLS of the SM's
    // 512 columns); the occupancy query reports one CTA per SM for kernels that allocate tensor memory
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    const int by_smem = smem_sm / (int)(C::SMEM + 1024);
    per_sm = std::max(1, std::min(std::min(by_smem, 16), 512 / (int)C::TMEM_COLS));
  }
  const unsigned char* img = reinterpret_cast<const unsigned char*>(inv);
  const float* mu = reinterpret_cast<const float*>(img + g.n_cells * (int64_t)C::CELL_Q);
  const int64_t tiles = (g.n_cells + C::CPT - 1) / C::CPT;
  const int64_t grid = std::min<int64_t>(tiles, (int64_t)sms * per_sm);
  const cudaError_t e = launch_k(k, dim3((unsigned)grid), dim3(128), C::SMEM, s, r, u, img, mu, g, mt, cs, cd, status,
                                 nslab, ss);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int DIM, int N, int NT>
cudaError_t eig_tc_t(const float* r, float* u, const void* inv, const GridDesc& g, const ModeTab<float>& mt,
                     const float* cs, float* cd, int* status, int nslab, int64_t ss, cudaStream_t s) {
  if (!status || nslab > 8) return cudaErrorInvalidValue;
  return nslab > 1 ? eig_tc_launch<DIM, N, NT, 8>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s)
                   : eig_tc_launch<DIM, N, NT, 1>(r, u, inv, g, mt, cs, cd, status, 1, ss, s);
}

template <int DIM, int N>
cudaError_t eig_setup_t(const GridDesc& g, const double* geo64, const LocalTab& lt, void* out, int prec,
                        cudaStream_t s) {
  constexpr int NB = DIM == 3 ? N * N * N : N * N;
  const size_t smem = (size_t)3 * NB * NB * sizeof(double);
  auto k = eig_setup_kernel<DIM, N>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)g.n_cells, kEigThreads, smem, s>>>(g, geo64, lt, reinterpret_cast<unsigned char*>(out), prec);
  return cudaGetLastError();
}

template <int DIM, int N, int NT, typename T, typename TI, bool MULTI>
cudaError_t eig_launch(const T* r, T* u, const void* inv, const GridDesc& g, const ModeTab<T>& mt, const T* cs, T* cd,
                       int* status, int nslab, int64_t ss, cudaStream_t s) {
  using C = EigCfg<DIM, N, NT, TI>;
  auto k = eig_apply_kernel<DIM, N, NT, T, TI, MULTI>;
  static int per_sm = 0, sms = 0;
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
  const cudaError_t e = launch_k(k, dim3((unsigned)grid), dim3(C::THREADS), C::SMEM, s, r, u,
                                 reinterpret_cast<const unsigned char*>(inv), g, mt, cs, cd, status, nslab, ss);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

template <int DIM, int N, int NT, typename T, typename TI>
cudaError_t eig_apply_t(const T* r, T* u, const void* inv, const GridDesc& g, const ModeTab<T>& mt, const T* cs, T* cd,
                        int* status, int nslab, int64_t ss, cudaStream_t s) {
  if (!status) return cudaErrorInvalidValue;
  return nslab > 1 ? eig_launch<DIM, N, NT, T, TI, true>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s)
                   : eig_launch<DIM, N, NT, T, TI, false>(r, u, inv, g, mt, cs, cd, status, 1, ss, s);
}

}  // namespace

int64_t eig_cell_bytes(int dim, int n, int esz) { return eig_cell_bytes_c(dim == 3 ? n * n * n : n * n, esz); }

int64_t eig_tc_bytes(int dim, int n, int64_t n_cells) {
  const int nb = dim == 3 ? n * n * n : n * n;
  if (nb > 64) return -1;
  const int nq = eig_tc_nq(nb);
  return n_cells * ((int64_t)nq * nq * 2 + (int64_t)nq * 4);
}

cudaError_t launch_eig_setup(int dim, int n, const GridDesc& g, const double* geo64, const LocalTab& lt, void* out,
                             int prec, cudaStream_t s) {
  if (prec < 0 || prec > 3) return cudaErrorInvalidValue;
  if (prec == 3 && (dim == 3 ? n * n * n : n * n) > 64) return cudaErrorInvalidValue;
  if (dim == 3) {
    if (n == 2) return eig_setup_t<3, 2>(g, geo64, lt, out, prec, s);
    if (n == 3) return eig_setup_t<3, 3>(g, geo64, lt, out, prec, s);
    if (n == 4) return eig_setup_t<3, 4>(g, geo64, lt, out, prec, s);
  } else {
    if (n == 2) return eig_setup_t<2, 2>(g, geo64, lt, out, prec, s);
    if (n == 3) return eig_setup_t<2, 3>(g, geo64, lt, out, prec, s);
    if (n == 4) return eig_setup_t<2, 4>(g, geo64, lt, out, prec, s);
    if (n == 5) return eig_setup_t<2, 5>(g, geo64, lt, out, prec, s);
  }
  return cudaErrorInvalidValue;
}

#define STMG_EIG_CASE(DIM, N, NT)                                                                            \
  if (dim == DIM && n == N && nt == NT) {                                                                    \
    if (prec == 0) return eig_apply_t<DIM, N, NT, T, double>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s); \
    if (prec == 1) return eig_apply_t<DIM, N, NT, T, float>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s);  \
    return eig_apply_t<DIM, N, NT, T, __nv_bfloat16>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s);         \
  }

template <typename T>
cudaError_t launch_eig_apply(int dim, int n, int nt, const T* r, T* u, const void* inv, int prec, const GridDesc& g,
                             const ModeTab<T>& mt, const T* cs, T* cd, int* status, int nslab, int64_t ss,
                             cudaStream_t s) {
  STMG_EIG_CASE(3, 2, 1) STMG_EIG_CASE(3, 2, 2) STMG_EIG_CASE(3, 2, 3) STMG_EIG_CASE(3, 2, 4)
  STMG_EIG_CASE(3, 3, 1) STMG_EIG_CASE(3, 3, 2) STMG_EIG_CASE(3, 3, 3) STMG_EIG_CASE(3, 3, 4)
  STMG_EIG_CASE(3, 4, 1) STMG_EIG_CASE(3, 4, 2) STMG_EIG_CASE(3, 4, 3) STMG_EIG_CASE(3, 4, 4)
  STMG_EIG_CASE(2, 2, 1) STMG_EIG_CASE(2, 2, 2) STMG_EIG_CASE(2, 2, 3) STMG_EIG_CASE(2, 2, 4)
  STMG_EIG_CASE(2, 3, 1) STMG_EIG_CASE(2, 3, 2) STMG_EIG_CASE(2, 3, 3) STMG_EIG_CASE(2, 3, 4)
  STMG_EIG_CASE(2, 4, 1) STMG_EIG_CASE(2, 4, 2) STMG_EIG_CASE(2, 4, 3) STMG_EIG_CASE(2, 4, 4)
  STMG_EIG_CASE(2, 5, 1) STMG_EIG_CASE(2, 5, 2) STMG_EIG_CASE(2, 5, 3) STMG_EIG_CASE(2, 5, 4)
  return cudaErrorInvalidValue;
}

template cudaError_t launch_eig_apply<float>(int, int, int, const float*, float*, const void*, int, const GridDesc&,
                                             const ModeTab<float>&, const float*, float*, int*, int, int64_t,
                                             cudaStream_t);
template cudaError_t launch_eig_apply<double>(int, int, int, const double*, double*, const void*, int, const GridDesc&,
                                              const ModeTab<double>&, const double*, double*, int*, int, int64_t,
                                              cudaStream_t);

}  // namespace stmg

namespace stmg {

#define STMG_EIG_TC_CASE(DIM, N, NT) \
  if (dim == DIM && n == N && nt == NT) return eig_tc_t<DIM, N, NT>(r, u, inv, g, mt, cs, cd, status, nslab, ss, s);

cudaError_t launch_eig_tc_apply(int dim, int n, int nt, const float* r, float* u, const void* inv, const GridDesc& g,
                                const ModeTab<float>& mt, const float* cs, float* cd, int* status, int nslab,
                                int64_t ss, cudaStream_t s) {
  STMG_EIG_TC_CASE(3, 2, 1) STMG_EIG_TC_CASE(3, 2, 2) STMG_EIG_TC_CASE(3, 2, 3) STMG_EIG_TC_CASE(3, 2, 4)
  STMG_EIG_TC_CASE(3, 3, 1) STMG_EIG_TC_CASE(3, 3, 2) STMG_EIG_TC_CASE(3, 3, 3) STMG_EIG_TC_CASE(3, 3, 4)
  STMG_EIG_TC_CASE(3, 4, 1) STMG_EIG_TC_CASE(3, 4, 2) STMG_EIG_TC_CASE(3, 4, 3) STMG_EIG_TC_CASE(3, 4, 4)
  STMG_EIG_TC_CASE(2, 2, 1) STMG_EIG_TC_CASE(2, 2, 2) STMG_EIG_TC_CASE(2, 2, 3) STMG_EIG_TC_CASE(2, 2, 4)
  STMG_EIG_TC_CASE(2, 3, 1) STMG_EIG_TC_CASE(2, 3, 2) STMG_EIG_TC_CASE(2, 3, 3) STMG_EIG_TC_CASE(2, 3, 4)
  STMG_EIG_TC_CASE(2, 4, 1) STMG_EIG_TC_CASE(2, 4, 2) STMG_EIG_TC_CASE(2, 4, 3) STMG_EIG_TC_CASE(2, 4, 4)
  STMG_EIG_TC_CASE(2, 5, 1) STMG_EIG_TC_CASE(2, 5, 2) STMG_EIG_TC_CASE(2, 5, 3) STMG_EIG_TC_CASE(2, 5, 4)
  return cudaErrorInvalidValue;
}

}  // namespace stmg
