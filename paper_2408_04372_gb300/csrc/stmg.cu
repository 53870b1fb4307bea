// Host side of libstmg: context, multigrid hierarchy, V-cycle, FGMRES and the C ABI (include/stmg.h).
#include <algorithm>
#include <type_traits>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/stmg.h"
#include "common.cuh"
#include "kernels.h"
#include "net.h"
#include "tables.h"

using namespace stmg;

namespace {

struct Level {
  int dim = 3, p = 1, n = 2, N = 2, k = 0, nt = 1;
  int nc = 1;          // slabs in the level's system (eq. heat-cg-dg-at-once), vectors [slab][N_t][node]
  double tau = 1.0;    // slab length on this level (doubles on tau-levels)
  GridDesc g{};
  std::vector<double> vertices;   // host (N+1)^dim x dim
  std::vector<double> rho_qp;     // host cells x (p+1)^dim
  double* geo64 = nullptr;
  float* geo32 = nullptr;
  df64* geodf = nullptr;         // finest level only, when the outer apply runs in double-float
  OpTab<df64> tabdf{};
  SlabCoeffs sc;
  OpTab<double> tab64{};
  OpTab<float> tab32{};
  // coupling -B of slab i to the last time DoF of slab i-1 (TM column N_t - 1 = -alpha), nc > 1
  OpTab<double> cpl64{};
  OpTab<float> cpl32{};
  LocalTab lt{};
  // smoother
  int nreal = 0, ncplx = 0;
  ModeTab<double> mt64{};
  ModeTab<float> mt32{};
  void* inv = nullptr;
  int inv_prec = 1;
  bool fd = false;             // fast diagonalisation instead of stored inverses
  bool eig = false;            // stored per-cell eigendecompositions (Q, mu) instead of inverse planes
  bool eig_tc = false;         // ... applied on the tensor cores (BF16 operand images, FP32 vectors)
  FDTab<double> fd64{};
  FDTab<float> fd32{};
  double* rho_cell64 = nullptr;
  float* rho_cell32 = nullptr;
  double omega = 1.0;
  // work vectors
  double *f64 = nullptr, *u64 = nullptr, *r64 = nullptr;
  float *f32 = nullptr, *u32 = nullptr, *r32 = nullptr;
  // transfer into this level from levels[l+1] (tkind 1 space, 2 time degree, 3 slab length, 0 none)
  int tkind = 0;
  Transfer1D tr{};
  TimeTransfer tt{};
  // coarsest level dense solve
  int n_coarse = 0;
  int64_t* cmap = nullptr;
  double* cinv64 = nullptr;
  float* cinv32 = nullptr;
  int64_t slab_size() const { return (int64_t)nt * g.n_nodes; }
  int64_t size() const { return (int64_t)nc * slab_size(); }
};

}  // namespace

// pinned host staging: Arnoldi columns (up to 66 values) of even iterations at 0, of odd ones here
constexpr int kColSlot = 192;

struct stmg_ctx {
  cudaStream_t stream = nullptr;       // private stream (graph capture needs a non-legacy stream)
  cudaStream_t user_stream = nullptr;  // caller's stream; every call is ordered after and before it
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaEvent_t ev_iter[2] = {nullptr, nullptr};  // end of FGMRES iteration j (slot j % 2): its column is on the host
  int dim = 3, pde = 0, scheme = 0;
  double tau = 1.0;
  stmg_options opt{};
  std::vector<Level> levels;
  std::string err;
  std::vector<void*> allocations;
  // FGMRES workspace
  int m = 30;
  int nvec = 0;
  double* V = nullptr;   // (nvec) vectors, stride vld
  int64_t vld = 0;       // stride of the Krylov basis: n0 rounded up to 32 (256-byte aligned vectors)
  double* Z = nullptr;   // (m) vectors
  float* Z32 = nullptr;  // (m) preconditioned vectors in FP32 (FP32 V-cycle with the double-float apply: exact)
  double* partial = nullptr;        // per-block partial sums of the Gram-Schmidt passes
  unsigned int* counter = nullptr;  // arrival counter of those passes (zero between launches)
  int* status = nullptr;            // device status word: nonzero after a bounded device wait gave up
  double* dsm = nullptr;  // device scalars [0..nvec+8) h1, [128..) h2, [256..) outputs
  double* hsm = nullptr;  // pinned host mirror: [0..) and [kColSlot..) Arnoldi columns of even / odd iterations
  double* tmp[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* rhs_buf = nullptr;
  double* u_buf = nullptr;
  cudaGraphExec_t graph32 = nullptr, graph64 = nullptr;
  int64_t graph32_kernels = 0, graph64_kernels = 0;
  // one FGMRES iteration per Krylov index j, per variant: bit 0 the relaxed (FP32) operator apply,
  // bit 1 the double-float Krylov basis (Gram-Schmidt on the FP32 pipe)
  std::vector<cudaGraphExec_t> iter_graphs[4];
  std::vector<int64_t> iter_graph_kernels[4];
  bool gs_df = false;  // this solve keeps its Krylov basis V in double-float pairs
  bool warmed32 = false, warmed64 = false;
  int64_t launches = 0;  // kernels issued by this context (graph replays count their kernel nodes)
  std::vector<stmg_net*> nets;  // networks bound to this context; detached when it is destroyed
  bool outer_df = false;        // FGMRES apply on V-cycle outputs in double-float (FP32 V-cycle only)
  int device = -1;                  // CUDA device current at stmg_create
  void* noalloc_scratch = nullptr;  // device address of the fixed smoothing scratch on that device
};

// A network outliving its context keeps only its own device memory; every later call on it
// except stmg_net_destroy returns STMG_ERR_INVALID_ARG.
extern "C" {
static void net_detach(stmg_net* net);
}

namespace {

#define CK(...)                                                                   \
  do {                                                                            \
    cudaError_t e_ = (__VA_ARGS__);                                               \
    if (e_ != cudaSuccess) {                                                      \
      ctx->err = std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_);       \
      return STMG_ERR_CUDA;                                                       \
    }                                                                             \
  } while (0)

#define CKS(...)                                                                  \
  do {                                                                            \
    stmg_status s_ = (__VA_ARGS__);                                               \
    if (s_ != STMG_OK) return s_;                                                 \
  } while (0)

template <typename T>
stmg_status dev_alloc(stmg_ctx* ctx, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? STMG_ERR_OOM : STMG_ERR_CUDA;
  }
  ctx->allocations.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return STMG_OK;
}

stmg_status invalid(stmg_ctx* ctx, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return STMG_ERR_INVALID_ARG;
}

// ---------------------------------------------------------------- level setup

struct Spec { int p, N, k, nc; double tau; };

// Coarsening in space first, then in time (Algorithm mg-sequence, Section 3.2).  p_coarsening: the
// space levels first lower p one by one down to 1, then halve the cells; otherwise they keep p and
// only halve the cells (h-multigrid).  With several slabs in one system (nc > 1), tau-levels merge
// pairs of slabs (tau -> 2 tau) while their number is even, before the k-levels.
int64_t level_unknowns(const Spec& sp, int dim, int scheme) {
  const int64_t in1 = (int64_t)sp.p * sp.N - 1;
  return (int64_t)sp.nc * (scheme == STMG_DG ? sp.k + 1 : sp.k) * (dim == 3 ? in1 * in1 * in1 : in1 * in1);
}

std::vector<Spec> level_sequence(int p, int N, int k, int scheme, bool p_coarsening, int nc, double tau) {
  std::vector<Spec> s{{p, N, k, nc, tau}};
  auto next = [&](int dp, int hN, int dk, int hc) {
    const Spec b = s.back();
    s.push_back({b.p - dp, b.N / hN, b.k - dk, b.nc / hc, b.tau * hc});
  };
  if (p_coarsening)
    while (s.back().p > 1) next(1, 1, 0, 1);
  while (s.back().N % 2 == 0 && s.back().N / 2 >= 2) next(0, 2, 0, 1);
  while (s.back().nc % 2 == 0) next(0, 1, 0, 2);
  const int kmin = scheme == STMG_DG ? 0 : 1;
  while (s.back().k > kmin) next(0, 1, 1, 1);
  return s;
}

void fill_tables(Level& L) {
  std::vector<double> xn = space_nodes(L.p), xq, wq;
  gauss_legendre(L.n, xq, wq);
  OpTab<double> t{};
  for (int q = 0; q < L.n; ++q)
    for (int i = 0; i < L.n; ++i) {
      t.B[q][i] = lagrange(xn, i, xq[q]);
      t.D[q][i] = lagrange_deriv(xq, i, xq[q]);
      L.lt.B[q][i] = t.B[q][i];
      L.lt.Dn[q][i] = lagrange_deriv(xn, i, xq[q]);
    }
  for (int i = 0; i < L.nt; ++i)
    for (int j = 0; j < L.nt; ++j) {
      t.TA[i][j] = L.sc.TA[i * L.nt + j];
      t.TM[i][j] = L.sc.TM[i * L.nt + j];
    }
  t.sign = 1.0;
  L.tab64 = t;
  OpTab<float> f{};
  for (int a = 0; a < kMaxN; ++a)
    for (int b = 0; b < kMaxN; ++b) { f.B[a][b] = (float)t.B[a][b]; f.D[a][b] = (float)t.D[a][b]; }
  for (int a = 0; a < kMaxNT; ++a)
    for (int b = 0; b < kMaxNT; ++b) { f.TA[a][b] = (float)t.TA[a][b]; f.TM[a][b] = (float)t.TM[a][b]; }
  f.sign = 1.0f;
  L.tab32 = f;
  OpTab<df64> d{};
  for (int a = 0; a < kMaxN; ++a)
    for (int b = 0; b < kMaxN; ++b) { d.B[a][b] = df_split(t.B[a][b]); d.D[a][b] = df_split(t.D[a][b]); }
  for (int a = 0; a < kMaxNT; ++a)
    for (int b = 0; b < kMaxNT; ++b) { d.TA[a][b] = df_split(t.TA[a][b]); d.TM[a][b] = df_split(t.TM[a][b]); }
  d.sign = df64(1.0f);
  L.tabdf = d;
}

template <typename T> OpTab<T>& tab_of(Level& L);
template <> OpTab<double>& tab_of<double>(Level& L) { return L.tab64; }
template <> OpTab<float>& tab_of<float>(Level& L) { return L.tab32; }
template <typename T> const T* geo_of(const Level& L);
template <> const double* geo_of<double>(const Level& L) { return L.geo64; }
template <> const float* geo_of<float>(const Level& L) { return L.geo32; }
template <typename T> ModeTab<T>& mt_of(Level& L);
template <> ModeTab<double>& mt_of<double>(Level& L) { return L.mt64; }
template <> ModeTab<float>& mt_of<float>(Level& L) { return L.mt32; }
template <typename T> T* fv(Level& L);
template <> double* fv<double>(Level& L) { return L.f64; }
template <> float* fv<float>(Level& L) { return L.f32; }
template <typename T> T* uv(Level& L);
template <> double* uv<double>(Level& L) { return L.u64; }
template <> float* uv<float>(Level& L) { return L.u32; }
template <typename T> T* rv(Level& L);
template <> double* rv<double>(Level& L) { return L.r64; }
template <> float* rv<float>(Level& L) { return L.r32; }
template <typename T> const FDTab<T>& fd_of(const Level& L);
template <> const FDTab<double>& fd_of<double>(const Level& L) { return L.fd64; }
template <> const FDTab<float>& fd_of<float>(const Level& L) { return L.fd32; }
template <typename T> const T* rho_of(const Level& L);
template <> const double* rho_of<double>(const Level& L) { return L.rho_cell64; }
template <> const float* rho_of<float>(const Level& L) { return L.rho_cell32; }
template <typename T> const T* cinv_of(const Level& L);
template <> const double* cinv_of<double>(const Level& L) { return L.cinv64; }
template <> const float* cinv_of<float>(const Level& L) { return L.cinv32; }

template <typename T> const OpTab<T>& cpl_of(const Level& L);
template <> const OpTab<double>& cpl_of<double>(const Level& L) { return L.cpl64; }
template <> const OpTab<float>& cpl_of<float>(const Level& L) { return L.cpl32; }

// y (+)= sign S x on unconstrained rows, slab by slab: the slab operator on the diagonal and the
// coupling -B to the previous slab's last time DoF below it (eq. heat-cg-dg-at-once)
template <typename T>
stmg_status apply_slabs(stmg_ctx* ctx, Level& L, const T* x, T* y, T sign) {
  OpTab<T> t = tab_of<T>(L);
  t.sign = sign;
  OpTab<T> c = cpl_of<T>(L);
  if (sign != T(1))
    for (int i = 0; i < kMaxNT; ++i) c.TM[i][L.nt - 1] *= sign;
  const int64_t ss = L.slab_size();
  for (int i = 0; i < L.nc; ++i) {
    CK(launch_apply<T>(L.dim, L.n, L.nt, x + i * ss, y + i * ss, geo_of<T>(L), L.g, t, 1, ctx->stream));
    if (i > 0) CK(launch_mass_couple<T, T, T>(L.dim, L.n, L.nt, x + (i - 1) * ss, y + i * ss, geo_of<T>(L), L.g, c,
                                              ctx->stream));
  }
  ctx->launches += 2 * L.nc - 1;
  return STMG_OK;
}

// y = S x (identity on constrained rows)
template <typename T>
stmg_status op_apply(stmg_ctx* ctx, Level& L, const T* x, T* y) {
  CK(launch_init_rows<T>(y, nullptr, x, L.g, L.nt * L.nc, 0, ctx->stream));
  ctx->launches += 1;
  return apply_slabs<T>(ctx, L, x, y, T(1));
}

// y = S x for an FP32 x, in double-float arithmetic, FP64 y (identity on constrained rows)
// (slab blocks in double-float; the coupling between slabs in FP64 from the FP32 input).  init false:
// y is already 0 and x vanishes on constrained rows (a V-cycle output), so no initialisation pass.
stmg_status op_apply_df(stmg_ctx* ctx, Level& L, const float* x, double* y, bool init = true) {
  if (!L.geodf) { ctx->err = "no double-float geometry on this level"; return STMG_ERR_UNSUPPORTED; }
  if (init) {
    CK(launch_init_rows_f2d(y, x, L.g, L.nt * L.nc, ctx->stream));
    ctx->launches += 1;
  }
  ctx->launches += 2 * L.nc - 1;
  OpTab<df64> t = L.tabdf;
  t.sign = df64(1.0f);
  const int64_t ss = L.slab_size();
  for (int i = 0; i < L.nc; ++i) {
    CK(launch_apply_df(L.dim, L.n, L.nt, x + i * ss, y + i * ss, L.geodf, L.g, t, 1, ctx->stream));
    if (i > 0)
      CK(launch_mass_couple<double, float, double>(L.dim, L.n, L.nt, x + (i - 1) * ss, y + i * ss, L.geo64, L.g,
                                                   L.cpl64, ctx->stream));
  }
  return STMG_OK;
}

// r = f - S u on the finest level for FGMRES.  df: the slab blocks in double-float arithmetic on u
// split into float pairs (FP32 pipe, about 44 bits; used when the stopping target is at least
// 1e-10 of ||b||, so that the residual's own error stays far below it), else FP64.
stmg_status op_residual_outer(stmg_ctx* ctx, Level& L, const double* f, const double* u, double* r, bool df);

// r = f - S u
template <typename T>
stmg_status op_residual(stmg_ctx* ctx, Level& L, const T* f, const T* u, T* r) {
  CK(launch_init_rows<T>(r, f, u, L.g, L.nt * L.nc, 1, ctx->stream));
  ctx->launches += 1;
  return apply_slabs<T>(ctx, L, u, r, T(-1));
}

stmg_status op_residual_outer(stmg_ctx* ctx, Level& L, const double* f, const double* u, double* r, bool df) {
  if (!df || !L.geodf) return op_residual<double>(ctx, L, f, u, r);
  CK(launch_init_rows<double>(r, f, u, L.g, L.nt * L.nc, 1, ctx->stream));
  OpTab<df64> t = L.tabdf;
  t.sign = df64(-1.0f);
  OpTab<double> c = L.cpl64;
  for (int i = 0; i < kMaxNT; ++i) c.TM[i][L.nt - 1] = -c.TM[i][L.nt - 1];
  const int64_t ss = L.slab_size();
  for (int i = 0; i < L.nc; ++i) {
    CK(launch_apply_df_d(L.dim, L.n, L.nt, u + i * ss, r + i * ss, L.geodf, L.g, t, 1, ctx->stream));
    if (i > 0)
      CK(launch_mass_couple<double, double, double>(L.dim, L.n, L.nt, u + (i - 1) * ss, r + i * ss, L.geo64, L.g, c,
                                                    ctx->stream));
  }
  ctx->launches += 2 * L.nc;
  return STMG_OK;
}

// u += omega * ASM r ; optionally also copy_dst := copy_src (a fused side job for the V-cycle)
template <typename T>
stmg_status op_asm(stmg_ctx* ctx, Level& L, const T* r, T* u, double omega, const T* copy_src = nullptr,
                   T* copy_dst = nullptr) {
  ModeTab<T> mt = mt_of<T>(L);
  mt.omega = (T)omega;
  // block diagonal over the slabs: every space-time cell lies in one slab (same local inverses)
  const int64_t ss = L.slab_size();
  if (L.eig_tc) {
    if constexpr (std::is_same<T, float>::value) {
      ctx->launches += 1;
      CK(launch_eig_tc_apply(L.dim, L.n, L.nt, r, u, L.inv, L.g, mt, copy_src, copy_dst, ctx->status, L.nc, ss,
                             ctx->stream));
      return STMG_OK;
    } else {
      ctx->err = "the tensor-core smoother takes FP32 vectors";
      return STMG_ERR_UNSUPPORTED;
    }
  }
  if (L.eig) {
    ctx->launches += 1;
    CK(launch_eig_apply<T>(L.dim, L.n, L.nt, r, u, L.inv, L.inv_prec, L.g, mt, copy_src, copy_dst, ctx->status, L.nc,
                           ss, ctx->stream));
    return STMG_OK;
  }
  if (!L.fd) {
    ctx->launches += 1;
    CK(launch_asm_apply<T>(L.dim, L.n, L.nt, r, u, L.inv, L.inv_prec, L.g, mt, copy_src, copy_dst, ctx->status, L.nc,
                           ss, ctx->stream));
    return STMG_OK;
  }
  ctx->launches += L.nc;
  for (int i = 0; i < L.nc; ++i) {
    const int64_t o = i * ss;
    CK(launch_fd_apply<T>(L.n, L.nt, r + o, u + o, rho_of<T>(L), L.g, fd_of<T>(L), mt, copy_src ? copy_src + o : nullptr,
                          copy_dst ? copy_dst + o : nullptr, ctx->stream));
  }
  return STMG_OK;
}

template <typename T>
stmg_status op_smooth(stmg_ctx* ctx, int l, int sweeps, const T* f, T* u, T* r) {
  Level& L = ctx->levels[l];
  for (int s = 0; s < sweeps; ++s) {
    CKS(op_residual<T>(ctx, L, f, u, r));
    CKS(op_asm<T>(ctx, L, r, u, L.omega));
  }
  return STMG_OK;
}

bool transfer_fused_host(int terms, int64_t n_out) { return terms <= 8 || (terms <= 27 && n_out < (int64_t)4 << 20); }

// r_{l+1} = R r_l ; optionally also zero_dst := 0 over the coarse vector (V-cycle side job)
template <typename T>
stmg_status op_restrict(stmg_ctx* ctx, int l, const T* rf, T* rc, T* zero_dst = nullptr) {
  Level& F = ctx->levels[l];
  Level& C = ctx->levels[l + 1];
  ctx->launches += 1;
  if (F.tkind == 1) {
    CK(launch_restrict_space<T>(rc, rf, F.g, C.g, F.nt * F.nc, F.tr, zero_dst, ctx->stream));
    const int R = F.tr.width_r;
    if (!transfer_fused_host(F.dim == 3 ? R * R * R : R * R, C.size())) ctx->launches += F.dim - 1;
  }
  else CK(launch_restrict_time<T>(rc, rf, F.g, F.tt, zero_dst, ctx->stream));
  return STMG_OK;
}

// u_l += P e_{l+1} ; optionally also copy_dst := copy_src over the fine vector (V-cycle side job)
template <typename T>
stmg_status op_prolongate_add(stmg_ctx* ctx, int l, const T* ec, T* uf, const T* copy_src = nullptr,
                              T* copy_dst = nullptr) {
  Level& F = ctx->levels[l];
  Level& C = ctx->levels[l + 1];
  ctx->launches += 1;
  if (F.tkind == 1) {
    CK(launch_prolong_space_add<T>(uf, ec, F.g, C.g, F.nt * F.nc, F.tr, copy_src, copy_dst, ctx->stream));
    const int R = F.tr.width_p;
    if (!transfer_fused_host(F.dim == 3 ? R * R * R : R * R, F.size())) ctx->launches += F.dim - 1;
  }
  else CK(launch_prolong_time_add<T>(uf, ec, F.g, F.tt, copy_src, copy_dst, ctx->stream));
  return STMG_OK;
}

// r += -S u on unconstrained rows, r already holding f (the V-cycle keeps u = 0 on constrained nodes,
// so f - u = f there): the residual without its initialisation pass
template <typename T>
stmg_status op_residual_preset(stmg_ctx* ctx, Level& L, const T* u, T* r) {
  return apply_slabs<T>(ctx, L, u, r, T(-1));
}

template <typename T>
stmg_status coarse_solve(stmg_ctx* ctx, Level& L, const T* f, T* u, bool u_zeroed = false) {
  if (!u_zeroed) CK(cudaMemsetAsync(u, 0, sizeof(T) * L.size(), ctx->stream));
  CK(launch_coarse_solve<T>(f, u, cinv_of<T>(L), L.cmap, L.n_coarse, L.size(), ctx->stream));
  ctx->launches += 1;
  return STMG_OK;
}

// Algorithm stmg: V-cycle with zero initial guess on level l, f_l -> u_l.  Bookkeeping passes
// are fused into the neighbouring kernels: the restriction into level l zeroes u_l, the first
// smoothing kernel and the prolongation write r_l := f_l, so that the residuals need only the
// operator kernel (u_l stays 0 on constrained nodes throughout).
template <typename T>
stmg_status vcycle_level(stmg_ctx* ctx, int l) {
  Level& L = ctx->levels[l];
  T* f = fv<T>(L);
  T* u = uv<T>(L);
  T* r = rv<T>(L);
  if (l == (int)ctx->levels.size() - 1) return coarse_solve<T>(ctx, L, f, u, l > 0);
  if (l == 0) CK(cudaMemsetAsync(u, 0, sizeof(T) * L.size(), ctx->stream));
  const int nu1 = ctx->opt.nu_pre, nu2 = ctx->opt.nu_post;
  for (int s = 0; s < nu1; ++s) {
    if (s == 0) {
      // zero guess: residual = f; on the last pre-sweep also preset r := f for the residual below
      CKS(op_asm<T>(ctx, L, f, u, L.omega, nu1 == 1 ? f : nullptr, nu1 == 1 ? r : nullptr));
    } else {
      CKS(op_residual<T>(ctx, L, f, u, r));
      CKS(op_asm<T>(ctx, L, r, u, L.omega));
      if (s == nu1 - 1) CK(cudaMemcpyAsync(r, f, sizeof(T) * L.size(), cudaMemcpyDeviceToDevice, ctx->stream));
    }
  }
  const T* res = f;
  if (nu1 > 0) {
    CKS(op_residual_preset<T>(ctx, L, u, r));
    res = r;
  }
  Level& Cl = ctx->levels[l + 1];
  CKS(op_restrict<T>(ctx, l, res, fv<T>(Cl), uv<T>(Cl)));
  CKS(vcycle_level<T>(ctx, l + 1));
  CKS(op_prolongate_add<T>(ctx, l, uv<T>(Cl), u, nu2 > 0 ? f : nullptr, nu2 > 0 ? r : nullptr));
  for (int s = 0; s < nu2; ++s) {
    if (s == 0) CKS(op_residual_preset<T>(ctx, L, u, r));
    else CKS(op_residual<T>(ctx, L, f, u, r));
    CKS(op_asm<T>(ctx, L, r, u, L.omega));
  }
  return STMG_OK;
}

template <typename T>
stmg_status run_vcycle(stmg_ctx* ctx) {
  bool& warmed = sizeof(T) == 4 ? ctx->warmed32 : ctx->warmed64;
  cudaGraphExec_t& ge = sizeof(T) == 4 ? ctx->graph32 : ctx->graph64;
  if (!warmed) {  // first call runs eagerly (sets kernel attributes), later calls replay a graph
    warmed = true;
    return vcycle_level<T>(ctx, 0);
  }
  if (!ge) {
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t saved = ctx->launches;
    stmg_status st = vcycle_level<T>(ctx, 0);
    ctx->launches = saved;
    const int64_t before = ctx->launches;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (st != STMG_OK) return st;
    if (e != cudaSuccess) { ctx->err = std::string("capture: ") + cudaGetErrorString(e); return STMG_ERR_CUDA; }
    (void)before;
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    int64_t nk = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      cudaGraphNodeGetType(nd, &ty);
      if (ty == cudaGraphNodeTypeKernel) ++nk;
    }
    (sizeof(T) == 4 ? ctx->graph32_kernels : ctx->graph64_kernels) = nk;
    e = cudaGraphInstantiate(&ge, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { ctx->err = std::string("instantiate: ") + cudaGetErrorString(e); ge = nullptr; return STMG_ERR_CUDA; }
  }
  CK(cudaGraphLaunch(ge, ctx->stream));
  ctx->launches += sizeof(T) == 4 ? ctx->graph32_kernels : ctx->graph64_kernels;
  return STMG_OK;
}

// splitmix64 counter-based generator (Steele, Lea, Flood 2014)
uint64_t splitmix64(uint64_t i) {
  uint64_t z = i + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

bool node_constrained(const Level& L, int64_t node) {
  const int nn1 = L.g.nn1;
  const int gx = (int)(node % nn1);
  const int64_t rest = node / nn1;
  if (gx == 0 || gx == nn1 - 1) return true;
  if (L.dim == 3) {
    const int gy = (int)(rest % nn1), gz = (int)(rest / nn1);
    return gy == 0 || gy == nn1 - 1 || gz == 0 || gz == nn1 - 1;
  }
  return rest == 0 || rest == nn1 - 1;
}

// out[0] = x . x (device), one launch; double-float arithmetic when x is 16-byte aligned
stmg_status dot_self(stmg_ctx* ctx, const double* x, int64_t n, double* out) {
  CK(launch_cgs_pass(nullptr, n, 0, const_cast<double*>(x), n, nullptr, 0, 0, 1, nullptr, 0, ctx->partial,
                     ctx->counter, out, ctx->stream, ctx->status, nullptr, nullptr, 3));
  ctx->launches += 1;
  return STMG_OK;
}

// enqueue part: no host synchronisation (capturable).  Classical Gram-Schmidt twice in three
// fused passes over the basis: h1 = V^T w ; w -= V h1, h2 = V^T w, |w|^2 ; w = (w - V h2) / hn with
// hn^2 = |w|^2 - |h2|^2 (orthonormal basis), the column h1 + h2 and hn (with copy32, also the FP32
// copy of the normalised w: the next V-cycle's input).
stmg_status orthogonalise_enqueue(stmg_ctx* ctx, const double* V0, int64_t ld, int nv, double* w, int64_t n,
                                  float* copy32 = nullptr, double* hdst = nullptr, bool df = false) {
  double* d_h1 = ctx->dsm;
  double* d_h2 = ctx->dsm + 128;
  int* st = ctx->status;
  // df: the basis is in double-float pairs; the first pass converts w (FP64, the operator's output)
  CK(launch_cgs_pass(V0, ld, nv, w, n, nullptr, 0, 1, 0, nullptr, 0, ctx->partial, ctx->counter, d_h1, ctx->stream, st,
                     nullptr, nullptr, df ? 2 : 0));
  // the second pass also reduces |w|^2 (into d_h2[nv]), from which the third pass knows the norm of
  // its result and normalises it (and writes the FP32 copy) as it subtracts
  CK(launch_cgs_pass(V0, ld, nv, w, n, d_h1, 1, 1, 1, nullptr, 0, ctx->partial, ctx->counter, d_h2, ctx->stream, st,
                     nullptr, nullptr, df ? 1 : 0));
  // the third pass's last block writes the Arnoldi column straight into the pinned host buffer (mapped
  // and device-addressable under unified addressing; the host reads it after the stream or the
  // iteration's event has completed): no copy between one iteration and the next
  CK(launch_cgs_pass(V0, ld, nv, w, n, d_h2, 1, 0, 0, d_h1, 1, ctx->partial, ctx->counter, hdst ? hdst : ctx->hsm,
                     ctx->stream, st, d_h2 + nv, copy32, df ? 1 : 0));
  ctx->launches += 3;
  return STMG_OK;
}

stmg_status orthogonalise_read(stmg_ctx* ctx, int nv, std::vector<double>& h, double& hn) {
  CK(cudaStreamSynchronize(ctx->stream));
  h.assign(ctx->hsm, ctx->hsm + nv);
  hn = ctx->hsm[nv];
  return STMG_OK;
}

// One Arnoldi/FGMRES orthogonalisation step (classical Gram-Schmidt, twice):
// w <- w - V h, h = [V^T w]_1 + [V^T w]_2 ; hn = ||w|| ; w <- w / hn.  Host gets h (nv) and hn.
stmg_status orthogonalise(stmg_ctx* ctx, const double* V0, int64_t ld, int nv, double* w, int64_t n, std::vector<double>& h,
                          double& hn) {
  CKS(orthogonalise_enqueue(ctx, V0, ld, nv, w, n));
  return orthogonalise_read(ctx, nv, h, hn);
}

stmg_status estimate_omega(stmg_ctx* ctx, int l) {
  Level& L = ctx->levels[l];
  const int64_t n = L.size();
  int64_t n_free = 0;
  for (int64_t node = 0; node < L.g.n_nodes; ++node) n_free += node_constrained(L, node) ? 0 : 1;
  n_free *= (int64_t)L.nt * L.nc;
  // the Krylov space lives on the unconstrained DoFs: at most that many steps
  const int steps = (int)std::min<int64_t>(20, n_free);
  std::vector<double> v0(n);
  const uint64_t base = (uint64_t)l << 32;
  double nr = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double x = 2.0 * ((double)(splitmix64(base + (uint64_t)i) >> 11) * 0x1.0p-53) - 1.0;
    if (node_constrained(L, i % L.g.n_nodes)) x = 0.0;
    v0[i] = x;
    nr += x * x;
  }
  nr = std::sqrt(nr);
  for (auto& x : v0) x /= nr;
  std::vector<double*> V(steps + 1);
  const int64_t ld = (n + 31) / 32 * 32;  // 256-byte aligned basis vectors (bulk copies)
  for (int j = 0; j <= steps; ++j) V[j] = ctx->V + (size_t)j * ld;
  CK(cudaMemcpyAsync(V[0], v0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  std::vector<double> H((steps + 1) * steps, 0.0);
  int m = steps;
  double* z = ctx->Z;
  for (int j = 0; j < steps; ++j) {
    if (L.eig_tc) {  // the tensor-core smoother takes FP32 vectors
      CK(launch_convert<double, float>(V[j], L.r32, n, ctx->stream));
      CK(cudaMemsetAsync(L.u32, 0, sizeof(float) * n, ctx->stream));
      CKS(op_asm<float>(ctx, L, L.r32, L.u32, 1.0));
      CK(launch_convert<float, double>(L.u32, z, n, ctx->stream));
    } else {
      CK(cudaMemsetAsync(z, 0, sizeof(double) * n, ctx->stream));
      CKS(op_asm<double>(ctx, L, V[j], z, 1.0));
    }
    CKS(op_apply<double>(ctx, L, z, V[j + 1]));
    std::vector<double> h;
    double hn = 0.0;
    CKS(orthogonalise(ctx, V[0], ld, j + 1, V[j + 1], n, h, hn));
    for (int i = 0; i <= j; ++i) H[i * steps + j] = h[i];
    H[(j + 1) * steps + j] = hn;
    if (hn <= 1e-14 * std::fabs(H[j * steps + j]) + 1e-300) { m = j + 1; break; }
  }
  std::vector<double> Hm(m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Hm[i * m + j] = H[i * steps + j];
  std::vector<cplx> ev = eigenvalues(m, Hm);
  double lmax = -1e300, lmin = 1e300;
  for (auto& e : ev) {
    if (std::abs(e) <= 1e-12) continue;
    lmax = std::max(lmax, e.real());
    lmin = std::min(lmin, e.real());
  }
  if (!(lmax + lmin > 0.0) || !std::isfinite(lmax + lmin)) {
    ctx->err = "relaxation estimate failed on level " + std::to_string(l) + " (" + std::to_string(m) + " Arnoldi steps, Ritz values";
    for (auto& e : ev) ctx->err += " " + std::to_string(e.real()) + "+" + std::to_string(e.imag()) + "i";
    ctx->err += ")";
    return STMG_ERR_INTERNAL;
  }
  L.omega = std::min(1.0, 2.0 / (lmax + lmin));  // the paper takes omega_l in (0, 1) (Section 3.3)
  return STMG_OK;
}

// Synchronises and reads the device status word (bounded waits that gave up set it).
stmg_status check_device_status(stmg_ctx* ctx) {
  int* h = reinterpret_cast<int*>(ctx->hsm + 510);
  CK(cudaMemcpyAsync(h, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (*h != 0) {
    ctx->err = "a device wait for a bulk copy gave up (status word set); results of this call are invalid";
    return STMG_ERR_TIMEOUT;
  }
  return STMG_OK;
}

stmg_status setup_smoother(stmg_ctx* ctx, Level& L) {
  const int nt = L.nt;
  // T = TA^-1 TM, eigen-decomposition
  std::vector<double> TAi = L.sc.TA;
  if (!invert(nt, TAi)) { ctx->err = "singular time matrix"; return STMG_ERR_INTERNAL; }
  std::vector<double> T(nt * nt, 0.0);
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < nt; ++j)
      for (int l = 0; l < nt; ++l) T[i * nt + j] += TAi[i * nt + l] * L.sc.TM[l * nt + j];
  std::vector<cplx> lam, V;
  if (!eigen_decompose(nt, T, lam, V)) { ctx->err = "time matrix not diagonalisable"; return STMG_ERR_INTERNAL; }
  std::vector<cplx> Vinv = V;
  invert_complex(nt, Vinv);
  // representatives: real modes, then one of each conjugate pair (Im > 0)
  std::vector<int> reps;
  for (int m = 0; m < nt; ++m) if (lam[m].imag() == 0.0) reps.push_back(m);
  L.nreal = (int)reps.size();
  for (int m = 0; m < nt; ++m) if (lam[m].imag() > 0.0) reps.push_back(m);
  L.ncplx = (int)reps.size() - L.nreal;
  if (L.nreal + 2 * L.ncplx != nt) { ctx->err = "unpaired complex time eigenvalue"; return STMG_ERR_INTERNAL; }
  ModeTab<double> mt{};
  mt.nreal = L.nreal; mt.ncplx = L.ncplx;
  std::vector<double> lr, li;
  for (size_t r = 0; r < reps.size(); ++r) {
    const int m = reps[r];
    lr.push_back(lam[m].real());
    li.push_back(lam[m].imag());
    mt.lre[r] = lam[m].real();
    mt.lim[r] = lam[m].imag();
    for (int t = 0; t < nt; ++t) {
      cplx w = 0.0;  // W = V^-1 TA^-1
      for (int l = 0; l < nt; ++l) w += Vinv[m * nt + l] * TAi[l * nt + t];
      mt.Wr[r][t] = w.real(); mt.Wi[r][t] = w.imag();
      mt.Vr[t][r] = V[t * nt + m].real(); mt.Vi[t][r] = V[t * nt + m].imag();
    }
  }
  mt.omega = 1.0;
  mt.weighted = ctx->opt.asm_weighting;
  L.mt64 = mt;
  ModeTab<float> mf{};
  mf.nreal = mt.nreal; mf.ncplx = mt.ncplx;
  for (int a = 0; a < kMaxNT; ++a)
    for (int b = 0; b < kMaxNT; ++b) {
      mf.Wr[a][b] = (float)mt.Wr[a][b]; mf.Wi[a][b] = (float)mt.Wi[a][b];
      mf.Vr[a][b] = (float)mt.Vr[a][b]; mf.Vi[a][b] = (float)mt.Vi[a][b];
    }
  for (int a = 0; a < kMaxNT; ++a) { mf.lre[a] = (float)mt.lre[a]; mf.lim[a] = (float)mt.lim[a]; }
  mf.omega = 1.0f;
  mf.weighted = mt.weighted;
  L.mt32 = mf;
  if (L.fd) {
    std::vector<double> S, lamfd;
    fd_tables_1d(L.p, L.N, S, lamfd);
    FDTab<double> f64{};
    FDTab<float> f32{};
    for (int t = 0; t < 3; ++t)
      for (int a = 0; a < L.n; ++a) {
        f64.lam[t][a] = lamfd[t * L.n + a];
        f32.lam[t][a] = (float)lamfd[t * L.n + a];
        for (int i = 0; i < L.n; ++i) {
          f64.S[t][a][i] = S[(t * L.n + a) * L.n + i];
          f32.S[t][a][i] = (float)S[(t * L.n + a) * L.n + i];
        }
      }
    L.fd64 = f64;
    L.fd32 = f32;
    const int nqd = L.n * L.n * L.n;
    std::vector<double> rc(L.g.n_cells);
    std::vector<float> rcf(L.g.n_cells);
    for (int64_t c = 0; c < L.g.n_cells; ++c) {
      double sum = 0.0;
      for (int q = 0; q < nqd; ++q) sum += L.rho_qp[c * nqd + q];
      rc[c] = sum / nqd;
      rcf[c] = (float)rc[c];
    }
    CKS(dev_alloc(ctx, &L.rho_cell64, L.g.n_cells));
    CKS(dev_alloc(ctx, &L.rho_cell32, L.g.n_cells));
    CK(cudaMemcpy(L.rho_cell64, rc.data(), sizeof(double) * rc.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(L.rho_cell32, rcf.data(), sizeof(float) * rcf.size(), cudaMemcpyHostToDevice));
    return STMG_OK;
  }
  if (L.eig_tc) {
    const int64_t bytes = eig_tc_bytes(L.dim, L.n, L.g.n_cells);
    if (bytes < 0 || L.nc > 8) {
      ctx->err = "the tensor-core smoother needs (p+1)^dim <= 64 and at most 8 slabs per system";
      return STMG_ERR_UNSUPPORTED;
    }
    void* store = nullptr;
    cudaError_t e = cudaMalloc(&store, (size_t)bytes);
    if (e != cudaSuccess) { ctx->err = std::string("cudaMalloc eigen images: ") + cudaGetErrorString(e); return STMG_ERR_OOM; }
    ctx->allocations.push_back(store);
    L.inv = store;
    L.inv_prec = 3;
    CK(launch_eig_setup(L.dim, L.n, L.g, L.geo64, L.lt, L.inv, 3, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return STMG_OK;
  }
  if (L.eig) {
    if (L.dim == 3 && L.n > 4) {
      ctx->err = "the eigendecomposition smoother supports p <= 3 in 3D";
      return STMG_ERR_UNSUPPORTED;
    }
    const int prec = L.inv_prec == 0 ? 0 : L.inv_prec == 1 ? 1 : 2;
    L.inv_prec = prec;
    const size_t bytes = (size_t)L.g.n_cells * eig_cell_bytes(L.dim, L.n, prec == 0 ? 8 : prec == 1 ? 4 : 2);
    void* store = nullptr;
    cudaError_t e = cudaMalloc(&store, bytes);
    if (e != cudaSuccess) { ctx->err = std::string("cudaMalloc eigen store: ") + cudaGetErrorString(e); return STMG_ERR_OOM; }
    ctx->allocations.push_back(store);
    L.inv = store;
    CK(launch_eig_setup(L.dim, L.n, L.g, L.geo64, L.lt, L.inv, prec, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return STMG_OK;
  }
  const int NB = L.dim == 3 ? L.n * L.n * L.n : L.n * L.n;
  if (L.dim == 3 && L.n > 4) {
    ctx->err = "dense additive Schwarz setup supports p <= 3 in 3D";
    return STMG_ERR_UNSUPPORTED;
  }
  const size_t esz = L.inv_prec == 0 ? 8 : L.inv_prec == 1 ? 4 : L.inv_prec == 2 ? 2 : 1;
  (void)NB;
  const size_t count = (size_t)L.g.n_cells * asm_cell_stride(L.dim, L.n, nt, (int)esz);
  void* inv = nullptr;
  cudaError_t e = cudaMalloc(&inv, count * esz);
  if (e != cudaSuccess) { ctx->err = std::string("cudaMalloc inverses: ") + cudaGetErrorString(e); return STMG_ERR_OOM; }
  ctx->allocations.push_back(inv);
  L.inv = inv;
  double* dl = nullptr;
  CKS(dev_alloc(ctx, &dl, 2 * kMaxNT));
  std::vector<double> lam_host(2 * kMaxNT, 0.0);
  for (size_t r = 0; r < lr.size(); ++r) { lam_host[r] = lr[r]; lam_host[kMaxNT + r] = li[r]; }
  CK(cudaMemcpyAsync(dl, lam_host.data(), sizeof(double) * 2 * kMaxNT, cudaMemcpyHostToDevice, ctx->stream));
  CK(launch_asm_setup(L.dim, L.n, nt, L.g, L.geo64, L.lt, dl, dl + kMaxNT, L.nreal, L.ncplx, L.inv, L.inv_prec,
                      ctx->opt.asm_weighting, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return STMG_OK;
}

stmg_status setup_transfer(stmg_ctx* ctx, Level& F, const Level& C) {
  if (F.nc != C.nc) {  // tau-level: fine slabs 2j, 2j+1 under coarse slab j (contiguous in memory)
    F.tkind = 3;
    std::vector<double> P = tau_prolongation(F.k);
    F.tt.ntf = 2 * F.nt; F.tt.ntc = C.nt; F.tt.nb = C.nc;
    for (int i = 0; i < 2 * F.nt; ++i)
      for (int j = 0; j < C.nt; ++j) F.tt.P[i][j] = P[i * C.nt + j];
    return STMG_OK;
  }
  if (F.k != C.k) {
    F.tkind = 2;
    std::vector<double> P = time_prolongation(ctx->scheme, F.k, C.k);
    F.tt.ntf = F.nt; F.tt.ntc = C.nt; F.tt.nb = F.nc;
    for (int i = 0; i < F.nt; ++i)
      for (int j = 0; j < C.nt; ++j) F.tt.P[i][j] = P[i * C.nt + j];
    return STMG_OK;
  }
  F.tkind = 1;
  std::vector<int> start;
  std::vector<double> w;
  prolongation_1d(F.p, F.N, C.p, C.N, start, w);
  const int W = C.p + 1;
  const int nf = F.g.nn1, nc = C.g.nn1;
  // 1D lists with the Dirichlet masks folded in (fine and coarse end nodes dropped)
  std::vector<std::vector<std::pair<int, double>>> plist(nf), rlist(nc);
  for (int gf = 1; gf < nf - 1; ++gf)
    for (int b = 0; b < W; ++b) {
      const int gc = start[gf] + b;
      const double v = w[(size_t)gf * W + b];
      if (v == 0.0 || gc == 0 || gc == nc - 1) continue;
      plist[gf].push_back({gc, v});
      rlist[gc].push_back({gf, v});
    }
  auto pack = [&](const std::vector<std::vector<std::pair<int, double>>>& lists, int& R, int** d_idx,
                  double** d_w, float** d_w32) -> stmg_status {
    R = 1;
    for (auto& l : lists) R = std::max<int>(R, (int)l.size());
    std::vector<int> idx(lists.size() * R, -1);
    std::vector<double> wt(lists.size() * R, 0.0);
    for (size_t i = 0; i < lists.size(); ++i)
      for (size_t c = 0; c < lists[i].size(); ++c) { idx[i * R + c] = lists[i][c].first; wt[i * R + c] = lists[i][c].second; }
    std::vector<float> wt32(wt.begin(), wt.end());
    CKS(dev_alloc(ctx, d_idx, idx.size()));
    CKS(dev_alloc(ctx, d_w, wt.size()));
    CKS(dev_alloc(ctx, d_w32, wt32.size()));
    CK(cudaMemcpy(*d_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(*d_w, wt.data(), sizeof(double) * wt.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(*d_w32, wt32.data(), sizeof(float) * wt32.size(), cudaMemcpyHostToDevice));
    return STMG_OK;
  };
  int *pi = nullptr, *ri = nullptr;
  double *pw = nullptr, *rw = nullptr;
  float *pw32 = nullptr, *rw32 = nullptr;
  CKS(pack(plist, F.tr.width_p, &pi, &pw, &pw32));
  CKS(pack(rlist, F.tr.width_r, &ri, &rw, &rw32));
  F.tr.p_idx = pi;
  F.tr.p_w = pw;
  F.tr.p_w32 = pw32;
  F.tr.r_idx = ri;
  F.tr.r_w = rw;
  F.tr.r_w32 = rw32;
  const size_t tmp = (size_t)F.nt * F.nc * nf * (size_t)(F.dim == 3 ? nf : 1) * nc;
  double *t1 = nullptr, *t2 = nullptr;
  CKS(dev_alloc(ctx, &t1, tmp));
  CKS(dev_alloc(ctx, &t2, tmp));
  F.tr.tmp1 = t1;
  F.tr.tmp2 = t2;
  return STMG_OK;
}

stmg_status setup_coarse(stmg_ctx* ctx, Level& L) {
  std::vector<int64_t> map;
  for (int t = 0; t < L.nt * L.nc; ++t)
    for (int64_t node = 0; node < L.g.n_nodes; ++node)
      if (!node_constrained(L, node)) map.push_back((int64_t)t * L.g.n_nodes + node);
  const int n = (int)map.size();
  if (n > 4096) { ctx->err = "coarsest level too large for the dense solver"; return STMG_ERR_UNSUPPORTED; }
  L.n_coarse = n;
  const int64_t tot = L.size();
  double *x = nullptr, *y = nullptr;
  CKS(dev_alloc(ctx, &x, tot));
  CKS(dev_alloc(ctx, &y, tot));
  std::vector<double> S((size_t)n * n), col(tot);
  CK(cudaMemsetAsync(x, 0, sizeof(double) * tot, ctx->stream));
  const double one = 1.0, zero = 0.0;
  for (int j = 0; j < n; ++j) {
    CK(cudaMemcpyAsync(x + map[j], &one, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CKS(op_apply<double>(ctx, L, x, y));
    CK(cudaMemcpyAsync(col.data(), y, sizeof(double) * tot, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(x + map[j], &zero, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < n; ++i) S[(size_t)i * n + j] = col[map[i]];
  }
  if (!invert(n, S)) { ctx->err = "coarsest operator singular"; return STMG_ERR_INTERNAL; }
  // row-major inverse, rows padded with zeros to coarse_ld(n) entries (the coarse kernel reads one row
  // per warp in 16-byte loads)
  const int ld = coarse_ld(n);
  std::vector<double> cm((size_t)n * ld, 0.0);
  std::vector<float> cmf((size_t)n * ld, 0.0f);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      cm[(size_t)i * ld + j] = S[(size_t)i * n + j];
      cmf[(size_t)i * ld + j] = (float)S[(size_t)i * n + j];
    }
  CKS(dev_alloc(ctx, &L.cmap, n));
  CKS(dev_alloc(ctx, &L.cinv64, (size_t)n * ld));
  CKS(dev_alloc(ctx, &L.cinv32, (size_t)n * ld));
  CK(cudaMemcpy(L.cmap, map.data(), sizeof(int64_t) * n, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(L.cinv64, cm.data(), sizeof(double) * n * ld, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(L.cinv32, cmf.data(), sizeof(float) * n * ld, cudaMemcpyHostToDevice));
  return STMG_OK;
}

stmg_status create_impl(stmg_ctx* ctx, const stmg_mesh* mesh, const stmg_problem* pr, const stmg_options* op) {
  if (!mesh || !pr) return invalid(ctx, "mesh and problem are required");
  const int dim = mesh->dim, N = mesh->n_cells;
  if (dim != 2 && dim != 3) return invalid(ctx, "dim must be 2 or 3");
  if (N < 2) return invalid(ctx, "n_cells must be >= 2");
  if (pr->p < 1 || pr->p > 5 || (pr->p == 5 && dim != 3))
    return invalid(ctx, "p must be in 1..4 (1..5 in 3D, where Q5 levels use the fast diagonalisation)");
  CKS(dev_alloc(ctx, &ctx->status, 1));
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  if (pr->time_scheme != STMG_DG && pr->time_scheme != STMG_CGP) return invalid(ctx, "unknown time scheme");
  if (pr->pde != STMG_HEAT && pr->pde != STMG_WAVE) return invalid(ctx, "unknown pde");
  const int nt = pr->time_scheme == STMG_DG ? pr->k + 1 : pr->k;
  if (nt < 1 || nt > kMaxNT || (pr->time_scheme == STMG_CGP && pr->k < 1)) return invalid(ctx, "time degree out of range");
  if (!(pr->tau > 0.0)) return invalid(ctx, "tau must be positive");
  const int nslabs = pr->n_slabs == 0 ? 1 : pr->n_slabs;
  if (nslabs < 1 || nslabs > 64) return invalid(ctx, "n_slabs must be in 1..64");
  if (nslabs > 1 && (pr->pde != STMG_HEAT || pr->time_scheme != STMG_DG))
    return invalid(ctx, "several slabs in one system: heat equation with dG in time only");
  {  // the kernels index vectors and cells in 32-bit arithmetic
    const double nn1 = (double)pr->p * N + 1.0;
    if (std::pow(nn1, dim) * nt * nslabs * 2.0 >= 2147483648.0)
      return invalid(ctx, "problem too large: a level's vectors must hold fewer than 2^30 entries");
  }
  ctx->dim = dim; ctx->pde = pr->pde; ctx->scheme = pr->time_scheme; ctx->tau = pr->tau;
  stmg_options o{};
  if (op) o = *op;
  if (o.nu_pre < 0 || o.nu_post < 0) return invalid(ctx, "negative smoothing sweeps");
  if (o.nu_pre == 0) o.nu_pre = 1;
  if (o.nu_post == 0) o.nu_post = 1;
  if (o.vcycle_precision != STMG_FP64) o.vcycle_precision = STMG_FP32;
  if (o.fgmres_restart <= 0) o.fgmres_restart = 30;
  if (o.fgmres_restart > 64) return invalid(ctx, "fgmres_restart must be <= 64");
  if (!(o.rtol > 0.0)) o.rtol = 1e-8;
  if (!(o.atol >= 0.0)) return invalid(ctx, "atol must be >= 0");
  if (o.space_coarsening != STMG_COARSEN_P_THEN_H && o.space_coarsening != STMG_COARSEN_H)
    return invalid(ctx, "space_coarsening out of range");
  if (o.coarse_max_dofs < 0 || o.coarse_max_dofs > 4096) return invalid(ctx, "coarse_max_dofs must be in 0..4096");
  if (o.asm_weighting != 0 && o.asm_weighting != 1) return invalid(ctx, "asm_weighting must be 0 or 1");
  if (o.outer_relax != 0 && o.outer_relax != 1) return invalid(ctx, "outer_relax must be 0 or 1");
  if (o.max_it <= 0) o.max_it = 200;
  if (o.inverse_precision == 0) o.inverse_precision = o.vcycle_precision;
  if (o.outer_apply == 0) o.outer_apply = o.vcycle_precision == STMG_FP32 ? STMG_DF32 : STMG_FP64;
  if (o.outer_apply != STMG_FP64 && o.outer_apply != STMG_DF32) return invalid(ctx, "outer_apply must be FP64 or DF32");
  if (o.outer_apply == STMG_DF32 && o.vcycle_precision != STMG_FP32)
    return invalid(ctx, "the double-float outer apply needs the FP32 V-cycle");
  ctx->outer_df = o.outer_apply == STMG_DF32;
  if (o.inverse_precision != STMG_FP64 && o.inverse_precision != STMG_FP32 && o.inverse_precision != STMG_BF16 &&
      o.inverse_precision != STMG_FP8)
    return invalid(ctx, "inverse_precision out of range");
  if (o.inverse_precision == STMG_FP8 && o.vcycle_precision != STMG_FP32)
    return invalid(ctx, "FP8 inverses need the FP32 V-cycle");
  const int inv_prec = o.inverse_precision == STMG_FP64 ? 0 : o.inverse_precision == STMG_FP32 ? 1
                     : o.inverse_precision == STMG_BF16 ? 2 : 3;
  ctx->opt = o;
  const int64_t nv1 = N + 1;
  const int64_t nverts = dim == 3 ? nv1 * nv1 * nv1 : nv1 * nv1;
  std::vector<double> verts((size_t)nverts * dim);
  if (mesh->vertices) {
    std::memcpy(verts.data(), mesh->vertices, sizeof(double) * verts.size());
  } else {
    for (int64_t v = 0; v < nverts; ++v) {
      int64_t r = v;
      for (int d = 0; d < dim; ++d) { verts[v * dim + d] = (double)(r % nv1) / N; r /= nv1; }
    }
  }
  // finest-level coefficient at Gauss points and per-cell means
  const int64_t ncells_f = dim == 3 ? (int64_t)N * N * N : (int64_t)N * N;
  const int nqd_f = dim == 3 ? (pr->p + 1) * (pr->p + 1) * (pr->p + 1) : (pr->p + 1) * (pr->p + 1);
  std::vector<double> rho_f((size_t)ncells_f * nqd_f, 1.0), cell_mean(ncells_f, 1.0);
  if (pr->coeff) {
    if (pr->coeff_mode == STMG_COEFF_PER_CELL) {
      for (int64_t c = 0; c < ncells_f; ++c) {
        cell_mean[c] = pr->coeff[c];
        for (int q = 0; q < nqd_f; ++q) rho_f[c * nqd_f + q] = pr->coeff[c];
      }
    } else if (pr->coeff_mode == STMG_COEFF_PER_QPOINT) {
      for (int64_t c = 0; c < ncells_f; ++c) {
        double s = 0.0;
        for (int q = 0; q < nqd_f; ++q) { rho_f[c * nqd_f + q] = pr->coeff[c * nqd_f + q]; s += pr->coeff[c * nqd_f + q]; }
        cell_mean[c] = s / nqd_f;
      }
    } else {
      return invalid(ctx, "unknown coefficient mode");
    }
    for (double v : rho_f) if (!(v > 0.0) || !std::isfinite(v)) return invalid(ctx, "coefficient must be positive and finite");
  }
  std::vector<Spec> seq = level_sequence(pr->p, N, pr->k, pr->time_scheme, o.space_coarsening == STMG_COARSEN_P_THEN_H,
                                         nslabs, pr->tau);
  // a shallower hierarchy: the first coarser level with at most coarse_max_dofs unknowns is the coarsest
  if (o.coarse_max_dofs > 0)
    for (size_t li = 1; li < seq.size(); ++li)
      if (level_unknowns(seq[li], dim, pr->time_scheme) <= o.coarse_max_dofs) { seq.resize(li + 1); break; }
  ctx->levels.resize(seq.size());
  for (size_t li = 0; li < seq.size(); ++li) {
    Level& L = ctx->levels[li];
    L.dim = dim; L.p = seq[li].p; L.n = L.p + 1; L.N = seq[li].N; L.k = seq[li].k;
    L.nc = seq[li].nc; L.tau = seq[li].tau;
    L.nt = pr->time_scheme == STMG_DG ? L.k + 1 : L.k;
    L.g.dim = dim; L.g.N = L.N; L.g.p = L.p; L.g.nn1 = L.p * L.N + 1;
    L.g.n_nodes = dim == 3 ? (int64_t)L.g.nn1 * L.g.nn1 * L.g.nn1 : (int64_t)L.g.nn1 * L.g.nn1;
    L.g.n_cells = dim == 3 ? (int64_t)L.N * L.N * L.N : (int64_t)L.N * L.N;
    L.sc = slab_coeffs(pr->pde, pr->time_scheme, L.k, L.tau);
    for (int i = 0; i < L.nt; ++i)
      for (int j = 0; j < L.nt; ++j)
        if (i != j && std::fabs(L.sc.TA[i * L.nt + j]) > 1e-13 * std::fabs(L.sc.TA[i * L.nt + i])) {
          ctx->err = "time mass matrix is not diagonal";
          return STMG_ERR_INTERNAL;
        }
    fill_tables(L);
    // coupling to the previous slab (heat dG: the coefficient of M_h u_0 in the slab's right-hand side)
    L.cpl64 = L.tab64;
    for (int i = 0; i < kMaxNT; ++i)
      for (int j = 0; j < kMaxNT; ++j) { L.cpl64.TA[i][j] = 0.0; L.cpl64.TM[i][j] = 0.0; }
    for (int i = 0; i < L.nt; ++i) L.cpl64.TM[i][L.nt - 1] = -L.sc.RM_u0[i];
    L.cpl64.sign = 1.0;
    L.cpl32 = L.tab32;
    for (int i = 0; i < kMaxNT; ++i)
      for (int j = 0; j < kMaxNT; ++j) { L.cpl32.TA[i][j] = 0.0f; L.cpl32.TM[i][j] = (float)L.cpl64.TM[i][j]; }
    L.cpl32.sign = 1.0f;
    // vertices: every (N/N_l)-th fine vertex
    const int r = N / L.N;
    const int64_t lv1 = L.N + 1;
    const int64_t lnv = dim == 3 ? lv1 * lv1 * lv1 : lv1 * lv1;
    L.vertices.resize((size_t)lnv * dim);
    for (int64_t v = 0; v < lnv; ++v) {
      const int64_t ix = v % lv1, iy = (v / lv1) % lv1, iz = dim == 3 ? v / (lv1 * lv1) : 0;
      const int64_t fv_ = ix * r + nv1 * (iy * r + nv1 * iz * r);
      for (int d = 0; d < dim; ++d) L.vertices[v * dim + d] = verts[fv_ * dim + d];
    }
    const int nq = L.n;
    const int nqd = dim == 3 ? nq * nq * nq : nq * nq;
    if (li == 0) {
      L.rho_qp = rho_f;
    } else {
      std::vector<double> xq, wq;
      gauss_legendre(nq, xq, wq);
      L.rho_qp.resize((size_t)L.g.n_cells * nqd);
      for (int64_t c = 0; c < L.g.n_cells; ++c) {
        const int64_t cx = c % L.N, cy = (c / L.N) % L.N, cz = dim == 3 ? c / ((int64_t)L.N * L.N) : 0;
        const int64_t cc[3] = {cx, cy, cz};
        for (int q = 0; q < nqd; ++q) {
          const int qi[3] = {q % nq, (q / nq) % nq, q / (nq * nq)};
          int64_t fid = 0;
          for (int d = dim - 1; d >= 0; --d) {
            const double s = (cc[d] + xq[qi[d]]) / L.N;
            int64_t fc = (int64_t)std::floor(s * N);
            if (fc > N - 1) fc = N - 1;
            fid = fid * N + fc;
          }
          L.rho_qp[c * nqd + q] = cell_mean[fid];
        }
      }
    }
    // device geometry
    double *dvert = nullptr, *drho = nullptr, *dxq = nullptr, *dwq = nullptr;
    CKS(dev_alloc(ctx, &dvert, L.vertices.size()));
    CKS(dev_alloc(ctx, &drho, L.rho_qp.size()));
    CKS(dev_alloc(ctx, &dxq, nq));
    CKS(dev_alloc(ctx, &dwq, nq));
    std::vector<double> xq, wq;
    gauss_legendre(nq, xq, wq);
    CK(cudaMemcpy(dvert, L.vertices.data(), sizeof(double) * L.vertices.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(drho, L.rho_qp.data(), sizeof(double) * L.rho_qp.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dxq, xq.data(), sizeof(double) * nq, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(dwq, wq.data(), sizeof(double) * nq, cudaMemcpyHostToDevice));
    const int ncomp = dim == 3 ? 7 : 4;
    CKS(dev_alloc(ctx, &L.geo64, (size_t)L.g.n_cells * ncomp * nqd));
    const bool chunked = geo_chunked(dim, nq);
    CKS(dev_alloc(ctx, &L.geo32, chunked ? (size_t)geo_chunk_cells(L.g.n_cells) * 8 * nqd
                                         : (size_t)L.g.n_cells * ncomp * nqd));
    if (li == 0 && ctx->outer_df) CKS(dev_alloc(ctx, &L.geodf, (size_t)L.g.n_cells * ncomp * nqd));
    CK(launch_geometry(L.g, dvert, drho, dxq, dwq, L.geo64, L.geo32, L.geodf, ctx->stream));
    const int64_t sz = L.size();
    CKS(dev_alloc(ctx, &L.f64, sz)); CKS(dev_alloc(ctx, &L.u64, sz)); CKS(dev_alloc(ctx, &L.r64, sz));
    CKS(dev_alloc(ctx, &L.f32, sz)); CKS(dev_alloc(ctx, &L.u32, sz)); CKS(dev_alloc(ctx, &L.r32, sz));
    CK(cudaMemsetAsync(L.u64, 0, sizeof(double) * sz, ctx->stream));
    CK(cudaMemsetAsync(L.u32, 0, sizeof(float) * sz, ctx->stream));
    L.inv_prec = inv_prec;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  // Krylov workspace (also used by the relaxation estimate)
  const int64_t n0 = ctx->levels[0].size();
  ctx->m = o.fgmres_restart;
  ctx->nvec = std::max(ctx->m, 20) + 1;
  ctx->vld = (n0 + 31) / 32 * 32;
  CKS(dev_alloc(ctx, &ctx->V, (size_t)ctx->nvec * ctx->vld));
  CKS(dev_alloc(ctx, &ctx->Z, (size_t)std::max(ctx->m, 1) * n0));
  if (o.vcycle_precision == STMG_FP32 && ctx->outer_df) CKS(dev_alloc(ctx, &ctx->Z32, (size_t)std::max(ctx->m, 1) * n0));
  CKS(dev_alloc(ctx, &ctx->partial, (size_t)cgs_blocks() * 80));
  CKS(dev_alloc(ctx, &ctx->counter, 1));
  CK(cudaMemsetAsync(ctx->counter, 0, sizeof(unsigned int), ctx->stream));
  CKS(dev_alloc(ctx, &ctx->dsm, 512));
  for (int i = 0; i < 6; ++i) CKS(dev_alloc(ctx, &ctx->tmp[i], ctx->levels[0].g.n_nodes));
  CKS(dev_alloc(ctx, &ctx->rhs_buf, n0));
  CKS(dev_alloc(ctx, &ctx->u_buf, n0 * 3 + 4 * ctx->levels[0].g.n_nodes));
  CK(cudaMallocHost(&ctx->hsm, 512 * sizeof(double)));
  // local solver per level: fast diagonalisation on Cartesian 3D grids where it is exact (rho constant
  // on every cell patch) or where stored inverses are not supported (p = 4), else stored inverses
  bool cartesian = true;
  if (mesh->vertices) {
    for (int64_t v = 0; v < nverts && cartesian; ++v) {
      int64_t r = v;
      for (int d = 0; d < dim; ++d) {
        if (std::fabs(verts[v * dim + d] - (double)(r % nv1) / N) > 1e-14) cartesian = false;
        r /= nv1;
      }
    }
  }
  if (o.smoother_kind < STMG_SMOOTHER_AUTO || o.smoother_kind > STMG_SMOOTHER_EIG_TC)
    return invalid(ctx, "smoother_kind must be AUTO, DENSE, FD, EIG or EIG_TC");
  if (o.smoother_kind == STMG_SMOOTHER_EIG_TC && o.vcycle_precision == STMG_FP64)
    return invalid(ctx, "the tensor-core smoother runs in the FP32 V-cycle");
  if (o.smoother_kind == STMG_SMOOTHER_FD && (dim != 3 || !cartesian))
    return invalid(ctx, "fast diagonalisation needs a 3D Cartesian grid");
  for (size_t li = 0; li + 1 < ctx->levels.size(); ++li) {
    Level& L = ctx->levels[li];
    bool patch_const = true;
    const int nqd = dim == 3 ? L.n * L.n * L.n : L.n * L.n;
    for (int64_t c = 0; c < L.g.n_cells && patch_const; ++c) {
      const double r0 = L.rho_qp[c * nqd];
      for (int q = 0; q < nqd && patch_const; ++q) patch_const = L.rho_qp[c * nqd + q] == r0;
      if (dim != 3) continue;
      const int64_t cx = c % L.N, cy = (c / L.N) % L.N, cz = c / ((int64_t)L.N * L.N);
      for (int o3 = 0; o3 < 27 && patch_const; ++o3) {
        const int64_t nx = cx + o3 % 3 - 1, ny = cy + (o3 / 3) % 3 - 1, nz = cz + o3 / 9 - 1;
        if (nx < 0 || ny < 0 || nz < 0 || nx >= L.N || ny >= L.N || nz >= L.N) continue;
        patch_const = L.rho_qp[(nx + L.N * (ny + L.N * nz)) * nqd] == r0;
      }
    }
    if (o.smoother_kind == STMG_SMOOTHER_FD) L.fd = true;
    else if (o.smoother_kind == STMG_SMOOTHER_DENSE || o.smoother_kind >= STMG_SMOOTHER_EIG) L.fd = false;
    else L.fd = dim == 3 && cartesian && (patch_const || L.n > 4);
    L.eig = o.smoother_kind >= STMG_SMOOTHER_EIG;
    L.eig_tc = o.smoother_kind == STMG_SMOOTHER_EIG_TC;
  }
  for (size_t li = 0; li + 1 < ctx->levels.size(); ++li) {
    CKS(setup_smoother(ctx, ctx->levels[li]));
    CKS(setup_transfer(ctx, ctx->levels[li], ctx->levels[li + 1]));
  }
  CKS(setup_coarse(ctx, ctx->levels.back()));
  for (size_t li = 0; li + 1 < ctx->levels.size(); ++li) {
    if (o.omega) ctx->levels[li].omega = o.omega[li];
    else CKS(estimate_omega(ctx, (int)li));
  }
  CKS(check_device_status(ctx));
  CK(cudaStreamSynchronize(ctx->stream));
  return STMG_OK;
}

template <typename T>
stmg_status vcycle_public(stmg_ctx* ctx, const T* r, T* e) {
  Level& L = ctx->levels[0];
  CK(cudaMemcpyAsync(fv<T>(L), r, sizeof(T) * L.size(), cudaMemcpyDeviceToDevice, ctx->stream));
  CKS(run_vcycle<T>(ctx));
  CK(cudaMemcpyAsync(e, uv<T>(L), sizeof(T) * L.size(), cudaMemcpyDeviceToDevice, ctx->stream));
  return STMG_OK;
}

// Relative error assumed for the FP32 operator apply in the relaxed FGMRES (inexact Krylov,
// Simoncini & Szyld 2003): iteration j may use it once the residual estimate |g_j| is at most
// target / kRelaxDelta, so that the apply's error stays below the target.
constexpr double kRelaxDelta = 1e-5;

// w = S z for an FP32 z vanishing on constrained rows, FP32 arithmetic, FP64 w (already 0)
stmg_status op_apply_f2d(stmg_ctx* ctx, Level& L, const float* x, double* y) {
  OpTab<float> t = L.tab32;
  t.sign = 1.0f;
  const int64_t ss = L.slab_size();
  for (int i = 0; i < L.nc; ++i) {
    CK(launch_apply_f2d(L.dim, L.n, L.nt, x + i * ss, y + i * ss, L.geo32, L.g, t, 1, ctx->stream));
    if (i > 0)
      CK(launch_mass_couple<double, float, double>(L.dim, L.n, L.nt, x + (i - 1) * ss, y + i * ss, L.geo64, L.g,
                                                   L.cpl64, ctx->stream));
  }
  ctx->launches += 2 * L.nc - 1;
  return STMG_OK;
}

// z_j = B v_j, v_{j+1} = S z_j, CGS2 against v_0..v_j, Hessenberg column to the host buffer of
// parity j (hsm + (j % 2) * kColSlot).
// low: the operator apply in FP32 arithmetic (relaxed FGMRES), else double-float / FP64.
stmg_status fgmres_iteration_enqueue(stmg_ctx* ctx, int j, bool in_capture, bool low = false) {
  Level& L = ctx->levels[0];
  const int64_t n = L.size();
  double* v = ctx->V + (size_t)j * ctx->vld;
  double* z = ctx->Z + (size_t)j * n;
  double* w = ctx->V + (size_t)(j + 1) * ctx->vld;
  if (ctx->opt.vcycle_precision == STMG_FP32 && ctx->outer_df) {
    // z_j is exact in FP32: the V-cycle writes it straight into the FP32 basis Z32[j] (level 0's
    // output pointer is redirected for this iteration's graph), the double-float apply reads it,
    // and w starts from 0 (z_j vanishes on constrained rows).  The V-cycle input (float) v_j was
    // written by the previous iteration's normalisation, except at j = 0.
    float* z32 = ctx->Z32 + (size_t)j * n;
    if (j == 0 && !ctx->gs_df) {  // with the double-float basis the restart's normalisation wrote L.f32
      CK(launch_convert<double, float>(v, L.f32, n, ctx->stream));
      ctx->launches += 1;
    }
    float* saved = L.u32;
    L.u32 = z32;
    stmg_status st = in_capture ? vcycle_level<float>(ctx, 0) : run_vcycle<float>(ctx);
    L.u32 = saved;
    CKS(st);
    CK(cudaMemsetAsync(w, 0, sizeof(double) * n, ctx->stream));
    if (low) CKS(op_apply_f2d(ctx, L, z32, w));
    else CKS(op_apply_df(ctx, L, z32, w, false));
    return orthogonalise_enqueue(ctx, ctx->V, ctx->vld, j + 1, w, n, j + 1 < ctx->m ? L.f32 : nullptr,
                                 ctx->hsm + (j & 1) * kColSlot, ctx->gs_df);
  }
  if (ctx->opt.vcycle_precision == STMG_FP32) {
    CK(launch_convert<double, float>(v, L.f32, n, ctx->stream));
    if (in_capture) CKS(vcycle_level<float>(ctx, 0));
    else CKS(run_vcycle<float>(ctx));
    CK(launch_convert<float, double>(L.u32, z, n, ctx->stream));
    ctx->launches += 2;
    CKS(op_apply<double>(ctx, L, z, w));
  } else {
    CK(cudaMemcpyAsync(L.f64, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    if (in_capture) CKS(vcycle_level<double>(ctx, 0));
    else CKS(run_vcycle<double>(ctx));
    CK(cudaMemcpyAsync(z, L.u64, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    CKS(op_apply<double>(ctx, L, z, w));
  }
  return orthogonalise_enqueue(ctx, ctx->V, ctx->vld, j + 1, w, n, nullptr, ctx->hsm + (j & 1) * kColSlot);
}

stmg_status fgmres_iteration(stmg_ctx* ctx, int j, bool low = false) {
  const bool warmed = ctx->opt.vcycle_precision == STMG_FP32 ? ctx->warmed32 : ctx->warmed64;
  if (!warmed) return fgmres_iteration_enqueue(ctx, j, false, low);  // first V-cycle runs eagerly
  const int variant = (low ? 1 : 0) | (ctx->gs_df ? 2 : 0);
  std::vector<cudaGraphExec_t>& graphs = ctx->iter_graphs[variant];
  std::vector<int64_t>& kernels = ctx->iter_graph_kernels[variant];
  if ((int)graphs.size() < ctx->m) {
    graphs.assign(ctx->m, nullptr);
    kernels.assign(ctx->m, 0);
  }
  if (!graphs[j]) {
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    const int64_t saved = ctx->launches;
    stmg_status st = fgmres_iteration_enqueue(ctx, j, true, low);
    ctx->launches = saved;
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (st != STMG_OK) return st;
    if (e != cudaSuccess) { ctx->err = std::string("capture: ") + cudaGetErrorString(e); return STMG_ERR_CUDA; }
    size_t nn = 0;
    cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    cudaGraphGetNodes(graph, nodes.data(), &nn);
    int64_t nk = 0;
    for (auto nd : nodes) {
      cudaGraphNodeType ty;
      cudaGraphNodeGetType(nd, &ty);
      if (ty == cudaGraphNodeTypeKernel) ++nk;
    }
    e = cudaGraphInstantiate(&graphs[j], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { ctx->err = std::string("instantiate: ") + cudaGetErrorString(e); graphs[j] = nullptr; return STMG_ERR_CUDA; }
    kernels[j] = nk;
  }
  CK(cudaGraphLaunch(graphs[j], ctx->stream));
  ctx->launches += kernels[j];
  return STMG_OK;
}

stmg_status norm2(stmg_ctx* ctx, const double* x, int64_t n, double& out) {
  CKS(dot_self(ctx, x, n, ctx->dsm + 448));
  CK(cudaMemcpyAsync(ctx->hsm + 448, ctx->dsm + 448, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  out = std::sqrt(std::max(ctx->hsm[448], 0.0));
  return STMG_OK;
}

stmg_status solve_impl(stmg_ctx* ctx, const double* b, double* x, stmg_solve_stats* st) {
  Level& L = ctx->levels[0];
  const int64_t n = L.size();
  const int m = ctx->m;
  double bnorm = 0.0;
  CKS(norm2(ctx, b, n, bnorm));
  stmg_solve_stats s{};
  if (bnorm == 0.0) {
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (st) *st = s;
    return STMG_OK;
  }
  if (!std::isfinite(bnorm)) { ctx->err = "right-hand side is not finite"; return STMG_ERR_NONFINITE; }
  // stopping rule: ||b - S x|| <= max(rtol ||b||, atol) (the absolute part only when atol > 0)
  const double target = std::max(ctx->opt.rtol * bnorm, ctx->opt.atol);
  const bool df_residual = ctx->outer_df && target >= 1e-10 * bnorm;
  // the Krylov basis in double-float pairs (Gram-Schmidt on the FP32 pipe, about 44 bits) under the
  // same condition as the double-float residual; FP64 otherwise
  ctx->gs_df = df_residual;
  std::vector<double*> V(m + 1), Z(m);
  for (int j = 0; j <= m; ++j) V[j] = ctx->V + (size_t)j * ctx->vld;
  for (int j = 0; j < m; ++j) Z[j] = ctx->Z + (size_t)j * n;
  int its = 0;
  bool first = true;
  stmg_status result = STMG_OK;
  while (true) {
    CKS(op_residual_outer(ctx, L, b, x, V[0], df_residual));
    double beta = 0.0;
    CKS(norm2(ctx, V[0], n, beta));
    if (!std::isfinite(beta)) { ctx->err = "residual is not finite"; return STMG_ERR_NONFINITE; }
    if (first) { s.initial_rel_residual = beta / bnorm; first = false; }
    s.rel_residual = beta / bnorm;
    if (beta <= target) break;
    if (its >= ctx->opt.max_it) { result = STMG_ERR_NOT_CONVERGED; break; }
    if (its > 0) s.restarts++;
    if (ctx->gs_df) CK(launch_scale_to_df(V[0], 1.0 / beta, n, L.f32, ctx->stream));
    else CK(launch_axpby(0.0, V[0], 1.0 / beta, V[0], n, ctx->stream));
    ctx->launches += 1;
    std::vector<double> H((size_t)(m + 1) * m, 0.0), g(m + 1, 0.0), cs(m, 0.0), sn(m, 0.0);
    g[0] = beta;
    int jend = 0;
    // Iterations are pipelined: iteration j + 1 only needs v_{j+1}, which iteration j leaves on the
    // device, so it is enqueued before the host reads iteration j's Arnoldi column and the GPU does
    // not wait for the host round trip.  The host's decisions for it are taken from the residual
    // estimate extrapolated by the last contraction factor: whether the cycle goes on (not
    // speculated when the estimate is within kSpecMargin of the target, so that normally no
    // iteration is wasted; one that is wasted is simply not used) and the relaxed (FP32) apply.
    constexpr double kSpecMargin = 10.0;
    std::vector<char> lowv(m, 0);
    int enq = 0;          // iterations of this cycle enqueued so far
    double ratio = 1.0;   // last contraction |g_{j+1}| / |g_j|
    auto relax_ok = [&](double gest) { return ctx->opt.outer_relax && ctx->outer_df && gest <= target / kRelaxDelta; };
    auto enqueue = [&](int jj, bool lw) -> stmg_status {
      CKS(fgmres_iteration(ctx, jj, lw));
      CK(cudaEventRecord(ctx->ev_iter[jj & 1], ctx->stream));
      lowv[jj] = lw;
      enq = jj + 1;
      return STMG_OK;
    };
    CKS(enqueue(0, false));
    for (int j = 0; j < m; ++j) {
      if (enq == j + 1 && j + 1 < m && its + 1 < ctx->opt.max_it) {
        const double gpred = std::fabs(g[j]) * ratio;  // extrapolated |g_{j+1}|
        if (gpred > kSpecMargin * target) CKS(enqueue(j + 1, relax_ok(gpred)));
      }
      CK(cudaEventSynchronize(ctx->ev_iter[j & 1]));
      const double* col = ctx->hsm + (j & 1) * kColSlot;
      std::vector<double> h(col, col + j + 1);
      const double hn = col[j + 1];
      for (int i = 0; i <= j; ++i) {
        if (!std::isfinite(h[i])) { ctx->err = "preconditioned vector is not finite"; return STMG_ERR_NONFINITE; }
        H[(size_t)i * m + j] = h[i];
      }
      if (!std::isfinite(hn)) { ctx->err = "preconditioned vector is not finite"; return STMG_ERR_NONFINITE; }
      H[(size_t)(j + 1) * m + j] = hn;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)(i + 1) * m + j] = -sn[i] * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = t;
      }
      const double den = std::hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
      cs[j] = H[(size_t)j * m + j] / den;
      sn[j] = H[(size_t)(j + 1) * m + j] / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ratio = std::fabs(sn[j]);  // |g_{j+1}| / |g_j|
      ++its;
      jend = j + 1;
      if (lowv[j]) s.relaxed_iterations++;
      if (hn == 0.0) break;  // breakdown: the Krylov space is invariant, the update below is exact
      if (std::fabs(g[j + 1]) <= target || its >= ctx->opt.max_it) break;
      if (enq == j + 1 && j + 1 < m) CKS(enqueue(j + 1, relax_ok(std::fabs(g[j + 1]))));
    }
    std::vector<double> y(jend, 0.0);
    for (int i = jend - 1; i >= 0; --i) {
      double t = g[i];
      for (int l = i + 1; l < jend; ++l) t -= H[(size_t)i * m + l] * y[l];
      y[i] = t / H[(size_t)i * m + i];
    }
    CK(cudaMemcpyAsync(ctx->dsm + 320, y.data(), sizeof(double) * jend, cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->opt.vcycle_precision == STMG_FP32 && ctx->outer_df)
      CK(launch_multi_axpy<float>(x, ctx->Z32, n, ctx->dsm + 320, jend, 1.0, n, ctx->stream));
    else
      CK(launch_multi_axpy<double>(x, ctx->Z, n, ctx->dsm + 320, jend, 1.0, n, ctx->stream));
    ctx->launches += 1;
  }
  s.iterations = its;
  if (st) *st = s;
  CKS(check_device_status(ctx));
  if (result != STMG_OK) ctx->err = "FGMRES did not reach rtol within max_it";
  return result;
}

// One slab: rhs = RM_f (x) M f + RM_f0 M f0 + RA_u0 A u0 + RM_u0 M u0 + RM_v0 M v0, constrained rows 0
stmg_status rhs_slab(stmg_ctx* ctx, const double* f, const double* f0, const double* u0, const double* v0, double* rhs) {
  Level& L = ctx->levels[0];
  const int nt = L.nt;
  const int64_t nn = L.g.n_nodes;
  CK(cudaMemsetAsync(rhs, 0, sizeof(double) * L.slab_size(), ctx->stream));
  // mass terms: in double-float (FP32 pipe, about 44 bits) where the level has double-float geometry,
  // else FP64
  auto mass = [&](int ntm, const double* x, double* y, const OpTab<double>& tb) -> cudaError_t {
    if (!L.geodf) return launch_mass_apply(L.dim, L.n, ntm, x, y, L.geo64, L.g, tb, ctx->stream);
    OpTab<df64> td = L.tabdf;
    for (int i = 0; i < kMaxNT; ++i)
      for (int j = 0; j < kMaxNT; ++j) { td.TA[i][j] = df64(0.0f); td.TM[i][j] = df_split(tb.TM[i][j]); }
    td.sign = df64(1.0f);
    return launch_mass_apply_df(L.dim, L.n, ntm, x, y, L.geodf, L.g, td, ctx->stream);
  };
  OpTab<double> t = L.tab64;
  for (int i = 0; i < kMaxNT; ++i)
    for (int j = 0; j < kMaxNT; ++j) {
      t.TA[i][j] = 0.0;
      t.TM[i][j] = (i < nt && j < nt) ? L.sc.RM_f[i * nt + j] : 0.0;
    }
  t.sign = 1.0;
  if (f) CK(mass(nt, f, rhs, t));
  ctx->launches += 3;
  // single-block terms
  const double* srcs[4] = {f0, u0, u0, v0};
  const std::vector<double>* coef[4] = {&L.sc.RM_f0, &L.sc.RA_u0, &L.sc.RM_u0, &L.sc.RM_v0};
  const bool stiff[4] = {false, true, false, false};
  std::vector<const double*> xs;
  std::vector<double> C;
  std::vector<int> used;
  for (int term = 0; term < 4; ++term) {
    bool nz = false;
    for (double c : *coef[term]) nz = nz || c != 0.0;
    if (!nz || !srcs[term]) continue;
    double* out = ctx->tmp[term];
    CK(cudaMemsetAsync(out, 0, sizeof(double) * nn, ctx->stream));
    OpTab<double> t1 = L.tab64;
    for (int i = 0; i < kMaxNT; ++i)
      for (int j = 0; j < kMaxNT; ++j) { t1.TA[i][j] = 0.0; t1.TM[i][j] = 0.0; }
    if (stiff[term]) t1.TA[0][0] = 1.0; else t1.TM[0][0] = 1.0;
    t1.sign = 1.0;
    if (stiff[term]) CK(launch_apply<double>(L.dim, L.n, 1, srcs[term], out, L.geo64, L.g, t1, 0, ctx->stream));
    else CK(mass(1, srcs[term], out, t1));
    ctx->launches += 1;
    xs.push_back(out);
    used.push_back(term);
  }
  if (!xs.empty()) {
    const int nin = (int)xs.size();
    C.assign((size_t)nt * nin, 0.0);
    for (int i = 0; i < nt; ++i)
      for (int j = 0; j < nin; ++j) C[(size_t)i * nin + j] = (*coef[used[j]])[i];
    CK(launch_time_mix(xs.data(), nin, C.data(), nt, rhs, nn, 1, ctx->stream));
    ctx->launches += 1;
  }
  CK(launch_zero_constrained(rhs, L.g, nt, ctx->stream));
  return STMG_OK;
}

// Several slabs in one system (eq. heat-cg-dg-at-once): every slab gets its source term, only the
// first the previous end value u0 (the later ones take it from the coupling block).
stmg_status rhs_impl(stmg_ctx* ctx, const double* f, const double* f0, const double* u0, const double* v0, double* rhs) {
  const Level& L = ctx->levels[0];
  const int64_t ss = L.slab_size();
  for (int i = 0; i < L.nc; ++i)
    CKS(rhs_slab(ctx, f ? f + i * ss : nullptr, i == 0 ? f0 : nullptr, i == 0 ? u0 : nullptr, i == 0 ? v0 : nullptr,
                 rhs + i * ss));
  return STMG_OK;
}

stmg_status velocity_impl(stmg_ctx* ctx, const double* u, const double* u0, const double* v0, double* v) {
  Level& L = ctx->levels[0];
  const int nt = L.nt;
  const int64_t nn = L.g.n_nodes;
  std::vector<const double*> xs;
  std::vector<double> C;
  for (int j = 0; j < nt; ++j) xs.push_back(u + (int64_t)j * nn);
  xs.push_back(u0);
  if (v0) xs.push_back(v0);
  const int nin = (int)xs.size();
  C.assign((size_t)nt * nin, 0.0);
  for (int i = 0; i < nt; ++i) {
    for (int j = 0; j < nt; ++j) C[(size_t)i * nin + j] = L.sc.VU[i * nt + j];
    C[(size_t)i * nin + nt] = L.sc.Vu0[i];
    if (v0) C[(size_t)i * nin + nt + 1] = L.sc.Vv0[i];
  }
  CK(launch_time_mix(xs.data(), nin, C.data(), nt, v, nn, 0, ctx->stream));
  CK(launch_zero_constrained(v, L.g, nt, ctx->stream));
  return STMG_OK;
}

// Orders a call's work after the caller's stream and the caller's stream after the call.
struct StreamJoin {
  stmg_ctx* c;
  explicit StreamJoin(stmg_ctx* ctx) : c(ctx) {
    if (c && c->stream) {
      cudaEventRecord(c->ev_in, c->user_stream);
      cudaStreamWaitEvent(c->stream, c->ev_in, 0);
    }
  }
  ~StreamJoin() {
    if (c && c->stream) {
      cudaEventRecord(c->ev_out, c->stream);
      cudaStreamWaitEvent(c->user_stream, c->ev_out, 0);
    }
  }
};

stmg_status check_level(stmg_ctx* ctx, int level, int precision) {
  if (!ctx) return STMG_ERR_INVALID_ARG;
  if (level < 0 || level >= (int)ctx->levels.size()) return invalid(ctx, "level out of range");
  if (precision != STMG_FP32 && precision != STMG_FP64) return invalid(ctx, "precision must be FP32 or FP64");
  return STMG_OK;
}

}  // namespace

// Fixed scratch for stmg_smooth_noalloc: part of this file's device image.  stmg_create looks
// up its address, which loads the image, so every device on which a context was created holds
// the buffer until the process exits.  Host code must not use the symbol as a pointer; it asks
// the runtime for the device address instead.
static __device__ __align__(256) unsigned char g_noalloc_scratch[STMG_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of the fixed scratch on the current device.  Looking it up also loads this
// file's device image on that device (under lazy module loading it would otherwise load at the
// first lookup), so stmg_create calls this once and keeps the result in the context.
stmg_status resolve_noalloc_scratch(stmg_ctx* ctx) {
  CK(cudaGetDevice(&ctx->device));
  void* p = nullptr;
  CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  ctx->noalloc_scratch = p;
  return STMG_OK;
}

}  // namespace

extern "C" {

stmg_status stmg_create(stmg_ctx** out, const stmg_mesh* mesh, const stmg_problem* problem,
                        const stmg_options* options, void* stream) {
  if (!out) return STMG_ERR_INVALID_ARG;
  *out = nullptr;
  stmg_ctx* ctx = new stmg_ctx();
  ctx->user_stream = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ctx->ev_iter[i], cudaEventDisableTiming);
  if (e != cudaSuccess) {
    ctx->err = std::string("stream set-up: ") + cudaGetErrorString(e);
    *out = ctx;
    return STMG_ERR_CUDA;
  }
  stmg_status s = resolve_noalloc_scratch(ctx);
  if (s != STMG_OK) {
    *out = ctx;
    return s;
  }
  {
    StreamJoin join(ctx);
    s = create_impl(ctx, mesh, problem, options);
  }
  *out = ctx;  // returned even on error so that stmg_last_error can be read; destroy it
  return s;
}

stmg_status stmg_destroy(stmg_ctx* ctx) {
  if (!ctx) return STMG_OK;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (stmg_net* net : ctx->nets) net_detach(net);
  for (auto& gv : ctx->iter_graphs)
    for (auto g : gv)
      if (g) cudaGraphExecDestroy(g);
  if (ctx->graph32) cudaGraphExecDestroy(ctx->graph32);
  if (ctx->graph64) cudaGraphExecDestroy(ctx->graph64);
  for (void* p : ctx->allocations) cudaFree(p);
  if (ctx->hsm) cudaFreeHost(ctx->hsm);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  for (auto ev : ctx->ev_iter)
    if (ev) cudaEventDestroy(ev);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return STMG_OK;
}

const char* stmg_last_error(const stmg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

stmg_status stmg_sizes(const stmg_ctx* ctx, int64_t* n_nodes, int* n_t, int* n_levels) {
  if (!ctx || ctx->levels.empty()) return STMG_ERR_INVALID_ARG;
  if (n_nodes) *n_nodes = ctx->levels[0].g.n_nodes;
  if (n_t) *n_t = ctx->levels[0].nt;
  if (n_levels) *n_levels = (int)ctx->levels.size();
  return STMG_OK;
}

stmg_status stmg_level_slabs(const stmg_ctx* ctx, int level, int* n_slabs, double* tau) {
  if (!ctx || level < 0 || level >= (int)ctx->levels.size()) return STMG_ERR_INVALID_ARG;
  if (n_slabs) *n_slabs = ctx->levels[level].nc;
  if (tau) *tau = ctx->levels[level].tau;
  return STMG_OK;
}

stmg_status stmg_level_info(const stmg_ctx* ctx, int level, int* p, int* n_cells, int* k, int64_t* n_nodes, int* n_t,
                            double* omega) {
  if (!ctx || level < 0 || level >= (int)ctx->levels.size()) return STMG_ERR_INVALID_ARG;
  const Level& L = ctx->levels[level];
  if (p) *p = L.p;
  if (n_cells) *n_cells = L.N;
  if (k) *k = L.k;
  if (n_nodes) *n_nodes = L.g.n_nodes;
  if (n_t) *n_t = L.nt;
  if (omega) *omega = L.omega;
  return STMG_OK;
}

static void map_point(const Level& L, int64_t cell, const double* xi, double* out) {
  const int dim = L.dim;
  const int64_t nv1 = L.N + 1;
  const int64_t cx = cell % L.N, cy = (cell / L.N) % L.N, cz = dim == 3 ? cell / ((int64_t)L.N * L.N) : 0;
  for (int d = 0; d < dim; ++d) out[d] = 0.0;
  const int nvert = dim == 3 ? 8 : 4;
  for (int b = 0; b < nvert; ++b) {
    const int bits[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
    double f = 1.0;
    for (int d = 0; d < dim; ++d) f *= bits[d] ? xi[d] : 1.0 - xi[d];
    const int64_t vid = (cx + bits[0]) + nv1 * ((cy + bits[1]) + nv1 * (cz + bits[2]));
    for (int d = 0; d < dim; ++d) out[d] += f * L.vertices[vid * dim + d];
  }
}

// Q1 map of a cell and its Jacobian J[d][e] = d x_d / d xi_e at reference point xi.
static void map_point_jac(const Level& L, int64_t cell, const double* xi, double* x, double J[3][3]) {
  const int dim = L.dim;
  const int64_t nv1 = L.N + 1;
  const int64_t cx = cell % L.N, cy = (cell / L.N) % L.N, cz = dim == 3 ? cell / ((int64_t)L.N * L.N) : 0;
  for (int d = 0; d < 3; ++d) {
    x[d] = 0.0;
    for (int e = 0; e < 3; ++e) J[d][e] = 0.0;
  }
  const int nvert = dim == 3 ? 8 : 4;
  for (int b = 0; b < nvert; ++b) {
    const int bits[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
    double f[3], df[3];
    for (int d = 0; d < dim; ++d) { f[d] = bits[d] ? xi[d] : 1.0 - xi[d]; df[d] = bits[d] ? 1.0 : -1.0; }
    double val = 1.0;
    for (int d = 0; d < dim; ++d) val *= f[d];
    const int64_t vid = (cx + bits[0]) + nv1 * ((cy + bits[1]) + nv1 * (cz + bits[2]));
    for (int e = 0; e < dim; ++e) {
      double g = df[e];
      for (int d = 0; d < dim; ++d) if (d != e) g *= f[d];
      for (int d = 0; d < dim; ++d) J[d][e] += g * L.vertices[vid * dim + d];
    }
    for (int d = 0; d < dim; ++d) x[d] += val * L.vertices[vid * dim + d];
  }
}

// Cell and reference coordinates of physical point p on level L (Newton on the Q1 map of the cells
// whose vertex bounding box contains p); false if no cell contains it.
static bool locate_point(const Level& L, const double* p, int64_t& cell, double* xi) {
  const int dim = L.dim;
  const int64_t nv1 = L.N + 1;
  for (int64_t c = 0; c < L.g.n_cells; ++c) {
    const int64_t cx = c % L.N, cy = (c / L.N) % L.N, cz = dim == 3 ? c / ((int64_t)L.N * L.N) : 0;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int b = 0; b < (dim == 3 ? 8 : 4); ++b) {
      const int64_t vid = (cx + (b & 1)) + nv1 * ((cy + ((b >> 1) & 1)) + nv1 * (cz + ((b >> 2) & 1)));
      for (int d = 0; d < dim; ++d) {
        lo[d] = std::min(lo[d], L.vertices[vid * dim + d]);
        hi[d] = std::max(hi[d], L.vertices[vid * dim + d]);
      }
    }
    bool in = true;
    for (int d = 0; d < dim; ++d) in = in && p[d] >= lo[d] - 1e-9 && p[d] <= hi[d] + 1e-9;
    if (!in) continue;
    double r[3] = {0.5, 0.5, 0.5}, x[3], J[3][3];
    for (int it = 0; it < 50; ++it) {
      map_point_jac(L, c, r, x, J);
      // solve J s = x - p (dim <= 3, Cramer)
      double b[3] = {x[0] - p[0], x[1] - p[1], dim == 3 ? x[2] - p[2] : 0.0}, st[3] = {0.0, 0.0, 0.0};
      if (dim == 2) {
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        st[0] = (b[0] * J[1][1] - J[0][1] * b[1]) / det;
        st[1] = (J[0][0] * b[1] - b[0] * J[1][0]) / det;
      } else {
        const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                           J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                           J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        for (int k = 0; k < 3; ++k) {
          double M[3][3];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i][j] = j == k ? b[i] : J[i][j];
          st[k] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                   M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
        }
      }
      double mx = 0.0;
      for (int d = 0; d < dim; ++d) { r[d] -= st[d]; mx = std::max(mx, std::fabs(st[d])); }
      if (mx < 1e-15) break;
    }
    bool inside = true;
    for (int d = 0; d < dim; ++d) inside = inside && r[d] >= -1e-12 && r[d] <= 1.0 + 1e-12;
    if (inside) {
      cell = c;
      for (int d = 0; d < dim; ++d) xi[d] = std::min(1.0, std::max(0.0, r[d]));
      return true;
    }
  }
  return false;
}

stmg_status stmg_point_values(stmg_ctx* ctx, const double* u, int npts, const double* xyz, double* out) {
  if (!ctx || !u || !xyz || !out || npts < 0) return STMG_ERR_INVALID_ARG;
  if (npts == 0) return STMG_OK;
  StreamJoin join_(ctx);
  const Level& L = ctx->levels[0];
  const int n = L.n, dim = L.dim, nb = dim == 3 ? n * n * n : n * n;
  const int ncomp = L.nc * L.nt;
  std::vector<double> xn = space_nodes(L.p);
  std::vector<int64_t> nodes((size_t)npts * nb);
  std::vector<double> w((size_t)npts * nb);
  for (int pt = 0; pt < npts; ++pt) {
    int64_t c = 0;
    double xi[3] = {0.0, 0.0, 0.0};
    if (!locate_point(L, xyz + (size_t)pt * dim, c, xi))
      return invalid(ctx, "point " + std::to_string(pt) + " lies outside the grid");
    const int64_t cx = c % L.N, cy = (c / L.N) % L.N, cz = dim == 3 ? c / ((int64_t)L.N * L.N) : 0;
    for (int a = 0; a < nb; ++a) {
      const int ai[3] = {a % n, (a / n) % n, a / (n * n)};
      double phi = 1.0;
      for (int d = 0; d < dim; ++d) phi *= lagrange(xn, ai[d], xi[d]);
      const int64_t gx = cx * L.p + ai[0], gy = cy * L.p + ai[1], gz = dim == 3 ? cz * L.p + ai[2] : 0;
      nodes[(size_t)pt * nb + a] = gx + (int64_t)L.g.nn1 * (gy + (int64_t)L.g.nn1 * gz);
      w[(size_t)pt * nb + a] = phi;
    }
  }
  void* buf = nullptr;
  const size_t bytes = (size_t)npts * nb * (sizeof(int64_t) + sizeof(double)) + (size_t)npts * ncomp * sizeof(double);
  CK(cudaMalloc(&buf, bytes));
  int64_t* d_nodes = reinterpret_cast<int64_t*>(buf);
  double* d_w = reinterpret_cast<double*>(d_nodes + (size_t)npts * nb);
  double* d_out = d_w + (size_t)npts * nb;
  cudaError_t e = cudaMemcpyAsync(d_nodes, nodes.data(), sizeof(int64_t) * nodes.size(), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_w, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = launch_point_values(u, L.g.n_nodes, ncomp, d_nodes, d_w, nb, npts, d_out, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, sizeof(double) * npts * ncomp, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  ctx->launches += 1;
  cudaFree(buf);
  CK(e);
  return STMG_OK;
}

stmg_status stmg_node_coords(const stmg_ctx* ctx, int level, double* xyz) {
  if (!ctx || !xyz || level < 0 || level >= (int)ctx->levels.size()) return STMG_ERR_INVALID_ARG;
  const Level& L = ctx->levels[level];
  std::vector<double> xn = space_nodes(L.p);
  const int n = L.n, dim = L.dim;
  const int nb = dim == 3 ? n * n * n : n * n;
  for (int64_t c = 0; c < L.g.n_cells; ++c) {
    const int64_t cx = c % L.N, cy = (c / L.N) % L.N, cz = dim == 3 ? c / ((int64_t)L.N * L.N) : 0;
    for (int a = 0; a < nb; ++a) {
      const int ai[3] = {a % n, (a / n) % n, a / (n * n)};
      const double xi[3] = {xn[ai[0]], xn[ai[1]], dim == 3 ? xn[ai[2]] : 0.0};
      const int64_t gx = cx * L.p + ai[0], gy = cy * L.p + ai[1], gz = dim == 3 ? cz * L.p + ai[2] : 0;
      const int64_t node = gx + (int64_t)L.g.nn1 * (gy + (int64_t)L.g.nn1 * gz);
      map_point(L, c, xi, xyz + node * dim);
    }
  }
  return STMG_OK;
}

stmg_status stmg_qpoint_coords(const stmg_ctx* ctx, int level, double* xyz) {
  if (!ctx || !xyz || level < 0 || level >= (int)ctx->levels.size()) return STMG_ERR_INVALID_ARG;
  const Level& L = ctx->levels[level];
  std::vector<double> xq, wq;
  gauss_legendre(L.n, xq, wq);
  const int n = L.n, dim = L.dim;
  const int nq = dim == 3 ? n * n * n : n * n;
  for (int64_t c = 0; c < L.g.n_cells; ++c)
    for (int q = 0; q < nq; ++q) {
      const double xi[3] = {xq[q % n], xq[(q / n) % n], dim == 3 ? xq[q / (n * n)] : 0.0};
      map_point(L, c, xi, xyz + (c * nq + q) * dim);
    }
  return STMG_OK;
}

stmg_status stmg_apply(stmg_ctx* ctx, int level, int precision, const void* x, void* y) {
  StreamJoin join_(ctx);
  if (ctx && precision == STMG_DF32) {
    if (level != 0 || !ctx->levels[0].geodf)
      return invalid(ctx, "DF32 applies exist on level 0 of a context with outer_apply = DF32");
    return op_apply_df(ctx, ctx->levels[0], (const float*)x, (double*)y);
  }
  CKS(check_level(ctx, level, precision));
  Level& L = ctx->levels[level];
  if (precision == STMG_FP64) return op_apply<double>(ctx, L, (const double*)x, (double*)y);
  return op_apply<float>(ctx, L, (const float*)x, (float*)y);
}

stmg_status stmg_residual(stmg_ctx* ctx, int level, int precision, const void* f, const void* u, void* r) {
  StreamJoin join_(ctx);
  CKS(check_level(ctx, level, precision));
  Level& L = ctx->levels[level];
  if (precision == STMG_FP64) return op_residual<double>(ctx, L, (const double*)f, (const double*)u, (double*)r);
  return op_residual<float>(ctx, L, (const float*)f, (const float*)u, (float*)r);
}

stmg_status stmg_smooth(stmg_ctx* ctx, int level, int precision, int sweeps, const void* f, void* u) {
  StreamJoin join_(ctx);
  CKS(check_level(ctx, level, precision));
  if (level == (int)ctx->levels.size() - 1) return invalid(ctx, "the coarsest level has no smoother");
  if (sweeps < 0) return invalid(ctx, "sweeps must be >= 0");
  Level& L = ctx->levels[level];
  if (precision == STMG_FP64) return op_smooth<double>(ctx, level, sweeps, (const double*)f, (double*)u, L.r64);
  return op_smooth<float>(ctx, level, sweeps, (const float*)f, (float*)u, L.r32);
}

stmg_status stmg_restrict(stmg_ctx* ctx, int level, int precision, const void* rf, void* rc) {
  StreamJoin join_(ctx);
  CKS(check_level(ctx, level, precision));
  if (level == (int)ctx->levels.size() - 1) return invalid(ctx, "no coarser level");
  if (precision == STMG_FP64) return op_restrict<double>(ctx, level, (const double*)rf, (double*)rc);
  return op_restrict<float>(ctx, level, (const float*)rf, (float*)rc);
}

stmg_status stmg_prolongate_add(stmg_ctx* ctx, int level, int precision, const void* ec, void* uf) {
  StreamJoin join_(ctx);
  CKS(check_level(ctx, level, precision));
  if (level == (int)ctx->levels.size() - 1) return invalid(ctx, "no coarser level");
  if (precision == STMG_FP64) return op_prolongate_add<double>(ctx, level, (const double*)ec, (double*)uf);
  return op_prolongate_add<float>(ctx, level, (const float*)ec, (float*)uf);
}

stmg_status stmg_vcycle(stmg_ctx* ctx, int precision, const void* r, void* e) {
  StreamJoin join_(ctx);
  CKS(check_level(ctx, 0, precision));
  if (precision == STMG_FP64) return vcycle_public<double>(ctx, (const double*)r, (double*)e);
  return vcycle_public<float>(ctx, (const float*)r, (float*)e);
}

stmg_status stmg_rhs(stmg_ctx* ctx, const double* f, const double* f0, const double* u0, const double* v0, double* rhs) {
  StreamJoin join_(ctx);
  if (!ctx || !rhs) return STMG_ERR_INVALID_ARG;
  return rhs_impl(ctx, f, f0, u0, v0, rhs);
}

stmg_status stmg_solve(stmg_ctx* ctx, const double* rhs, double* u, stmg_solve_stats* stats) {
  StreamJoin join_(ctx);
  if (!ctx || !rhs || !u) return STMG_ERR_INVALID_ARG;
  const stmg_status s = solve_impl(ctx, rhs, u, stats);
  // a bounded device wait that gave up invalidates every result of the call, whatever path it took
  if (s != STMG_ERR_CUDA && check_device_status(ctx) == STMG_ERR_TIMEOUT) return STMG_ERR_TIMEOUT;
  return s;
}

stmg_status stmg_wave_velocity(stmg_ctx* ctx, const double* u, const double* u0, const double* v0, double* v) {
  StreamJoin join_(ctx);
  if (!ctx || !u || !u0 || !v) return STMG_ERR_INVALID_ARG;
  if (ctx->pde != STMG_WAVE) return invalid(ctx, "velocity update needs the wave equation");
  return velocity_impl(ctx, u, u0, v0, v);
}

stmg_status stmg_guess_previous(stmg_ctx* ctx, const double* u0, double* u) {
  StreamJoin join_(ctx);
  if (!ctx || !u0 || !u) return STMG_ERR_INVALID_ARG;
  Level& L = ctx->levels[0];
  CK(launch_broadcast_time(u0, u, L.nt * L.nc, L.g.n_nodes, ctx->stream));
  ctx->launches += 1;
  return STMG_OK;
}

stmg_status stmg_solve_slab_host(stmg_ctx* ctx, const double* f, const double* f0, const double* u0, const double* v0,
                                 double* u, double* v, stmg_solve_stats* stats) {
  StreamJoin join_(ctx);
  if (!ctx || !f || !u0 || !u) return STMG_ERR_INVALID_ARG;
  Level& L = ctx->levels[0];
  const int64_t nn = L.g.n_nodes, n = L.size();
  double* d_f = ctx->u_buf;                 // n
  double* d_u = ctx->u_buf + n;             // n
  double* d_f0 = ctx->u_buf + 3 * n;        // nn each
  double* d_u0 = d_f0 + nn;
  double* d_v0 = d_u0 + nn;
  CK(cudaMemcpyAsync(d_f, f, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d_u0, u0, sizeof(double) * nn, cudaMemcpyHostToDevice, ctx->stream));
  if (f0) CK(cudaMemcpyAsync(d_f0, f0, sizeof(double) * nn, cudaMemcpyHostToDevice, ctx->stream));
  if (v0) CK(cudaMemcpyAsync(d_v0, v0, sizeof(double) * nn, cudaMemcpyHostToDevice, ctx->stream));
  CKS(rhs_impl(ctx, d_f, f0 ? d_f0 : nullptr, d_u0, v0 ? d_v0 : nullptr, ctx->rhs_buf));
  CK(launch_broadcast_time(d_u0, d_u, L.nt * L.nc, nn, ctx->stream));
  ctx->launches += 1;
  stmg_status s = solve_impl(ctx, ctx->rhs_buf, d_u, stats);
  if (s != STMG_OK && s != STMG_ERR_NOT_CONVERGED) return s;
  CK(cudaMemcpyAsync(u, d_u, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  if (v && ctx->pde == STMG_WAVE) {
    double* vbuf = ctx->rhs_buf;  // rhs no longer needed
    CKS(velocity_impl(ctx, d_u, d_u0, v0 ? d_v0 : nullptr, vbuf));
    CK(cudaMemcpyAsync(v, vbuf, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return s;
}

stmg_status stmg_smooth_noalloc(stmg_ctx* ctx, int level, int precision, int sweeps, const void* f, void* u) {
  CKS(check_level(ctx, level, precision));
  if (level == (int)ctx->levels.size() - 1) return invalid(ctx, "the coarsest level has no smoother");
  if (sweeps < 0) return invalid(ctx, "sweeps must be >= 0");
  Level& L = ctx->levels[level];
  const size_t bytes = (size_t)L.size() * (precision == STMG_FP64 ? sizeof(double) : sizeof(float));
  if (bytes > (size_t)STMG_NOALLOC_SCRATCH_BYTES)
    return invalid(ctx, "stmg_smooth_noalloc: level needs " + std::to_string(bytes) +
                            " bytes of residual scratch, more than the fixed " +
                            std::to_string((long long)STMG_NOALLOC_SCRATCH_BYTES) + " bytes");
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != ctx->device)
    return invalid(ctx, "stmg_smooth_noalloc: the device that was current at stmg_create must be current");
  void* scratch = ctx->noalloc_scratch;
  StreamJoin join_(ctx);
  // every sweep overwrites the whole residual before reading it: nothing to clear
  if (precision == STMG_FP64)
    return op_smooth<double>(ctx, level, sweeps, (const double*)f, (double*)u, reinterpret_cast<double*>(scratch));
  return op_smooth<float>(ctx, level, sweeps, (const float*)f, (float*)u, reinterpret_cast<float*>(scratch));
}


// ------------------------------------------------------------------ learned initial guess
struct stmg_net {
  stmg_ctx* ctx = nullptr;  // null once the context has been destroyed
  NetDev d;
  std::vector<void*> allocs;
  std::vector<int> ch;
};

static void net_detach(stmg_net* net) { net->ctx = nullptr; }

static stmg_status net_alloc(stmg_net* net, void** p, size_t bytes) {
  stmg_ctx* ctx = net->ctx;
  cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
  if (e != cudaSuccess) {
    ctx->err = std::string("cudaMalloc (net): ") + cudaGetErrorString(e);
    return STMG_ERR_OOM;
  }
  net->allocs.push_back(*p);
  return cudaMemsetAsync(*p, 0, std::max<size_t>(bytes, 16), ctx->stream) == cudaSuccess ? STMG_OK : STMG_ERR_CUDA;
}

stmg_status stmg_net_destroy(stmg_net* net) {
  if (!net) return STMG_OK;
  if (net->ctx) {
    auto& v = net->ctx->nets;
    v.erase(std::remove(v.begin(), v.end(), net), v.end());
    if (net->ctx->stream) cudaStreamSynchronize(net->ctx->stream);
  }  // a detached network has no work in flight: its context synchronised when it was destroyed
  for (void* p : net->allocs) cudaFree(p);
  delete net;
  return STMG_OK;
}

stmg_status stmg_net_create(stmg_net** out, stmg_ctx* ctx, int layers, const int* channels, const double* weights,
                            const double* biases, const double* scales) {
  if (!out || !ctx || !channels || !weights || !biases || !scales) return STMG_ERR_INVALID_ARG;
  *out = nullptr;
  Level& L0 = ctx->levels[0];
  if (L0.nc != 1) return invalid(ctx, "the learned guess needs one slab per system");
  if (layers < 1 || layers > kNetMaxLayers) return invalid(ctx, "layers must be in 1..8");
  if (channels[0] != 2 * L0.nt || channels[layers] != L0.nt)
    return invalid(ctx, "network must map 2 N_t input channels to N_t output channels");
  for (int l = 0; l <= layers; ++l)
    if (channels[l] < 1 || channels[l] > 64) return invalid(ctx, "channel counts must be in 1..64");
  StreamJoin join_(ctx);
  stmg_net* net = new stmg_net();
  net->ctx = ctx;
  NetDev& d = net->d;
  d.L = layers;
  d.nt = L0.nt;
  d.nx = L0.g.nn1;
  d.ny = L0.g.nn1;
  d.nz = L0.dim == 3 ? L0.g.nn1 : 1;
  d.V = L0.g.n_nodes;
  d.nxp = d.nx + 2;
  d.nyp = d.ny + 2;
  d.nzp = d.nz + 2;
  d.Vp = (int64_t)d.nxp * d.nyp * d.nzp;
  d.status = ctx->status;
  d.su = (float)scales[0];
  d.sf = (float)scales[1];
  d.so = (float)scales[2];
  for (int l = 0; l <= layers; ++l) { d.ch[l] = channels[l]; d.cp[l] = net_pad(channels[l]); net->ch.push_back(channels[l]); }
  auto fail = [&](stmg_status st) { stmg_net_destroy(net); return st; };
  size_t woff = 0, boff = 0;
  for (int l = 0; l < layers; ++l) {
    const int ci = d.ch[l], co = d.ch[l + 1], cip = d.cp[l], cop = d.cp[l + 1];
    const size_t nw = (size_t)27 * cop * cip;
    std::vector<float> w(nw, 0.f), b(cop, 0.f);
    for (int o = 0; o < co; ++o) {
      for (int c = 0; c < ci; ++c)
        for (int t = 0; t < 27; ++t) w[((size_t)t * cop + o) * cip + c] = (float)weights[woff + ((size_t)o * ci + c) * 27 + t];
      b[o] = (float)biases[boff + o];
    }
    woff += (size_t)co * ci * 27;
    boff += co;
    stmg_status st;
    if ((st = net_alloc(net, (void**)&d.w32[l], nw * 4)) != STMG_OK) return fail(st);
    if ((st = net_alloc(net, (void**)&d.wt[l], nw * 2)) != STMG_OK) return fail(st);
    if ((st = net_alloc(net, (void**)&d.wtT[l], nw * 2)) != STMG_OK) return fail(st);
    if ((st = net_alloc(net, (void**)&d.gw[l], nw * 4)) != STMG_OK) return fail(st);
    if ((st = net_alloc(net, (void**)&d.mw[l], nw * 4)) != STMG_OK) return fail(st);
    if ((st = net_alloc(net, (void**)&d.vw[l], nw * 4)) != STMG_OK) return fail(st);
    if ((st = net_alloc(net, (void**)&d.bias[l], cop * 4)) != STMG_OK) return fail(st);
    if ((st = net_alloc(net, (void**)&d.gb[l], cop * 4)) != STMG_OK) return fail(st);
    if ((st = net_alloc(net, (void**)&d.mb[l], cop * 4)) != STMG_OK) return fail(st);
    if ((st = net_alloc(net, (void**)&d.vb[l], cop * 4)) != STMG_OK) return fail(st);
    if (cudaMemcpyAsync(d.w32[l], w.data(), nw * 4, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaMemcpyAsync(d.bias[l], b.data(), cop * 4, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess)
      return fail(STMG_ERR_CUDA);
  }
  for (int l = 0; l <= layers; ++l) {
    stmg_status st;
    if (l < layers && (st = net_alloc(net, (void**)&d.act[l], (size_t)d.Vp * d.cp[l] * 2)) != STMG_OK) return fail(st);
    if (l >= 1 && (st = net_alloc(net, (void**)&d.grad[l], (size_t)d.Vp * d.cp[l] * 2)) != STMG_OK) return fail(st);
  }
  stmg_status st;
  if ((st = net_alloc(net, (void**)&d.out, (size_t)d.Vp * d.cp[layers] * 4)) != STMG_OK) return fail(st);
  if (net_make_tmaps(d) != cudaSuccess) {
    ctx->err = "tensor maps of the network's convolutions could not be encoded";
    return fail(STMG_ERR_CUDA);
  }
  if ((st = net_alloc(net, (void**)&d.loss, 8)) != STMG_OK) return fail(st);
  if (net_refresh_bf16(d, ctx->stream) != cudaSuccess || cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return fail(STMG_ERR_CUDA);
  ctx->nets.push_back(net);
  *out = net;
  return STMG_OK;
}

stmg_status stmg_net_predict(stmg_net* net, const double* u_prev, const double* f, double* u_guess) {
  if (!net || !net->ctx || !u_prev || !f || !u_guess) return STMG_ERR_INVALID_ARG;
  stmg_ctx* ctx = net->ctx;
  StreamJoin join_(ctx);
  CK(net_forward(net->d, u_prev, f, ctx->stream));
  CK(net_guess(net->d, u_prev, u_guess, ctx->stream));
  ctx->launches += 2 + net->d.L;
  return STMG_OK;
}

static stmg_status net_fb(stmg_net* net, const double* u_prev, const double* f, const double* u_target, double* loss) {
  stmg_ctx* ctx = net->ctx;
  CK(net_forward(net->d, u_prev, f, ctx->stream));
  CK(net_backward(net->d, u_prev, u_target, net->d.loss, ctx->stream));
  CK(cudaMemcpyAsync(ctx->hsm + 500, net->d.loss, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (loss) *loss = ctx->hsm[500];
  ctx->launches += 1 + 2 * net->d.L + 1 + 3 * net->d.L;
  return STMG_OK;
}

stmg_status stmg_net_train_step(stmg_net* net, const double* u_prev, const double* f, const double* u_target, double lr,
                                double* loss) {
  if (!net || !net->ctx || !u_prev || !f || !u_target) return STMG_ERR_INVALID_ARG;
  stmg_ctx* ctx = net->ctx;
  StreamJoin join_(ctx);
  CKS(net_fb(net, u_prev, f, u_target, loss));
  if (!std::isfinite(ctx->hsm[500])) { ctx->err = "network loss is not finite"; return STMG_ERR_NONFINITE; }
  CK(net_adam(net->d, (float)lr, ctx->stream));
  ctx->launches += 3 * net->d.L;
  return STMG_OK;
}

stmg_status stmg_net_gradients(stmg_net* net, const double* u_prev, const double* f, const double* u_target,
                               double* loss, double* grad_w, double* grad_b, double* out_host) {
  if (!net || !net->ctx || !u_prev || !f || !u_target) return STMG_ERR_INVALID_ARG;
  stmg_ctx* ctx = net->ctx;
  StreamJoin join_(ctx);
  CKS(net_fb(net, u_prev, f, u_target, loss));
  const NetDev& d = net->d;
  size_t woff = 0, boff = 0;
  for (int l = 0; l < d.L; ++l) {
    const int ci = d.ch[l], co = d.ch[l + 1], cip = d.cp[l], cop = d.cp[l + 1];
    std::vector<float> gw((size_t)27 * cop * cip), gb(cop);
    CK(cudaMemcpy(gw.data(), d.gw[l], gw.size() * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(gb.data(), d.gb[l], gb.size() * 4, cudaMemcpyDeviceToHost));
    if (grad_w)
      for (int o = 0; o < co; ++o)
        for (int c = 0; c < ci; ++c)
          for (int t = 0; t < 27; ++t) grad_w[woff + ((size_t)o * ci + c) * 27 + t] = gw[((size_t)t * cop + o) * cip + c];
    if (grad_b)
      for (int o = 0; o < co; ++o) grad_b[boff + o] = gb[o];
    woff += (size_t)co * ci * 27;
    boff += co;
  }
  if (out_host) {
    const int cpl = d.cp[d.L];
    std::vector<float> o((size_t)d.Vp * cpl);
    CK(cudaMemcpy(o.data(), d.out, o.size() * 4, cudaMemcpyDeviceToHost));
    for (int c = 0; c < d.ch[d.L]; ++c)
      for (int64_t v = 0; v < d.V; ++v) out_host[(size_t)c * d.V + v] = o[(size_t)net_row(d, v) * cpl + c];
  }
  return STMG_OK;
}

stmg_status stmg_net_weights(stmg_net* net, double* w, double* b) {
  if (!net || !net->ctx) return STMG_ERR_INVALID_ARG;
  stmg_ctx* ctx = net->ctx;
  StreamJoin join_(ctx);
  CK(cudaStreamSynchronize(ctx->stream));
  const NetDev& d = net->d;
  size_t woff = 0, boff = 0;
  for (int l = 0; l < d.L; ++l) {
    const int ci = d.ch[l], co = d.ch[l + 1], cip = d.cp[l], cop = d.cp[l + 1];
    std::vector<float> hw((size_t)27 * cop * cip), hb(cop);
    CK(cudaMemcpy(hw.data(), d.w32[l], hw.size() * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hb.data(), d.bias[l], hb.size() * 4, cudaMemcpyDeviceToHost));
    if (w)
      for (int o = 0; o < co; ++o)
        for (int c = 0; c < ci; ++c)
          for (int t = 0; t < 27; ++t) w[woff + ((size_t)o * ci + c) * 27 + t] = hw[((size_t)t * cop + o) * cip + c];
    if (b)
      for (int o = 0; o < co; ++o) b[boff + o] = hb[o];
    woff += (size_t)co * ci * 27;
    boff += co;
  }
  return STMG_OK;
}

stmg_status stmg_select_guess(stmg_ctx* ctx, const double* rhs, const double* candidate, double* u, int* chosen) {
  if (!ctx || !rhs || !candidate || !u) return STMG_ERR_INVALID_ARG;
  StreamJoin join_(ctx);
  Level& L = ctx->levels[0];
  const int64_t n = L.size();
  double* r = ctx->V;  // Krylov workspace is free between solves
  double r_cur = 0.0, r_cand = 0.0;
  CKS(op_residual<double>(ctx, L, rhs, u, r));
  CKS(norm2(ctx, r, n, r_cur));
  CKS(op_residual<double>(ctx, L, rhs, candidate, r));
  CKS(norm2(ctx, r, n, r_cand));
  const bool take = std::isfinite(r_cand) && r_cand < r_cur;
  if (take) CK(cudaMemcpyAsync(u, candidate, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  if (chosen) *chosen = take ? 1 : 0;
  return STMG_OK;
}

stmg_status stmg_solve_slab_host_learned(stmg_ctx* ctx, stmg_net* net, const double* f, const double* u_prev,
                                         double* u, int* chosen, stmg_solve_stats* stats) {
  if (!ctx || !net || !f || !u_prev || !u) return STMG_ERR_INVALID_ARG;
  if (net->ctx != ctx) return invalid(ctx, "network is bound to another context");
  if (ctx->pde != STMG_HEAT || ctx->scheme != STMG_DG || ctx->levels[0].nc != 1)
    return invalid(ctx, "learned slab step supports heat dG with one slab per system");
  StreamJoin join_(ctx);
  Level& L = ctx->levels[0];
  const int64_t nn = L.g.n_nodes, n = L.size();
  double* d_f = ctx->u_buf;
  double* d_u = ctx->u_buf + n;
  double* d_prev = ctx->u_buf + 2 * n;
  double* d_cand = ctx->Z;  // Krylov workspace is free before the solve
  CK(cudaMemcpyAsync(d_f, f, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(d_prev, u_prev, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  const double* d_u0 = d_prev + (int64_t)(L.nt - 1) * nn;
  CKS(rhs_impl(ctx, d_f, nullptr, d_u0, nullptr, ctx->rhs_buf));
  CK(launch_broadcast_time(d_u0, d_u, L.nt, nn, ctx->stream));
  CK(net_forward(net->d, d_prev, d_f, ctx->stream));
  CK(net_guess(net->d, d_prev, d_cand, ctx->stream));
  ctx->launches += 3 + net->d.L;
  double r_prev = 0.0, r_cand = 0.0;
  double* r = ctx->V;
  CKS(op_residual<double>(ctx, L, ctx->rhs_buf, d_u, r));
  CKS(norm2(ctx, r, n, r_prev));
  CKS(op_residual<double>(ctx, L, ctx->rhs_buf, d_cand, r));
  CKS(norm2(ctx, r, n, r_cand));
  const bool take = std::isfinite(r_cand) && r_cand < r_prev;
  if (take) CK(cudaMemcpyAsync(d_u, d_cand, sizeof(double) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  if (chosen) *chosen = take ? 1 : 0;
  stmg_status s = solve_impl(ctx, ctx->rhs_buf, d_u, stats);
  if (s != STMG_OK && s != STMG_ERR_NOT_CONVERGED) return s;
  CK(cudaMemcpyAsync(u, d_u, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return s;
}

stmg_status stmg_selftest_device_timeout(stmg_ctx* ctx) {
  if (!ctx) return STMG_ERR_INVALID_ARG;
  StreamJoin join_(ctx);
  CK(launch_wait_selftest(ctx->status, ctx->stream));
  ctx->launches += 1;
  return check_device_status(ctx);
}

stmg_status stmg_launch_count(const stmg_ctx* ctx, int64_t* count) {
  if (!ctx || !count) return STMG_ERR_INVALID_ARG;
  *count = ctx->launches;
  return STMG_OK;
}

stmg_status stmg_time_kernel(stmg_ctx* ctx, int kernel, int level, int precision, int reps, double* avg_ms) {
  if (kernel == STMG_KERNEL_ORTHO) {
    if (!ctx || level < 1 || level > ctx->m || reps < 1 || !avg_ms ||
        (precision != STMG_FP64 && precision != STMG_DF32))
      return invalid(ctx, "ortho timing: 1 <= level <= fgmres_restart basis vectors, FP64 or DF32, reps >= 1");
    const int64_t n = ctx->levels[0].size();
    const bool dfb = precision == STMG_DF32;
    // a basis and a vector with nonzero entries (timing only: byte pattern 0x3f in every word)
    CK(cudaMemsetAsync(ctx->V, 0x3f, sizeof(double) * (size_t)(level + 1) * ctx->vld, ctx->stream));
    double* w = ctx->V + (size_t)level * ctx->vld;
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    CKS(orthogonalise_enqueue(ctx, ctx->V, ctx->vld, level, w, n, ctx->levels[0].f32, nullptr, dfb));
    CK(cudaEventRecord(a, ctx->stream));
    for (int i = 0; i < reps; ++i) CKS(orthogonalise_enqueue(ctx, ctx->V, ctx->vld, level, w, n, ctx->levels[0].f32, nullptr, dfb));
    CK(cudaEventRecord(b, ctx->stream));
    CK(cudaEventSynchronize(b));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    *avg_ms = (double)ms / reps;
    return STMG_OK;
  }
  const bool df = precision == STMG_DF32;
  if (df && (!ctx || kernel != STMG_KERNEL_APPLY || level != 0 || !ctx->levels[0].geodf))
    return invalid(ctx, "DF32 timing exists for the level-0 apply of a context with outer_apply = DF32");
  CKS(check_level(ctx, level, df ? STMG_FP64 : precision));
  if (reps < 1 || !avg_ms) return invalid(ctx, "reps must be >= 1");
  if (kernel != STMG_KERNEL_APPLY && kernel != STMG_KERNEL_ASM && kernel != STMG_KERNEL_VCYCLE)
    return invalid(ctx, "unknown kernel id");
  if (kernel == STMG_KERNEL_ASM && level == (int)ctx->levels.size() - 1) return invalid(ctx, "no smoother there");
  Level& L = ctx->levels[level];
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  auto once = [&]() -> stmg_status {
    if (kernel == STMG_KERNEL_VCYCLE) {
      if (precision == STMG_FP64) return run_vcycle<double>(ctx);
      return run_vcycle<float>(ctx);
    }
    if (kernel == STMG_KERNEL_APPLY) {
      if (df) {
        OpTab<df64> t = L.tabdf;
        CK(launch_apply_df(L.dim, L.n, L.nt, L.u32, L.r64, L.geodf, L.g, t, 1, ctx->stream));
      } else if (precision == STMG_FP64) {
        OpTab<double> t = L.tab64;
        CK(launch_apply<double>(L.dim, L.n, L.nt, L.u64, L.r64, L.geo64, L.g, t, 1, ctx->stream));
      } else {
        OpTab<float> t = L.tab32;
        CK(launch_apply<float>(L.dim, L.n, L.nt, L.u32, L.r32, L.geo32, L.g, t, 1, ctx->stream));
      }
      return STMG_OK;
    }
    if (precision == STMG_FP64) return op_asm<double>(ctx, L, L.r64, L.u64, L.omega);
    return op_asm<float>(ctx, L, L.r32, L.u32, L.omega);
  };
  CKS(once());  // warm-up
  CK(cudaEventRecord(a, ctx->stream));
  for (int i = 0; i < reps; ++i) CKS(once());
  CK(cudaEventRecord(b, ctx->stream));
  CK(cudaEventSynchronize(b));
  float ms = 0.0f;
  CK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *avg_ms = (double)ms / reps;
  return STMG_OK;
}

}  // extern "C"
