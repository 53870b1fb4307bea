// Host-callable launchers of the STMG device kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "common.cuh"
#include "df64.cuh"

namespace stmg {

// ---- operator (apply.cu) ----
template <typename T>
cudaError_t launch_apply(int dim, int n, int nt, const T* x, T* y, const T* geo, const GridDesc& g,
                         const OpTab<T>& tab, int mask_input, cudaStream_t s);
// Mass part only, y += (TM (x) M_h) x in FP64 (TA ignored, no input masking): right-hand sides.
cudaError_t launch_mass_apply(int dim, int n, int nt, const double* x, double* y, const double* geo, const GridDesc& g,
                              const OpTab<double>& tab, cudaStream_t s);
// Mass part with constrained input nodes read as 0, y += (TM (x) M_h) x in arithmetic T from TI to TO:
// the coupling -B u_{i-1} between consecutive slabs of eq. heat-cg-dg-at-once (TM holds the column
// of the previous slab's last time DoF).  Instances <float,float,float>, <double,double,double>,
// <double,float,double>.
template <typename T, typename TI, typename TO>
cudaError_t launch_mass_couple(int dim, int n, int nt, const TI* x, TO* y, const T* geo, const GridDesc& g,
                               const OpTab<T>& tab, cudaStream_t s);
// Same operator in double-float arithmetic (df64.cuh) for an FP32 input vector, accumulated into
// an FP64 output: the FGMRES apply on V-cycle outputs, which are exact in FP32.
cudaError_t launch_apply_df(int dim, int n, int nt, const float* x, double* y, const df64* geo, const GridDesc& g,
                            const OpTab<df64>& tab, int mask_input, cudaStream_t s);
// Mass part in double-float on an FP64 input split into float pairs (right-hand sides on level 0).
cudaError_t launch_mass_apply_df(int dim, int n, int nt, const double* x, double* y, const df64* geo, const GridDesc& g,
                                 const OpTab<df64>& tab, cudaStream_t s);
// FP32 arithmetic on an FP32 input, accumulated into an FP64 output: the relaxed FGMRES apply once
// the residual is small enough for its rounding (inexact Krylov).
cudaError_t launch_apply_f2d(int dim, int n, int nt, const float* x, double* y, const float* geo, const GridDesc& g,
                             const OpTab<float>& tab, int mask_input, cudaStream_t s);
// Same for an FP64 input vector, split into two floats per entry (the FGMRES residual on level 0).
cudaError_t launch_apply_df_d(int dim, int n, int nt, const double* x, double* y, const df64* geo, const GridDesc& g,
                              const OpTab<df64>& tab, int mask_input, cudaStream_t s);
// y = constrained ? x : 0 for an FP32 x and FP64 y (initialisation for launch_apply_df)
cudaError_t launch_init_rows_f2d(double* y, const float* x, const GridDesc& g, int nt, cudaStream_t s);
// mode 0: y = constrained ? x : 0 ; mode 1: y = constrained ? f - x : f ; mode 2: y = 0
template <typename T>
cudaError_t launch_init_rows(T* y, const T* f, const T* x, const GridDesc& g, int nt, int mode, cudaStream_t s);

// ---- geometry (setup.cu) ----
// geo64 [cell][7 or 4][nq^dim]: rho w |J| J^-1 J^-T (upper triangle) and w |J|; geo32 the same in
// FP32, geodf (may be NULL) as double-float pairs.  geo32 uses the chunked layout where
// geo_chunked(dim, nq) holds (common.cuh) and then holds geo_chunk_cells(n_cells) cells x 8 components.
cudaError_t launch_geometry(const GridDesc& g, const double* vertices, const double* rho_qp, const double* xq,
                            const double* wq, double* geo64, float* geo32, df64* geodf, cudaStream_t s);

// ---- additive Schwarz (asm.cu) ----
struct LocalTab {        // 1D tables of the nodal basis at Gauss points (setup in FP64)
  double B[kMaxN][kMaxN];   // value of node basis i at Gauss point q: B[q][i]
  double Dn[kMaxN][kMaxN];  // derivative of node basis i at Gauss point q
};
// Builds, per cell and time mode, the inverse of (A_K + lambda_m M_K) with A_K, M_K the
// global matrices restricted to the cell's nodes; writes planes of the storage type.  weighted:
// row a scaled by 1 / (number of cells containing node a), the weighted Schwarz sum.
cudaError_t launch_asm_setup(int dim, int n, int nt, const GridDesc& g, const double* geo64, const LocalTab& lt,
                             const double* lam_re, const double* lam_im, int nreal, int ncplx, void* inv,
                             int inv_prec, int weighted, cudaStream_t s);
// elements per cell in the inverse store (N_t planes, padded to a 16-byte multiple)
int64_t asm_cell_stride(int dim, int n, int nt, int esz);
// Local solves through a per-cell generalized eigendecomposition A_K Q = M_K Q diag(mu) (eig.cu):
// bytes per cell of the store (Q as NB x NBP entries of esz bytes, then NBP FP32 eigenvalues),
// the set-up (prec 0 FP64, 1 FP32, 2 BF16 storage of Q) and the smoother sweep (same contract as
// launch_asm_apply; the weighted sum's factors are applied by the kernel).
int64_t eig_cell_bytes(int dim, int n, int esz);
cudaError_t launch_eig_setup(int dim, int n, const GridDesc& g, const double* geo64, const LocalTab& lt, void* out,
                             int prec, cudaStream_t s);
// Tensor-core variant (BF16 Q images padded to 16, 32 or 64 rows, swizzled as the operand layout wants,
// then FP32 eigenvalues; (p+1)^dim <= 64; FP32 vectors; at most 8 slabs per system): store bytes
// (-1 when unsupported), set-up with prec 3, sweep.
int64_t eig_tc_bytes(int dim, int n, int64_t n_cells);
cudaError_t launch_eig_tc_apply(int dim, int n, int nt, const float* r, float* u, const void* inv, const GridDesc& g,
                                const ModeTab<float>& mt, const float* cs, float* cd, int* status, int nslab,
                                int64_t ss, cudaStream_t s);
template <typename T>
cudaError_t launch_eig_apply(int dim, int n, int nt, const T* r, T* u, const void* inv, int prec, const GridDesc& g,
                             const ModeTab<T>& mt, const T* cs, T* cd, int* status, int nslab, int64_t ss,
                             cudaStream_t s);
// copy_src/copy_dst (may be NULL): side job for the V-cycle, copy_dst := copy_src on every node of every cell.
// status (device int, may be NULL): with it the inverses arrive by bulk copies (TMA) into shared memory and
// a timed-out wait stores STMG_DEVICE_TIMEOUT there; without it each thread streams its rows itself.
// nslab slabs of slab_stride entries each share the inverses (one bulk copy serves all of them).
template <typename T>
cudaError_t launch_asm_apply(int dim, int n, int nt, const T* r, T* u, const void* inv, int inv_prec,
                             const GridDesc& g, const ModeTab<T>& mt, const T* copy_src, T* copy_dst, int* status,
                             int nslab, int64_t slab_stride, cudaStream_t s);

// Test hook: a bounded device wait that cannot complete; about one second later *status holds
// STMG_DEVICE_TIMEOUT.
cudaError_t launch_wait_selftest(int* status, cudaStream_t s);

// ---- fast diagonalisation local solves (fd.cu), 3D Cartesian cells ----
template <typename T>
cudaError_t launch_fd_apply(int n, int nt, const T* r, T* u, const T* rho_cell, const GridDesc& g, const FDTab<T>& fd,
                            const ModeTab<T>& mt, const T* copy_src, T* copy_dst, cudaStream_t s);

// ---- transfers (transfer.cu) ----
// 1D lists of the separable transfers, Dirichlet masks folded in: prolongation rows of fine
// boundary nodes and columns of coarse boundary nodes are dropped, likewise for the restriction.
struct Transfer1D {
  int width_p;           // max coarse entries per fine node
  int width_r;           // max fine entries per coarse node
  const int* p_idx;      // [nn1_f][width_p]  (coarse index, -1 padding)
  const double* p_w;     // [nn1_f][width_p]
  const int* r_idx;      // [nn1_c][width_r]  (fine index, -1 padding)
  const double* r_w;     // [nn1_c][width_r]
  const float* p_w32;    // the weights in FP32 for the FP32 V-cycle (converting per use would take the
  const float* r_w32;    // FP64 pipe, which is slow on this GPU)
  void* tmp1;            // scratch: nt * nn1_f^2 * nn1_c doubles each
  void* tmp2;
};
// Side jobs for the V-cycle (pointers may be NULL): prolongations also copy copy_src -> copy_dst over
// the fine vector, restrictions also zero zero_dst over the coarse vector.
template <typename T>
cudaError_t launch_prolong_space_add(T* uf, const T* ec, const GridDesc& gf, const GridDesc& gc, int nt,
                                     const Transfer1D& t, const T* copy_src, T* copy_dst, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict_space(T* rc, const T* rf, const GridDesc& gf, const GridDesc& gc, int nt,
                                  const Transfer1D& t, T* zero_dst, cudaStream_t s);
// Time transfers act on nb blocks of consecutive time components, the fine block b being components
// [b ntf, (b+1) ntf) and the coarse one [b ntc, (b+1) ntc) of a [component][node] vector.  k-levels:
// P_k per slab (ntf, ntc = N_t of the two levels, nb = slabs).  tau-levels: two consecutive fine slabs
// form one fine block (ntf = 2 N_t) under one coarse slab of twice the length (ntc = N_t, nb = coarse slabs).
struct TimeTransfer { int ntf, ntc, nb; double P[2 * kMaxNT][kMaxNT]; };
template <typename T>
cudaError_t launch_prolong_time_add(T* uf, const T* ec, const GridDesc& g, const TimeTransfer& t, const T* copy_src,
                                    T* copy_dst, cudaStream_t s);
template <typename T>
cudaError_t launch_restrict_time(T* rc, const T* rf, const GridDesc& g, const TimeTransfer& t, T* zero_dst,
                                 cudaStream_t s);

// ---- vectors, reductions, coarse solve (vec.cu) ----
template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin* x, Tout* y, int64_t n, cudaStream_t s);
cudaError_t launch_axpby(double a, const double* x, double b, double* y, int64_t n, cudaStream_t s);
// One classical Gram-Schmidt pass over V_0..V_{nv-1} (nv <= 64), single launch, bit-reproducible:
// optionally w -= sum_j c[j] V_j, then s_j = V_j . w and/or s_nv = w . w; fin 0 writes s to out,
// fin 1 the Arnoldi column out[j] = h_prev[j] + c[j], out[nv] = ||w||, out[nv+1] = 1/||w||.
// partial: (K+1) x cgs_blocks() doubles; counter: one zero-initialised unsigned int per stream,
// left at zero on return.  status (device int, may be NULL): with it, and 16-byte aligned w, V0 and
// stride, the vectors arrive by bulk copies (TMA) and a timed-out wait is recorded there.
cudaError_t launch_cgs_pass(const double* V0, int64_t stride, int nv, double* w, int64_t n, const double* c, int sub,
                            int dot, int norm, const double* h_prev, int fin, double* partial, unsigned int* counter,
                            double* out, cudaStream_t s, int* status = nullptr, const double* nrm2 = nullptr,
                            float* copy32 = nullptr, int vfmt = 0);
// vfmt: 0 FP64 vectors; 1 the basis and w as double-float pairs (hi, lo) in their 8 bytes per entry,
// double-float arithmetic; 2 the same with w arriving in FP64 (converted and written back as pairs);
// 3 w in FP64, read only, double-float arithmetic (no basis: a norm; the FP64 pass when w is unaligned).
// r = x * scale as double-float pairs written over x (FP64 in), and its FP32 copy (the V-cycle input).
cudaError_t launch_scale_to_df(double* x, double scale, int64_t n, float* copy32, cudaStream_t s);
int cgs_blocks();
// w += sign * sum_j h[j] V_j  (h on the device, V_j = V0 + j * stride; V in FP64 or FP32)
template <typename TV>
cudaError_t launch_multi_axpy(double* w, const TV* V0, int64_t stride, const double* h, int nv, double sign,
                              int64_t n, cudaStream_t s);
cudaError_t launch_broadcast_time(const double* u0, double* u, int nt, int64_t n_nodes, cudaStream_t s);
// out[pt][c] = sum_a w[pt][a] u[c n_nodes + nodes[pt][a]] for npts points, ncomp components, nb nodes each
cudaError_t launch_point_values(const double* u, int64_t n_nodes, int ncomp, const int64_t* nodes, const double* w,
                                int nb, int npts, double* out, cudaStream_t s);
// y[i][node] = sum_j C[i][j] x_j[node] over nin vectors (time-only mixing)
cudaError_t launch_time_mix(const double* const* xs, int nin, const double* C, int nout, double* y,
                            int64_t n_nodes, int accumulate, cudaStream_t s);
// inv: n rows of coarse_ld(n) entries (zero padding), row-major
inline int coarse_ld(int n) { return (n + 3) / 4 * 4; }
template <typename T>
cudaError_t launch_coarse_solve(const T* f, T* u, const T* inv, const int64_t* map, int n, int64_t total,
                                cudaStream_t s);
cudaError_t launch_zero_constrained(double* y, const GridDesc& g, int nt, cudaStream_t s);

}  // namespace stmg
