// Matrix-free space-time operator y (+)= sign * (TA (x) A_h + TM (x) M_h) x   (Section 3.1):
// FP32 and FP64 instances of the kernels in apply_kernels.cuh, and the row initialisation.
#include "apply_kernels.cuh"

namespace stmg {

namespace {

using apply_detail::launch_apply_t;

// init_apply: y = 0 on unconstrained rows, y = x on constrained rows (identity).
// init_residual: r = f on unconstrained rows, r = f - x on constrained rows.
template <typename T, typename TX = T>
__global__ void init_rows_kernel(T* __restrict__ y, const T* __restrict__ f, const TX* __restrict__ x,
                                 GridDesc g, int nt, int mode) {
  pdl_wait();
  pdl_trigger();
  const int64_t total = g.n_nodes * nt;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t node = (uint32_t)idx % (uint32_t)g.n_nodes;
    int gx, gy, gz;
    node_xyz(node, g.nn1, gx, gy, gz);
    bool bnd = on_boundary(gx, g.nn1) || on_boundary(gy, g.nn1);
    if (g.dim == 3) bnd = bnd || on_boundary(gz, g.nn1);
    T v;
    if (mode == 0) v = bnd ? (T)x[idx] : T(0);
    else if (mode == 1) v = bnd ? f[idx] - (T)x[idx] : f[idx];
    else v = T(0);
    y[idx] = v;
  }
}

}  // namespace

#define STMG_APPLY_CASE(DIM, N, NT)                                              \
  if (dim == DIM && n == N && nt == NT) return launch_apply_t<DIM, N, NT>(x, y, geo, g, tab, mask_input, s);

template <typename T>
cudaError_t launch_apply(int dim, int n, int nt, const T* x, T* y, const T* geo, const GridDesc& g,
                         const OpTab<T>& tab, int mask_input, cudaStream_t s) {
  STMG_APPLY_CASE(3, 2, 1) STMG_APPLY_CASE(3, 2, 2) STMG_APPLY_CASE(3, 2, 3) STMG_APPLY_CASE(3, 2, 4)
  STMG_APPLY_CASE(3, 3, 1) STMG_APPLY_CASE(3, 3, 2) STMG_APPLY_CASE(3, 3, 3) STMG_APPLY_CASE(3, 3, 4)
  STMG_APPLY_CASE(3, 4, 1) STMG_APPLY_CASE(3, 4, 2) STMG_APPLY_CASE(3, 4, 3) STMG_APPLY_CASE(3, 4, 4)
  STMG_APPLY_CASE(3, 5, 1) STMG_APPLY_CASE(3, 5, 2) STMG_APPLY_CASE(3, 5, 3) STMG_APPLY_CASE(3, 5, 4)
  STMG_APPLY_CASE(3, 2, 5) STMG_APPLY_CASE(3, 3, 5) STMG_APPLY_CASE(3, 4, 5) STMG_APPLY_CASE(3, 5, 5)
  STMG_APPLY_CASE(3, 6, 1) STMG_APPLY_CASE(3, 6, 5)
  STMG_APPLY_CASE(2, 2, 1) STMG_APPLY_CASE(2, 2, 2) STMG_APPLY_CASE(2, 2, 3) STMG_APPLY_CASE(2, 2, 4)
  STMG_APPLY_CASE(2, 3, 1) STMG_APPLY_CASE(2, 3, 2) STMG_APPLY_CASE(2, 3, 3) STMG_APPLY_CASE(2, 3, 4)
  STMG_APPLY_CASE(2, 4, 1) STMG_APPLY_CASE(2, 4, 2) STMG_APPLY_CASE(2, 4, 3) STMG_APPLY_CASE(2, 4, 4)
  STMG_APPLY_CASE(2, 5, 1) STMG_APPLY_CASE(2, 5, 2) STMG_APPLY_CASE(2, 5, 3) STMG_APPLY_CASE(2, 5, 4)
  return cudaErrorInvalidValue;
}

#define STMG_MASS_CASE(DIM, N, NT)                                              \
  if (dim == DIM && n == N && nt == NT) return launch_apply_t<DIM, N, NT, double, double, double, true>(x, y, geo, g, tab, 0, s);

cudaError_t launch_mass_apply(int dim, int n, int nt, const double* x, double* y, const double* geo, const GridDesc& g,
                              const OpTab<double>& tab, cudaStream_t s) {
  STMG_MASS_CASE(3, 2, 1) STMG_MASS_CASE(3, 2, 2) STMG_MASS_CASE(3, 2, 3) STMG_MASS_CASE(3, 2, 4)
  STMG_MASS_CASE(3, 3, 1) STMG_MASS_CASE(3, 3, 2) STMG_MASS_CASE(3, 3, 3) STMG_MASS_CASE(3, 3, 4)
  STMG_MASS_CASE(3, 4, 1) STMG_MASS_CASE(3, 4, 2) STMG_MASS_CASE(3, 4, 3) STMG_MASS_CASE(3, 4, 4)
  STMG_MASS_CASE(3, 5, 1) STMG_MASS_CASE(3, 5, 2) STMG_MASS_CASE(3, 5, 3) STMG_MASS_CASE(3, 5, 4)
  STMG_MASS_CASE(3, 2, 5) STMG_MASS_CASE(3, 3, 5) STMG_MASS_CASE(3, 4, 5) STMG_MASS_CASE(3, 5, 5)
  STMG_MASS_CASE(3, 6, 1) STMG_MASS_CASE(3, 6, 5)
  STMG_MASS_CASE(2, 2, 1) STMG_MASS_CASE(2, 2, 2) STMG_MASS_CASE(2, 2, 3) STMG_MASS_CASE(2, 2, 4)
  STMG_MASS_CASE(2, 3, 1) STMG_MASS_CASE(2, 3, 2) STMG_MASS_CASE(2, 3, 3) STMG_MASS_CASE(2, 3, 4)
  STMG_MASS_CASE(2, 4, 1) STMG_MASS_CASE(2, 4, 2) STMG_MASS_CASE(2, 4, 3) STMG_MASS_CASE(2, 4, 4)
  STMG_MASS_CASE(2, 5, 1) STMG_MASS_CASE(2, 5, 2) STMG_MASS_CASE(2, 5, 3) STMG_MASS_CASE(2, 5, 4)
  return cudaErrorInvalidValue;
}

#define STMG_F2D_CASE(DIM, N, NT)                                              \
  if (dim == DIM && n == N && nt == NT) return launch_apply_t<DIM, N, NT, float, float, double>(x, y, geo, g, tab, mask_input, s);

cudaError_t launch_apply_f2d(int dim, int n, int nt, const float* x, double* y, const float* geo, const GridDesc& g,
                             const OpTab<float>& tab, int mask_input, cudaStream_t s) {
  STMG_F2D_CASE(3, 2, 1) STMG_F2D_CASE(3, 2, 2) STMG_F2D_CASE(3, 2, 3) STMG_F2D_CASE(3, 2, 4)
  STMG_F2D_CASE(3, 3, 1) STMG_F2D_CASE(3, 3, 2) STMG_F2D_CASE(3, 3, 3) STMG_F2D_CASE(3, 3, 4)
  STMG_F2D_CASE(3, 4, 1) STMG_F2D_CASE(3, 4, 2) STMG_F2D_CASE(3, 4, 3) STMG_F2D_CASE(3, 4, 4)
  STMG_F2D_CASE(3, 5, 1) STMG_F2D_CASE(3, 5, 2) STMG_F2D_CASE(3, 5, 3) STMG_F2D_CASE(3, 5, 4)
  STMG_F2D_CASE(3, 2, 5) STMG_F2D_CASE(3, 3, 5) STMG_F2D_CASE(3, 4, 5) STMG_F2D_CASE(3, 5, 5) STMG_F2D_CASE(3, 6, 5)
  STMG_F2D_CASE(2, 2, 1) STMG_F2D_CASE(2, 2, 2) STMG_F2D_CASE(2, 2, 3) STMG_F2D_CASE(2, 2, 4)
  STMG_F2D_CASE(2, 3, 1) STMG_F2D_CASE(2, 3, 2) STMG_F2D_CASE(2, 3, 3) STMG_F2D_CASE(2, 3, 4)
  STMG_F2D_CASE(2, 4, 1) STMG_F2D_CASE(2, 4, 2) STMG_F2D_CASE(2, 4, 3) STMG_F2D_CASE(2, 4, 4)
  STMG_F2D_CASE(2, 5, 1) STMG_F2D_CASE(2, 5, 2) STMG_F2D_CASE(2, 5, 3) STMG_F2D_CASE(2, 5, 4)
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t launch_init_rows(T* y, const T* f, const T* x, const GridDesc& g, int nt, int mode, cudaStream_t s) {
  const int64_t total = g.n_nodes * nt;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  { const cudaError_t e_ = launch_k(init_rows_kernel<T>, dim3(blocks), dim3(256), 0, s, y, f, x, g, nt, mode); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

cudaError_t launch_init_rows_f2d(double* y, const float* x, const GridDesc& g, int nt, cudaStream_t s) {
  const int64_t total = g.n_nodes * nt;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  if (blocks < 1) blocks = 1;
  { const cudaError_t e_ = launch_k(init_rows_kernel<double, float>, dim3(blocks), dim3(256), 0, s, y, nullptr, x, g, nt, 0); if (e_ != cudaSuccess) return e_; }
  return cudaGetLastError();
}

template cudaError_t launch_apply<float>(int, int, int, const float*, float*, const float*, const GridDesc&,
                                         const OpTab<float>&, int, cudaStream_t);
template cudaError_t launch_apply<double>(int, int, int, const double*, double*, const double*, const GridDesc&,
                                          const OpTab<double>&, int, cudaStream_t);
template cudaError_t launch_init_rows<float>(float*, const float*, const float*, const GridDesc&, int, int, cudaStream_t);
template cudaError_t launch_init_rows<double>(double*, const double*, const double*, const GridDesc&, int, int,
                                              cudaStream_t);

}  // namespace stmg
