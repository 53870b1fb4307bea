// Double-float instances of the operator kernels (apply_kernels.cuh) for an FP64 input vector:
// each entry is split into two floats at the gather, the arithmetic runs in double-float with
// double-float tables and geometry, the output is FP64.  The FGMRES residual b - S x on the finest
// level (x in FP64) runs in these instead of the FP64 pipe.
#include "apply_kernels.cuh"

namespace stmg {

using apply_detail::launch_apply_t;

#define STMG_APPLY_CASE(DIM, N, NT)                                              \
  if (dim == DIM && n == N && nt == NT) return launch_apply_t<DIM, N, NT>(x, y, geo, g, tab, mask_input, s);

cudaError_t launch_apply_df_d(int dim, int n, int nt, const double* x, double* y, const df64* geo, const GridDesc& g,
                              const OpTab<df64>& tab, int mask_input, cudaStream_t s) {
  STMG_APPLY_CASE(3, 2, 1) STMG_APPLY_CASE(3, 2, 2) STMG_APPLY_CASE(3, 2, 3) STMG_APPLY_CASE(3, 2, 4)
  STMG_APPLY_CASE(3, 3, 1) STMG_APPLY_CASE(3, 3, 2) STMG_APPLY_CASE(3, 3, 3) STMG_APPLY_CASE(3, 3, 4)
  STMG_APPLY_CASE(3, 4, 1) STMG_APPLY_CASE(3, 4, 2) STMG_APPLY_CASE(3, 4, 3) STMG_APPLY_CASE(3, 4, 4)
  STMG_APPLY_CASE(3, 5, 1) STMG_APPLY_CASE(3, 5, 2) STMG_APPLY_CASE(3, 5, 3) STMG_APPLY_CASE(3, 5, 4)
  STMG_APPLY_CASE(3, 2, 5) STMG_APPLY_CASE(3, 3, 5) STMG_APPLY_CASE(3, 4, 5) STMG_APPLY_CASE(3, 5, 5) STMG_APPLY_CASE(3, 6, 5)
  STMG_APPLY_CASE(2, 2, 1) STMG_APPLY_CASE(2, 2, 2) STMG_APPLY_CASE(2, 2, 3) STMG_APPLY_CASE(2, 2, 4)
  STMG_APPLY_CASE(2, 3, 1) STMG_APPLY_CASE(2, 3, 2) STMG_APPLY_CASE(2, 3, 3) STMG_APPLY_CASE(2, 3, 4)
  STMG_APPLY_CASE(2, 4, 1) STMG_APPLY_CASE(2, 4, 2) STMG_APPLY_CASE(2, 4, 3) STMG_APPLY_CASE(2, 4, 4)
  STMG_APPLY_CASE(2, 5, 1) STMG_APPLY_CASE(2, 5, 2) STMG_APPLY_CASE(2, 5, 3) STMG_APPLY_CASE(2, 5, 4)
  return cudaErrorInvalidValue;
}

#define STMG_MASS_DFD_CASE(DIM, N, NT)                                              \
  if (dim == DIM && n == N && nt == NT) return launch_apply_t<DIM, N, NT, df64, double, double, true>(x, y, geo, g, tab, 0, s);

cudaError_t launch_mass_apply_df(int dim, int n, int nt, const double* x, double* y, const df64* geo, const GridDesc& g,
                                 const OpTab<df64>& tab, cudaStream_t s) {
  STMG_MASS_DFD_CASE(3, 2, 1) STMG_MASS_DFD_CASE(3, 2, 2) STMG_MASS_DFD_CASE(3, 2, 3) STMG_MASS_DFD_CASE(3, 2, 4)
  STMG_MASS_DFD_CASE(3, 3, 1) STMG_MASS_DFD_CASE(3, 3, 2) STMG_MASS_DFD_CASE(3, 3, 3) STMG_MASS_DFD_CASE(3, 3, 4)
  STMG_MASS_DFD_CASE(3, 4, 1) STMG_MASS_DFD_CASE(3, 4, 2) STMG_MASS_DFD_CASE(3, 4, 3) STMG_MASS_DFD_CASE(3, 4, 4)
  STMG_MASS_DFD_CASE(3, 5, 1) STMG_MASS_DFD_CASE(3, 5, 2) STMG_MASS_DFD_CASE(3, 5, 3) STMG_MASS_DFD_CASE(3, 5, 4)
  STMG_MASS_DFD_CASE(3, 2, 5) STMG_MASS_DFD_CASE(3, 3, 5) STMG_MASS_DFD_CASE(3, 4, 5) STMG_MASS_DFD_CASE(3, 5, 5)
  STMG_MASS_DFD_CASE(3, 6, 1) STMG_MASS_DFD_CASE(3, 6, 5)
  STMG_MASS_DFD_CASE(2, 2, 1) STMG_MASS_DFD_CASE(2, 2, 2) STMG_MASS_DFD_CASE(2, 2, 3) STMG_MASS_DFD_CASE(2, 2, 4)
  STMG_MASS_DFD_CASE(2, 3, 1) STMG_MASS_DFD_CASE(2, 3, 2) STMG_MASS_DFD_CASE(2, 3, 3) STMG_MASS_DFD_CASE(2, 3, 4)
  STMG_MASS_DFD_CASE(2, 4, 1) STMG_MASS_DFD_CASE(2, 4, 2) STMG_MASS_DFD_CASE(2, 4, 3) STMG_MASS_DFD_CASE(2, 4, 4)
  STMG_MASS_DFD_CASE(2, 5, 1) STMG_MASS_DFD_CASE(2, 5, 2) STMG_MASS_DFD_CASE(2, 5, 3) STMG_MASS_DFD_CASE(2, 5, 4)
  return cudaErrorInvalidValue;
}

}  // namespace stmg
