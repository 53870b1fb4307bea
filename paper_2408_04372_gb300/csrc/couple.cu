// Coupling between consecutive slabs of the at-once system (eq. heat-cg-dg-at-once):
// y_i += (TM (x) M_h) x_{i-1}, with TM holding -alpha in the column of the last time DoF of the
// previous slab, constrained input nodes read as 0 (the constrained columns of B are zero).
// Mass-only instances of the operator kernels in apply_kernels.cuh.
#include "apply_kernels.cuh"

namespace stmg {

using apply_detail::launch_apply_t;

#define STMG_COUPLE_CASE(DIM, N, NT)                                                                     \
  if (dim == DIM && n == N && nt == NT) return launch_apply_t<DIM, N, NT, T, TI, TO, true>(x, y, geo, g, tab, 1, s);

template <typename T, typename TI, typename TO>
cudaError_t launch_mass_couple(int dim, int n, int nt, const TI* x, TO* y, const T* geo, const GridDesc& g,
                               const OpTab<T>& tab, cudaStream_t s) {
  STMG_COUPLE_CASE(3, 2, 1) STMG_COUPLE_CASE(3, 2, 2) STMG_COUPLE_CASE(3, 2, 3) STMG_COUPLE_CASE(3, 2, 4)
  STMG_COUPLE_CASE(3, 3, 1) STMG_COUPLE_CASE(3, 3, 2) STMG_COUPLE_CASE(3, 3, 3) STMG_COUPLE_CASE(3, 3, 4)
  STMG_COUPLE_CASE(3, 4, 1) STMG_COUPLE_CASE(3, 4, 2) STMG_COUPLE_CASE(3, 4, 3) STMG_COUPLE_CASE(3, 4, 4)
  STMG_COUPLE_CASE(3, 5, 1) STMG_COUPLE_CASE(3, 5, 2) STMG_COUPLE_CASE(3, 5, 3) STMG_COUPLE_CASE(3, 5, 4)
  STMG_COUPLE_CASE(2, 2, 1) STMG_COUPLE_CASE(2, 2, 2) STMG_COUPLE_CASE(2, 2, 3) STMG_COUPLE_CASE(2, 2, 4)
  STMG_COUPLE_CASE(2, 3, 1) STMG_COUPLE_CASE(2, 3, 2) STMG_COUPLE_CASE(2, 3, 3) STMG_COUPLE_CASE(2, 3, 4)
  STMG_COUPLE_CASE(2, 4, 1) STMG_COUPLE_CASE(2, 4, 2) STMG_COUPLE_CASE(2, 4, 3) STMG_COUPLE_CASE(2, 4, 4)
  STMG_COUPLE_CASE(2, 5, 1) STMG_COUPLE_CASE(2, 5, 2) STMG_COUPLE_CASE(2, 5, 3) STMG_COUPLE_CASE(2, 5, 4)
  return cudaErrorInvalidValue;
}

template cudaError_t launch_mass_couple<float, float, float>(int, int, int, const float*, float*, const float*,
                                                             const GridDesc&, const OpTab<float>&, cudaStream_t);
template cudaError_t launch_mass_couple<double, double, double>(int, int, int, const double*, double*, const double*,
                                                                const GridDesc&, const OpTab<double>&, cudaStream_t);
template cudaError_t launch_mass_couple<double, float, double>(int, int, int, const float*, double*, const double*,
                                                               const GridDesc&, const OpTab<double>&, cudaStream_t);

}  // namespace stmg
