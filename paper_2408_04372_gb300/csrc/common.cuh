// Shared device-side definitions of the STMG library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <utility>

namespace stmg {

// Programmatic dependent launch.  Kernels of the solve path start with pdl_wait(): launched with
// the programmatic-serialisation attribute, a kernel may be scheduled while its predecessor drains,
// and griddepcontrol.wait blocks until the predecessor grid has completed and its writes are
// visible (without the attribute it returns at once).  pdl_trigger() lets the next kernel be
// scheduled as soon as every CTA of this one has started.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launch with programmatic stream serialisation (graph capture turns it into programmatic edges).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr int kMaxN = 6;    // p <= 5
constexpr int STMG_DEVICE_TIMEOUT = 1;  // device status word: a bounded wait gave up
constexpr int kMaxNT = 5;   // time DoFs per slab

// Tables of one operator evaluation, passed by value (constant bank).
//   B[q][i]  : 1D nodal (Gauss-Lobatto) basis i at Gauss point q
//   D[q][r]  : derivative at Gauss point q of the Lagrange basis through the Gauss points (collocation)
//   TA, TM   : time matrices of S = TA (x) A_h + TM (x) M_h
template <typename T>
struct OpTab {
  T B[kMaxN][kMaxN];
  T D[kMaxN][kMaxN];
  T TA[kMaxNT][kMaxNT];
  T TM[kMaxNT][kMaxNT];
  T sign;
};

// Structured-grid description of one level.
struct GridDesc {
  int dim;
  int N;          // cells per direction
  int p;
  int nn1;        // nodes per direction = p*N + 1
  int64_t n_nodes;
  int64_t n_cells;
};

__host__ __device__ inline bool on_boundary(int g, int nn1) { return g == 0 || g == nn1 - 1; }

// Coordinates of a cell or node index, in 32-bit unsigned division: every index of a level is below
// 2^31 (checked when a context is created), and 32-bit division costs a fraction of 64-bit division.
__device__ __forceinline__ void cell_xyz(int64_t cell, const GridDesc& g, int& cx, int& cy, int& cz) {
  const uint32_t c = (uint32_t)cell, n = (uint32_t)g.N;
  const uint32_t r = c / n;
  cx = (int)(c - r * n);
  cy = (int)(r % n);
  cz = (int)(r / n);
}
__device__ __forceinline__ void node_xyz(int64_t node, int nn1, int& gx, int& gy, int& gz) {
  const uint32_t c = (uint32_t)node, n = (uint32_t)nn1;
  const uint32_t r = c / n;
  gx = (int)(c - r * n);
  gy = (int)(r % n);
  gz = (int)(r / n);
}

// Geometry layout.  The FP32 geometry of 3D levels with at most three nodes per direction is read
// by the register-resident operator kernel (one thread per cell and time DoF), whose warps read
// consecutive cells with 16-byte loads: it is stored in chunks of kGeoChunk cells,
// [cell / 32][Gauss point][part][cell % 32][4], part 0 = (G00, G01, G02, G11), part 1 = (G12, G22, m, 0).
// Every other geometry array is [cell][component][point].
constexpr int kGeoChunk = 32;
__host__ __device__ constexpr bool geo_chunked(int dim, int n) { return dim == 3 && n <= 3; }
__host__ __device__ inline int64_t geo_chunk_cells(int64_t n_cells) {
  return (n_cells + kGeoChunk - 1) / kGeoChunk * kGeoChunk;
}

// Time diagonalisation of the local space-time matrices for the additive
// Schwarz smoother: modes m = 0..nreal-1 are real, then ncplx complex modes
// (one representative per conjugate pair).  W = V^-1 TA^-1 (rows = modes),
// V[t][m] (columns = eigenvectors).
template <typename T>
struct ModeTab {
  int nreal, ncplx;
  T Wr[kMaxNT][kMaxNT], Wi[kMaxNT][kMaxNT];
  T Vr[kMaxNT][kMaxNT], Vi[kMaxNT][kMaxNT];
  T lre[kMaxNT], lim[kMaxNT];   // eigenvalues of the representative modes
  T omega;
  int weighted;  // fast diagonalisation: each cell's correction at a node divided by the node's cell count
                 // (stored inverses carry the factor in their rows)
};

// 1 / (number of cells that contain an unconstrained node) on the structured grid: a factor 1/2 for
// every direction in which the node index is a multiple of p (a face shared by two cells)
template <typename T>
__device__ __forceinline__ T node_weight(int gx, int gy, int gz, int dim, int p) {
  T w = T(1);
  if (gx % p == 0) w *= T(0.5);
  if (gy % p == 0) w *= T(0.5);
  if (dim == 3 && gz % p == 0) w *= T(0.5);
  return w;
}

// Fast diagonalisation tables for the three 1D cell types (first, interior, last cell):
// S[t][a][i] = component a of the M1-orthonormal eigenvector i, lam[t][i] its eigenvalue.
template <typename T>
struct FDTab {
  T S[3][kMaxN][kMaxN];
  T lam[3][kMaxN];
};

template <typename T> __device__ inline T to_t(float v);
template <> __device__ inline float to_t<float>(float v) { return v; }
template <> __device__ inline double to_t<double>(float v) { return (double)v; }

template <typename T> __device__ inline T load_as(const T* p) { return *p; }
__device__ inline float load_f(const float* p) { return __ldg(p); }
__device__ inline double load_f(const double* p) { return __ldg(p); }
__device__ inline float load_f(const __nv_bfloat16* p) { return __bfloat162float(*p); }

}  // namespace stmg
