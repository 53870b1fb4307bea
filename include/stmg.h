/*
 * stmg.h -- C ABI of the GB300 space-time multigrid (STMG) library, libstmg.so.
 *
 * The library solves the slab systems of tensor-product space-time finite
 * elements (continuous Q_p in space on a structured, Q1-mapped grid; dG(k) or
 * cGP(k) in time) for the heat equation and the acoustic wave equation:
 *
 *     S u = rhs,   S = T_A (x) A_h + T_M (x) M_h            (Section 2)
 *
 * heat dG  (eq. heat-cg-dg):  T_A = M_tau, T_M = A_tau
 * heat cGP (eq. heat-cg-cg):  T_A = M_tau, T_M = A_tau
 * wave dG/cGP (eqs. wave-cg-dg, wave-cg-cg, condensed to u):
 *                             T_A = M_tau, T_M = A_tau M_tau^-1 A_tau
 * with M_h, A_h the Q_p mass and rho-weighted stiffness matrices
 * (eq. space-matrices), by FGMRES preconditioned with one space-time multigrid
 * V-cycle (Algorithm stmg) whose smoother is the space-time cell-wise additive
 * Schwarz method (eqs. vanka0, vanka) and whose levels coarsen first in space
 * (p, then h) and then in time (k) (Algorithm mg-sequence, Section 3.2).
 *
 * Conventions for every vector argument:
 *   - caller-owned DEVICE memory (unless the function name ends in _host);
 *   - layout [N_t][n_nodes]: N_t time-major blocks of all spatial nodes;
 *   - nodes lexicographic, x fastest: node (gx, gy, gz) ->
 *       gx + (p*N+1) * (gy + (p*N+1) * gz);
 *   - nodes on the boundary of the domain carry homogeneous Dirichlet
 *     conditions: operators act as the identity on those rows and ignore
 *     those columns; right-hand sides and corrections are zero there;
 *   - element type double for precision STMG_FP64 and float for STMG_FP32.
 * Calls are asynchronous on the stream passed to stmg_create unless stated.
 * No call throws; every call returns a status and, on error, stores a message
 * readable with stmg_last_error.  After STMG_ERR_CUDA the context must be
 * destroyed.  A context is not thread safe.
 */
#ifndef STMG_H
#define STMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stmg_ctx stmg_ctx;

typedef enum {
  STMG_OK = 0,
  STMG_ERR_INVALID_ARG = 1,   /* a size, pointer or option is out of range */
  STMG_ERR_CUDA = 2,          /* a CUDA runtime call failed; destroy the context */
  STMG_ERR_OOM = 3,           /* device allocation failed */
  STMG_ERR_NOT_CONVERGED = 4, /* FGMRES hit max_it before rtol */
  STMG_ERR_BREAKDOWN = 5,     /* Krylov breakdown before convergence */
  STMG_ERR_TIMEOUT = 6,       /* a bounded device wait gave up (reported by stmg_solve); destroy the context */
  STMG_ERR_NONFINITE = 7,     /* NaN/Inf met in a residual or preconditioner output */
  STMG_ERR_INTERNAL = 8,
  STMG_ERR_UNSUPPORTED = 9    /* valid request outside the compiled kernel set */
} stmg_status;

enum { STMG_HEAT = 0, STMG_WAVE = 1 };                 /* PDE, eqs. heat, wave */
enum { STMG_DG = 0, STMG_CGP = 1 };                    /* time discretisation, Sections 2.1 / 2.2 */
enum { STMG_COEFF_PER_CELL = 0, STMG_COEFF_PER_QPOINT = 1 };
/* STMG_DF32 = double-float: FP32 input vector, arithmetic on pairs of FP32 numbers (about 44
 * significand bits), FP64 output; only for the finest-level operator (outer_apply, stmg_apply). */
/* STMG_FP8: e4m3 with one FP32 scale per stored plane (Schwarz inverses only, FP32 V-cycle). */
enum { STMG_FP64 = 1, STMG_FP32 = 2, STMG_BF16 = 3, STMG_DF32 = 4, STMG_FP8 = 5 };   /* 0 in an option = default */
/* Local solvers of the additive Schwarz smoother (eqs. vanka0, vanka), all exact up to rounding:
 *   DENSE: per cell and time mode the inverse plane (A_K + lambda_m M_K)^-1 (N_t planes per cell);
 *   FD:    fast diagonalisation on 3D Cartesian cells (separable 1D eigenvectors; exact for a
 *          coefficient constant on the cell patch, a cell-mean approximation otherwise);
 *   EIG:   per cell the generalized eigendecomposition A_K Q = M_K Q diag(mu), Q^T M_K Q = I, so that
 *          (A_K + lambda_m M_K)^-1 = Q diag(1 / (mu + lambda_m)) Q^T for every time mode: one matrix Q
 *          and (p+1)^dim eigenvalues per cell instead of N_t planes (inverse_precision FP64, FP32 or
 *          BF16 for Q; FP8 stores BF16); any grid, p <= 3 in 3D, p <= 4 in 2D.
 *   EIG_TC: EIG with Q in BF16 and both products Q^T s and Q z_hat on the tensor cores (tcgen05, FP32
 *          accumulation; right-hand sides split into two BF16 parts); FP32 V-cycle only,
 *          (p+1)^dim <= 64, at most 8 slabs per system; stmg_smooth with FP64 vectors returns
 *          STMG_ERR_UNSUPPORTED.
 *   AUTO:  FD on 3D Cartesian grids where it is exact (or p = 4), DENSE elsewhere. */
enum { STMG_SMOOTHER_AUTO = 0, STMG_SMOOTHER_DENSE = 1, STMG_SMOOTHER_FD = 2, STMG_SMOOTHER_EIG = 3,
       STMG_SMOOTHER_EIG_TC = 4 };

/* Structured grid of n_cells^dim cells.  vertices: HOST array of
 * (n_cells+1)^dim x dim coordinates (lexicographic, x fastest), copied at
 * create; NULL means the Cartesian grid of [0,1]^dim.  Boundary vertices must
 * lie on the boundary of the unit box (homogeneous Dirichlet on all of it). */
typedef struct {
  int dim;                 /* 2 or 3 */
  int n_cells;             /* cells per direction, >= 2 */
  const double* vertices;  /* host, may be NULL */
} stmg_mesh;

/* The slab problem (Section 2).  p: spatial degree 1..4 (1..5 in 3D, where Q5 levels need the fast
 * diagonalisation, i.e. a Cartesian grid with a constant coefficient); k: time degree
 * (dG: 0..4, N_t = k+1; cGP: 1..5, N_t = k; N_t = 5 only in 3D with the fast diagonalisation);
 * tau: slab length.
 * n_slabs (0 = 1): consecutive slabs solved as one system, heat equation with dG
 * only (eq. heat-cg-dg-at-once: the slab operator S on the block diagonal, the
 * coupling -B = -1 (x) alpha (x) M_h to the previous slab's last time DoF below it).
 * Vectors of such a system are [slab][N_t][n_nodes]; the hierarchy adds
 * tau-levels (pairs of slabs merged, tau -> 2 tau, while their number is even)
 * between the space and the k levels (Algorithm mg-sequence).  1..64.
 * Size limit: 2 n_slabs N_t (p n_cells + 1)^dim < 2^31 (the kernels index in 32-bit arithmetic);
 * larger problems are refused with STMG_ERR_INVALID_ARG.
 * coeff (HOST, copied at create): rho of eq. space-matrices, either one value
 * per finest cell (PER_CELL) or one per finest-level Gauss point
 * ([cell][(p+1)^dim points, x fastest], PER_QPOINT); NULL means rho = 1.
 * Coarse levels sample the finest cell means at their Gauss points by logical
 * (reference-grid) position. */
typedef struct {
  int pde;
  int time_scheme;
  int p;
  int k;
  double tau;
  int coeff_mode;
  const double* coeff;
  int n_slabs;
} stmg_problem;

/* Solver options.  Zero-initialised fields take the defaults in brackets.
 * omega: HOST array with one relaxation weight per smoothed level (all levels
 * but the coarsest), copied at create; NULL estimates each by eq. relaxation
 * (20-step Arnoldi on S_l B_l, omega = min(1, 2/(Re lambda_max + Re lambda_min)):
 * the paper takes omega_l in (0, 1)). */
typedef struct {
  int nu_pre;              /* pre-smoothing sweeps nu_1 of Algorithm stmg [1] */
  int nu_post;             /* post-smoothing sweeps nu_2 [1] */
  int vcycle_precision;    /* STMG_FP32 (mixed) or STMG_FP64 (plain) [FP32] */
  int inverse_precision;   /* storage of dense local inverses: FP64/FP32/BF16/FP8 [same as V-cycle] */
  int smoother_kind;       /* AUTO, DENSE, FD, EIG or EIG_TC (see above) [AUTO] */
  const double* omega;     /* host, may be NULL */
  int fgmres_restart;      /* [30] */
  double rtol;             /* relative residual target of stmg_solve [1e-8] */
  int max_it;              /* [200] */
  int outer_apply;         /* arithmetic of the FGMRES operator apply on V-cycle outputs: STMG_FP64, or
                              STMG_DF32 (FP32 V-cycle only; its outputs are exact in FP32) [DF32 with
                              the FP32 V-cycle, else FP64].  Residuals b - S x always use FP64. */
  double atol;             /* absolute residual target: stmg_solve stops at ||rhs - S u||_2 <=
                              max(rtol ||rhs||_2, atol) [0: relative test only] */
  int space_coarsening;    /* spatial levels of the hierarchy: STMG_COARSEN_P_THEN_H lowers p one by one
                              down to 1, then halves the cells; STMG_COARSEN_H keeps p and halves the
                              cells; time coarsening (k) follows either way [P_THEN_H] */
  int coarse_max_dofs;     /* 1..4096: the hierarchy ends at the first coarser level with at most this many
                              unknowns, solved exactly by its dense inverse; 0: the full sequence down to
                              2^dim cells and the lowest time degree [0] */
  int asm_weighting;       /* 0: the additive Schwarz sum of eq. vanka0 as printed; 1: each cell's
                              correction at a node divided by the number of cells that contain the
                              node (a partition of unity; with it the omega estimate reaches the cap 1
                              on the coarse levels) [0] */
  int outer_relax;         /* 1: relaxed FGMRES (inexact Krylov, Simoncini & Szyld 2003; FP32 V-cycle with
                              the DF32 outer apply only): an iteration whose residual estimate is at most
                              1e5 x the stopping target applies S in FP32 arithmetic (relative error about
                              1e-5); the stopping test stays on the accurate residual [0] */
} stmg_options;

enum { STMG_COARSEN_P_THEN_H = 0, STMG_COARSEN_H = 1 };

typedef struct {
  int iterations;          /* FGMRES iterations (= V-cycles) */
  int restarts;
  double rel_residual;     /* ||rhs - S u||_2 / ||rhs||_2 computed in FP64 at exit */
  double initial_rel_residual;
  int relaxed_iterations;  /* iterations that used the FP32 operator apply (outer_relax) */
} stmg_solve_stats;

/* Builds all levels, geometry, smoother inverses, transfers and the coarse
 * solver on the device; *out receives the context.  stream: a cudaStream_t
 * (NULL = legacy default stream).  Synchronous. */
stmg_status stmg_create(stmg_ctx** out, const stmg_mesh* mesh, const stmg_problem* problem,
                        const stmg_options* options, void* stream);
stmg_status stmg_destroy(stmg_ctx* ctx);
const char* stmg_last_error(const stmg_ctx* ctx);

/* Sizes of the finest level and number of levels (level 0 = finest). */
stmg_status stmg_sizes(const stmg_ctx* ctx, int64_t* n_nodes, int* n_t, int* n_levels);
/* Slabs in the system of a level and their length (tau-levels halve the one, double the other). */
stmg_status stmg_level_slabs(const stmg_ctx* ctx, int level, int* n_slabs, double* tau);
/* Per-level data: degree p, cells per direction, time degree k, nodes, N_t (per slab), omega. */
stmg_status stmg_level_info(const stmg_ctx* ctx, int level, int* p, int* n_cells, int* k,
                            int64_t* n_nodes, int* n_t, double* omega);
/* Physical node coordinates of a level (HOST output, n_nodes x dim).  Synchronous. */
stmg_status stmg_node_coords(const stmg_ctx* ctx, int level, double* xyz);
/* Point values (goal quantities of the structural-health-monitoring example, Section 4.3): the
 * finest-level finite-element function u (DEVICE, [n_slabs][N_t][n_nodes]) evaluated at npts physical
 * points (HOST xyz, npts x dim) for every slab and time DoF -> out (HOST, npts x n_slabs N_t).  Each
 * point is located by Newton on the Q1 map of the cells; STMG_ERR_INVALID_ARG if a point lies outside
 * the grid.  Synchronous. */
stmg_status stmg_point_values(stmg_ctx* ctx, const double* u, int npts, const double* xyz, double* out);
/* Physical Gauss-point coordinates of a level (HOST output, cells x (p+1)^dim x dim). */
stmg_status stmg_qpoint_coords(const stmg_ctx* ctx, int level, double* xyz);

/* y = S_l x on level l (matrix-free, sum factorisation, Section 3.1).  precision STMG_DF32
 * (level 0 of a context created with outer_apply = STMG_DF32): x is float*, y is double*. */
stmg_status stmg_apply(stmg_ctx* ctx, int level, int precision, const void* x, void* y);
/* r = f - S_l u. */
stmg_status stmg_residual(stmg_ctx* ctx, int level, int precision, const void* f, const void* u, void* r);
/* sweeps of u <- u + omega_l sum_T R_T^T D_T [R_T S_l R_T^T]^-1 R_T (f - S_l u)  (eqs. vanka0, vanka;
 * D_T = I, or with asm_weighting the inverse number of cells containing each node). */
stmg_status stmg_smooth(stmg_ctx* ctx, int level, int precision, int sweeps, const void* f, void* u);
/* r_{l+1} = P_l^T r_l (restriction from level l to level l+1, Section 3.2). */
stmg_status stmg_restrict(stmg_ctx* ctx, int level, int precision, const void* r_fine, void* r_coarse);
/* u_l += P_l e_{l+1} (prolongation and correction, Section 3.2). */
stmg_status stmg_prolongate_add(stmg_ctx* ctx, int level, int precision, const void* e_coarse, void* u_fine);
/* e = V-cycle(r) with zero initial guess on the finest level (Algorithm stmg). */
stmg_status stmg_vcycle(stmg_ctx* ctx, int precision, const void* r, void* e);

/* Right-hand side of the slab (FP64): rhs = M_tau(x)M_h f + [known-data terms of
 * eqs. heat-cg-dg / heat-cg-cg / wave-cg-dg / wave-cg-cg]; f: nodal source
 * values [N_t][n_nodes] at the free time nodes of the slab; f0: source at the
 * slab start (cGP only, else ignored, may be NULL); u0, v0: end values of the
 * previous slab (v0 wave only).  Rows of boundary nodes are set to 0.  With
 * n_slabs > 1, f is [slab][N_t][n_nodes] and u0 enters the first slab only. */
stmg_status stmg_rhs(stmg_ctx* ctx, const double* f, const double* f0, const double* u0,
                     const double* v0, double* rhs);
/* FGMRES (right preconditioned, one V-cycle per iteration) on the finest level
 * in FP64 until ||rhs - S u|| <= rtol ||rhs||; u holds the initial guess on entry.
 * Synchronous (reads the Krylov scalars each iteration).  stats may be NULL. */
stmg_status stmg_solve(stmg_ctx* ctx, const double* rhs, double* u, stmg_solve_stats* stats);
/* Wave only: velocity of the slab from the condensed solution,
 * v = M_tau^-1 (A_tau u + alpha u0 - beta v0) (cGP) / M_tau^-1 (A_tau u - alpha u0) (dG). */
stmg_status stmg_wave_velocity(stmg_ctx* ctx, const double* u, const double* u0, const double* v0,
                               double* v);
/* Broadcast of the previous slab's end value to all time DoFs (of every slab of the system):
 * the plain initial guess. */
stmg_status stmg_guess_previous(stmg_ctx* ctx, const double* u0, double* u);

/* End-to-end slab step from HOST buffers: uploads f [N_t][n], f0, u0, v0 (may be
 * NULL as above), builds the right-hand side, solves from the previous-slab
 * guess and downloads u [N_t][n] (and v for the wave equation, may be NULL).
 * With n_slabs > 1, f and u are [slab][N_t][n].  Synchronous. */
stmg_status stmg_solve_slab_host(stmg_ctx* ctx, const double* f, const double* f0, const double* u0,
                                 const double* v0, double* u, double* v, stmg_solve_stats* stats);

/* ---- Learned initial guess (not in the paper) ----
 * A chain of `layers` 3x3x3 convolutions on the finest node grid (zero padding),
 * ReLU between layers, BF16 activations and weights with FP32 accumulation on the
 * tensor cores; trained with Adam on FP32 master weights by the library's own
 * forward and backward kernels.  Input channels: the previous slab's N_t time
 * blocks times scales[0] and the slab's source at its N_t time nodes times
 * scales[1]; output: N_t channels c, the guess is u_prev_end + c / scales[2] on
 * unconstrained nodes (u_prev_end = last time block of the previous slab).
 * channels: layers+1 counts (channels[0] = 2 N_t, channels[layers] = N_t, all <= 64);
 * weights: HOST FP64, per layer [co][ci][27] concatenated, tap = (dx+1)+3(dy+1)+9(dz+1);
 * biases: HOST FP64, per layer [co] concatenated.  All vectors: device FP64 [N_t][n_nodes]. */
typedef struct stmg_net stmg_net;
stmg_status stmg_net_create(stmg_net** out, stmg_ctx* ctx, int layers, const int* channels, const double* weights,
                            const double* biases, const double* scales);
/* Frees the network.  Destroying its context first is allowed: the network is then detached,
 * every later call on it returns STMG_ERR_INVALID_ARG, and stmg_net_destroy still frees it. */
stmg_status stmg_net_destroy(stmg_net* net);
/* u_guess = network guess for the slab after u_prev, from the slab's source f. */
stmg_status stmg_net_predict(stmg_net* net, const double* u_prev, const double* f, double* u_guess);
/* One Adam step (lr) on the mean squared error against the scaled target
 * (u_target - u_prev_end) * scales[2] over unconstrained nodes; *loss (host) receives the loss
 * before the step.  Synchronous. */
stmg_status stmg_net_train_step(stmg_net* net, const double* u_prev, const double* f, const double* u_target,
                                double lr, double* loss);
/* Loss, parameter gradients (HOST, same layouts as weights/biases) and the raw network output
 * (HOST [N_t][n_nodes], before scaling back) without updating; any output may be NULL.  Synchronous. */
stmg_status stmg_net_gradients(stmg_net* net, const double* u_prev, const double* f, const double* u_target,
                               double* loss, double* grad_w, double* grad_b, double* out);
/* Keeps the better of two initial guesses: u holds the default guess (e.g. the previous-slab
 * guess) on entry; if ||rhs - S candidate|| < ||rhs - S u|| (FP64), u becomes candidate.
 * *chosen (host, may be NULL) = 1 when the candidate was taken.  Synchronous. */
stmg_status stmg_select_guess(stmg_ctx* ctx, const double* rhs, const double* candidate, double* u, int* chosen);
/* End-to-end learned slab step (heat dG) from HOST buffers: uploads f [N_t][n] and the previous
 * slab u_prev [N_t][n], builds the right-hand side, predicts the network guess, keeps it only if
 * its FP64 residual is below the previous-slab guess's (*chosen = 1, may be NULL), solves with
 * FGMRES and downloads u [N_t][n].  Synchronous. */
stmg_status stmg_solve_slab_host_learned(stmg_ctx* ctx, stmg_net* net, const double* f, const double* u_prev,
                                         double* u, int* chosen, stmg_solve_stats* stats);
/* Current FP32 master parameters (HOST, FP64 arrays in the layouts of stmg_net_create). */
stmg_status stmg_net_weights(stmg_net* net, double* weights, double* biases);

/* Smoothing without any device allocation.  Same result as stmg_smooth, but the
 * residual f - S_l u of each sweep is kept in a fixed buffer of
 * STMG_NOALLOC_SCRATCH_BYTES bytes that is part of the library's device image
 * instead of the context's per-level work vectors.  Meant for callers that may
 * not call cudaMalloc (or any allocating routine) on the path that smooths, for
 * example code whose device memory is fully handed to another allocator once
 * the context exists, or code that must not touch the context's own scratch.
 * The paper has no counterpart; this is an interface variant only.
 * - stmg_create looks up the buffer's device address on the device current at
 *   create time; that lookup loads the library's device image there, so the
 *   buffer is taken when the context is created, not at the first smoothing
 *   call.  Every device on which a context was created holds it until the
 *   process exits.  The same device must be current at every call
 *   (STMG_ERR_INVALID_ARG otherwise).
 * - Returns STMG_ERR_INVALID_ARG, before any device work, when N_t * n_nodes of
 *   the level times the element size (8 for FP64, 4 for FP32) exceeds the buffer.
 * - All calls share the one buffer and it keeps the last call's contents:
 *   calls that overlap on the GPU (other streams, other contexts, other
 *   threads) race; order them on one stream. */
#define STMG_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)
stmg_status stmg_smooth_noalloc(stmg_ctx* ctx, int level, int precision, int sweeps, const void* f, void* u);

/* Number of kernels this context has launched so far (a captured V-cycle graph
 * counts its kernel nodes at every replay).  Host-side counter, no device work. */
stmg_status stmg_launch_count(const stmg_ctx* ctx, int64_t* count);

/* Measurement hook: runs `reps` back-to-back launches of one kernel on the
 * context's own stream over the level's work vectors (contents are
 * overwritten) and returns the mean duration from CUDA events recorded on that
 * stream.  kernel: STMG_KERNEL_APPLY (the operator kernel alone, no row
 * initialisation), STMG_KERNEL_ASM (one additive Schwarz application) or
 * STMG_KERNEL_VCYCLE (one whole V-cycle from level 0; level must be 0).  Synchronous.
 * precision STMG_DF32 times the double-float level-0 apply (outer_apply = STMG_DF32).
 * STMG_KERNEL_ORTHO: one FGMRES orthogonalisation (the three Gram-Schmidt passes) of a level-0
 * vector against `level` basis vectors (1..fgmres_restart), the basis in FP64 (precision
 * STMG_FP64) or in double-float pairs (STMG_DF32); the Krylov workspace is overwritten. */
enum { STMG_KERNEL_APPLY = 1, STMG_KERNEL_ASM = 2, STMG_KERNEL_VCYCLE = 3, STMG_KERNEL_ORTHO = 4 };
/* Test hook for failure detection (no counterpart in the paper).  Runs one kernel whose bounded
 * device wait cannot complete: it gives up after about one second and records the timeout in the
 * context's device status word, exactly as a bulk copy that never lands would.  Nothing faults.
 * Returns STMG_ERR_TIMEOUT; from then on the bulk-copy kernels of this context skip their work and
 * stmg_solve returns STMG_ERR_TIMEOUT.  Destroy the context afterwards.  Synchronous. */
stmg_status stmg_selftest_device_timeout(stmg_ctx* ctx);
stmg_status stmg_time_kernel(stmg_ctx* ctx, int kernel, int level, int precision, int reps, double* avg_ms);

#ifdef __cplusplus
}
#endif

#endif /* STMG_H */
