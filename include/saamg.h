/*
 * saamg.h -- C ABI of the GB300 (sm_103a) SAAMG-PCG library.
 *
 * Conjugate gradients on the finite-difference Poisson system of an irregular 3-D
 * pipe domain, preconditioned by one smoothed-aggregation AMG V-cycle per iteration
 * (Adelmann, Arbenz, Ineichen, "A Fast Parallel Poisson Solver on Irregular Domains
 * Applied to Beam Dynamic Simulations").
 *
 * Conventions for every call:
 *   - Every function returns a saamg_status (0 = OK, 1 = not converged, < 0 = error),
 *     never aborts, throws or exits.  saamg_last_error() gives a message for the
 *     calling thread's last failure.
 *   - Device pointers are caller-owned and must stay valid until the work enqueued on
 *     `stream` has finished.  `stream` is a cudaStream_t (NULL = legacy default
 *     stream); all GPU work of a call is enqueued on it.  Calls that must return a
 *     host-visible result (sizes, iteration counts) synchronise that stream.
 *   - Handles (saamg_operator, saamg_hierarchy) are library-owned and released by
 *     saamg_free().  An operator must outlive every hierarchy set up from it.
 *   - Box arrays: nx*ny*nz doubles, node (i,j,k) at index i + nx*(j + ny*k), node
 *     position origin + (i*h[0], j*h[1], k*h[2]).  Compact arrays: one entry per
 *     unknown, unknowns numbered in ascending box index.
 *   - Device memory is taken from the allocator installed by saamg_set_allocator
 *     (cudaMalloc/cudaFree when none is installed).
 */
#ifndef SAAMG_H
#define SAAMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SAAMG_MAX_LEVELS 16

typedef enum {
  SAAMG_OK = 0,
  SAAMG_NOT_CONVERGED = 1,   /* maxit reached; the best iterate is returned */
  SAAMG_NOT_READY = 2,       /* saamg_solve_test: the solve is still running */
  SAAMG_EINVAL = -1,         /* invalid argument */
  SAAMG_ENOMEM = -2,         /* the allocator returned NULL */
  SAAMG_ECUDA = -3,          /* a CUDA runtime call failed */
  SAAMG_NUMERICAL = -4,      /* NaN/Inf or a zero pivot / breakdown */
  SAAMG_DEVICE_TIMEOUT = -5, /* a bounded device-side wait gave up */
  SAAMG_UNIMPLEMENTED = -6
} saamg_status;

/* Dirichlet treatment on the pipe wall Gamma_1 (Sec. 2, Eqs. (7), (8), (9)-(10)). */
typedef enum {
  SAAMG_BC_CONSTANT = 0,
  SAAMG_BC_LINEAR = 1,
  SAAMG_BC_QUADRATIC = 2
} saamg_boundary_mode;

/* Treatment of the two end planes Gamma_2: Robin (Eq. (5), Eq. (11)) or zero Dirichlet. */
typedef enum { SAAMG_Z_ROBIN = 0, SAAMG_Z_DIRICHLET = 1 } saamg_zbc;

/* Arithmetic of the V-cycle.  The outer CG, its residual, dot products, search
 * direction and the coarsest-level solve are FP64 in every mode. */
typedef enum {
  SAAMG_PREC_FP64 = 0,      /* whole method in FP64 */
  SAAMG_PREC_FP32 = 1,      /* V-cycle in FP32, coarse operators stored FP32 */
  SAAMG_PREC_FP32_BF16 = 2  /* V-cycle in FP32, coarse operators stored BF16 */
} saamg_precision;

/* Aggregation of the tentative prolongator (Sec. 3.2, "Prolongation operator").
 * MIS2: aggregates grown from a distance-2 maximal independent set of the graph of A_l
 * (hashed priorities; identical on any launch configuration).
 * CUBES: the paper's own "decoupled" aggregation: aggregates are the cubes of 3 x 3 x 3
 * lattice nodes (fewer where the domain boundary cuts a cube); the coarse nodes are the
 * cubes, so every level is again a lattice with ceil(n/3) nodes per axis. */
typedef enum { SAAMG_AGG_MIS2 = 0, SAAMG_AGG_CUBES = 1 } saamg_aggregation;

/* Coarsest-level solver (Sec. 3.2, "Coarse level solver"): an exact solve by dense LU
 * with partial pivoting (applied as an explicit inverse), or coarse_sweeps symmetric
 * Gauss-Seidel steps from zero. */
typedef enum { SAAMG_COARSE_LU = 0, SAAMG_COARSE_GS = 1 } saamg_coarse_solver;

/* Domain Omega (Sec. 2, Sec. 4.1): an elliptic pipe along z, cross-section
 * ((x-cx)/(a s))^2 + ((y-cy)/(b s))^2 < 1 where s = 1 at the first z-plane of the grid
 * and s = taper at the last, linear in between (taper = 1: straight pipe).  The first
 * and last z-planes of the grid are Gamma_2. */
typedef struct {
  double a, b;
  double taper;
  double cx, cy;
  int zbc;               /* saamg_zbc */
  int symmetrize_gamma2; /* 1: halve Robin rows (and rhs) so that constant and linear
                            modes give a symmetric matrix; 0: the raw rows */
} saamg_domain;

typedef struct {
  int n[3];
  double h[3];
  double origin[3];
} saamg_grid;

typedef struct {
  int cheb_degree;    /* Chebyshev steps per pre- and post-smoothing (default 2) */
  double cheb_ratio;  /* lambda_hi / lambda_lo of the smoothing interval (30) */
  double cheb_safety; /* lambda_hi = safety * lambda_hat (1.1) */
  int max_coarse;     /* stop coarsening at <= max_coarse unknowns (1000, Table 1) */
  int max_levels;     /* including the finest level (10) */
  int power_iters;    /* power-iteration steps for lambda_hat (10) */
  int precision;      /* saamg_precision (FP64) */
  int beta_rule;      /* 0: r'z ratio (Fletcher-Reeves form), 1: Polak-Ribiere (0) */
  int maxit;          /* PCG iteration limit (1000) */
  int aggregation;    /* saamg_aggregation (MIS-2) */
  int coarse_solver;  /* saamg_coarse_solver (dense LU) */
  int coarse_sweeps;  /* Gauss-Seidel steps per coarse solve (3, Sec. 3.2) */
  int device_loop;    /* 1: saamg_solve / saamg_solve_host run the PCG loop on the device (the
                         graph of saamg_solve_async: no host round trip per iteration); 0: a
                         host-driven loop with one synchronisation per iteration.  Both run the
                         same kernels in the same order and give the same bits. (1) */
} saamg_params;

typedef struct {
  int iters;          /* products A p */
  int converged;      /* 1 when ||r|| <= rtol ||b|| */
  double relres;      /* recursive residual ||r||/||b|| of the scaled system */
  double relres_true; /* recomputed ||b - A x|| / ||b|| of the scaled system */
  double solve_ms;    /* wall time of the call */
} saamg_solve_info;

typedef struct {
  int levels;
  int n[SAAMG_MAX_LEVELS];          /* unknowns per level */
  long long nnz[SAAMG_MAX_LEVELS];  /* nonzeros of A_l (level 0: explicit CSR) */
  long long nnz_p[SAAMG_MAX_LEVELS];/* nonzeros of P_l (0 on the coarsest level) */
  double lambda[SAAMG_MAX_LEVELS];  /* power-iteration estimate of lambda_max(D^-1 A_l) */
  long long device_bytes;           /* device memory held by the hierarchy */
  double setup_ms;                  /* wall time of saamg_setup */
  int sell_index_bytes[SAAMG_MAX_LEVELS]; /* smoother layout of A_l: 0 CSR (level 0: the
                                             stencil), 4 SELL with 32-bit columns, 2 SELL
                                             with 16-bit column offsets from the row */
} saamg_hierarchy_info;

typedef struct saamg_operator saamg_operator;
typedef struct saamg_hierarchy saamg_hierarchy;

/* Allocator hook: alloc(bytes, stream, ctx) -> device pointer or NULL; free(ptr, stream, ctx). */
typedef void *(*saamg_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*saamg_free_fn)(void *ptr, void *stream, void *ctx);

/* Fills *p with the defaults listed above.  EINVAL if p is NULL. */
saamg_status saamg_params_default(saamg_params *p);

/* Installs a process-wide device allocator (both NULL: back to cudaMalloc/cudaFree).
 * Handles keep the allocator that created them.  Not thread-safe against concurrent
 * allocation. */
saamg_status saamg_set_allocator(saamg_alloc_fn alloc, saamg_free_fn free_fn, void *ctx);

/* Builds the scaled operator D^-1/2 A D^-1/2 of Sec. 2 (Eqs. (5)-(12) and the scaling
 * paragraph after Eq. (12)) on the device: inside test and boundary fractions of every
 * lattice node, the rows of the constant / linear / quadratic extrapolation, Robin rows
 * on Gamma_2, the diagonal scaling, a matrix-free stencil description and an explicit
 * CSR copy for the AMG setup.  mode: saamg_boundary_mode.
 * Errors: EINVAL (NULL pointers, sizes < 1, nz < 2 (Robin) or < 3 (Dirichlet), h <= 0,
 * a, b, taper <= 0, more than 2^31 nonzeros, more than 30000 nodes along x, a lattice line
 * whose inside nodes are not contiguous), ENOMEM, ECUDA. */
saamg_status saamg_build_operator(const saamg_domain *domain, const saamg_grid *grid,
                                  int mode, void *stream, saamg_operator **out);

/* Number of unknowns and nonzeros of the scaled operator. */
saamg_status saamg_operator_size(const saamg_operator *op, int *n_unknowns, long long *nnz);

/* Copies the operator to HOST buffers (any may be NULL): node_of_row[n] (box index),
 * scale[n] (s_i = a_ii^-1/2), rowptr[n+1], col[nnz], val[nnz] (scaled values), and
 * is_regular[n] (1 when the row is applied with the constant interior stencil). */
saamg_status saamg_operator_copy(const saamg_operator *op, int *node_of_row, double *scale,
                                 int *rowptr, int *col, double *val, unsigned char *is_regular,
                                 void *stream);

/* y = Ahat x on compact device vectors (matrix-free stencil, Eq. (6) with the boundary rows). */
saamg_status saamg_operator_apply(const saamg_operator *op, const double *x, double *y,
                                  void *stream);

/* inv = A^-1 for a dense n x n matrix: the coarsest-level direct solver of Sec. 3.2 ("Coarse
 * level solver") on its own.  a and inv are device arrays stored by rows (a[i * n + j] =
 * A(i, j)); a is only read, and inv must not overlap it.  Gauss-Jordan elimination with the
 * pivot choice of an LU with partial pivoting (largest |a_ik| among the rows not yet
 * pivoted, the lowest row on ties; a NaN is never chosen), FP64 throughout.  Temporary
 * device memory: 2 n^2 doubles.  Synchronises the stream (it reads the pivot flag).
 * Errors: EINVAL (n < 0 or n > 16384, NULL array with n > 0), ENOMEM, ECUDA, NUMERICAL (a
 * pivot column without a nonzero finite candidate). */
saamg_status saamg_dense_inverse(int n, const double *a, double *inv, void *stream);

/* Sets up the SA-AMG hierarchy of Sec. 3.2 on the device: MIS-2 aggregation of the
 * adjacency graph of A_l, tentative prolongator, lambda_hat by power iteration, damped-
 * Jacobi smoothed prolongator P_l, R_l = P_l^T, Galerkin A_{l+1} = R_l A_l P_l, and a
 * dense LU (partial pivoting) with explicit inverse of the coarsest matrix.
 * params NULL = defaults.  Errors: EINVAL, ENOMEM, ECUDA, NUMERICAL (zero pivot,
 * coarsest level larger than 16384 because coarsening stalled). */
saamg_status saamg_setup(const saamg_operator *op, const saamg_params *params, void *stream,
                         saamg_hierarchy **out);

/* Setup that reuses the aggregation hierarchy of `prev` (Sec. 5.2, "Reusing the aggregation
 * hierarchy"; Table 6): for a new operator whose matrix has the same pattern as the one
 * prev was built on (same unknowns; e.g. another boundary mode or other grid spacings on
 * the same lattice of unknowns), the aggregates and the number of levels of prev are kept
 * and only lambda_hat, the smoothed prolongators, the Galerkin operators and the coarse LU
 * are rebuilt from the new values.  Aggregation depends on the pattern only, so the result
 * equals a fresh saamg_setup on op.  params NULL = prev's parameters (max_coarse and
 * max_levels are ignored: prev fixes the levels).  prev stays valid and independent.
 * EINVAL when the patterns differ. */
saamg_status saamg_setup_reuse(const saamg_operator *op, const saamg_hierarchy *prev,
                               const saamg_params *params, void *stream, saamg_hierarchy **out);

/* A work set of h: a second hierarchy handle over h's levels with work vectors of its own,
 * so that solves of one geometry (successive right-hand sides, Sec. 5.2) can be in flight
 * at the same time.  It reads h's level matrices, prolongators, restrictions, aggregates,
 * smoother coefficients and coarse solver without copying them (h's owner, if h is itself a
 * work set) and allocates only its V-cycle vectors (FP64 or FP32 by h's precision), the PCG
 * vectors and the reduction partials; its device-loop graph is its own.  Every solve call
 * accepts it like a hierarchy and gives the same bits as on h.  saamg_set_cheb_degree and
 * saamg_autotune_cheb_degree change the handle they are given only.  Free it with
 * saamg_free; the shared levels are released when the hierarchy that owns them and all of its
 * work sets have been freed (in any order).  device_bytes and setup_ms of its info count
 * its own vectors and its creation.  Errors: EINVAL, ENOMEM, ECUDA. */
saamg_status saamg_hierarchy_work_set(const saamg_hierarchy *h, void *stream,
                                      saamg_hierarchy **out);

saamg_status saamg_hierarchy_get_info(const saamg_hierarchy *h, saamg_hierarchy_info *info);

/* Copies level l to HOST buffers (any may be NULL): A_l as CSR (rowptr[n_l+1], col, val),
 * aggregate index agg[n_l] and root flags root[n_l] (levels below the coarsest), P_l as
 * CSR (p_rowptr[n_l+1], p_col, p_val) and R_l (r_rowptr[n_{l+1}+1], r_col, r_val). */
saamg_status saamg_hierarchy_copy_level(const saamg_hierarchy *h, int l, int *rowptr, int *col,
                                        double *val, int *agg, unsigned char *root,
                                        int *p_rowptr, int *p_col, double *p_val,
                                        int *r_rowptr, int *r_col, double *r_val, void *stream);

/* z = M r: one V-cycle (Algorithm 1) on compact device vectors of level 0. */
saamg_status saamg_vcycle(const saamg_hierarchy *h, const double *r, double *z, void *stream);

/* Solves A phi = rho (Sec. 3.1, PCG preconditioned by one V-cycle per iteration) on BOX
 * device arrays: rho = rho/epsilon_0 sampled at the nodes (read at unknowns only), phi
 * holds the initial guess on entry (warm start, Sec. 4) and the solution on exit, zero
 * at non-unknowns.  Stops when ||r||_2 <= rtol ||b||_2 for the scaled system.
 * Returns OK, NOT_CONVERGED (maxit reached), NUMERICAL (NaN/Inf or breakdown), EINVAL. */
saamg_status saamg_solve(saamg_hierarchy *h, const double *rho, double *phi, double rtol,
                         void *stream, saamg_solve_info *info);

/* Same as saamg_solve with HOST box arrays; the host<->device transfers are part of the call.
 * Page-locked (pinned) arrays are read by the gather and written by the scatter kernels
 * directly through their mapped device addresses (each value crosses the host link once, no
 * staging copy); pageable arrays are staged through device box arrays allocated for the call. */
saamg_status saamg_solve_host(saamg_hierarchy *h, const double *rho_host, double *phi_host,
                              double rtol, void *stream, saamg_solve_info *info);

/* Same solve as saamg_solve, enqueued as ONE CUDA graph and returning at once: the whole
 * PCG loop (Sec. 3.1) runs on the device in a conditional while node whose test kernel
 * ends the loop (no host round trip per iteration).  Gather, the graph, the copy of the
 * result scalars and the scatter are enqueued on `stream`.  The first call on a hierarchy
 * captures the graph (about one solve's worth of launches; make it outside any capture).
 * rho and phi must stay valid until saamg_solve_wait or saamg_solve_test reports the end.
 * A hierarchy holds one solve's work vectors: do not start a second solve on the same
 * hierarchy before the first has finished (saamg_solve_batched orders them for you). */
saamg_status saamg_solve_async(saamg_hierarchy *h, const double *rho, double *phi, double rtol,
                               void *stream);

/* OK when the hierarchy's last asynchronous solve has finished, NOT_READY otherwise. */
saamg_status saamg_solve_test(const saamg_hierarchy *h);

/* Waits for the hierarchy's last asynchronous solve and returns its status and info
 * (solve_ms is left 0). */
saamg_status saamg_solve_wait(saamg_hierarchy *h, saamg_solve_info *info);

/* Many solves in one call (batched serving of many geometries): count right-hand sides
 * rho[j] -> phi[j] (device box arrays; phi[j] holds the initial guess) on hierarchies hs[j]
 * of any sizes, precisions and Chebyshev degrees; several may share a hierarchy.  The batch
 * runs as ONE CUDA graph launch, in one of two forms that give the same bits as saamg_solve
 * for every solve:
 *   merged: every solve gets its own work vectors, and each operation of a PCG iteration
 *     (every smoothing step, residual, transfer and coarse solve of the V-cycles, the CG
 *     products, dot products and updates) is one kernel launch over all solves that are still
 *     iterating, the solves split into up to 8 sub-batches that run side by side;
 *   per-solve: one device-loop graph per solve (as saamg_solve_async), solves of one
 *     hierarchy in order on one of up to 32 concurrent branches.
 * The graph is built on the first call for a set of (hierarchy, rho, phi, rtol) and kept
 * for later calls with the same set (two sets are kept; saamg_release_batch_cache frees
 * them).  The first call with a set runs the merged form, the second the per-solve form, and
 * later calls the one whose first run was faster (saamg_batch_last reports both times).
 * Batches with a single solve, a hierarchy without unknowns or a Gauss-Seidel coarse solver
 * always take the per-solve form.  Joins back into `stream` and returns when all are done;
 * infos[j] per solve (solve_ms = the wall time of the whole batch).  Returns the worst
 * status. */
saamg_status saamg_solve_batched(saamg_hierarchy *const *hs, const double *const *rho,
                                 double *const *phi, int count, double rtol, void *stream,
                                 saamg_solve_info *infos);

/* The form the most recent saamg_solve_batched call ran (merged: 1 merged, 0 per-solve) and
 * the wall times in ms of the first run of each form with that set of solves (-1: not run). */
saamg_status saamg_batch_last(int *merged, double *ms_merged, double *ms_graphs);

/* Frees the graphs and work vectors that saamg_solve_batched keeps for repeated batches
 * (they are otherwise held until they are replaced, and never freed at process exit, when
 * the allocator hook may no longer be callable). */
saamg_status saamg_release_batch_cache(void);

/* Launch shape of the level-0 stencil passes of one precision (the Chebyshev steps, the
 * residual and the matrix-free prolongation; the passes with a reduction keep a fixed shape
 * so that their partial sums never change).  Every row is computed the same way under every
 * shape, so results are identical; only the time changes. */
typedef struct saamg_stencil_config {
  int chunks_per_step; /* chunks of 32 rows per warp step: 1, 2 or 4 */
  int packed;          /* 1: 32 regular-run rows per warp from the row list, then the table
                          rows; 0: the line chunks (<= 32 unknowns of one x-line) */
  int block;           /* threads per block: 128 or 256 */
  int blocks_per_sm;   /* grid = SMs x this (fewer when the rows run out): 8, 16 or 32 */
} saamg_stencil_config;

/* The shape op uses for precision 0 (FP64 passes) or 1 (FP32 passes, also the BF16 mode's). */
saamg_status saamg_stencil_config_get(const saamg_operator *op, int precision,
                                      saamg_stencil_config *cfg);
/* Sets it (cfg NULL: the default); EINVAL for a shape outside the sets above.  Hierarchies
 * set up later, and solve graphs captured later, use it; graphs captured before keep theirs. */
saamg_status saamg_stencil_config_set(saamg_operator *op, int precision,
                                      const saamg_stencil_config *cfg);
/* Autotuner of the launch shape: times the level-0 Chebyshev step of precision 0 or 1 under
 * all 36 shapes on scratch vectors of op's size (allocated and freed here), sets the fastest
 * on op and returns it with its time in microseconds (median of three launches). */
saamg_status saamg_autotune_stencil(saamg_operator *op, int precision, void *stream,
                                    saamg_stencil_config *best, double *best_us);

/* Changes the Chebyshev degree of every smoothed level (coefficients from the stored
 * lambda_hat; the hierarchy is otherwise unchanged).  EINVAL outside 1..16. */
saamg_status saamg_set_cheb_degree(saamg_hierarchy *h, int degree);

/* Autotuner: times a device-loop solve of rho (device box array) for every Chebyshev
 * degree lo..hi, keeps the degree with the shortest converged solve and returns it and
 * its time.  Allocates one box array for the trial solutions. */
saamg_status saamg_autotune_cheb_degree(saamg_hierarchy *h, const double *rho, int lo, int hi,
                                        double rtol, void *stream, int *best_degree,
                                        double *best_ms);

/* Deterministic MIS-2 aggregation of a symmetric graph given as CSR on the device
 * (rowptr[n+1], col[nnz], self loops allowed), distinct node ids ids[n] (NULL: the row
 * index) and a 32-bit seed.  The priority of node v is fmix32(id_v ^ seed), a bijection,
 * so distinct ids never tie.  Outputs (device):
 * root[n] (1 = aggregate root) and agg[n] (aggregate index, roots numbered by ascending
 * row).  *n_agg receives the number of aggregates.  Same rule as the hierarchy's setup. */
saamg_status saamg_mis2_aggregate(int n, const int *rowptr, const int *col, const uint32_t *ids,
                                  uint32_t seed, unsigned char *root, int *agg, int *n_agg,
                                  void *stream);

/* saamg_mis2_aggregate without any device allocation (the paper has no counterpart; it
 * exists for callers that cannot allocate device memory at the point of the call, such as
 * code inside a fixed memory pool or a callback that must not re-enter the allocator).
 * Same arguments, rule and results as saamg_mis2_aggregate.  Its scratch is one static
 * device array of about 5.8 MB per device that loads the library, held until the process
 * exits; graphs with more than 262,144 nodes are rejected with EINVAL.  Every call looks up
 * the array's device address (cudaGetSymbolAddress, which allocates nothing); the first call
 * on a device also loads the library's device code there, so make that first call before
 * any stream capture.  Calls share the array: two calls whose GPU work
 * overlaps (other streams, other host threads) race and give undefined results.  Nothing
 * from an earlier call is read: every call initialises the parts it uses. */
saamg_status saamg_mis2_aggregate_noalloc(int n, const int *rowptr, const int *col,
                                          const uint32_t *ids, uint32_t seed, unsigned char *root,
                                          int *agg, int *n_agg, void *stream);

/* --- Around the solve in a PIC time step (Sec. 1, Sec. 4.1) --------------------------
 * Box arrays follow saamg_solve's layout (i fastest, nx*ny*nz FP64, device memory).
 * Particles are structure-of-arrays: x, y, z, q, np entries each, device memory. */

/* Cloud-in-cell deposition (Sec. 4.1, the charge density from the particles):
 * rho(node) = sum_p q_p W(x_p - x_node) / (hx hy hz), W the product of the 1-D hat
 * functions of width h; each particle reaches the 8 nodes of its cell, nodes outside the
 * box are dropped.  rho is overwritten.  Deterministic: every contribution is rounded once
 * to a 64-bit fixed-point value scaled from sum |q|, so the result does not depend on the
 * order of the atomic additions (relative accuracy about np * 2^-61 of sum|q| / V).
 * rho is NaN everywhere when a charge is not finite.  EINVAL on NULL arrays with np > 0. */
saamg_status saamg_deposit_cic(const saamg_grid *grid, int np, const double *x, const double *y,
                               const double *z, const double *q, double *rho, void *stream);

/* E = -grad phi (Sec. 1, the self field from the potential) on the box: at the unknowns of
 * op, second-order differences that take phi = 0 at the wall point of an outside neighbour
 * (boundary fraction of Sec. 2, the operator's clamped s; the derivative of the quadratic
 * through the three points), and on a Robin end plane the z-derivative of the Robin
 * condition (-phi/d outward); 0 at all other box nodes.  phi: box, e.g. saamg_solve's
 * output; ex, ey, ez: box, overwritten. */
saamg_status saamg_field_gradient(const saamg_operator *op, const double *phi, double *ex,
                                  double *ey, double *ez, void *stream);

/* The nodal field at the particles with the deposition's weights (the CIC pair that
 * conserves momentum): epx[p] = sum over the 8 nodes of W * ex(node), likewise y, z. */
saamg_status saamg_gather_cic(const saamg_grid *grid, const double *ex, const double *ey,
                              const double *ez, int np, const double *x, const double *y,
                              const double *z, double *epx, double *epy, double *epz,
                              void *stream);

/* Kernel classes for saamg_kernel_timing_read. */
typedef enum {
  SAAMG_KT_STENCIL_SMOOTH = 0, /* level-0 Chebyshev step fused with the residual (full step) */
  SAAMG_KT_STENCIL_APPLY = 1,  /* level-0 A x, and A p with p'Ap in PCG */
  SAAMG_KT_COARSE = 2,         /* smoother / residual on level 1 (rows = matrix entries) */
  SAAMG_KT_TRANSFER = 3,       /* CSR restriction / prolongation between levels 0 and 1 (entries) */
  SAAMG_KT_SPGEMM = 4,         /* sparse products of the setup */
  SAAMG_KT_STENCIL_RESID = 5,  /* level-0 residual b - A x */
  SAAMG_KT_STENCIL_FIRST = 6,  /* first Chebyshev steps on level 0 (from zero, or c1 = 0) */
  SAAMG_KT_PIC = 7,            /* CIC deposition and gather (rows = particles) */
  SAAMG_KT_PROLONG0 = 8,       /* matrix-free level-0 prolongation of the FP32 V-cycle */
  SAAMG_KT_COARSE_DEEP = 9,    /* SAAMG_KT_COARSE on levels >= 2 */
  SAAMG_KT_TRANSFER_DEEP = 10, /* SAAMG_KT_TRANSFER between levels >= 1 */
  SAAMG_KT_COUNT = 11
} saamg_kernel_class;

/* Number of kernels this library has launched in the calling process. */
long long saamg_kernel_launches(void);

/* enable != 0: record a CUDA event pair on the launching stream around every launch of
 * the classes above (adds two event records per launch); 0: stop recording. */
saamg_status saamg_kernel_timing(int enable);

/* Waits for the recorded events of class kclass and returns their summed duration, the
 * number of launches and the rows they processed since the last read; then resets the
 * class.  EINVAL for an unknown class. */
saamg_status saamg_kernel_timing_read(int kclass, double *total_ms, long long *launches,
                                      long long *rows);

/* Releases an operator or a hierarchy (NULL is ignored).  Waits for the handle's
 * outstanding work first.  The levels of a hierarchy with live work sets stay allocated
 * until the last of them is freed. */
void saamg_free(void *handle);

/* Message of the calling thread's last error ("" if none). */
const char *saamg_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SAAMG_H */
