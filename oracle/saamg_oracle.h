/*
 * saamg_oracle.h -- plain, slow, single-threaded FP64 CPU oracle for SAAMG-PCG.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the only thing the two sides
 * have in common are the seeded input arrays the tests hand to both.
 *
 * Method: Adelmann, Arbenz, Ineichen, "A Fast Parallel Poisson Solver on
 * Irregular Domains Applied to Beam Dynamic Simulations".
 *   - Sec. 2, Eqs. (5)-(11): finite-difference Poisson system on an irregular
 *     domain with constant / linear / quadratic Dirichlet extrapolation on the
 *     pipe wall and a Robin condition on the open ends; Eq. (12) and the
 *     paragraph after it: symmetric diagonal scaling D^-1/2 A D^-1/2.
 *   - Sec. 3.1: conjugate gradients; Sec. 3.2, Algorithm 1: V-cycle with
 *     R = P^T, tentative prolongator from aggregates, damped-Jacobi smoothed
 *     prolongator, Chebyshev smoother, direct coarse solve.
 *
 * Every array is owned by the oracle; getters copy into caller buffers.
 */
#ifndef SAAMG_ORACLE_H
#define SAAMG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_op orc_op;
typedef struct orc_hier orc_hier;

/* Boundary modes (Sec. 2, Eqs. (7), (8), (9)-(10)). */
enum { ORC_CONSTANT = 0, ORC_LINEAR = 1, ORC_QUADRATIC = 2 };
/* Treatment of the two z-planes: Robin (Eq. (5), third line; Eq. (11)) or Dirichlet. */
enum { ORC_Z_ROBIN = 0, ORC_Z_DIRICHLET = 1 };

/* Build the unscaled and scaled operator of Sec. 2 on the box grid
 * node(i,j,k) = origin + (i hx, j hy, k hz), 0 <= i < nx etc.
 * Domain: elliptic cross-section with semi-axes a*sigma(z), b*sigma(z) about (cx, cy);
 * sigma is 1 at the first z-plane and `taper` at the last, linear in between.
 * Returns NULL on invalid arguments. */
orc_op *orc_build_operator(int nx, int ny, int nz, double hx, double hy, double hz,
                           double ox, double oy, double oz, double a, double b,
                           double taper, double cx, double cy, int zbc,
                           int symmetrize_gamma2, int mode);
void orc_op_free(orc_op *op);
int orc_op_n(const orc_op *op);
long orc_op_nnz(const orc_op *op);
/* node_of_row[n]: box index i + nx (j + ny k); scale[n]: s_i = d_i^-1/2;
 * bfac[n]: 0.5 on symmetrised Robin-plane rows, else 1;
 * rowptr[n+1], col[nnz], aval[nnz] (unscaled A), ahat[nnz] (scaled). Any may be NULL. */
void orc_op_get(const orc_op *op, int *node_of_row, double *scale, double *bfac,
                int *rowptr, int *col, double *aval, double *ahat);
/* Boundary fractions per row: frac[6*n] for directions (-x,+x,-y,+y,-z,+z);
 * -1 where the neighbour is an unknown or the side is a virtual Robin point. */
void orc_op_fractions(const orc_op *op, double *frac);
/* Inside test of one box node (1 = unknown). */
int orc_node_inside(const orc_op *op, int i, int j, int k);

/* The steps on either side of the solve in a PIC time step (Sec. 1, Sec. 4.1).
 * Particles: coordinate arrays x, y, z and charges q of length np.  Box arrays of the
 * nx x ny x nz node lattice node(i,j,k) = origin + (i hx, j hy, k hz), i fastest. */
void orc_deposit_cic(int nx, int ny, int nz, double hx, double hy, double hz, double ox,
                     double oy, double oz, int np, const double *x, const double *y,
                     const double *z, const double *q, double *rho);
void orc_field_gradient(const orc_op *op, const double *phi, double *ex, double *ey,
                        double *ez);
void orc_gather_cic(int nx, int ny, int nz, double hx, double hy, double hz, double ox,
                    double oy, double oz, const double *ex, const double *ey, const double *ez,
                    int np, const double *x, const double *y, const double *z, double *epx,
                    double *epy, double *epz);

/* SA-AMG hierarchy (Sec. 3.2). */
orc_hier *orc_setup(const orc_op *op, int cheb_degree, double cheb_ratio,
                    double cheb_safety, int max_coarse, int max_levels,
                    int power_iters);
/* Aggregation kinds: MIS-2 seeded (default) or cubes of 3^3 lattice nodes (Sec. 3.2). */
enum { ORC_AGG_MIS2 = 0, ORC_AGG_CUBES = 1 };
orc_hier *orc_setup_agg(const orc_op *op, int cheb_degree, double cheb_ratio,
                        double cheb_safety, int max_coarse, int max_levels,
                        int power_iters, int aggregation);
/* Coarsest-level solver: dense LU (default) or symmetric Gauss-Seidel steps (Sec. 3.2). */
enum { ORC_COARSE_LU = 0, ORC_COARSE_GS = 1 };
orc_hier *orc_setup_ex(const orc_op *op, int cheb_degree, double cheb_ratio,
                       double cheb_safety, int max_coarse, int max_levels, int power_iters,
                       int aggregation, int coarse_solver, int coarse_sweeps);
/* Colouring of the coarsest level (Gauss-Seidel); returns the number of colours or 0. */
int orc_hier_colours(const orc_hier *h, int *colour);
void orc_hier_free(orc_hier *h);
int orc_hier_levels(const orc_hier *h);
int orc_hier_n(const orc_hier *h, int l);
long orc_hier_nnz(const orc_hier *h, int l);
long orc_hier_nnz_p(const orc_hier *h, int l);
/* Status of setup: 0 ok, nonzero error (e.g. coarse level too large). */
int orc_hier_status(const orc_hier *h);
void orc_hier_get_a(const orc_hier *h, int l, int *rowptr, int *col, double *val);
void orc_hier_get_agg(const orc_hier *h, int l, int *agg, unsigned char *is_root);
void orc_hier_get_p(const orc_hier *h, int l, int *rowptr, int *col, double *val);
void orc_hier_get_r(const orc_hier *h, int l, int *rowptr, int *col, double *val);
double orc_hier_lambda(const orc_hier *h, int l);
double orc_hier_omega(const orc_hier *h, int l);

/* Building blocks, exposed so that each can be pinned on its own. */
unsigned int orc_fmix32(unsigned int h);
void orc_mis2(int n, const int *rowptr, const int *col, const unsigned int *ids,
              unsigned int seed, unsigned char *is_root);
int orc_aggregate(int n, const int *rowptr, const int *col, const unsigned int *ids,
                  unsigned int seed, const unsigned char *is_root, int *agg);
/* Cubes of 3 x 3 x 3 lattice nodes (ids on a dims[0] x dims[1] x dims[2] lattice); fills
 * agg, is_root (smallest row of each aggregate), next_ids (cube index of each aggregate)
 * and next_dims (the cube lattice); any output may be NULL except agg. */
int orc_cube_aggregate(int n, const unsigned int *ids, const int dims[3], int *agg,
                       unsigned char *is_root, unsigned int *next_ids, int next_dims[3]);
/* Multicolouring by synchronous rounds of local key maxima (colour = round). */
int orc_colour(int n, const int *rowptr, const int *col, const unsigned int *ids,
               unsigned int seed, int *colour);
/* `steps` symmetric multicolour Gauss-Seidel steps from x = 0. */
void orc_sgs(int n, const int *rowptr, const int *col, const double *val, const double *invd,
             const int *colour, int ncolours, int steps, const double *b, double *x);
double orc_power_lambda(int n, const int *rowptr, const int *col, const double *val,
                        const unsigned int *ids, int iters);
void orc_cheb_smooth(int n, const int *rowptr, const int *col, const double *val,
                     const double *invd, double lambda_hat, double ratio, double safety,
                     int degree, const double *b, double *x, int x_is_zero);
int orc_dense_lu_solve(int n, const double *a, const double *b, double *x);

/* Preconditioner application z = M r on level 0 (one V-cycle, Algorithm 1). */
void orc_vcycle(const orc_hier *h, const double *r, double *z);
/* PCG on the scaled system (Sec. 3.1).  beta_rule 0: Fletcher-Reeves (r'z ratio),
 * 1: Polak-Ribiere.  Returns 0 converged, 1 not converged, -1 numerical breakdown. */
int orc_pcg(const orc_hier *h, const double *bhat, double *xhat, double rtol, int maxit,
            int beta_rule, int *iters, double *relres);
/* Full solve on box arrays: rho (box) -> phi (box), phi holds the initial guess
 * on entry (warm start, Sec. 4), zero outside the unknowns on exit. */
int orc_solve(const orc_hier *h, const double *rho_box, double *phi_box, double rtol,
              int maxit, int beta_rule, int *iters, double *relres, double *relres_true);

#ifdef __cplusplus
}
#endif
#endif
