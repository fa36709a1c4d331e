/*
 * saamg_oracle.c -- plain FP64 CPU oracle for SAAMG-PCG (test infrastructure).
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg use
 * this file.  It is deliberately slow and sequential: every step is written in
 * the order the paper gives it, so that it can be checked against the paper by
 * eye.  Compile with -ffp-contract=off: the geometric decisions (which node is
 * an unknown, the boundary fractions s, t) must be taken with the same IEEE
 * operations, in the same order, as any implementation compared against this one.
 *
 * The same source also builds, with -fopenmp, a multi-threaded CPU baseline (never
 * the parity reference): row loops and vector loops are split into static chunks
 * (every row still summed in the order written here, so those results are bitwise
 * those of the sequential build), and a dot product adds its chunk sums in thread
 * order, which makes it reproducible for a given thread count but not bitwise equal
 * to the sequential sum.  Without -fopenmp the pragmas are ignored.
 *
 * Paper: Adelmann, Arbenz, Ineichen, "A Fast Parallel Poisson Solver on Irregular
 * Domains Applied to Beam Dynamic Simulations" (J. Comput. Phys.).
 *
 * Readings of points the paper leaves open are marked READING.
 */
#include "saamg_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------- */
/* Small CSR container                                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
  int n, m; /* rows, cols */
  long nnz;
  int *rowptr; /* n+1 (int: every workload here stays below 2^31 nonzeros) */
  int *col;
  double *val;
} csr_t;

static void csr_free(csr_t *a) {
  free(a->rowptr);
  free(a->col);
  free(a->val);
  memset(a, 0, sizeof(*a));
}

static void csr_alloc(csr_t *a, int n, int m, long nnz) {
  a->n = n;
  a->m = m;
  a->nnz = nnz;
  a->rowptr = (int *)calloc((size_t)n + 1, sizeof(int));
  a->col = (int *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int));
  a->val = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
}

/* y = A x, each row summed in column order. */
static void csr_spmv(const csr_t *a, const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < a->n; ++i) {
    double acc = 0.0;
    for (int p = a->rowptr[i]; p < a->rowptr[i + 1]; ++p) acc += a->val[p] * x[a->col[p]];
    y[i] = acc;
  }
}

static double dot(int n, const double *x, const double *y) {
#ifdef _OPENMP
  /* multi-threaded baseline build: static chunks summed in index order, then the chunk
   * sums in thread order */
  double part[1024];
  int nt = omp_get_max_threads();
  if (nt > 1024) nt = 1024;
#pragma omp parallel num_threads(nt)
  {
    int t = omp_get_thread_num(), T = omp_get_num_threads();
    long lo = (long)n * t / T, hi = (long)n * (t + 1) / T;
    double a = 0.0;
    for (long i = lo; i < hi; ++i) a += x[i] * y[i];
    part[t] = a;
#pragma omp barrier
#pragma omp single
    nt = T;
  }
  double acc = 0.0;
  for (int t = 0; t < nt; ++t) acc += part[t];
  return acc;
#else
  double acc = 0.0;
  for (int i = 0; i < n; ++i) acc += x[i] * y[i];
  return acc;
#endif
}

/* ------------------------------------------------------------------------- */
/* Operator (Sec. 2)                                                          */
/* ------------------------------------------------------------------------- */
struct orc_op {
  int nx, ny, nz;
  double hx, hy, hz, ox, oy, oz;
  double a, b, taper, cx, cy;
  int zbc, symmetrize, mode;
  int n;              /* unknowns */
  int *node_of_row;   /* box index of each unknown, ascending */
  int *row_of_node;   /* -1 for box nodes that are not unknowns */
  double *scale;      /* s_i = 1 / sqrt(a_ii) */
  double *bfac;       /* 0.5 on symmetrised Robin rows, 1 elsewhere */
  double *frac;       /* 6 per row: boundary fraction or -1 */
  csr_t A;            /* unscaled */
  csr_t Ahat;         /* D^-1/2 A D^-1/2 */
};

static double node_coord(double o, int i, double h) { return o + (double)i * h; }

/* z-range of the domain: the two planes Gamma_2 are the first and last z-plane. */
static double zlo(const orc_op *op) { return op->oz; }
static double zhi(const orc_op *op) { return op->oz + (double)(op->nz - 1) * op->hz; }

/* Cross-section scale sigma(z): 1 at the first plane, `taper` at the last (Sec. 4.1
 * uses elliptic cylinders; the taper is the same cylinder with a linear cone). */
static double taper_sigma(const orc_op *op, double z) {
  if (op->taper == 1.0 || op->nz < 2) return 1.0;
  double tau = (z - zlo(op)) / (zhi(op) - zlo(op));
  return 1.0 + (op->taper - 1.0) * tau;
}

/* Implicit function of the elliptic wall Gamma_1 (Sec. 4.1): F < 0 inside. */
static double wall_F(const orc_op *op, double x, double y, double z) {
  double sg = taper_sigma(op, z);
  double u = (x - op->cx) / (op->a * sg);
  double v = (y - op->cy) / (op->b * sg);
  return (u * u + v * v) - 1.0;
}

/* Omega_h (Sec. 2): lattice points of Omega plus the Robin planes.  With Dirichlet
 * z-ends the first and last plane carry known zeros and are not unknowns. */
int orc_node_inside(const orc_op *op, int i, int j, int k) {
  if (i < 0 || j < 0 || k < 0 || i >= op->nx || j >= op->ny || k >= op->nz) return 0;
  if (op->zbc == ORC_Z_DIRICHLET && (k == 0 || k == op->nz - 1)) return 0;
  double x = node_coord(op->ox, i, op->hx);
  double y = node_coord(op->oy, j, op->hy);
  double z = node_coord(op->oz, k, op->hz);
  return wall_F(op, x, y, z) < 0.0;
}

static int box_index(const orc_op *op, int i, int j, int k) {
  return i + op->nx * (j + op->ny * k);
}

static int is_unknown(const orc_op *op, int i, int j, int k) {
  if (i < 0 || j < 0 || k < 0 || i >= op->nx || j >= op->ny || k >= op->nz) return 0;
  return op->row_of_node[box_index(op, i, j, k)] >= 0;
}

static double clamp_frac(double s) {
  /* READING: the paper needs 0 < s <= 1 (Sec. 2, definition of x*); the clamp only
   * guards against rounding and against a wall farther than one step (box face). */
  const double smin = 9.5367431640625e-07; /* 2^-20 */
  if (s < smin) s = smin;
  if (s > 1.0) s = 1.0;
  return s;
}

/* Boundary fraction s of Sec. 2 (Fig. 2): x* = x - s h e_i is the wall point between
 * the node and its outside neighbour closest to the node.  dir in 0..5 = -x,+x,-y,+y,-z,+z. */
static double boundary_fraction(const orc_op *op, int i, int j, int k, int dir) {
  double x = node_coord(op->ox, i, op->hx);
  double y = node_coord(op->oy, j, op->hy);
  double z = node_coord(op->oz, k, op->hz);
  double sg = taper_sigma(op, z);
  if (dir == 0 || dir == 1) {
    double v = (y - op->cy) / (op->b * sg);
    double w = (op->a * sg) * sqrt(1.0 - v * v);
    double s = (dir == 0) ? (x - (op->cx - w)) / op->hx : ((op->cx + w) - x) / op->hx;
    return clamp_frac(s);
  }
  if (dir == 2 || dir == 3) {
    double u = (x - op->cx) / (op->a * sg);
    double w = (op->b * sg) * sqrt(1.0 - u * u);
    double s = (dir == 2) ? (y - (op->cy - w)) / op->hy : ((op->cy + w) - y) / op->hy;
    return clamp_frac(s);
  }
  /* z: the wall crosses a z-line only for a taper, where sigma(z*) = q. */
  if (op->taper == 1.0 || op->nz < 2) return 1.0;
  double u0 = (x - op->cx) / op->a;
  double v0 = (y - op->cy) / op->b;
  double q = sqrt(u0 * u0 + v0 * v0);
  double tstar = (q - 1.0) / (op->taper - 1.0);
  double zstar = zlo(op) + tstar * (zhi(op) - zlo(op));
  if (dir == 4) {
    if (zstar < z) return clamp_frac((z - zstar) / op->hz);
    return 1.0; /* neighbour is outside because of an end plane, at distance h */
  }
  if (zstar > z) return clamp_frac((zstar - z) / op->hz);
  return 1.0;
}

/* One coordinate direction of one row: contribution dd to the diagonal and the
 * couplings to the minus / plus neighbours (0 when that neighbour is not an unknown).
 * Sec. 2: substitute the extrapolated value of the outside neighbour into the
 * difference star Eq. (6), with g = 0:
 *   constant  Eq. (7):  u(x') := 0
 *   linear    Eq. (8):  u(x') := (1 - 1/s) u(x)
 *   quadratic Eq. (9):  u(x') := 2(s-1)/s u(x) - (s-1)/(s+1) u(x'')
 *             Eq. (10): both neighbours outside, fractions s and t.
 * The algebra of each substitution is written next to its case. */
static void direction_row(int mode, double c, int in_m, int in_p, double s, double t,
                          double *dd, double *om, double *opp) {
  *om = 0.0;
  *opp = 0.0;
  if (in_m && in_p) { /* interior direction, Eq. (6) */
    *dd = 2.0 * c;
    *om = -c;
    *opp = -c;
    return;
  }
  if (!in_m && !in_p) {
    if (mode == ORC_CONSTANT) {
      *dd = 2.0 * c; /* 2u - 0 - 0 */
    } else if (mode == ORC_LINEAR) {
      /* READING: Eq. (8) on each side: 2u - (1-1/s)u - (1-1/t)u = (1/s + 1/t) u */
      *dd = (1.0 / s + 1.0 / t) * c;
    } else {
      /* Eq. (10): 2u - [(s-1)(t+1) + (s+1)(t-1)]/(st) u = 2/(st) u */
      *dd = (2.0 / (s * t)) * c;
    }
    return;
  }
  /* one side outside with fraction f, the other (inside) neighbour gets the coupling */
  double f = in_m ? t : s;
  double dgl, off;
  if (mode == ORC_CONSTANT) {
    dgl = 2.0 * c; /* 2u - 0 - u'' */
    off = -c;
  } else if (mode == ORC_LINEAR) {
    dgl = (1.0 + 1.0 / f) * c; /* 2u - (1-1/f)u - u'' */
    off = -c;
  } else {
    /* Eq. (9): 2u - 2(f-1)/f u + (f-1)/(f+1) u'' - u'' = (2/f) u - 2/(f+1) u'' */
    dgl = (2.0 / f) * c;
    off = -(2.0 / (f + 1.0)) * c;
  }
  *dd = dgl;
  if (in_m) *om = off;
  else *opp = off;
}

orc_op *orc_build_operator(int nx, int ny, int nz, double hx, double hy, double hz,
                           double ox, double oy, double oz, double a, double b,
                           double taper, double cx, double cy, int zbc,
                           int symmetrize_gamma2, int mode) {
  if (nx < 1 || ny < 1 || nz < 2 || !(hx > 0) || !(hy > 0) || !(hz > 0) || !(a > 0) ||
      !(b > 0) || !(taper > 0) || mode < 0 || mode > 2 || zbc < 0 || zbc > 1)
    return NULL;
  if (zbc == ORC_Z_DIRICHLET && nz < 3) return NULL;
  orc_op *op = (orc_op *)calloc(1, sizeof(orc_op));
  op->nx = nx; op->ny = ny; op->nz = nz;
  op->hx = hx; op->hy = hy; op->hz = hz;
  op->ox = ox; op->oy = oy; op->oz = oz;
  op->a = a; op->b = b; op->taper = taper; op->cx = cx; op->cy = cy;
  op->zbc = zbc; op->symmetrize = symmetrize_gamma2; op->mode = mode;

  long nbox = (long)nx * ny * nz;
  op->row_of_node = (int *)malloc((size_t)nbox * sizeof(int));
  /* inside test of every node, then rows numbered in ascending box index */
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i)
        op->row_of_node[box_index(op, i, j, k)] = orc_node_inside(op, i, j, k) ? 0 : -1;
  int n = 0;
  for (long q = 0; q < nbox; ++q)
    if (op->row_of_node[q] >= 0) op->row_of_node[q] = n++;
  op->n = n;
  op->node_of_row = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
  for (long q = 0; q < nbox; ++q)
    if (op->row_of_node[q] >= 0) op->node_of_row[op->row_of_node[q]] = (int)q;

  op->scale = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  op->bfac = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  op->frac = (double *)malloc((size_t)(n > 0 ? 6 * n : 1) * sizeof(double));
  csr_alloc(&op->A, n, n, 7L * n);

  const double cdir[3] = {1.0 / (hx * hx), 1.0 / (hy * hy), 1.0 / (hz * hz)};
  /* Robin distance d: half the extent of Omega in z (Sec. 2, after Eq. (5)). */
  const double dist = 0.5 * ((double)(nz - 1) * hz);
  /* row r takes the diagonal and one entry per neighbour that is an unknown */
#pragma omp parallel for schedule(static)
  for (int r = 0; r < n; ++r) {
    int q = op->node_of_row[r];
    int i = q % nx, j = (q / nx) % ny, k = q / (nx * ny);
    op->A.rowptr[r + 1] = 1 + is_unknown(op, i - 1, j, k) + is_unknown(op, i + 1, j, k) +
                          is_unknown(op, i, j - 1, k) + is_unknown(op, i, j + 1, k) +
                          is_unknown(op, i, j, k - 1) + is_unknown(op, i, j, k + 1);
  }
  op->A.rowptr[0] = 0;
  for (int r = 0; r < n; ++r) op->A.rowptr[r + 1] += op->A.rowptr[r];
#pragma omp parallel for schedule(static)
  for (int r = 0; r < n; ++r) {
    long p = op->A.rowptr[r];
    int q = op->node_of_row[r];
    int i = q % nx, j = (q / nx) % ny, k = q / (nx * ny);
    int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k},
                    {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
    double off[6] = {0, 0, 0, 0, 0, 0};
    double dd[3];
    int gamma2 = (zbc == ORC_Z_ROBIN) && (k == 0 || k == nz - 1);
    for (int dir = 0; dir < 6; ++dir) op->frac[6 * r + dir] = -1.0;
    for (int ax = 0; ax < 3; ++ax) {
      int dm = 2 * ax, dp = 2 * ax + 1;
      int in_m = is_unknown(op, nb[dm][0], nb[dm][1], nb[dm][2]);
      int in_p = is_unknown(op, nb[dp][0], nb[dp][1], nb[dp][2]);
      if (ax == 2 && gamma2) {
        /* Robin end plane, Eq. (11): u(x') = u(x'') - (2h/d) u(x) for the virtual
         * point x' beyond the plane; substituted into Eq. (6):
         *   2u - u(x'') + (2h/d)u - u(x'') = (2 + 2h/d) u - 2 u(x''). */
        int inner_is_p = (k == 0);
        int in_inner = inner_is_p ? in_p : in_m;
        double c = cdir[2];
        if (in_inner) {
          dd[2] = (2.0 + (2.0 * hz) / dist) * c;
          if (inner_is_p) off[dp] = -2.0 * c;
          else off[dm] = -2.0 * c;
        } else {
          /* READING: the inner neighbour x'' is itself outside the wall (only possible
           * with a taper).  It is replaced by the one-sided extrapolation of its side
           * (constant: 0; linear and quadratic: (1 - 1/t) u(x), the quadratic rule
           * needing the virtual point), then Eq. (11) gives
           *   2u - 2u(x'') + (2h/d) u. */
          int dinner = inner_is_p ? dp : dm;
          double t = boundary_fraction(op, i, j, k, dinner);
          op->frac[6 * r + dinner] = t;
          if (op->mode == ORC_CONSTANT) dd[2] = (2.0 + (2.0 * hz) / dist) * c;
          else dd[2] = ((2.0 * hz) / dist + 2.0 / t) * c;
        }
        continue;
      }
      double s = 1.0, t = 1.0;
      if (!in_m) {
        s = boundary_fraction(op, i, j, k, dm);
        op->frac[6 * r + dm] = s;
      }
      if (!in_p) {
        t = boundary_fraction(op, i, j, k, dp);
        op->frac[6 * r + dp] = t;
      }
      direction_row(mode, cdir[ax], in_m, in_p, s, t, &dd[ax], &off[dm], &off[dp]);
    }
    /* Sec. 2: "must be applied to all of them" -- the directions add up. */
    double diag = (dd[0] + dd[1]) + dd[2];
    double bf = 1.0;
    if (gamma2 && op->symmetrize) {
      /* READING: the Robin rows are halved (row and right-hand side) so that the
       * constant and linear matrices are symmetric, as Sec. 2 states they are. */
      diag *= 0.5;
      for (int d6 = 0; d6 < 6; ++d6) off[d6] *= 0.5;
      bf = 0.5;
    }
    op->bfac[r] = bf;
    /* CSR row in ascending column order: -z, -y, -x, self, +x, +y, +z */
    const int order[7] = {4, 2, 0, -1, 1, 3, 5};
    for (int o = 0; o < 7; ++o) {
      int d6 = order[o];
      if (d6 < 0) {
        op->A.col[p] = r;
        op->A.val[p] = diag;
        ++p;
        continue;
      }
      if (!is_unknown(op, nb[d6][0], nb[d6][1], nb[d6][2])) continue;
      op->A.col[p] = op->row_of_node[box_index(op, nb[d6][0], nb[d6][1], nb[d6][2])];
      op->A.val[p] = off[d6];
      ++p;
    }
    op->scale[r] = 1.0 / sqrt(diag);
  }
  long p = op->A.rowptr[n];
  op->A.nnz = p;

  /* Symmetric diagonal scaling (Sec. 2, last paragraph): ahat_ij = a_ij (s_i s_j). */
  csr_alloc(&op->Ahat, n, n, p);
  memcpy(op->Ahat.rowptr, op->A.rowptr, (size_t)(n + 1) * sizeof(int));
  memcpy(op->Ahat.col, op->A.col, (size_t)(p > 0 ? p : 1) * sizeof(int));
#pragma omp parallel for schedule(static)
  for (int r = 0; r < n; ++r)
    for (int e = op->A.rowptr[r]; e < op->A.rowptr[r + 1]; ++e)
      op->Ahat.val[e] = op->A.val[e] * (op->scale[r] * op->scale[op->A.col[e]]);
  return op;
}

void orc_op_free(orc_op *op) {
  if (!op) return;
  free(op->node_of_row);
  free(op->row_of_node);
  free(op->scale);
  free(op->bfac);
  free(op->frac);
  csr_free(&op->A);
  csr_free(&op->Ahat);
  free(op);
}

int orc_op_n(const orc_op *op) { return op->n; }
long orc_op_nnz(const orc_op *op) { return op->A.nnz; }

void orc_op_get(const orc_op *op, int *node_of_row, double *scale, double *bfac,
                int *rowptr, int *col, double *aval, double *ahat) {
  int n = op->n;
  long nnz = op->A.nnz;
  if (node_of_row) memcpy(node_of_row, op->node_of_row, (size_t)n * sizeof(int));
  if (scale) memcpy(scale, op->scale, (size_t)n * sizeof(double));
  if (bfac) memcpy(bfac, op->bfac, (size_t)n * sizeof(double));
  if (rowptr) memcpy(rowptr, op->A.rowptr, (size_t)(n + 1) * sizeof(int));
  if (col) memcpy(col, op->A.col, (size_t)nnz * sizeof(int));
  if (aval) memcpy(aval, op->A.val, (size_t)nnz * sizeof(double));
  if (ahat) memcpy(ahat, op->Ahat.val, (size_t)nnz * sizeof(double));
}

void orc_op_fractions(const orc_op *op, double *frac) {
  memcpy(frac, op->frac, (size_t)op->n * 6 * sizeof(double));
}

/* ------------------------------------------------------------------------- */
/* Around the solve in the PIC step: CIC deposition, E = -grad phi, CIC gather */
/* ------------------------------------------------------------------------- */
/* Cloud-in-cell weights of one coordinate: cell index c = floor((x - o) / h) and the
 * weights (1 - f, f) of the nodes c and c + 1, f = (x - o) / h - c. */
static void cic_axis(double x, double o, double h, long *c, double *f) {
  double u = (x - o) / h;
  double fl = floor(u);
  *c = (long)fl;
  *f = u - fl;
}

/* Sec. 4.1 (the charge density comes from the particles by cloud-in-cell area weighting):
 * rho(node) = sum_p q_p W(x_p - x_node) / (hx hy hz), W the product of the three 1-D hat
 * weights.  Each particle adds ((q / V) wx) wy) wz to its 8 surrounding nodes, in particle
 * order, z-slab, y-row, x-node (c, b, a = 0, 1); nodes outside the box are dropped. */
void orc_deposit_cic(int nx, int ny, int nz, double hx, double hy, double hz, double ox,
                     double oy, double oz, int np, const double *x, const double *y,
                     const double *z, const double *q, double *rho) {
  const double vol = (hx * hy) * hz;
  for (long v = 0; v < (long)nx * ny * nz; ++v) rho[v] = 0.0;
  for (int p = 0; p < np; ++p) {
    long ci, cj, ck;
    double fx, fy, fz;
    cic_axis(x[p], ox, hx, &ci, &fx);
    cic_axis(y[p], oy, hy, &cj, &fy);
    cic_axis(z[p], oz, hz, &ck, &fz);
    const double qv = q[p] / vol;
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          long i = ci + a, j = cj + b, k = ck + c;
          if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) continue;
          double wx = a ? fx : 1.0 - fx, wy = b ? fy : 1.0 - fy, wz = c ? fz : 1.0 - fz;
          rho[i + nx * (j + (long)ny * k)] += ((qv * wx) * wy) * wz;
        }
  }
}

/* Derivative at a node from the node value p0 and its neighbours along one axis, at
 * distances h (inside) or s h (wall point, value 0, s = boundary fraction): the derivative
 * of the quadratic through the three points.  in_m / in_p: neighbour is an unknown. */
static double axis_derivative(double h, int in_m, int in_p, double pm, double p0, double pp,
                              double t, double s) {
  if (in_m && in_p) return (pp - pm) / (2.0 * h);
  if (in_m) /* wall at +s h */
    return (-(s * s) * pm + (s * s - 1.0) * p0) / (h * s * (1.0 + s));
  if (in_p) /* wall at -t h */
    return ((t * t) * pp - (t * t - 1.0) * p0) / (h * t * (1.0 + t));
  return p0 * (s - t) / (h * s * t); /* walls at -t h and +s h */
}

/* E = -grad phi (the self field of the beam, Sec. 1) at the unknowns, 0 elsewhere.
 * READING: second-order differences that use the wall value phi = 0 at the boundary
 * fraction of Sec. 2 (the same clamped s as the operator); on a Robin end plane the
 * z-derivative is the one the Robin condition prescribes (outward normal derivative
 * = -phi / d with d = (nz - 1) hz / 2). */
void orc_field_gradient(const orc_op *op, const double *phi, double *ex, double *ey,
                        double *ez) {
  const int nx = op->nx, ny = op->ny, nz = op->nz;
  const double dist = 0.5 * ((double)(nz - 1) * op->hz);
  const double h[3] = {op->hx, op->hy, op->hz};
  double *E[3] = {ex, ey, ez};
  for (long v = 0; v < (long)nx * ny * nz; ++v) ex[v] = ey[v] = ez[v] = 0.0;
  for (int r = 0; r < op->n; ++r) {
    long q = op->node_of_row[r];
    int i = (int)(q % nx), j = (int)((q / nx) % ny), k = (int)(q / ((long)nx * ny));
    int nb[6][3] = {{i - 1, j, k}, {i + 1, j, k}, {i, j - 1, k},
                    {i, j + 1, k}, {i, j, k - 1}, {i, j, k + 1}};
    const double p0 = phi[q];
    for (int ax = 0; ax < 3; ++ax) {
      int dm = 2 * ax, dp = 2 * ax + 1;
      double d;
      if (ax == 2 && op->zbc == ORC_Z_ROBIN && (k == 0 || k == nz - 1)) {
        d = (k == 0 ? 1.0 : -1.0) * p0 / dist;
      } else {
        int in_m = is_unknown(op, nb[dm][0], nb[dm][1], nb[dm][2]);
        int in_p = is_unknown(op, nb[dp][0], nb[dp][1], nb[dp][2]);
        double pm = in_m ? phi[nb[dm][0] + nx * (nb[dm][1] + (long)ny * nb[dm][2])] : 0.0;
        double pp = in_p ? phi[nb[dp][0] + nx * (nb[dp][1] + (long)ny * nb[dp][2])] : 0.0;
        double t = in_m ? 1.0 : boundary_fraction(op, i, j, k, dm);
        double s = in_p ? 1.0 : boundary_fraction(op, i, j, k, dp);
        d = axis_derivative(h[ax], in_m, in_p, pm, p0, pp, t, s);
      }
      E[ax][q] = -d;
    }
  }
}

/* The field at the particles with the deposition's weights (momentum-conserving pair of
 * the CIC scheme): E_p = sum over the 8 nodes of ((wx wy) wz) E(node), in the deposition's
 * node order; nodes outside the box contribute nothing. */
void orc_gather_cic(int nx, int ny, int nz, double hx, double hy, double hz, double ox,
                    double oy, double oz, const double *ex, const double *ey, const double *ez,
                    int np, const double *x, const double *y, const double *z, double *epx,
                    double *epy, double *epz) {
  for (int p = 0; p < np; ++p) {
    long ci, cj, ck;
    double fx, fy, fz;
    cic_axis(x[p], ox, hx, &ci, &fx);
    cic_axis(y[p], oy, hy, &cj, &fy);
    cic_axis(z[p], oz, hz, &ck, &fz);
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          long i = ci + a, j = cj + b, k = ck + c;
          if (i < 0 || j < 0 || k < 0 || i >= nx || j >= ny || k >= nz) continue;
          double w = ((a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy)) * (c ? fz : 1.0 - fz);
          long v = i + nx * (j + (long)ny * k);
          sx += w * ex[v];
          sy += w * ey[v];
          sz += w * ez[v];
        }
    epx[p] = sx;
    epy[p] = sy;
    epz[p] = sz;
  }
}

/* ------------------------------------------------------------------------- */
/* Hashed priorities                                                          */
/* ------------------------------------------------------------------------- */
/* MurmurHash3 32-bit finaliser (Appleby, public domain): xor-shift 16, multiply by
 * 0x85ebca6b, xor-shift 13, multiply by 0xc2b2ae35, xor-shift 16.  A bijection of
 * 32-bit words, used as a reproducible pseudo-random priority. */
unsigned int orc_fmix32(unsigned int h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

/* Strict total order of nodes: hash in the high word, id in the low word. */
static uint64_t node_key(unsigned int id, unsigned int seed) {
  return ((uint64_t)orc_fmix32(id ^ seed) << 32) | (uint64_t)id;
}

/* ------------------------------------------------------------------------- */
/* Aggregation (Sec. 3.2, "Prolongation operator")                           */
/* ------------------------------------------------------------------------- */
typedef struct {
  uint64_t key;
  int row;
} keyrow_t;

static int cmp_key_desc(const void *pa, const void *pb) {
  uint64_t a = ((const keyrow_t *)pa)->key, b = ((const keyrow_t *)pb)->key;
  return (a < b) - (a > b);
}

/* Nodes by decreasing key.  The keys are distinct, so every correct sort gives the same
 * order; the multi-threaded baseline build sorts static chunks in parallel and merges them
 * pairwise. */
static void sort_keys_desc(keyrow_t *a, int n) {
#ifdef _OPENMP
  int T = omp_get_max_threads();
  if (T > 64) T = 64;
  if (T > 1 && n >= 65536) {
    long b[65];
    for (int t = 0; t <= T; ++t) b[t] = (long)n * t / T;
#pragma omp parallel for num_threads(T) schedule(static, 1)
    for (int t = 0; t < T; ++t) qsort(a + b[t], (size_t)(b[t + 1] - b[t]), sizeof(keyrow_t), cmp_key_desc);
    keyrow_t *src = a, *dst = (keyrow_t *)malloc((size_t)n * sizeof(keyrow_t));
    for (int w = 1; w < T; w *= 2) {
#pragma omp parallel for schedule(static, 1)
      for (int t = 0; t < T; t += 2 * w) {
        long lo = b[t], mid = b[t + w < T ? t + w : T], hi = b[t + 2 * w < T ? t + 2 * w : T];
        long i = lo, j = mid, o = lo;
        while (i < mid && j < hi) dst[o++] = src[i].key > src[j].key ? src[i++] : src[j++];
        while (i < mid) dst[o++] = src[i++];
        while (j < hi) dst[o++] = src[j++];
      }
      keyrow_t *tmp = src;
      src = dst;
      dst = tmp;
    }
    if (src != a) {
      memcpy(a, src, (size_t)n * sizeof(keyrow_t));
      free(src);
    } else {
      free(dst);
    }
    return;
  }
#endif
  qsort(a, (size_t)n, sizeof(keyrow_t), cmp_key_desc);
}

/* READING: the paper aggregates with per-processor 3^d cubes ("uncoupled", Sec. 3.2,
 * Table 1).  Here aggregates are seeded by a distance-2 maximal independent set of
 * the adjacency graph G_l of A_l (the graph named in Sec. 3.2), computed by the
 * sequential greedy rule: visit nodes by decreasing key; a node joins the set when
 * no node within graph distance 2 has joined. */
void orc_mis2(int n, const int *rowptr, const int *col, const unsigned int *ids,
              unsigned int seed, unsigned char *is_root) {
  keyrow_t *order = (keyrow_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(keyrow_t));
  unsigned char *blocked = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
  for (int i = 0; i < n; ++i) {
    order[i].key = node_key(ids[i], seed);
    order[i].row = i;
    is_root[i] = 0;
  }
  sort_keys_desc(order, n);
  for (int o = 0; o < n; ++o) {
    int v = order[o].row;
    if (blocked[v]) continue;
    is_root[v] = 1;
    blocked[v] = 1;
    for (int p = rowptr[v]; p < rowptr[v + 1]; ++p) {
      int u = col[p];
      blocked[u] = 1;
      for (int q = rowptr[u]; q < rowptr[u + 1]; ++q) blocked[col[q]] = 1;
    }
  }
  free(order);
  free(blocked);
}

/* Aggregates from the roots.  Phase 1: a root and its neighbours (disjoint, since
 * roots are at distance >= 3).  Phase 2: every other node joins the phase-1
 * aggregate of an adjacent phase-1 node, taking the root with the largest key.
 * Aggregates are numbered by ascending root row.  Returns the number of aggregates,
 * or -1 if a node could not be placed (impossible for a maximal set). */
int orc_aggregate(int n, const int *rowptr, const int *col, const unsigned int *ids,
                  unsigned int seed, const unsigned char *is_root, int *agg) {
  int *root1 = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
  int *rank = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
  int nagg = 0, bad = 0;
  for (int i = 0; i < n; ++i) root1[i] = -1;
  for (int r = 0; r < n; ++r) {
    rank[r] = -1;
    if (!is_root[r]) continue;
    rank[r] = nagg++;
    root1[r] = r;
    for (int p = rowptr[r]; p < rowptr[r + 1]; ++p) root1[col[p]] = r;
  }
  for (int i = 0; i < n; ++i) {
    int root = root1[i];
    if (root < 0) {
      uint64_t best = 0;
      for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int r = root1[col[p]];
        if (r < 0) continue;
        uint64_t kr = node_key(ids[r], seed);
        if (root < 0 || kr > best) {
          root = r;
          best = kr;
        }
      }
    }
    if (root < 0) {
      bad = 1;
      agg[i] = -1;
    } else {
      agg[i] = rank[root];
    }
  }
  free(root1);
  free(rank);
  return bad ? -1 : nagg;
}

/* ------------------------------------------------------------------------- */
/* Spectral bound (Sec. 3.2, "Smoothing operator": bounds for the spectrum)   */
/* ------------------------------------------------------------------------- */
/* READING: lambda_max(D^-1 A) estimated by `iters` power-iteration steps from the
 * start vector v_i = 0.5 + fmix32(id_i ^ 0xA5A5A5A5) / 2^32:
 *   v <- D^-1 A v / ||D^-1 A v||_2  (iters times);  lambda = ||D^-1 A v||_2. */
double orc_power_lambda(int n, const int *rowptr, const int *col, const double *val,
                        const unsigned int *ids, int iters) {
  if (n == 0) return 1.0;
  double *v = (double *)malloc((size_t)n * sizeof(double));
  double *w = (double *)malloc((size_t)n * sizeof(double));
  double *invd = (double *)malloc((size_t)n * sizeof(double));
  for (int i = 0; i < n; ++i) {
    v[i] = 0.5 + (double)orc_fmix32(ids[i] ^ 0xA5A5A5A5u) / 4294967296.0;
    double d = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
      if (col[p] == i) d = val[p];
    invd[i] = 1.0 / d;
  }
  double lam = 0.0;
  for (int it = 0; it <= iters; ++it) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) acc += val[p] * v[col[p]];
      w[i] = invd[i] * acc;
    }
    double nrm = sqrt(dot(n, w, w));
    lam = nrm;
    if (it == iters) break;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) v[i] = w[i] / nrm;
  }
  free(v);
  free(w);
  free(invd);
  return lam;
}

/* ------------------------------------------------------------------------- */
/* Chebyshev smoother (Sec. 3.2, "Smoothing operator")                       */
/* ------------------------------------------------------------------------- */
/* READING: Chebyshev acceleration (Saad, Iterative Methods for Sparse Linear Systems,
 * Alg. 12.1) applied to D^-1 A on the interval [lambda_hi / ratio, lambda_hi] with
 * lambda_hi = safety * lambda_hat.  `degree` steps; each step recomputes r = b - A x.
 *   theta = (hi + lo)/2, delta = (hi - lo)/2, sigma = theta/delta, rho_0 = 1/sigma
 *   step 0:  d = (D^-1 r) / theta;                                  x += d
 *   step k:  rho_k = 1/(2 sigma - rho_{k-1});
 *            d = rho_k rho_{k-1} d + (2 rho_k / delta) D^-1 r;       x += d */
void orc_cheb_smooth(int n, const int *rowptr, const int *col, const double *val,
                     const double *invd, double lambda_hat, double ratio, double safety,
                     int degree, const double *b, double *x, int x_is_zero) {
  double hi = safety * lambda_hat, lo = hi / ratio;
  double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo);
  double sigma = theta / delta;
  double rho_prev = 1.0 / sigma;
  double *r = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  double *d = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  csr_t a = {n, n, rowptr[n], (int *)rowptr, (int *)col, (double *)val};
  for (int step = 0; step < degree; ++step) {
    if (step == 0 && x_is_zero) {
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) r[i] = b[i];
    } else {
      csr_spmv(&a, x, r);
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
    }
    if (step == 0) {
      double c2 = 1.0 / theta;
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) d[i] = c2 * (invd[i] * r[i]);
    } else {
      double rho = 1.0 / (2.0 * sigma - rho_prev);
      double c1 = rho * rho_prev, c2 = (2.0 * rho) / delta;
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) d[i] = c1 * d[i] + c2 * (invd[i] * r[i]);
      rho_prev = rho;
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) x[i] = x[i] + d[i];
  }
  free(r);
  free(d);
}

/* ------------------------------------------------------------------------- */
/* Dense LU with partial pivoting (Sec. 3.2, "Coarse level solver")           */
/* ------------------------------------------------------------------------- */
typedef struct {
  int n;
  double *lu; /* row-major, L unit lower (below diagonal), U upper */
  int *perm;  /* row k of LU is row perm[k] of the original matrix */
} dense_lu_t;

/* READING: the paper factors the coarsest matrix with KLU; a dense LU with partial
 * pivoting (pivot = largest |a_ik|, lowest row on ties) gives the same solution to
 * rounding. Returns 0, or -1 on a zero pivot. */
static int dense_lu_factor(dense_lu_t *f, int n, const double *a) {
  f->n = n;
  f->lu = (double *)malloc((size_t)(n > 0 ? n : 1) * (size_t)(n > 0 ? n : 1) * sizeof(double));
  f->perm = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
  memcpy(f->lu, a, (size_t)n * n * sizeof(double));
  for (int i = 0; i < n; ++i) f->perm[i] = i;
  double *m = f->lu;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(m[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      double v = fabs(m[(size_t)i * n + k]);
      if (v > best) {
        best = v;
        p = i;
      }
    }
    if (best == 0.0) return -1;
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        double tmp = m[(size_t)k * n + j];
        m[(size_t)k * n + j] = m[(size_t)p * n + j];
        m[(size_t)p * n + j] = tmp;
      }
      int tp = f->perm[k];
      f->perm[k] = f->perm[p];
      f->perm[p] = tp;
    }
    double piv = m[(size_t)k * n + k];
#pragma omp parallel for schedule(static) if (n - k > 256)
    for (int i = k + 1; i < n; ++i) {
      double l = m[(size_t)i * n + k] / piv;
      m[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; ++j) m[(size_t)i * n + j] -= l * m[(size_t)k * n + j];
    }
  }
  return 0;
}

static void dense_lu_solve(const dense_lu_t *f, const double *b, double *x) {
  int n = f->n;
  const double *m = f->lu;
  for (int i = 0; i < n; ++i) {
    double acc = b[f->perm[i]];
    for (int j = 0; j < i; ++j) acc -= m[(size_t)i * n + j] * x[j];
    x[i] = acc;
  }
  for (int i = n - 1; i >= 0; --i) {
    double acc = x[i];
    for (int j = i + 1; j < n; ++j) acc -= m[(size_t)i * n + j] * x[j];
    x[i] = acc / m[(size_t)i * n + i];
  }
}

static void dense_lu_free(dense_lu_t *f) {
  free(f->lu);
  free(f->perm);
}

int orc_dense_lu_solve(int n, const double *a, const double *b, double *x) {
  dense_lu_t f;
  int rc = dense_lu_factor(&f, n, a);
  if (rc == 0) dense_lu_solve(&f, b, x);
  dense_lu_free(&f);
  return rc;
}

/* ------------------------------------------------------------------------- */
/* Sparse products for the Galerkin operator                                  */
/* ------------------------------------------------------------------------- */
static int cmp_int(const void *pa, const void *pb) {
  int a = *(const int *)pa, b = *(const int *)pb;
  return (a > b) - (a < b);
}

/* C = X Y, row by row (Gustavson).  Each entry is summed in the order the products
 * arise: X's row in column order, then Y's row in column order.  The pattern is
 * structural (an entry whose value cancels to zero is kept).  A first pass counts each
 * row's distinct columns, a second one forms the rows in place. */
static void csr_matmul(const csr_t *x, const csr_t *y, csr_t *c) {
  int n = x->n, m = y->m;
  int *rowptr = (int *)calloc((size_t)n + 1, sizeof(int));
#pragma omp parallel
  {
    int *mark = (int *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int));
    for (int j = 0; j < m; ++j) mark[j] = -1;
#pragma omp for schedule(static)
    for (int i = 0; i < n; ++i) {
      int cnt = 0;
      for (int p = x->rowptr[i]; p < x->rowptr[i + 1]; ++p) {
        int k = x->col[p];
        for (int q = y->rowptr[k]; q < y->rowptr[k + 1]; ++q) {
          int j = y->col[q];
          if (mark[j] != i) {
            mark[j] = i;
            ++cnt;
          }
        }
      }
      rowptr[i + 1] = cnt;
    }
    free(mark);
  }
  for (int i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
  long nnz = rowptr[n];
  int *ccol = (int *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int));
  double *cval = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
#pragma omp parallel
  {
    int *mark = (int *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int));
    double *acc = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    int *cols = (int *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int));
    for (int j = 0; j < m; ++j) mark[j] = -1;
#pragma omp for schedule(static)
    for (int i = 0; i < n; ++i) {
      int cnt = 0;
      for (int p = x->rowptr[i]; p < x->rowptr[i + 1]; ++p) {
        int k = x->col[p];
        double xv = x->val[p];
        for (int q = y->rowptr[k]; q < y->rowptr[k + 1]; ++q) {
          int j = y->col[q];
          if (mark[j] != i) {
            mark[j] = i;
            acc[j] = 0.0;
            cols[cnt++] = j;
          }
          acc[j] += xv * y->val[q];
        }
      }
      qsort(cols, (size_t)cnt, sizeof(int), cmp_int);
      long o = rowptr[i];
      for (int t = 0; t < cnt; ++t) {
        ccol[o + t] = cols[t];
        cval[o + t] = acc[cols[t]];
      }
    }
    free(mark);
    free(acc);
    free(cols);
  }
  c->n = n;
  c->m = m;
  c->nnz = nnz;
  c->rowptr = rowptr;
  c->col = ccol;
  c->val = cval;
}

/* Explicit transpose; each row of the result lists its columns in ascending order. */
static void csr_transpose(const csr_t *a, csr_t *t) {
  csr_alloc(t, a->m, a->n, a->nnz);
  for (long p = 0; p < a->nnz; ++p) t->rowptr[a->col[p] + 1]++;
  for (int j = 0; j < a->m; ++j) t->rowptr[j + 1] += t->rowptr[j];
  int *fill = (int *)malloc((size_t)(a->m > 0 ? a->m : 1) * sizeof(int));
  for (int j = 0; j < a->m; ++j) fill[j] = t->rowptr[j];
  for (int i = 0; i < a->n; ++i)
    for (int p = a->rowptr[i]; p < a->rowptr[i + 1]; ++p) {
      int q = fill[a->col[p]]++;
      t->col[q] = i;
      t->val[q] = a->val[p];
    }
  free(fill);
}

/* ------------------------------------------------------------------------- */
/* Cube ("decoupled") aggregation (Sec. 3.2)                                  */
/* ------------------------------------------------------------------------- */
/* The paper's own coarsening: aggregates are cubes of 3 x 3 x 3 lattice nodes, fewer where
 * the cube meets the domain boundary.  Node v carries the lattice id i + d0 (j + d1 k) of a
 * d0 x d1 x d2 lattice; its cube is (i/3, j/3, k/3) on the lattice of ceil(d/3) cubes per
 * axis.  Every cube that holds a node is one aggregate; aggregates are numbered by
 * ascending cube index, and the cube index is the coarse node's lattice id.
 * READING: a cube's nodes form one aggregate even when the domain boundary cuts the cube
 * into pieces that are not connected inside it.  The root of an aggregate (reported for
 * inspection only) is its member with the smallest row.  Returns the number of aggregates. */
int orc_cube_aggregate(int n, const unsigned int *ids, const int dims[3], int *agg,
                       unsigned char *is_root, unsigned int *next_ids, int next_dims[3]) {
  long c0 = (dims[0] + 2) / 3, c1 = (dims[1] + 2) / 3, c2 = (dims[2] + 2) / 3;
  long ncubes = c0 * c1 * c2;
  if (next_dims) {
    next_dims[0] = (int)c0;
    next_dims[1] = (int)c1;
    next_dims[2] = (int)c2;
  }
  long *cube = (long *)malloc((size_t)(n > 0 ? n : 1) * sizeof(long));
  int *rank = (int *)malloc((size_t)(ncubes > 0 ? ncubes : 1) * sizeof(int));
  for (long c = 0; c < ncubes; ++c) rank[c] = -1;
  for (int v = 0; v < n; ++v) {
    long id = (long)ids[v];
    long i = id % dims[0], j = (id / dims[0]) % dims[1], k = id / ((long)dims[0] * dims[1]);
    cube[v] = i / 3 + c0 * (j / 3 + c1 * (k / 3));
    rank[cube[v]] = 0; /* used */
  }
  int nagg = 0;
  for (long c = 0; c < ncubes; ++c)
    if (rank[c] == 0) {
      if (next_ids) next_ids[nagg] = (unsigned int)c;
      rank[c] = nagg++;
    }
  for (int v = 0; v < n; ++v) agg[v] = rank[cube[v]];
  if (is_root) {
    int *first = (int *)malloc((size_t)(nagg > 0 ? nagg : 1) * sizeof(int));
    for (int a = 0; a < nagg; ++a) first[a] = -1;
    for (int v = 0; v < n; ++v)
      if (first[agg[v]] < 0) first[agg[v]] = v;
    for (int v = 0; v < n; ++v) is_root[v] = (unsigned char)(first[agg[v]] == v);
    free(first);
  }
  free(cube);
  free(rank);
  return nagg;
}

/* ------------------------------------------------------------------------- */
/* Gauss-Seidel coarse solver (Sec. 3.2, "Coarse level solver")               */
/* ------------------------------------------------------------------------- */
/* READING: the paper applies three Gauss-Seidel steps on the coarsest level.  A step here is
 * a symmetric sweep (forward, then backward) in a multicolour order, from x = 0, which keeps
 * the V-cycle a symmetric operator for CG.  The colouring is the sequence of synchronous
 * rounds: in round c every uncoloured node whose key exceeds the keys of all its uncoloured
 * neighbours takes colour c; key(v) = (fmix32(id_v ^ seed), id_v), seed = 0x2545F491.  Rows
 * of one colour are never adjacent, so their updates within a sweep are independent. */
int orc_colour(int n, const int *rowptr, const int *col, const unsigned int *ids,
               unsigned int seed, int *colour) {
  for (int i = 0; i < n; ++i) colour[i] = -1;
  int left = n, c = 0;
  unsigned char *pick = (unsigned char *)malloc((size_t)(n > 0 ? n : 1));
  while (left > 0) {
    for (int i = 0; i < n; ++i) {
      pick[i] = 0;
      if (colour[i] >= 0) continue;
      uint64_t ki = ((uint64_t)orc_fmix32(ids[i] ^ seed) << 32) | ids[i];
      int best = 1;
      for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
        int j = col[p];
        if (j == i || colour[j] >= 0) continue;
        uint64_t kj = ((uint64_t)orc_fmix32(ids[j] ^ seed) << 32) | ids[j];
        if (kj > ki) best = 0;
      }
      pick[i] = (unsigned char)best;
    }
    for (int i = 0; i < n; ++i)
      if (pick[i]) {
        colour[i] = c;
        --left;
      }
    ++c;
  }
  free(pick);
  return c;
}

/* `steps` symmetric Gauss-Seidel steps from x = 0: forward over colours 0..C-1, then
 * backward over C-1..0; x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii with the sum in the
 * row's column order, the division as a multiply by invd_i = 1 / a_ii. */
void orc_sgs(int n, const int *rowptr, const int *col, const double *val, const double *invd,
             const int *colour, int ncolours, int steps, const double *b, double *x) {
  for (int i = 0; i < n; ++i) x[i] = 0.0;
  for (int st = 0; st < steps; ++st)
    for (int half = 0; half < 2; ++half)
      for (int cc = 0; cc < ncolours; ++cc) {
        int c = half == 0 ? cc : ncolours - 1 - cc;
        for (int i = 0; i < n; ++i) {
          if (colour[i] != c) continue;
          double acc = b[i];
          for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
            if (col[p] != i) acc -= val[p] * x[col[p]];
          x[i] = acc * invd[i];
        }
      }
}

/* ------------------------------------------------------------------------- */
/* Hierarchy (Sec. 3.2)                                                       */
/* ------------------------------------------------------------------------- */
#define ORC_MAX_LEVELS 32
#define ORC_MAX_DENSE 16384

typedef struct {
  csr_t A;
  double *invd;
  unsigned int *ids;
  int dims[3]; /* lattice of the ids (cube aggregation) */
  int *agg;
  unsigned char *root;
  double lambda, omega;
  csr_t P, R;
} level_t;

struct orc_hier {
  const orc_op *op;
  int nlev;
  int status;
  int degree;
  double ratio, safety;
  level_t lev[ORC_MAX_LEVELS];
  dense_lu_t coarse;
  int coarse_solver, coarse_sweeps; /* ORC_COARSE_*; Gauss-Seidel steps */
  int *colour, ncolours;            /* colouring of the coarsest level (Gauss-Seidel) */
  double **wb, **wx, **wr; /* per-level work vectors */
};

static double *diag_inverse(const csr_t *a) {
  double *invd = (double *)malloc((size_t)(a->n > 0 ? a->n : 1) * sizeof(double));
#pragma omp parallel for schedule(static)
  for (int i = 0; i < a->n; ++i) {
    double d = 0.0;
    for (int p = a->rowptr[i]; p < a->rowptr[i + 1]; ++p)
      if (a->col[p] == i) d = a->val[p];
    invd[i] = 1.0 / d;
  }
  return invd;
}

static void csr_copy(const csr_t *src, csr_t *dst) {
  csr_alloc(dst, src->n, src->m, src->nnz);
  memcpy(dst->rowptr, src->rowptr, (size_t)(src->n + 1) * sizeof(int));
  memcpy(dst->col, src->col, (size_t)(src->nnz > 0 ? src->nnz : 1) * sizeof(int));
  memcpy(dst->val, src->val, (size_t)(src->nnz > 0 ? src->nnz : 1) * sizeof(double));
}

/* Smoothed prolongator P = (I - omega D^-1 A) T = T - omega D^-1 (A T), with
 * T(i, agg(i)) = 1 the tentative prolongator (Sec. 3.2) and omega = 4 / (3 lambda).
 * (A T)_iJ sums a_ij over the row in column order for all j with agg(j) = J.  A first
 * pass counts each row's distinct aggregates, a second one forms the rows in place. */
static void smoothed_prolongator(const csr_t *a, const double *invd, const int *agg,
                                 int nagg, double omega, csr_t *p) {
  int n = a->n;
  int *rowptr = (int *)calloc((size_t)n + 1, sizeof(int));
#pragma omp parallel
  {
    int *mark = (int *)malloc((size_t)(nagg > 0 ? nagg : 1) * sizeof(int));
    for (int J = 0; J < nagg; ++J) mark[J] = -1;
#pragma omp for schedule(static)
    for (int i = 0; i < n; ++i) {
      int cnt = 0;
      for (int q = a->rowptr[i]; q < a->rowptr[i + 1]; ++q) {
        int J = agg[a->col[q]];
        if (mark[J] != i) {
          mark[J] = i;
          ++cnt;
        }
      }
      rowptr[i + 1] = cnt;
    }
    free(mark);
  }
  for (int i = 0; i < n; ++i) rowptr[i + 1] += rowptr[i];
  long nnz = rowptr[n];
  int *pcol = (int *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int));
  double *pval = (double *)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(double));
#pragma omp parallel
  {
    int *mark = (int *)malloc((size_t)(nagg > 0 ? nagg : 1) * sizeof(int));
    double *acc = (double *)calloc((size_t)(nagg > 0 ? nagg : 1), sizeof(double));
    int *cols = (int *)malloc((size_t)(nagg > 0 ? nagg : 1) * sizeof(int));
    for (int J = 0; J < nagg; ++J) mark[J] = -1;
#pragma omp for schedule(static)
    for (int i = 0; i < n; ++i) {
      int cnt = 0;
      for (int q = a->rowptr[i]; q < a->rowptr[i + 1]; ++q) {
        int J = agg[a->col[q]];
        if (mark[J] != i) {
          mark[J] = i;
          acc[J] = 0.0;
          cols[cnt++] = J;
        }
        acc[J] += a->val[q];
      }
      qsort(cols, (size_t)cnt, sizeof(int), cmp_int);
      double w = omega * invd[i];
      long o = rowptr[i];
      for (int t = 0; t < cnt; ++t) {
        int J = cols[t];
        double tij = (J == agg[i]) ? 1.0 : 0.0;
        pcol[o + t] = J;
        pval[o + t] = tij - w * acc[J];
      }
    }
    free(mark);
    free(acc);
    free(cols);
  }
  p->n = n;
  p->m = nagg;
  p->nnz = nnz;
  p->rowptr = rowptr;
  p->col = pcol;
  p->val = pval;
}

orc_hier *orc_setup(const orc_op *op, int cheb_degree, double cheb_ratio,
                    double cheb_safety, int max_coarse, int max_levels,
                    int power_iters) {
  return orc_setup_agg(op, cheb_degree, cheb_ratio, cheb_safety, max_coarse, max_levels,
                       power_iters, ORC_AGG_MIS2);
}

orc_hier *orc_setup_agg(const orc_op *op, int cheb_degree, double cheb_ratio,
                        double cheb_safety, int max_coarse, int max_levels,
                        int power_iters, int aggregation) {
  return orc_setup_ex(op, cheb_degree, cheb_ratio, cheb_safety, max_coarse, max_levels,
                      power_iters, aggregation, ORC_COARSE_LU, 3);
}

orc_hier *orc_setup_ex(const orc_op *op, int cheb_degree, double cheb_ratio,
                       double cheb_safety, int max_coarse, int max_levels, int power_iters,
                       int aggregation, int coarse_solver, int coarse_sweeps) {
  orc_hier *h = (orc_hier *)calloc(1, sizeof(orc_hier));
  h->coarse_solver = coarse_solver;
  h->coarse_sweeps = coarse_sweeps;
  h->op = op;
  h->degree = cheb_degree;
  h->ratio = cheb_ratio;
  h->safety = cheb_safety;
  if (max_levels > ORC_MAX_LEVELS) max_levels = ORC_MAX_LEVELS;
  if (max_levels < 1) max_levels = 1;

  level_t *L0 = &h->lev[0];
  csr_copy(&op->Ahat, &L0->A);
  L0->ids = (unsigned int *)malloc((size_t)(op->n > 0 ? op->n : 1) * sizeof(unsigned int));
  for (int i = 0; i < op->n; ++i) L0->ids[i] = (unsigned int)op->node_of_row[i];
  L0->dims[0] = op->nx;
  L0->dims[1] = op->ny;
  L0->dims[2] = op->nz;

  int l = 0;
  for (;;) {
    level_t *lv = &h->lev[l];
    lv->invd = diag_inverse(&lv->A);
    int n = lv->A.n;
    if (n <= max_coarse || l == max_levels - 1) break;
    /* MIS-2 seeds and aggregates on G_l, the structural off-diagonal graph of A_l
     * (the diagonal entry only adds the node itself to its own neighbourhood). */
    unsigned int seed = 0x9E3779B9u * (unsigned int)(l + 1);
    lv->root = (unsigned char *)malloc((size_t)(n > 0 ? n : 1));
    lv->agg = (int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int));
    unsigned int *next_ids = NULL;
    int next_dims[3] = {0, 0, 0};
    int nagg;
    if (aggregation == ORC_AGG_CUBES) {
      next_ids = (unsigned int *)malloc((size_t)(n > 0 ? n : 1) * sizeof(unsigned int));
      nagg = orc_cube_aggregate(n, lv->ids, lv->dims, lv->agg, lv->root, next_ids, next_dims);
    } else {
      orc_mis2(n, lv->A.rowptr, lv->A.col, lv->ids, seed, lv->root);
      nagg = orc_aggregate(n, lv->A.rowptr, lv->A.col, lv->ids, seed, lv->root, lv->agg);
    }
    if (nagg < 0) {
      free(next_ids);
      h->status = -2;
      break;
    }
    /* READING: stop when coarsening stalls (more than 90 % of the nodes remain). */
    if (10L * nagg > 9L * n) {
      free(next_ids);
      break;
    }
    lv->lambda = orc_power_lambda(n, lv->A.rowptr, lv->A.col, lv->A.val, lv->ids, power_iters);
    /* READING: omega = 4 / (3 lambda), the usual SA damping of Vanek, Mandel, Brezina. */
    lv->omega = 4.0 / (3.0 * lv->lambda);
    smoothed_prolongator(&lv->A, lv->invd, lv->agg, nagg, lv->omega, &lv->P);
    csr_transpose(&lv->P, &lv->R); /* R = P^T (Sec. 3.2) */
    csr_t ap;
    csr_matmul(&lv->A, &lv->P, &ap);
    level_t *nx = &h->lev[l + 1];
    csr_matmul(&lv->R, &ap, &nx->A); /* A_{l+1} = R A_l P */
    csr_free(&ap);
    if (next_ids) {
      /* cube aggregation: the coarse nodes are the cubes, ids on the cube lattice */
      nx->ids = next_ids;
      memcpy(nx->dims, next_dims, sizeof(next_dims));
    } else {
      nx->ids = (unsigned int *)malloc((size_t)(nagg > 0 ? nagg : 1) * sizeof(unsigned int));
      for (int J = 0; J < nagg; ++J) nx->ids[J] = (unsigned int)J;
    }
    ++l;
  }
  h->nlev = l + 1;
  /* The coarsest level needs a spectral bound only if it is smoothed; it is not. */
  level_t *lc = &h->lev[l];
  int nc = lc->A.n;
  if (h->status == 0 && h->coarse_solver == ORC_COARSE_GS) {
    h->colour = (int *)malloc((size_t)(nc > 0 ? nc : 1) * sizeof(int));
    h->ncolours = orc_colour(nc, lc->A.rowptr, lc->A.col, lc->ids, 0x2545F491u, h->colour);
  } else if (h->status == 0) {
    if (nc > ORC_MAX_DENSE) {
      h->status = -3;
    } else {
      double *dense = (double *)calloc((size_t)(nc > 0 ? nc : 1) * (size_t)(nc > 0 ? nc : 1), sizeof(double));
      for (int i = 0; i < nc; ++i)
        for (int p = lc->A.rowptr[i]; p < lc->A.rowptr[i + 1]; ++p)
          dense[(size_t)i * nc + lc->A.col[p]] = lc->A.val[p];
      if (dense_lu_factor(&h->coarse, nc, dense) != 0) h->status = -4;
      free(dense);
    }
  }
  h->wb = (double **)calloc((size_t)h->nlev, sizeof(double *));
  h->wx = (double **)calloc((size_t)h->nlev, sizeof(double *));
  h->wr = (double **)calloc((size_t)h->nlev, sizeof(double *));
  for (int q = 0; q < h->nlev; ++q) {
    size_t nq = (size_t)(h->lev[q].A.n > 0 ? h->lev[q].A.n : 1);
    h->wb[q] = (double *)calloc(nq, sizeof(double));
    h->wx[q] = (double *)calloc(nq, sizeof(double));
    h->wr[q] = (double *)calloc(nq, sizeof(double));
  }
  return h;
}

void orc_hier_free(orc_hier *h) {
  if (!h) return;
  for (int l = 0; l < ORC_MAX_LEVELS; ++l) {
    level_t *lv = &h->lev[l];
    csr_free(&lv->A);
    csr_free(&lv->P);
    csr_free(&lv->R);
    free(lv->invd);
    free(lv->ids);
    free(lv->agg);
    free(lv->root);
  }
  if (h->coarse.lu) dense_lu_free(&h->coarse);
  free(h->colour);
  for (int q = 0; q < h->nlev; ++q) {
    free(h->wb[q]);
    free(h->wx[q]);
    free(h->wr[q]);
  }
  free(h->wb);
  free(h->wx);
  free(h->wr);
  free(h);
}

int orc_hier_levels(const orc_hier *h) { return h->nlev; }
int orc_hier_colours(const orc_hier *h, int *colour) {
  if (!h->colour) return 0;
  if (colour) memcpy(colour, h->colour, (size_t)h->lev[h->nlev - 1].A.n * sizeof(int));
  return h->ncolours;
}
int orc_hier_status(const orc_hier *h) { return h->status; }
int orc_hier_n(const orc_hier *h, int l) { return h->lev[l].A.n; }
long orc_hier_nnz(const orc_hier *h, int l) { return h->lev[l].A.nnz; }
long orc_hier_nnz_p(const orc_hier *h, int l) { return h->lev[l].P.nnz; }
double orc_hier_lambda(const orc_hier *h, int l) { return h->lev[l].lambda; }
double orc_hier_omega(const orc_hier *h, int l) { return h->lev[l].omega; }

static void get_csr(const csr_t *a, int *rowptr, int *col, double *val) {
  if (rowptr) memcpy(rowptr, a->rowptr, (size_t)(a->n + 1) * sizeof(int));
  if (col) memcpy(col, a->col, (size_t)a->nnz * sizeof(int));
  if (val) memcpy(val, a->val, (size_t)a->nnz * sizeof(double));
}

void orc_hier_get_a(const orc_hier *h, int l, int *rowptr, int *col, double *val) {
  get_csr(&h->lev[l].A, rowptr, col, val);
}
void orc_hier_get_p(const orc_hier *h, int l, int *rowptr, int *col, double *val) {
  get_csr(&h->lev[l].P, rowptr, col, val);
}
void orc_hier_get_r(const orc_hier *h, int l, int *rowptr, int *col, double *val) {
  get_csr(&h->lev[l].R, rowptr, col, val);
}
void orc_hier_get_agg(const orc_hier *h, int l, int *agg, unsigned char *is_root) {
  int n = h->lev[l].A.n;
  if (agg && h->lev[l].agg) memcpy(agg, h->lev[l].agg, (size_t)n * sizeof(int));
  if (is_root && h->lev[l].root) memcpy(is_root, h->lev[l].root, (size_t)n);
}

/* ------------------------------------------------------------------------- */
/* V-cycle (Algorithm 1)                                                      */
/* ------------------------------------------------------------------------- */
static void mg_solve(const orc_hier *h, int l, const double *b, double *x) {
  const level_t *lv = &h->lev[l];
  int n = lv->A.n;
  if (l == h->nlev - 1) { /* DirectSolve, or Gauss-Seidel steps */
    if (h->coarse_solver == ORC_COARSE_GS)
      orc_sgs(n, lv->A.rowptr, lv->A.col, lv->A.val, lv->invd, h->colour, h->ncolours,
              h->coarse_sweeps, b, x);
    else
      dense_lu_solve(&h->coarse, b, x);
    return;
  }
  /* presmoothing from x = 0 */
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) x[i] = 0.0;
  orc_cheb_smooth(n, lv->A.rowptr, lv->A.col, lv->A.val, lv->invd, lv->lambda, h->ratio,
                  h->safety, h->degree, b, x, 1);
  /* residual r = b - A x */
  double *r = h->wr[l];
  csr_spmv(&lv->A, x, r);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
  /* restriction b_{l+1} = R r ; v_{l+1} = 0 ; recurse */
  double *bc = h->wb[l + 1], *vc = h->wx[l + 1];
  csr_spmv(&lv->R, r, bc);
  mg_solve(h, l + 1, bc, vc);
  /* coarse-grid correction x += P v */
  csr_spmv(&lv->P, vc, r);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) x[i] = x[i] + r[i];
  /* postsmoothing: same polynomial */
  orc_cheb_smooth(n, lv->A.rowptr, lv->A.col, lv->A.val, lv->invd, lv->lambda, h->ratio,
                  h->safety, h->degree, b, x, 0);
}

void orc_vcycle(const orc_hier *h, const double *r, double *z) { mg_solve(h, 0, r, z); }

/* ------------------------------------------------------------------------- */
/* Preconditioned conjugate gradients (Sec. 3.1, Sec. 3.2)                    */
/* ------------------------------------------------------------------------- */
/* Stopping rule ||r||_2 <= rtol ||b||_2 (Sec. 5.2).  The iteration count is the
 * number of products A p.  READING: for the mildly nonsymmetric quadratic matrix the
 * paper only says "CG"; beta_rule 0 is the usual ratio of successive r'z (Hestenes-
 * Stiefel / Fletcher-Reeves form), 1 is the Polak-Ribiere form z'(r - r_old)/r_old'z_old
 * for a variable preconditioner. */
int orc_pcg(const orc_hier *h, const double *bhat, double *xhat, double rtol, int maxit,
            int beta_rule, int *iters, double *relres) {
  const csr_t *a = &h->lev[0].A;
  int n = a->n;
  *iters = 0;
  *relres = 0.0;
  if (n == 0) return 0;
  double bnorm = sqrt(dot(n, bhat, bhat));
  if (bnorm == 0.0) {
    for (int i = 0; i < n; ++i) xhat[i] = 0.0;
    return 0;
  }
  double *r = (double *)malloc((size_t)n * sizeof(double));
  double *z = (double *)malloc((size_t)n * sizeof(double));
  double *p = (double *)malloc((size_t)n * sizeof(double));
  double *q = (double *)malloc((size_t)n * sizeof(double));
  csr_spmv(a, xhat, q);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) r[i] = bhat[i] - q[i];
  double rnorm = sqrt(dot(n, r, r));
  int rc = 1;
  if (rnorm <= rtol * bnorm) {
    rc = 0;
  } else {
    orc_vcycle(h, r, z);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) p[i] = z[i];
    double rz = dot(n, r, z);
    for (int it = 1; it <= maxit; ++it) {
      csr_spmv(a, p, q);
      double pq = dot(n, p, q);
      if (!(pq != 0.0) || !isfinite(pq) || !isfinite(rz)) {
        rc = -1;
        *iters = it;
        break;
      }
      double alpha = rz / pq;
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) {
        xhat[i] = xhat[i] + alpha * p[i];
        r[i] = r[i] - alpha * q[i];
      }
      rnorm = sqrt(dot(n, r, r));
      *iters = it;
      if (!isfinite(rnorm)) {
        rc = -1;
        break;
      }
      if (rnorm <= rtol * bnorm) {
        rc = 0;
        break;
      }
      orc_vcycle(h, r, z);
      double rz_new = dot(n, r, z);
      double beta;
      if (beta_rule == 1) {
        /* r_old = r + alpha q, so z'(r - r_old) = -alpha z'q */
        double zq = dot(n, z, q);
        beta = (-alpha * zq) / rz;
      } else {
        beta = rz_new / rz;
      }
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
      rz = rz_new;
    }
  }
  *relres = rnorm / bnorm;
  free(r);
  free(z);
  free(p);
  free(q);
  return rc;
}

/* Box arrays in, box array out; b = bfac * rho, bhat = S b, xhat = x / s, phi = S xhat.
 * relres is the recursive, relres_true the recomputed residual of the scaled system. */
int orc_solve(const orc_hier *h, const double *rho_box, double *phi_box, double rtol,
              int maxit, int beta_rule, int *iters, double *relres, double *relres_true) {
  const orc_op *op = h->op;
  int n = op->n;
  *iters = 0;
  *relres = 0.0;
  *relres_true = 0.0;
  if (h->status != 0) return -2;
  double *bhat = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  double *xhat = (double *)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
  for (int r = 0; r < n; ++r) {
    int q = op->node_of_row[r];
    bhat[r] = op->scale[r] * (op->bfac[r] * rho_box[q]);
    xhat[r] = phi_box[q] / op->scale[r];
  }
  int rc = orc_pcg(h, bhat, xhat, rtol, maxit, beta_rule, iters, relres);
  if (n > 0) {
    double *t = (double *)malloc((size_t)n * sizeof(double));
    csr_spmv(&h->lev[0].A, xhat, t);
    double num = 0.0, den = 0.0;
    for (int i = 0; i < n; ++i) {
      double e = bhat[i] - t[i];
      num += e * e;
      den += bhat[i] * bhat[i];
    }
    *relres_true = den > 0.0 ? sqrt(num) / sqrt(den) : 0.0;
    free(t);
  }
  long nbox = (long)op->nx * op->ny * op->nz;
  for (long q = 0; q < nbox; ++q) phi_box[q] = 0.0;
  for (int r = 0; r < n; ++r) phi_box[op->node_of_row[r]] = op->scale[r] * xhat[r];
  free(bhat);
  free(xhat);
  return rc;
}
