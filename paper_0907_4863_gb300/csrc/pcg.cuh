// Conjugate-gradient vector kernels (internal).
#pragma once

#include "common.cuh"

namespace saamg {

// Scalars of the CG recursion, kept on the device between kernels.
struct PcgCtl {
  double rz;      // r'z of the current direction
  double alpha;
  double beta;
  double pq;
  double rr;      // ||r||^2 after the last update
  double rz_new;
  double zq;
  double tol2;    // (rtol ||b||)^2
  int iters;
  int converged;
  int breakdown;
  int pad;
};

// partials[blockIdx] of sum a_i b_i (fixed grid kRedBlocks)
template <class TA, class TB>
void dot_partials(int n, const TA* a, const TB* b, double* partials, cudaStream_t s);

// ctl->pq = sum(partials); alpha = rz / pq (breakdown flag on 0/NaN)
void pcg_alpha(const double* partials, PcgCtl* ctl, cudaStream_t s);
// x += alpha p; r -= alpha q; partials of r'r
void pcg_update(int n, double* x, double* r, const double* p, const double* q, const PcgCtl* ctl,
                double* partials, cudaStream_t s);
// ctl->rr = sum(partials); converged = rr <= tol2; iters++
void pcg_check(const double* partials, PcgCtl* ctl, cudaStream_t s);
// rz_new = sum(part_rz); beta = rz_new / rz (rule 0) or -alpha zq / rz (rule 1, part_zq);
// rule -1 only stores rz (first direction)
void pcg_beta(const double* part_rz, const double* part_zq, int rule, PcgCtl* ctl,
              cudaStream_t s);
// p = z + beta p
template <class TZ>
void pcg_direction(int n, const TZ* z, double* p, const PcgCtl* ctl, cudaStream_t s);
// r = b - q, elementwise
void vec_sub(int n, const double* b, const double* q, double* r, cudaStream_t s);
template <class TZ>
void vec_copy_to_double(int n, const TZ* z, double* p, cudaStream_t s);

}  // namespace saamg
