// Conjugate-gradient vector kernels (internal).
#pragma once

#include "common.cuh"

namespace saamg {

// Scalars of the CG recursion, kept on the device between kernels.
struct PcgCtl {
  double rtol;    // stopping tolerance (device-loop solves read it here)
  double bb;      // ||b||^2
  double rr_true; // ||b - A x||^2 at exit
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
// partials of r'z and z'q in one sweep (bitwise the two dot_partials calls)
template <class TZ>
void dot2_partials(int n, const double* r, const TZ* z, const double* q, double* part_rz,
                   double* part_zq, cudaStream_t s);

// x += alpha p; r -= alpha q; partials of r'r; r32 (if not null) = FP32 copy of the new r
void pcg_update(int n, double* x, double* r, const double* p, const double* q, const PcgCtl* ctl,
                double* partials, cudaStream_t s, float* r32 = nullptr);
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

// --- device-loop PCG (one CUDA graph with a conditional while node) --------------
// prologue: ctl->bb = sum(part_bb), ctl->rr = sum(part_rr), tol2 = (rtol^2) bb; the loop
// condition is set to "not converged, no breakdown, maxit > 0"; x is zeroed when b = 0.
void pcg_graph_init(const double* part_bb, const double* part_rr, PcgCtl* ctl,
                    cudaGraphConditionalHandle cond, int maxit, double* x, int n, cudaStream_t s);
// beta of the device loop: 0 on the first pass (p = z), else rule 0 / rule 1
void pcg_graph_beta(const double* part_rz, const double* part_zq, int rule, PcgCtl* ctl,
                    cudaStream_t s);
// end of a pass: rr, iters, converged; clears the loop condition when done
void pcg_graph_check(const double* partials, PcgCtl* ctl, cudaGraphConditionalHandle cond,
                     int maxit, cudaStream_t s);
// ctl->rr_true = sum(partials)
void pcg_store_true(const double* partials, PcgCtl* ctl, cudaStream_t s);

}  // namespace saamg
