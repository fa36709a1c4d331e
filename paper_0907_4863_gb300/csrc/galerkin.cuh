// Hierarchy construction kernels (internal): spectral bound, prolongator, Galerkin product.
#pragma once

#include <vector>

#include "common.cuh"

namespace saamg {

// lambda_hat of D^-1 A by `iters` power-iteration steps from v_i = 0.5 + fmix32(id ^
// 0xA5A5A5A5)/2^32 (ids NULL: the row index).  Returns lambda_hat (synchronises).  With S
// given, D^-1 A is applied by the matrix-free level-0 stencil instead of the CSR; with As
// given (a SELL copy of A holding FP64 values), by the SELL kernel.
template <class T>
struct StencilDev;
struct DevSell;
double power_lambda(const DevCsr& A, const double* invd, const unsigned* ids, int iters,
                    cudaStream_t s, const StencilDev<double>* S = nullptr,
                    const DevSell* As = nullptr);
// The same in two halves, so that other work can run meanwhile: _start enqueues the steps on
// s (run keeps their buffers), _finish waits for s and returns lambda_hat.
struct PowerRun {
  int n = 0;
  Buf<double> v, w, part, nrm2;
};
void power_lambda_start(const DevCsr& A, const double* invd, const unsigned* ids, int iters,
                        cudaStream_t s, PowerRun& run, const StencilDev<double>* S = nullptr,
                        const DevSell* As = nullptr);
double power_lambda_finish(PowerRun& run, cudaStream_t s);

// C = X Y with a structural pattern (entries that cancel are kept), columns ascending in
// every row; every entry is summed in an order fixed by the row's product counts (X's
// entries in order within one lane group; the groups' partial sums in group order), so a
// product is bitwise reproducible.
void spgemm(const DevCsr& X, const DevCsr& Y, DevCsr& C, cudaStream_t s);

// The two phases of spgemm.  The symbolic phase reads the patterns of X and Y only and leaves
// C's row pointers, the rows binned by the numeric kernel class and the sorted columns of the
// hash rows in the plan; the numeric phase then needs matrices with those patterns and their
// values.  With `known` given (the C of an earlier product whose factors had the patterns of
// X and Y), C's pattern is taken from it and no symbolic pass runs; `known` must outlive the
// numeric phase.  Either way the numeric phase gives the bits of spgemm.
struct SpgemmPlan {
  int n = 0, m = 0;
  long long nnz = 0;
  double yavg = 0;
  Buf<int> rowptr;                 // C's row pointers
  Buf<int> nprod, cls, list, ctl;
  std::vector<int> hist, start;    // the numeric classes: row counts and list offsets
  Buf<int> soff, skeys;            // sorted columns the symbolic hash passes wrote
  const int* keys = nullptr;       // the sorted columns the numeric pass reads (or NULL) ...
  const int* koff = nullptr;       // ... and their row offsets
};
void spgemm_symbolic(const DevCsr& X, const DevCsr& Y, SpgemmPlan& plan, cudaStream_t s,
                     const DevCsr* known = nullptr);
void spgemm_numeric(const DevCsr& X, const DevCsr& Y, SpgemmPlan& plan, DevCsr& C, cudaStream_t s);

// P = (I - omega D^-1 A) T straight from A and the aggregates (T(i, agg(i)) = 1), without
// forming T or a general sparse product; nagg = the number of aggregates.
void prolongator(const DevCsr& A, const int* agg, int nagg, const double* invd, double omega,
                 DevCsr& P, cudaStream_t s);
// The same in two halves: _start forms A T (the part that does not depend on omega; `known`,
// a prolongator of the same pattern, spares the symbolic pass of the short-row path),
// _finish the values of P.
struct ProlongState {
  int n = 0, nagg = 0, G = 0;
  bool lists = false;              // rows of A longer than 8 entries: aggregate lists
  DevCsr AT;                       // short rows: A T; lists: P's row pointers and counts
  Buf<int> lcol;
  Buf<double> lval;
  const DevCsr* A = nullptr;
  const int* agg = nullptr;
  // set before _start when omega is known already: the level-0 row-at-a-time form then writes
  // P's values at once and _finish only hands P over
  const double* invd = nullptr;
  double omega = 0.0;
  bool final_values = false;
};
// stencil_rows: A is the level-0 operator (rows of at most 8 entries), whose A T is formed a
// row at a time, with the sums of the general product.
void prolongator_start(const DevCsr& A, const int* agg, int nagg, ProlongState& st,
                       cudaStream_t s, const DevCsr* known = nullptr, bool stencil_rows = false);
void prolongator_finish(ProlongState& st, const double* invd, double omega, DevCsr& P,
                        cudaStream_t s);

// R = P^T with ascending columns in every row.  Enqueued on s without any host wait (so it can
// run on a second stream beside other work).
void transpose(const DevCsr& P, DevCsr& R, cudaStream_t s);
// The same when R's pattern is known (`known`, the transpose of a P of the same pattern):
// the pattern is copied and every value moved to its place (a search in its row of R).
void transpose_known(const DevCsr& P, const DevCsr& known, DevCsr& R, cudaStream_t s);

}  // namespace saamg
