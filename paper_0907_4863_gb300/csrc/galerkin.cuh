// Hierarchy construction kernels (internal): spectral bound, prolongator, Galerkin product.
#pragma once

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

// P = (I - omega D^-1 A) T straight from A and the aggregates (T(i, agg(i)) = 1), without
// forming T or a general sparse product; nagg = the number of aggregates.
void prolongator(const DevCsr& A, const int* agg, int nagg, const double* invd, double omega,
                 DevCsr& P, cudaStream_t s);

// R = P^T with ascending columns in every row.
void transpose(const DevCsr& P, DevCsr& R, cudaStream_t s);

}  // namespace saamg
