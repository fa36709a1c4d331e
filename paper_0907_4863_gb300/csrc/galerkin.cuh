// Hierarchy construction kernels (internal): spectral bound, prolongator, Galerkin product.
#pragma once

#include "common.cuh"

namespace saamg {

// lambda_hat of D^-1 A by `iters` power-iteration steps from v_i = 0.5 + fmix32(id ^
// 0xA5A5A5A5)/2^32 (ids NULL: the row index).  Returns lambda_hat (synchronises).  With S
// given, D^-1 A is applied by the matrix-free level-0 stencil instead of the CSR.
template <class T>
struct StencilDev;
double power_lambda(const DevCsr& A, const double* invd, const unsigned* ids, int iters,
                    cudaStream_t s, const StencilDev<double>* S = nullptr);

// C = X Y with a structural pattern (entries that cancel are kept), columns ascending in
// every row, each entry summed in the order X's row (ascending columns) then Y's row.
void spgemm(const DevCsr& X, const DevCsr& Y, DevCsr& C, cudaStream_t s);

// Tentative prolongator T (one entry 1 per row at column agg(i)).
void tentative(const int* agg, int n, int nagg, DevCsr& T, cudaStream_t s);

// Smoothed prolongator from AT = A T:  P_iJ = [J == agg(i)] - (omega / a_ii) (AT)_iJ.
// P takes over AT's pattern; AT is consumed.
void smoothed_prolongator(DevCsr& AT, const int* agg, const double* invd, double omega,
                          DevCsr& P, cudaStream_t s);

// R = P^T with ascending columns in every row.
void transpose(const DevCsr& P, DevCsr& R, cudaStream_t s);

}  // namespace saamg
