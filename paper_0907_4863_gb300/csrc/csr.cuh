// CSR kernels of the coarse levels and the transfer operators (internal).
#pragma once

#include "common.cuh"

namespace saamg {

enum CsrMode {
  CSR_SPMV = 0,         // y = A x
  CSR_RESID = 1,        // y = b - A x
  CSR_CHEB = 2,         // r = b - A x; d = c1 d + c2 D^-1 r; y = x + d
  CSR_CHEB0 = 3,        // d = c2 D^-1 b; y = d
  CSR_ADD = 4,          // y += A x   (coarse-grid correction x += P v)
  CSR_SPMV_DINV_DOT = 5 // y = s D^-1 A x, partials of y.y (power iteration; s = *xscale or 1)
};

// Matrix values of type TM (double, float or bf16), vectors of type TV (double, float).
template <class TV, class TM>
void csr_apply(int mode, int n, const int* rowptr, const int* col, const TM* val, double avg_nnz,
               const TV* x, TV* y, const TV* b, TV* d, const TV* invd, TV c1, TV c2,
               double* partials, cudaStream_t s, int kclass = -1,
               const double* xscale = nullptr);

// The launch form csr_apply takes for a matrix of n rows with avg_nnz entries per row: 0 for
// a thread per (short) row, else the lanes G per row (2 .. 32).  dbl: FP64 vectors.
int csr_plan(int mode, int n, double avg_nnz, bool dbl);

// invd_i = 1 / a_ii (also the FP32 copy when invd32 is not null)
void csr_diag_inverse(const DevCsr& A, double* invd, float* invd32, cudaStream_t s);
void to_float(const double* in, float* out, size_t n, cudaStream_t s);
void to_bf16(const double* in, __nv_bfloat16* out, size_t n, cudaStream_t s);
void to_double(const float* in, double* out, size_t n, cudaStream_t s);

}  // namespace saamg
