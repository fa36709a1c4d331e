// Coarsest-level direct solver (internal).
#pragma once

#include "common.cuh"

namespace saamg {

struct CoarseSolver {
  int n = 0;
  int kind = 0;     // SAAMG_COARSE_LU or SAAMG_COARSE_GS
  Buf<double> inv;  // LU: A_L^-1, row-major
  // Gauss-Seidel: A_L (borrowed from the hierarchy), 1 / a_ii, rows sorted by colour
  const int* rowptr = nullptr;
  const int* col = nullptr;
  const double* val = nullptr;
  const double* invd = nullptr;
  Buf<int> colour, order, coff;
  int ncolours = 0, steps = 0;
  size_t bytes() const { return inv.bytes() + colour.bytes() + order.bytes() + coff.bytes(); }
};

// Dense LU with partial pivoting of A_L and its explicit inverse (synchronises).
void coarse_factor(const DevCsr& A, CoarseSolver& cs, cudaStream_t s);
// inv = A^-1 of the dense row-major n x n device matrix a, into row-major inv (synchronises;
// SAAMG_NUMERICAL on a zero pivot)
void dense_inverse(int n, const double* a, double* inv, cudaStream_t s);
// Gauss-Seidel coarse solver (Sec. 3.2): colours A_L's graph by synchronous rounds of local
// maxima of key(v) = (fmix32(id_v ^ 0x2545F491), id_v) (ids NULL: the row index) and sorts
// the rows by colour; each solve then runs `steps` symmetric multicolour sweeps from x = 0.
// A_L and invd must outlive cs.  n <= kCoarseGsMax (x and b live in one CTA's shared memory).
constexpr int kCoarseGsMax = 12288;
void coarse_gs_setup(const DevCsr& A, const double* invd, const unsigned* ids, int steps,
                     CoarseSolver& cs, cudaStream_t s);
// x = A_L^-1 b (LU) or the Gauss-Seidel steps (FP64 arithmetic for any vector type)
template <class TV>
void coarse_apply(const CoarseSolver& cs, const TV* b, TV* x, cudaStream_t s);

}  // namespace saamg
