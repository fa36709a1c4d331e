// Coarsest-level direct solver (internal).
#pragma once

#include "common.cuh"

namespace saamg {

struct CoarseSolver {
  int n = 0;
  Buf<double> inv;  // A_L^-1, column-major
};

// Dense LU with partial pivoting of A_L and its explicit inverse (synchronises).
void coarse_factor(const DevCsr& A, CoarseSolver& cs, cudaStream_t s);
// x = A_L^-1 b (FP64 accumulation for any vector type)
template <class TV>
void coarse_apply(const CoarseSolver& cs, const TV* b, TV* x, cudaStream_t s);

}  // namespace saamg
