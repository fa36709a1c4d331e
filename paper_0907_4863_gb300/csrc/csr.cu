// CSR kernels: coarse-level operator, Chebyshev smoother fused with the residual,
// restriction R r and prolongation x += P v (Algorithm 1), and D^-1 A x for the
// power iteration.  G lanes cooperate on one row (G chosen from the mean row length),
// partial row sums are combined with shuffles inside the G-lane group.
#include <cmath>

#include "csr.cuh"
#include "rows.cuh"

namespace saamg {

namespace {

template <class TV, class TM, int G, int MODE>
__global__ void __launch_bounds__(256) csr_k(int n, const int* __restrict__ rowptr,
                                             const int* __restrict__ col,
                                             const TM* __restrict__ val, const TV* __restrict__ x,
                                             TV* __restrict__ y, const TV* __restrict__ b,
                                             TV* __restrict__ d, const TV* __restrict__ invd,
                                             TV c1, TV c2, double* __restrict__ partials,
                                             const double* __restrict__ xscale) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int gl = lane % G;
  constexpr int kRowsPerWarp = 32 / G;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  double dacc = 0.0;
  if (MODE == CSR_SPMV_DINV_DOT) c2 = xscale ? (TV)*xscale : TV(1);
  // the trip count is uniform across the warp, so the group shuffles see all 32 lanes
  for (int wbase = warp * kRowsPerWarp; wbase < n; wbase += nwarps * kRowsPerWarp) {
    const int row = wbase + lane / G;
    rows::csr_group_row<TV, TM, G, MODE>(row, row < n, gl, rowptr, col, val, x, y, b, d, invd,
                                         c1, c2, dacc);
  }
  if (MODE == CSR_SPMV_DINV_DOT) {
    const double t = rows::block_sum(dacc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

// Thread per row for the short rows of the prolongators (a handful of entries each): the
// first kShortWin entries of a row are loaded under predicates, so all of the row's column,
// value and gather loads are in flight at once, and a warp keeps 32 rows in flight.  The
// row is summed in entry order; longer rows finish in a plain loop.
using rows::kShortWin;

template <class TV, class TM, int MODE>
__global__ void __launch_bounds__(256) csr_short_k(int n, const int* __restrict__ rowptr,
                                                   const int* __restrict__ col,
                                                   const TM* __restrict__ val,
                                                   const TV* __restrict__ x, TV* __restrict__ y) {
  pdl_wait();
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n;
       row += gridDim.x * blockDim.x)
    rows::csr_short_row<TV, TM, MODE>(row, rowptr, col, val, x, y);
}

template <class TV, class TM, int G>
void launch_g(int mode, int n, const int* rowptr, const int* col, const TM* val, const TV* x,
              TV* y, const TV* b, TV* d, const TV* invd, TV c1, TV c2, double* partials,
              cudaStream_t s, const double* xscale) {
  int blocks;
  if (mode == CSR_SPMV_DINV_DOT) {
    blocks = kRedBlocks;
  } else {
    long long need = ((long long)n * G + 255) / 256;
    blocks = (int)(need < sm_count() * 16 ? (need > 0 ? need : 1) : sm_count() * 16);
  }
#define SAAMG_CSR_CASE(M)                                                                  \
  case M:                                                                                  \
    launch_pdl(csr_k<TV, TM, G, M>, blocks, 256, 0, s, n, rowptr, col, val, x, y, b, d,   \
               invd, c1, c2, partials, xscale);                                            \
    break;
  switch (mode) {
    SAAMG_CSR_CASE(CSR_SPMV)
    SAAMG_CSR_CASE(CSR_RESID)
    SAAMG_CSR_CASE(CSR_CHEB)
    SAAMG_CSR_CASE(CSR_CHEB0)
    SAAMG_CSR_CASE(CSR_ADD)
    SAAMG_CSR_CASE(CSR_SPMV_DINV_DOT)
    default:
      fail(SAAMG_EINVAL, "bad csr mode");
  }
#undef SAAMG_CSR_CASE
  SAAMG_LAUNCH();
}

__global__ void diag_inverse_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                               const double* __restrict__ val, double* __restrict__ invd,
                               float* __restrict__ invd32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double dgl = 0.0;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
    if (col[p] == i) dgl = val[p];
  double v = 1.0 / dgl;
  invd[i] = v;
  if (invd32) invd32[i] = (float)v;
}

template <class TI, class TO>
__global__ void convert_k(const TI* __restrict__ in, TO* __restrict__ out, size_t n) {
  pdl_wait();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

__global__ void to_bf16_k(const double* __restrict__ in, __nv_bfloat16* __restrict__ out,
                          size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = __double2bfloat16(in[i]);
}

inline int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

int csr_plan(int mode, int n, double avg_nnz, bool dbl) {
  // the prolongators' short rows on a large level: a thread per row
  if ((mode == CSR_ADD || mode == CSR_SPMV) && avg_nnz <= kShortWin && n >= 100000) return 0;
  int g = dbl ? (avg_nnz <= 10.0 ? 2 : (avg_nnz <= 48.0 ? 4 : 8))
              : (avg_nnz <= 6.0 ? 2 : (avg_nnz <= 20.0 ? 4 : (avg_nnz <= 64.0 ? 8 : 16)));
  int gpar = 1;
  while (gpar < 32 && (long long)n * gpar < 150000) gpar <<= 1;
  // no more lanes than the row length needs: one entry per lane in FP32; in FP64, where a
  // warp-wide shuffle-add costs a full FP64 issue slot, up to 8 entries per lane (a level of
  // 9 k rows of 61 entries: 13.9 -> 9.8 us per smoothing step with 8 instead of 32 lanes)
  const double per_lane = dbl ? 8.0 : 1.0;
  int glen = 1;
  while (glen < 32 && glen * per_lane < avg_nnz) glen <<= 1;
  return std::max(g, std::min(gpar, glen));
}

template <class TV, class TM>
void csr_apply(int mode, int n, const int* rowptr, const int* col, const TM* val, double avg_nnz,
               const TV* x, TV* y, const TV* b, TV* d, const TV* invd, TV c1, TV c2,
               double* partials, cudaStream_t s, int kclass, const double* xscale) {
  if (n <= 0) {
    if (mode == CSR_SPMV_DINV_DOT) fill_double(partials, 0.0, kRedBlocks, s);
    return;
  }
  // timing unit of the sparse-matrix classes: matrix entries
  KernelTimer kt(kclass, std::llround(avg_nnz * n), s);
  // Lanes per row: FP64 shuffle-adds cost as much as the row's multiply-adds on this part, so
  // double vectors use few lanes (FP32 can afford wider groups for better coalescing) -- but
  // a small level (few rows, long rows: the deep levels of the hierarchy) needs wider groups
  // to fill the GPU at all: enough lanes for ~150 k threads, never more than the row length.
  const int g = csr_plan(mode, n, avg_nnz, sizeof(TV) == 8);
  if (g == 0) {
    const long long need = ((long long)n + 255) / 256;
    const int blocks = (int)(need < sm_count() * 16 ? need : sm_count() * 16);
    if (mode == CSR_ADD)
      launch_pdl(csr_short_k<TV, TM, CSR_ADD>, blocks, 256, 0, s, n, rowptr, col, val, x, y);
    else
      launch_pdl(csr_short_k<TV, TM, CSR_SPMV>, blocks, 256, 0, s, n, rowptr, col, val, x, y);
    SAAMG_LAUNCH();
    return;
  }
  switch (g) {
    case 2:
      launch_g<TV, TM, 2>(mode, n, rowptr, col, val, x, y, b, d, invd, c1, c2, partials, s, xscale);
      break;
    case 4:
      launch_g<TV, TM, 4>(mode, n, rowptr, col, val, x, y, b, d, invd, c1, c2, partials, s, xscale);
      break;
    case 8:
      launch_g<TV, TM, 8>(mode, n, rowptr, col, val, x, y, b, d, invd, c1, c2, partials, s, xscale);
      break;
    case 16:
      launch_g<TV, TM, 16>(mode, n, rowptr, col, val, x, y, b, d, invd, c1, c2, partials, s,
                           xscale);
      break;
    default:
      launch_g<TV, TM, 32>(mode, n, rowptr, col, val, x, y, b, d, invd, c1, c2, partials, s,
                           xscale);
  }
}

template void csr_apply<double, double>(int, int, const int*, const int*, const double*, double,
                                        const double*, double*, const double*, double*,
                                        const double*, double, double, double*, cudaStream_t, int,
                                        const double*);
template void csr_apply<float, float>(int, int, const int*, const int*, const float*, double,
                                      const float*, float*, const float*, float*, const float*,
                                      float, float, double*, cudaStream_t, int, const double*);
template void csr_apply<float, __nv_bfloat16>(int, int, const int*, const int*,
                                              const __nv_bfloat16*, double, const float*, float*,
                                              const float*, float*, const float*, float, float,
                                              double*, cudaStream_t, int, const double*);

void csr_diag_inverse(const DevCsr& A, double* invd, float* invd32, cudaStream_t s) {
  if (A.n == 0) return;
  diag_inverse_k<<<(A.n + 255) / 256, 256, 0, s>>>(A.n, A.rowptr.p, A.col.p, A.val.p, invd,
                                                   invd32);
  SAAMG_LAUNCH();
}

void to_float(const double* in, float* out, size_t n, cudaStream_t s) {
  if (!n) return;
  launch_pdl(convert_k<double, float>, grid_for(n), 256, 0, s, in, out, n);
  SAAMG_LAUNCH();
}

void to_double(const float* in, double* out, size_t n, cudaStream_t s) {
  if (!n) return;
  launch_pdl(convert_k<float, double>, grid_for(n), 256, 0, s, in, out, n);
  SAAMG_LAUNCH();
}

void to_bf16(const double* in, __nv_bfloat16* out, size_t n, cudaStream_t s) {
  if (!n) return;
  to_bf16_k<<<grid_for(n), 256, 0, s>>>(in, out, n);
  SAAMG_LAUNCH();
}

}  // namespace saamg
