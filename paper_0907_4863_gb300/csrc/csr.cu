// CSR kernels: coarse-level operator, Chebyshev smoother fused with the residual,
// restriction R r and prolongation x += P v (Algorithm 1), and D^-1 A x for the
// power iteration.  G lanes cooperate on one row (G chosen from the mean row length),
// partial row sums are combined with shuffles inside the G-lane group.
#include <cmath>

#include "csr.cuh"

namespace saamg {

namespace {

__device__ __forceinline__ double ld(const double* p, size_t i) { return p[i]; }
__device__ __forceinline__ float ld(const float* p, size_t i) { return p[i]; }
__device__ __forceinline__ float ld(const __nv_bfloat16* p, size_t i) {
  return __bfloat162float(p[i]);
}

template <class TV, class TM, int G, int MODE>
__global__ void __launch_bounds__(256) csr_k(int n, const int* __restrict__ rowptr,
                                             const int* __restrict__ col,
                                             const TM* __restrict__ val, const TV* __restrict__ x,
                                             TV* __restrict__ y, const TV* __restrict__ b,
                                             TV* __restrict__ d, const TV* __restrict__ invd,
                                             TV c1, TV c2, double* __restrict__ partials,
                                             const double* __restrict__ xscale) {
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
    const bool active = row < n;
    TV acc = TV(0);
    if (MODE != CSR_CHEB0 && active) {
      const int p0 = rowptr[row], p1 = rowptr[row + 1];
      int p = p0 + gl;
      // four independent (column, value) loads and gathers in flight per lane
      for (; p + 3 * G < p1; p += 4 * G) {
        const int k0 = col[p], k1 = col[p + G], k2 = col[p + 2 * G], k3 = col[p + 3 * G];
        const TV a0 = (TV)ld(val, p), a1 = (TV)ld(val, p + G), a2 = (TV)ld(val, p + 2 * G),
                 a3 = (TV)ld(val, p + 3 * G);
        const TV x0 = x[k0], x1 = x[k1], x2 = x[k2], x3 = x[k3];
        acc += a0 * x0;
        acc += a1 * x1;
        acc += a2 * x2;
        acc += a3 * x3;
      }
      for (; p < p1; p += G) acc += (TV)ld(val, p) * x[col[p]];
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o, G);
    if (active && gl == 0) {
      if (MODE == CSR_SPMV) {
        y[row] = acc;
      } else if (MODE == CSR_RESID) {
        y[row] = b[row] - acc;
      } else if (MODE == CSR_ADD) {
        y[row] = y[row] + acc;
      } else if (MODE == CSR_CHEB) {
        const TV r = b[row] - acc;
        const TV dprev = (c1 == TV(0)) ? TV(0) : c1 * d[row];
        const TV dv = dprev + c2 * (invd[row] * r);
        d[row] = dv;
        y[row] = x[row] + dv;
      } else if (MODE == CSR_CHEB0) {
        const TV dv = c2 * (invd[row] * b[row]);
        d[row] = dv;
        y[row] = dv;
      } else {  // CSR_SPMV_DINV_DOT: c2 carries the scale of x
        const TV w = (c2 * invd[row]) * acc;
        y[row] = w;
        dacc += (double)w * (double)w;
      }
    }
  }
  if (MODE == CSR_SPMV_DINV_DOT) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = dacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
      partials[blockIdx.x] = t;
    }
  }
}

// Thread per row for the short rows of the prolongators (a handful of entries each): the
// first kShortWin entries of a row are loaded under predicates, so all of the row's column,
// value and gather loads are in flight at once, and a warp keeps 32 rows in flight.  The
// row is summed in entry order; longer rows finish in a plain loop.
constexpr int kShortWin = 6;

template <class TV, class TM, int MODE>
__global__ void __launch_bounds__(256) csr_short_k(int n, const int* __restrict__ rowptr,
                                                   const int* __restrict__ col,
                                                   const TM* __restrict__ val,
                                                   const TV* __restrict__ x, TV* __restrict__ y) {
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n;
       row += gridDim.x * blockDim.x) {
    const int p0 = rowptr[row], p1 = rowptr[row + 1];
    const TV y0 = MODE == CSR_ADD ? y[row] : TV(0);
    int k[kShortWin];
    TV a[kShortWin];
#pragma unroll
    for (int q = 0; q < kShortWin; ++q) {
      const bool on = p0 + q < p1;
      k[q] = on ? col[p0 + q] : 0;
      a[q] = on ? (TV)ld(val, p0 + q) : TV(0);
    }
    TV acc = TV(0);
#pragma unroll
    for (int q = 0; q < kShortWin; ++q)
      if (p0 + q < p1) acc += a[q] * x[k[q]];
    for (int p = p0 + kShortWin; p < p1; ++p) acc += (TV)ld(val, p) * x[col[p]];
    y[row] = MODE == CSR_ADD ? y0 + acc : acc;
  }
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
    csr_k<TV, TM, G, M><<<blocks, 256, 0, s>>>(n, rowptr, col, val, x, y, b, d, invd, c1, c2, \
                                                partials, xscale);                         \
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
  // the prolongators' short rows on a large level: a thread per row
  if ((mode == CSR_ADD || mode == CSR_SPMV) && avg_nnz <= kShortWin && n >= 100000) {
    const long long need = ((long long)n + 255) / 256;
    const int blocks = (int)(need < sm_count() * 16 ? need : sm_count() * 16);
    if (mode == CSR_ADD)
      csr_short_k<TV, TM, CSR_ADD><<<blocks, 256, 0, s>>>(n, rowptr, col, val, x, y);
    else
      csr_short_k<TV, TM, CSR_SPMV><<<blocks, 256, 0, s>>>(n, rowptr, col, val, x, y);
    SAAMG_LAUNCH();
    return;
  }
  int g = sizeof(TV) == 8 ? (avg_nnz <= 10.0 ? 2 : (avg_nnz <= 48.0 ? 4 : 8))
                          : (avg_nnz <= 6.0 ? 2 : (avg_nnz <= 20.0 ? 4 : (avg_nnz <= 64.0 ? 8 : 16)));
  int gpar = 1;
  while (gpar < 32 && (long long)n * gpar < 150000) gpar <<= 1;
  int glen = 1;
  while (glen < 32 && glen < avg_nnz) glen <<= 1;
  g = std::max(g, std::min(gpar, glen));
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
  convert_k<double, float><<<grid_for(n), 256, 0, s>>>(in, out, n);
  SAAMG_LAUNCH();
}

void to_double(const float* in, double* out, size_t n, cudaStream_t s) {
  if (!n) return;
  convert_k<float, double><<<grid_for(n), 256, 0, s>>>(in, out, n);
  SAAMG_LAUNCH();
}

void to_bf16(const double* in, __nv_bfloat16* out, size_t n, cudaStream_t s) {
  if (!n) return;
  to_bf16_k<<<grid_for(n), 256, 0, s>>>(in, out, n);
  SAAMG_LAUNCH();
}

}  // namespace saamg
