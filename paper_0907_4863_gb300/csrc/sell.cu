// SELL-32-sigma kernels: layout construction from CSR and the V-cycle operations on it
// (Chebyshev step fused with the residual, residual, y = A x, y += A x).
#include "sell.cuh"
#include "rows.cuh"

namespace saamg {

namespace {

using rows::kSellCheb1;

// Block per window: stable rank of each row by decreasing length, from the window's
// lengths in shared memory.
__global__ void __launch_bounds__(kSellWindow) sell_rank_k(int n, const int* __restrict__ rowptr,
                                                           int* __restrict__ perm) {
  __shared__ int len[kSellWindow];
  const int t = threadIdx.x;
  const int base = blockIdx.x * kSellWindow;
  const int row = base + t;
  const int L = row < n ? rowptr[row + 1] - rowptr[row] : -1;
  len[t] = L;
  __syncthreads();
  if (row >= n) return;
  int r = 0;
  for (int j = 0; j < kSellWindow; ++j) {
    const int lj = len[j];
    r += (lj > L) | ((lj == L) & (j < t));
  }
  perm[base + r] = row;
}

// Entries of each slice: 32 x the length of its first (longest) row; windows hold whole
// slices, so a slice never mixes two windows.
__global__ void sell_width_k(int nslices, const int* __restrict__ rowptr,
                             const int* __restrict__ perm, int* __restrict__ size) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > nslices) return;
  if (s == nslices) {
    size[s] = 0;
    return;
  }
  const int r = perm[32 * s];
  size[s] = 32 * (rowptr[r + 1] - rowptr[r]);
}

__global__ void sell_fill_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                            const double* __restrict__ val, const int* __restrict__ perm,
                            const int* __restrict__ soff, int* __restrict__ scol,
                            short* __restrict__ sdcol, int* __restrict__ wide,
                            double* __restrict__ sval, float* __restrict__ sval32,
                            __nv_bfloat16* __restrict__ sval16) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int r = perm[p], s = p >> 5, lane = p & 31;
  const int w = (soff[s + 1] - soff[s]) >> 5;
  const int p0 = rowptr[r], len = rowptr[r + 1] - p0;
  const int padc = len > 0 ? col[p0 + len - 1] : 0;
  bool far = false;
  for (int k = 0; k < w; ++k) {
    const int e = soff[s] + 32 * k + lane;
    const bool real = k < len;
    const double v = real ? val[p0 + k] : 0.0;
    const int c = real ? col[p0 + k] : padc;
    scol[e] = c;
    const int d = c - r;
    far |= d < -32767 || d > 32767;
    sdcol[e] = (short)(far ? 0 : d);
    if (sval) sval[e] = v;
    if (sval32) sval32[e] = (float)v;
    if (sval16) sval16[e] = __double2bfloat16(v);
  }
  if (far) atomicOr(wide, 1);
}

// The value arrays of a layout whose structure is already in place (as sell_fill_k writes them).
__global__ void sell_values_k(int n, const int* __restrict__ rowptr, const double* __restrict__ val,
                              const int* __restrict__ perm, const int* __restrict__ soff,
                              double* __restrict__ sval, float* __restrict__ sval32,
                              __nv_bfloat16* __restrict__ sval16) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int r = perm[p], s = p >> 5, lane = p & 31;
  const int w = (soff[s + 1] - soff[s]) >> 5;
  const int p0 = rowptr[r], len = rowptr[r + 1] - p0;
  for (int k = 0; k < w; ++k) {
    const int e = soff[s] + 32 * k + lane;
    const double v = k < len ? val[p0 + k] : 0.0;
    if (sval) sval[e] = v;
    if (sval32) sval32[e] = (float)v;
    if (sval16) sval16[e] = __double2bfloat16(v);
  }
}

template <class TV, class TM, int MODE, bool REL>
__global__ void __launch_bounds__(256) sell_k(int n, int nslices, const int* __restrict__ perm,
                                              const int* __restrict__ soff,
                                              const int* __restrict__ col,
                                              const short* __restrict__ dcol,
                                              const TM* __restrict__ val, const TV* __restrict__ x,
                                              TV* __restrict__ y, const TV* __restrict__ b,
                                              TV* __restrict__ d, const TV* __restrict__ invd,
                                              TV c1, TV c2, double* __restrict__ partials,
                                              const double* __restrict__ xscale) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  double dacc = 0.0;
  if (MODE == CSR_SPMV_DINV_DOT) c2 = xscale ? (TV)*xscale : TV(1);
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < nslices; s += nw)
    rows::sell_row<TV, TM, MODE, REL>(s, lane, n, perm, soff, col, dcol, val, x, y, b, d, invd,
                                      c1, c2, dacc);
  if (MODE == CSR_SPMV_DINV_DOT) {  // fixed grid of kRedBlocks: the same partial sums every run
    const double t = rows::block_sum(dacc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

}  // namespace

void sell_from_csr(const DevCsr& A, DevSell& S, bool f64, bool f32, bool bf16, cudaStream_t s) {
  S.n = A.n;
  S.m = A.m;
  S.nnz = A.nnz;
  S.nslices = (A.n + 31) / 32;
  S.perm.alloc(A.n, s);
  S.soff.alloc(S.nslices + 1, s);
  if (A.n == 0) {
    fill_int(S.soff.p, 0, 1, s);
    S.nent = 0;
    S.col.alloc(0, s);
    return;
  }
  const int nwin = (A.n + kSellWindow - 1) / kSellWindow;
  sell_rank_k<<<nwin, kSellWindow, 0, s>>>(A.n, A.rowptr.p, S.perm.p);
  SAAMG_LAUNCH();
  Buf<int> size;
  size.alloc(S.nslices + 1, s);
  sell_width_k<<<(S.nslices + 1 + 255) / 256, 256, 0, s>>>(S.nslices, A.rowptr.p, S.perm.p,
                                                           size.p);
  SAAMG_LAUNCH();
  const long long nent = exclusive_scan(size.p, S.soff.p, S.nslices + 1, s);
  if (nent > 0x7fffffffLL) fail(SAAMG_EINVAL, "SELL layout above 2^31 entries");
  S.nent = nent;
  S.col.alloc(nent, s);
  S.dcol.alloc(nent, s);
  if (f64) S.val.alloc(nent, s);
  if (f32) S.val32.alloc(nent, s);
  if (bf16) S.val16.alloc(nent, s);
  Buf<int> wide;
  wide.alloc(1, s);
  fill_int(wide.p, 0, 1, s);
  sell_fill_k<<<(A.n + 255) / 256, 256, 0, s>>>(A.n, A.rowptr.p, A.col.p, A.val.p, S.perm.p,
                                                S.soff.p, S.col.p, S.dcol.p, wide.p,
                                                f64 ? S.val.p : nullptr,
                                                f32 ? S.val32.p : nullptr,
                                                bf16 ? S.val16.p : nullptr);
  SAAMG_LAUNCH();
  int hw = 0;
  d2h_sync(&hw, wide.p, sizeof(int), s);
  if (hw) {  // some column is more than 32767 rows away: 32-bit columns
    S.dcol.release();
    S.index_bytes = 4;
  } else {
    S.col.release();
    S.index_bytes = 2;
  }
}

void sell_like(const DevCsr& A, const DevSell& like, DevSell& S, bool f64, bool f32, bool bf16,
               cudaStream_t s) {
  if (like.n != A.n || like.nnz != A.nnz) fail(SAAMG_EINVAL, "SELL layout of another pattern");
  S.n = A.n;
  S.m = A.m;
  S.nnz = A.nnz;
  S.nslices = like.nslices;
  S.nent = like.nent;
  S.index_bytes = like.index_bytes;
  auto copy = [&](auto& dst, const auto& src, size_t count) {
    dst.alloc(count, s);
    if (count)
      SAAMG_CUDA(cudaMemcpyAsync(dst.p, src.p, count * sizeof(*src.p), cudaMemcpyDeviceToDevice,
                                 s));
  };
  copy(S.perm, like.perm, (size_t)A.n);
  copy(S.soff, like.soff, (size_t)like.nslices + 1);
  if (like.index_bytes == 2) copy(S.dcol, like.dcol, (size_t)like.nent);
  else copy(S.col, like.col, (size_t)like.nent);
  if (f64) S.val.alloc(S.nent, s);
  if (f32) S.val32.alloc(S.nent, s);
  if (bf16) S.val16.alloc(S.nent, s);
  if (A.n == 0) return;
  sell_values_k<<<(A.n + 255) / 256, 256, 0, s>>>(A.n, A.rowptr.p, A.val.p, S.perm.p, S.soff.p,
                                                  f64 ? S.val.p : nullptr,
                                                  f32 ? S.val32.p : nullptr,
                                                  bf16 ? S.val16.p : nullptr);
  SAAMG_LAUNCH();
}

template <class TV, class TM>
void sell_apply(int mode, const DevSell& S, const TM* val, const TV* x, TV* y, const TV* b,
                TV* d, const TV* invd, TV c1, TV c2, cudaStream_t s, int kclass,
                double* partials, const double* xscale) {
  if (S.n <= 0) {
    if (mode == CSR_SPMV_DINV_DOT) fill_double(partials, 0.0, kRedBlocks, s);
    return;
  }
  KernelTimer kt(kclass, S.nnz, s);  // timing unit of the SELL classes: matrix entries
  if (mode == CSR_CHEB && c1 == TV(0)) mode = kSellCheb1;
  const long long need = ((long long)S.nslices + 7) / 8;
  const int blocks =
      mode == CSR_SPMV_DINV_DOT ? kRedBlocks : (int)(need < sm_count() * 16 ? need : sm_count() * 16);
#define SAAMG_SELL_CASE(M)                                                                    \
  case M:                                                                                     \
    if (S.index_bytes == 2)                                                                   \
      launch_pdl(sell_k<TV, TM, M, true>, blocks, 256, 0, s, S.n, S.nslices, S.perm.p,       \
                 S.soff.p, nullptr, S.dcol.p, val, x, y, b, d, invd, c1, c2, partials,        \
                 xscale);                                                                     \
    else                                                                                      \
      launch_pdl(sell_k<TV, TM, M, false>, blocks, 256, 0, s, S.n, S.nslices, S.perm.p,      \
                 S.soff.p, S.col.p, nullptr, val, x, y, b, d, invd, c1, c2, partials,         \
                 xscale);                                                                     \
    break;
  switch (mode) {
    SAAMG_SELL_CASE(CSR_SPMV)
    SAAMG_SELL_CASE(CSR_RESID)
    SAAMG_SELL_CASE(CSR_CHEB)
    SAAMG_SELL_CASE(CSR_CHEB0)
    SAAMG_SELL_CASE(CSR_ADD)
    SAAMG_SELL_CASE(kSellCheb1)
    SAAMG_SELL_CASE(CSR_SPMV_DINV_DOT)
    default:
      fail(SAAMG_EINVAL, "bad SELL mode");
  }
#undef SAAMG_SELL_CASE
  SAAMG_LAUNCH();
}

template void sell_apply<double, double>(int, const DevSell&, const double*, const double*,
                                         double*, const double*, double*, const double*, double,
                                         double, cudaStream_t, int, double*, const double*);
template void sell_apply<float, float>(int, const DevSell&, const float*, const float*, float*,
                                       const float*, float*, const float*, float, float,
                                       cudaStream_t, int, double*, const double*);
template void sell_apply<float, __nv_bfloat16>(int, const DevSell&, const __nv_bfloat16*,
                                               const float*, float*, const float*, float*,
                                               const float*, float, float, cudaStream_t, int,
                                               double*, const double*);

}  // namespace saamg
