// Matrix-free level-0 operator: the 7-point star of Eq. (6) with the boundary rows of
// Sec. 2, scaled by D^-1/2 on both sides, applied on compact vectors.
//
// One warp per chunk of <= 32 consecutive unknowns of one x-line.  The x-neighbours are
// the adjacent compact rows; the y- and z-neighbours of lane i are the rows start' +
// (i - lo') of the neighbouring lines, so every warp load is a contiguous run.  Rows
// inside the line's regular run use the four interior coefficients held in registers;
// the remaining rows (near-boundary rows and their neighbours, about 5-8 % of all
// rows) read their 7 coefficients and 1/diag from the table.
#include "operator.cuh"

namespace saamg {

namespace {

template <class T>
__device__ __forceinline__ double to_d(T v) {
  return (double)v;
}

// One row of chunk c for this lane (x, b and the metadata are read-only; y and d are written).
template <class T, int MODE>
__device__ __forceinline__ void stencil_row(const StencilDev<T>& S, int c, int lane,
                                            const T* __restrict__ x, T* __restrict__ y,
                                            const T* __restrict__ b, T* __restrict__ d, T c1,
                                            T c2, T c2invd0, double& dacc) {
    const int2 ch = S.chunks[c];
    const int L = ch.x;
    const LineInfo me = S.lines[L];
    const int i = me.lo + ch.y + lane;
    if (i > me.hi) return;
    const int row = me.start + ch.y + lane;
    const bool reg = (i >= me.rlo) && (i <= me.rhi);
    T invd;
    const T* tb = nullptr;
    if (reg) {
      invd = S.invd0;
    } else {
      const int t = me.tstart + (i < me.rlo ? i - me.lo : (me.rlo - me.lo) + (i - me.rhi - 1));
      tb = S.table + 8 * (size_t)t;
      invd = tb[7];
    }
    if (MODE == ST_CHEB0) {
      T dv = (reg ? c2invd0 : c2 * invd) * b[row];
      d[row] = dv;
      y[row] = dv;
      return;
    }
    const T xc = x[row];
    // SPMV modes accumulate A x; RESID / CHEB accumulate r = b - A x directly (FP64 issue
    // slots bound this kernel in double precision, so every add is folded into an FMA)
    constexpr bool kResid = (MODE == ST_RESID || MODE == ST_CHEB || MODE == ST_CHEB1);
    T acc;
    if (reg) {
      // all six neighbours are unknowns
      const LineInfo ym = S.lines[L - 1], yp = S.lines[L + 1];
      const LineInfo zm = S.lines[L - S.ny], zp = S.lines[L + S.ny];
      const T sx = x[row - 1] + x[row + 1];
      const T sy = x[ym.start + (i - ym.lo)] + x[yp.start + (i - yp.lo)];
      const T sz = x[zm.start + (i - zm.lo)] + x[zp.start + (i - zp.lo)];
      if (kResid) {
        acc = fma(-S.c0, xc, b[row]);
        acc = fma(-S.cx, sx, acc);
        acc = fma(-S.cy, sy, acc);
        acc = fma(-S.cz, sz, acc);
      } else {
        acc = S.c0 * xc;
        acc = fma(S.cx, sx, acc);
        acc = fma(S.cy, sy, acc);
        acc = fma(S.cz, sz, acc);
      }
    } else {
      const int j = L % S.ny, k = L / S.ny;  // only boundary rows need the line's (j, k)
      acc = tb[0] * xc;
      if (i - 1 >= me.lo) acc = fma(tb[1], x[row - 1], acc);
      if (i + 1 <= me.hi) acc = fma(tb[2], x[row + 1], acc);
      if (j > 0) {
        const LineInfo l = S.lines[L - 1];
        if (i >= l.lo && i <= l.hi) acc = fma(tb[3], x[l.start + (i - l.lo)], acc);
      }
      if (j < S.ny - 1) {
        const LineInfo l = S.lines[L + 1];
        if (i >= l.lo && i <= l.hi) acc = fma(tb[4], x[l.start + (i - l.lo)], acc);
      }
      if (k > 0) {
        const LineInfo l = S.lines[L - S.ny];
        if (i >= l.lo && i <= l.hi) acc = fma(tb[5], x[l.start + (i - l.lo)], acc);
      }
      if (k < S.nz - 1) {
        const LineInfo l = S.lines[L + S.ny];
        if (i >= l.lo && i <= l.hi) acc = fma(tb[6], x[l.start + (i - l.lo)], acc);
      }
      if (kResid) acc = b[row] - acc;
    }
    if (MODE == ST_DINV_DOT) {
      const T w = invd * acc;
      y[row] = w;
      dacc = fma(to_d(w), to_d(w), dacc);
    } else if (MODE == ST_SPMV || MODE == ST_SPMV_DOT) {
      y[row] = acc;
      if (MODE == ST_SPMV_DOT) dacc = fma(to_d(xc), to_d(acc), dacc);
    } else if (MODE == ST_RESID) {
      y[row] = acc;
    } else {  // ST_CHEB / ST_CHEB1: d = c1 d + c2 D^-1 r; x_out = x + d
      const T c2i = reg ? c2invd0 : c2 * invd;
      const T dv = (MODE == ST_CHEB1) ? acc * c2i : fma(c1, d[row], acc * c2i);
      d[row] = dv;
      y[row] = xc + dv;
    }
}

// K chunks per warp iteration: the unrolled copies let the read-only loads of the next chunk
// be issued before the stores of the current one (more bytes in flight per warp).
template <class T, int MODE, int K>
__global__ void __launch_bounds__(256) stencil_k(StencilDev<T> S, const T* __restrict__ x,
                                                 T* __restrict__ y, const T* __restrict__ b,
                                                 T* __restrict__ d, T c1, T c2,
                                                 double* __restrict__ partials) {
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int nw = gridDim.x * wpb;
  const T c2invd0 = c2 * S.invd0;
  double dacc = 0.0;
  for (int c0 = (blockIdx.x * wpb + (threadIdx.x >> 5)) * K; c0 < S.nchunks; c0 += nw * K) {
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (c0 + k < S.nchunks)
        stencil_row<T, MODE>(S, c0 + k, lane, x, y, b, d, c1, c2, c2invd0, dacc);
  }
  if (MODE == ST_SPMV_DOT || MODE == ST_DINV_DOT) {
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
    if (lane == 0) sh[threadIdx.x >> 5] = dacc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < wpb; ++w) t += sh[w];
      partials[blockIdx.x] = t;
    }
  }
}

// chunks per warp iteration: FP32 is latency/HBM-bound and gains from more loads in flight;
// FP64 is bound by FP64 issue and keeps one
template <class T>
constexpr int kChunks() {
  return sizeof(T) == 4 ? 2 : 1;
}

}  // namespace

template <class T>
void stencil_apply(const StencilDev<T>& S, int mode, const T* x, T* y, const T* b, T* d, T c1,
                   T c2, double* partials, cudaStream_t s) {
  if (S.nchunks == 0) {
    if (mode == ST_SPMV_DOT || mode == ST_DINV_DOT) fill_double(partials, 0.0, kRedBlocks, s);
    return;
  }
  // the smoother class holds only the full Chebyshev step (fixed work per row); the
  // other modes of the same kernel are timed as "apply"
  // one timing class per kind of pass (each has a fixed amount of work per row)
  KernelTimer kt(mode == ST_CHEB                           ? SAAMG_KT_STENCIL_SMOOTH
                 : (mode == ST_SPMV || mode == ST_SPMV_DOT) ? SAAMG_KT_STENCIL_APPLY
                 : mode == ST_RESID                         ? SAAMG_KT_STENCIL_RESID
                 : (mode == ST_CHEB0 || mode == ST_CHEB1)   ? SAAMG_KT_STENCIL_FIRST
                                                            : -1,
                 S.n, s);
  // Reductions use the fixed grid so that partial sums are always taken the same way.
  int blocks = kRedBlocks;
  if (mode != ST_SPMV_DOT && mode != ST_DINV_DOT) {
    long long need = ((long long)S.nchunks + 8 * kChunks<T>() - 1) / (8 * kChunks<T>());
    blocks = (int)(need < 152 * 16 ? need : 152 * 16);
  }
  switch (mode) {
    case ST_SPMV:
      stencil_k<T, ST_SPMV, kChunks<T>()><<<blocks, 256, 0, s>>>(S, x, y, b, d, c1, c2, partials);
      break;
    case ST_SPMV_DOT:
      stencil_k<T, ST_SPMV_DOT, kChunks<T>()><<<blocks, 256, 0, s>>>(S, x, y, b, d, c1, c2, partials);
      break;
    case ST_RESID:
      stencil_k<T, ST_RESID, kChunks<T>()><<<blocks, 256, 0, s>>>(S, x, y, b, d, c1, c2, partials);
      break;
    case ST_CHEB:
      stencil_k<T, ST_CHEB, kChunks<T>()><<<blocks, 256, 0, s>>>(S, x, y, b, d, c1, c2, partials);
      break;
    case ST_CHEB0:
      stencil_k<T, ST_CHEB0, kChunks<T>()><<<blocks, 256, 0, s>>>(S, x, y, b, d, c1, c2, partials);
      break;
    case ST_CHEB1:
      stencil_k<T, ST_CHEB1, kChunks<T>()><<<blocks, 256, 0, s>>>(S, x, y, b, d, c1, c2, partials);
      break;
    case ST_DINV_DOT:
      stencil_k<T, ST_DINV_DOT, kChunks<T>()><<<blocks, 256, 0, s>>>(S, x, y, b, d, c1, c2, partials);
      break;
    default:
      fail(SAAMG_EINVAL, "bad stencil mode");
  }
  SAAMG_LAUNCH();
}

template void stencil_apply<double>(const StencilDev<double>&, int, const double*, double*,
                                    const double*, double*, double, double, double*,
                                    cudaStream_t);
template void stencil_apply<float>(const StencilDev<float>&, int, const float*, float*,
                                   const float*, float*, float, float, double*, cudaStream_t);

}  // namespace saamg
