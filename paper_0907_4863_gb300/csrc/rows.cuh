// Per-row and per-block arithmetic shared by the one-solve kernels and their batched forms
// (internal).  Both kinds of launch call these functions, so a row, a partial sum or a CG
// scalar comes out with the same bits whichever launch computes it.
#pragma once

#include "csr.cuh"

namespace saamg {
namespace rows {

__device__ __forceinline__ double ldv(const double* p, size_t i) { return p[i]; }
__device__ __forceinline__ float ldv(const float* p, size_t i) { return p[i]; }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p, size_t i) {
  return __bfloat162float(p[i]);
}

// --- CSR, G lanes per row ---------------------------------------------------------------
// Lane gl of the row's group sums entries gl, gl + G, ... (four loads in flight), the group
// combines its sums with shuffles (all 32 lanes of the warp take part), and lane 0 of the
// group applies MODE.  A row past n (active false) only joins the shuffles.
template <class TV, class TM, int G, int MODE>
__device__ __forceinline__ void csr_group_row(int row, bool active, int gl,
                                              const int* __restrict__ rowptr,
                                              const int* __restrict__ col,
                                              const TM* __restrict__ val,
                                              const TV* __restrict__ x, TV* __restrict__ y,
                                              const TV* __restrict__ b, TV* __restrict__ d,
                                              const TV* __restrict__ invd, TV c1, TV c2,
                                              double& dacc) {
  TV acc = TV(0);
  if (MODE != CSR_CHEB0 && active) {
    const int p0 = rowptr[row], p1 = rowptr[row + 1];
    int p = p0 + gl;
    for (; p + 7 * G < p1; p += 8 * G) {
      int kk[8];
      TV a[8], xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        kk[u] = col[p + u * G];
        a[u] = (TV)ldv(val, p + u * G);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = x[kk[u]];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += a[u] * xv[u];
    }
    for (; p + 3 * G < p1; p += 4 * G) {
      const int k0 = col[p], k1 = col[p + G], k2 = col[p + 2 * G], k3 = col[p + 3 * G];
      const TV a0 = (TV)ldv(val, p), a1 = (TV)ldv(val, p + G), a2 = (TV)ldv(val, p + 2 * G),
               a3 = (TV)ldv(val, p + 3 * G);
      const TV x0 = x[k0], x1 = x[k1], x2 = x[k2], x3 = x[k3];
      acc += a0 * x0;
      acc += a1 * x1;
      acc += a2 * x2;
      acc += a3 * x3;
    }
    for (; p < p1; p += G) acc += (TV)ldv(val, p) * x[col[p]];
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
      // written with explicit fma so that the compiler cannot contract it differently in
      // different kernels (c1 = 0: d is not read)
      const TV t = invd[row] * (b[row] - acc);
      const TV dv = (c1 == TV(0)) ? c2 * t : fma(c2, t, c1 * d[row]);
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

// --- CSR, a thread per short row ------------------------------------------------------------
constexpr int kShortWin = 6;

template <class TV, class TM, int MODE>
__device__ __forceinline__ void csr_short_row(int row, const int* __restrict__ rowptr,
                                              const int* __restrict__ col,
                                              const TM* __restrict__ val,
                                              const TV* __restrict__ x, TV* __restrict__ y) {
  const int p0 = rowptr[row], p1 = rowptr[row + 1];
  const TV y0 = MODE == CSR_ADD ? y[row] : TV(0);
  int k[kShortWin];
  TV a[kShortWin];
#pragma unroll
  for (int q = 0; q < kShortWin; ++q) {
    const bool on = p0 + q < p1;
    k[q] = on ? col[p0 + q] : 0;
    a[q] = on ? (TV)ldv(val, p0 + q) : TV(0);
  }
  TV acc = TV(0);
#pragma unroll
  for (int q = 0; q < kShortWin; ++q)
    if (p0 + q < p1) acc += a[q] * x[k[q]];
  for (int p = p0 + kShortWin; p < p1; ++p) acc += (TV)ldv(val, p) * x[col[p]];
  y[row] = MODE == CSR_ADD ? y0 + acc : acc;
}

// --- SELL-32, a thread per row of slice s ---------------------------------------------------
constexpr int kSellCheb1 = 6;  // CSR_CHEB with c1 = 0: d is not read

template <class TV, class TM, int MODE, bool REL>
__device__ __forceinline__ void sell_row(int s, int lane, int n, const int* __restrict__ perm,
                                         const int* __restrict__ soff,
                                         const int* __restrict__ col,
                                         const short* __restrict__ dcol,
                                         const TM* __restrict__ val, const TV* __restrict__ x,
                                         TV* __restrict__ y, const TV* __restrict__ b,
                                         TV* __restrict__ d, const TV* __restrict__ invd, TV c1,
                                         TV c2, double& dacc) {
  const int p = 32 * s + lane;
  if (p >= n) return;
  const int row = perm[p];
  TV acc = TV(0);
  if (MODE != CSR_CHEB0) {
    const int e0 = soff[s] + lane, w = (soff[s + 1] - soff[s]) >> 5;
    int k = 0;
    // eight independent (column, value, x) loads in flight per lane
    for (; k + 8 <= w; k += 8) {
      const int e = e0 + 32 * k;
      int kk[8];
      TV a[8], xv[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        kk[u] = REL ? row + dcol[e + 32 * u] : col[e + 32 * u];
        a[u] = (TV)ldv(val, e + 32 * u);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) xv[u] = x[kk[u]];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc = fma(a[u], xv[u], acc);
    }
    for (; k + 4 <= w; k += 4) {
      const int e = e0 + 32 * k;
      const int k0 = REL ? row + dcol[e] : col[e];
      const int k1 = REL ? row + dcol[e + 32] : col[e + 32];
      const int k2 = REL ? row + dcol[e + 64] : col[e + 64];
      const int k3 = REL ? row + dcol[e + 96] : col[e + 96];
      const TV a0 = (TV)ldv(val, e), a1 = (TV)ldv(val, e + 32), a2 = (TV)ldv(val, e + 64),
               a3 = (TV)ldv(val, e + 96);
      const TV x0 = x[k0], x1 = x[k1], x2 = x[k2], x3 = x[k3];
      acc = fma(a0, x0, acc);
      acc = fma(a1, x1, acc);
      acc = fma(a2, x2, acc);
      acc = fma(a3, x3, acc);
    }
    for (; k < w; ++k) {
      const int e = e0 + 32 * k;
      acc = fma((TV)ldv(val, e), x[REL ? row + dcol[e] : col[e]], acc);
    }
  }
  if (MODE == CSR_SPMV) {
    y[row] = acc;
  } else if (MODE == CSR_RESID) {
    y[row] = b[row] - acc;
  } else if (MODE == CSR_ADD) {
    y[row] = y[row] + acc;
  } else if (MODE == CSR_CHEB) {
    const TV dv = fma(c1, d[row], c2 * (invd[row] * (b[row] - acc)));
    d[row] = dv;
    y[row] = x[row] + dv;
  } else if (MODE == kSellCheb1) {
    const TV dv = c2 * (invd[row] * (b[row] - acc));
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

// --- coarse solve: row i of the explicit inverse times b, a warp per row -------------------
template <class TV>
__device__ __forceinline__ void gemv_row(int i, int n, int lane, const double* __restrict__ inv,
                                         const TV* __restrict__ b, TV* __restrict__ x) {
  const double* row = inv + (size_t)i * n;
  double acc = 0.0;
  for (int c = lane; c < n; c += 32) acc += row[c] * (double)b[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) x[i] = (TV)acc;
}

// --- reductions -----------------------------------------------------------------------------
// Sum over the block, valid in thread 0 (warp shuffles, then the warps in order).
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;
}

// Single-block ordered sum of kRedBlocks partials (kRedThreads threads), valid in all threads.
__device__ __forceinline__ double sum_fixed(const double* part) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < kRedBlocks; i += blockDim.x) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  double r = sh[0];
  __syncthreads();
  return r;
}

// Block `blk` of a fixed grid of kRedBlocks x kRedThreads: its partial of sum a_i b_i (loads
// of four grid strides in flight, the multiply-adds in index order).  Valid in thread 0.
template <class TA, class TB>
__device__ __forceinline__ double dot_block(int blk, int n, const TA* __restrict__ a,
                                            const TB* __restrict__ b) {
  double acc = 0.0;
  const int st = kRedBlocks * kRedThreads;
  int i = blk * kRedThreads + threadIdx.x;
  for (; i + 3 * st < n; i += 4 * st) {
    const double a0 = (double)a[i], a1 = (double)a[i + st], a2 = (double)a[i + 2 * st],
                 a3 = (double)a[i + 3 * st];
    const double b0 = (double)b[i], b1 = (double)b[i + st], b2 = (double)b[i + 2 * st],
                 b3 = (double)b[i + 3 * st];
    acc += a0 * b0;
    acc += a1 * b1;
    acc += a2 * b2;
    acc += a3 * b3;
  }
  for (; i < n; i += st) acc += (double)a[i] * (double)b[i];
  return block_sum(acc);
}

// r'z and z'q of block `blk` in one sweep; the same per-thread order and block tree as two
// dot_block calls.
template <class TZ>
__device__ __forceinline__ void dot2_block(int blk, int n, const double* __restrict__ r,
                                           const TZ* __restrict__ z,
                                           const double* __restrict__ q, double& t1,
                                           double& t2) {
  double a1 = 0.0, a2 = 0.0;
  const int st = kRedBlocks * kRedThreads;
  int i = blk * kRedThreads + threadIdx.x;
  // loads of four grid strides in flight (the fixed grid holds half the warps an SM can)
  for (; i + 3 * st < n; i += 4 * st) {
    double zz[4], rr[4], qq[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      zz[u] = (double)z[i + u * st];
      rr[u] = r[i + u * st];
      qq[u] = q[i + u * st];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a1 += rr[u] * zz[u];
      a2 += zz[u] * qq[u];
    }
  }
  for (; i < n; i += st) {
    const double zi = (double)z[i];
    a1 += r[i] * zi;
    a2 += zi * q[i];
  }
  t1 = block_sum(a1);
  __syncthreads();  // block_sum's shared array is reused
  t2 = block_sum(a2);
}

// x += alpha p; r -= alpha q; r32 = (float) r; block `blk`'s partial of r'r (thread 0).
__device__ __forceinline__ double update_block(int blk, int n, double a, double* __restrict__ x,
                                               double* __restrict__ r,
                                               const double* __restrict__ p,
                                               const double* __restrict__ q,
                                               float* __restrict__ r32) {
  double acc = 0.0;
  const int st = kRedBlocks * kRedThreads;
  int i = blk * kRedThreads + threadIdx.x;
  // two grid strides per step, every load before the stores
  for (; i + st < n; i += 2 * st) {
    const double x0 = x[i], x1 = x[i + st], p0 = p[i], p1 = p[i + st];
    const double rv0 = r[i], rv1 = r[i + st], q0 = q[i], q1 = q[i + st];
    x[i] = x0 + a * p0;
    const double ri0 = rv0 - a * q0;
    r[i] = ri0;
    if (r32) r32[i] = (float)ri0;
    acc += ri0 * ri0;
    x[i + st] = x1 + a * p1;
    const double ri1 = rv1 - a * q1;
    r[i + st] = ri1;
    if (r32) r32[i + st] = (float)ri1;
    acc += ri1 * ri1;
  }
  for (; i < n; i += st) {
    x[i] = x[i] + a * p[i];
    double ri = r[i] - a * q[i];
    r[i] = ri;
    if (r32) r32[i] = (float)ri;
    acc += ri * ri;
  }
  return block_sum(acc);
}

// --- the same blocks emulated by one warp ---------------------------------------------------
// A warp can stand in for a block of kRedThreads = 8 x 32 threads: lane l runs the loops of
// the block's threads 32 w + l (w = 0..7, the block's warps) one after the other with its own
// accumulator each, every accumulator is reduced by the warp's xor tree (the block's per-warp
// reduction), and the eight sums are added in warp order (the block's final loop).  The
// result has the bits of the block's partial, in every lane, without shared memory or
// barriers, and eight of these run side by side in a block.
constexpr int kVirtWarps = kRedThreads / 32;

__device__ __forceinline__ double warp_tree(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class TA, class TB>
__device__ __forceinline__ double dot_block_warp(int blk, int n, const TA* __restrict__ a,
                                                 const TB* __restrict__ b, int lane) {
  const int st = kRedBlocks * kRedThreads;
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kVirtWarps; ++w) {
    double acc = 0.0;
    int i = blk * kRedThreads + 32 * w + lane;
    for (; i + 3 * st < n; i += 4 * st) {
      const double a0 = (double)a[i], a1 = (double)a[i + st], a2 = (double)a[i + 2 * st],
                   a3 = (double)a[i + 3 * st];
      const double b0 = (double)b[i], b1 = (double)b[i + st], b2 = (double)b[i + 2 * st],
                   b3 = (double)b[i + 3 * st];
      acc += a0 * b0;
      acc += a1 * b1;
      acc += a2 * b2;
      acc += a3 * b3;
    }
    for (; i < n; i += st) acc += (double)a[i] * (double)b[i];
    t += warp_tree(acc);
  }
  return t;
}

template <class TZ>
__device__ __forceinline__ void dot2_block_warp(int blk, int n, const double* __restrict__ r,
                                                const TZ* __restrict__ z,
                                                const double* __restrict__ q, int lane,
                                                double& t1, double& t2) {
  const int st = kRedBlocks * kRedThreads;
  t1 = 0.0;
  t2 = 0.0;
#pragma unroll
  for (int w = 0; w < kVirtWarps; ++w) {
    double a1 = 0.0, a2 = 0.0;
    int i = blk * kRedThreads + 32 * w + lane;
    for (; i + st < n; i += 2 * st) {
      const double z0 = (double)z[i], z1 = (double)z[i + st];
      const double r0 = r[i], r1 = r[i + st], q0 = q[i], q1 = q[i + st];
      a1 += r0 * z0;
      a2 += z0 * q0;
      a1 += r1 * z1;
      a2 += z1 * q1;
    }
    for (; i < n; i += st) {
      const double zi = (double)z[i];
      a1 += r[i] * zi;
      a2 += zi * q[i];
    }
    t1 += warp_tree(a1);
    t2 += warp_tree(a2);
  }
}

__device__ __forceinline__ double update_block_warp(int blk, int n, double a,
                                                    double* __restrict__ x,
                                                    double* __restrict__ r,
                                                    const double* __restrict__ p,
                                                    const double* __restrict__ q,
                                                    float* __restrict__ r32, int lane) {
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kVirtWarps; ++w) {
    double acc = 0.0;
    for (int i = blk * kRedThreads + 32 * w + lane; i < n; i += kRedBlocks * kRedThreads) {
      x[i] = x[i] + a * p[i];
      double ri = r[i] - a * q[i];
      r[i] = ri;
      if (r32) r32[i] = (float)ri;
      acc += ri * ri;
    }
    t += warp_tree(acc);
  }
  return t;
}

}  // namespace rows
}  // namespace saamg
