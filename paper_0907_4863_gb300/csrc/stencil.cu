// Matrix-free level-0 operator: the 7-point star of Eq. (6) with the boundary rows of
// Sec. 2, scaled by D^-1/2 on both sides, applied on compact vectors.
//
// The x-neighbours of a row are the adjacent compact rows; its y- and z-neighbours are at a
// fixed offset per pair of lines (row + (start' - lo') - (start - lo)), so the loads of
// consecutive rows are contiguous runs.  Rows inside the line's regular run use the four
// interior coefficients held in registers; the remaining rows (near-boundary rows and their
// neighbours, about 5-8 % of all rows) read their 7 coefficients and 1/diag from the table.
// FP32 passes: one warp per chunk of <= 32 consecutive unknowns of one x-line.  FP64 passes
// (bound by FP64 issue): first 32 regular-run rows per warp from a (row, line) list, then
// 32 table rows per warp from the table-row list.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "operator.cuh"
#include "batch.cuh"
#include "rows.cuh"

namespace saamg {

namespace {

template <class T>
__device__ __forceinline__ double to_d(T v) {
  return (double)v;
}

// Bit test for a nonzero coefficient with integer instructions only (the FP64 pipe is the
// bottleneck of the double-precision kernel).
__device__ __forceinline__ bool nonzero(double v) {
  return (static_cast<unsigned long long>(__double_as_longlong(v)) << 1) != 0ull;
}
__device__ __forceinline__ bool nonzero(float v) { return (__float_as_uint(v) << 1) != 0u; }

// The 8 table entries of one row (64 B in double, 32 B in float, aligned to their size).
__device__ __forceinline__ void load8(const double* p, double v[8]) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const double2 t = q[k];
    v[2 * k] = t.x;
    v[2 * k + 1] = t.y;
  }
}
__device__ __forceinline__ void load8(const float* p, float v[8]) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const float4 t = q[k];
    v[4 * k] = t.x;
    v[4 * k + 1] = t.y;
    v[4 * k + 2] = t.z;
    v[4 * k + 3] = t.w;
  }
}

// One row of chunk c for this lane (x, b and the metadata are read-only; y and d are written).
// Every row runs the same seven-term arithmetic: a regular row takes the interior
// coefficients and the line's neighbour offsets; a table row (only its selection below
// diverges, and it holds no floating-point work) takes its own coefficients, and a missing
// neighbour (coefficient 0) points at the row itself.
// PACKED: chunk c is entries [32 c, 32 c + 32) of the list of regular-run rows, each lane
// finding its own line (no lane idles at the end of a line or on a table row); chunk c of the
// TABLE phase is the table rows [32 c, 32 c + 32), so no warp runs both kinds of row.
// Otherwise chunk c is the chunk record c.
template <class T, int MODE, bool PACKED, bool TABLE = false>
__device__ __forceinline__ void stencil_row(const StencilDev<T>& S, int c, int lane,
                                            const T* __restrict__ x, T* __restrict__ y,
                                            const T* __restrict__ b, T* __restrict__ d, T c1,
                                            T c2, T c2invd0, double& dacc,
                                            const int* __restrict__ agg) {
    int row;
    int ra = 0, rb = 0, tl = 0;  // chunk path: lanes of the regular run, table row of lane 0
    int4 nb;
    int t = -1;  // table row, if any
    if (TABLE) {
      t = 32 * c + lane;
      if (t >= S.ntable) return;
      row = S.trow[t];
      nb = S.nbr[S.rline[row]];
    } else if (PACKED) {
      const int k = 32 * c + lane;
      if (k >= S.nrun) return;
      const int2 rl = S.rrow[k];
      row = rl.x;
      nb = S.nbr[rl.y];
    } else {
      // the record as two 16-byte loads: (row0, tl, a | b << 16, n), then the offsets
      const int4* q = reinterpret_cast<const int4*>(S.crec + c);
      const int4 h0 = q[0];
      nb = q[1];
      if (lane >= h0.w) return;
      row = h0.x + lane;
      tl = h0.y;
      ra = (int)(short)(h0.z & 0xffff);
      rb = h0.z >> 16;
    }
    T a0 = S.c0, axm = S.cx, axp = S.cx, aym = S.cy, ayp = S.cy, azm = S.cz, azp = S.cz;
    T c2i = c2invd0;
    int oxm = -1, oxp = 1, oym = nb.x, oyp = nb.y, ozm = nb.z, ozp = nb.w;
    if (!TABLE && !PACKED && (lane < ra || lane > rb))
      t = tl + lane + (lane < ra ? 0 : ra - rb - 1);
    if (TABLE || (!PACKED && t >= 0)) {
      T tb[8];
      load8(S.table + 8 * (size_t)t, tb);
      a0 = tb[0];
      axm = tb[1];
      axp = tb[2];
      aym = tb[3];
      ayp = tb[4];
      azm = tb[5];
      azp = tb[6];
      c2i = c2 * tb[7];
      oxm = nonzero(axm) ? oxm : 0;
      oxp = nonzero(axp) ? oxp : 0;
      oym = nonzero(aym) ? oym : 0;
      oyp = nonzero(ayp) ? oyp : 0;
      ozm = nonzero(azm) ? ozm : 0;
      ozp = nonzero(azp) ? ozp : 0;
    }
    if (MODE == ST_CHEB0) {
      const T dv = c2i * b[row];
      d[row] = dv;
      y[row] = dv;
      return;
    }
    T xc, vxm, vxp, vym, vyp, vzm, vzp;
    if (MODE == ST_PROLONG) {  // x is the coarse vector, read through the aggregates: (T v)_j
      const int* ar = agg + row;
      xc = x[ar[0]];
      vxm = x[ar[oxm]];
      vxp = x[ar[oxp]];
      vym = x[ar[oym]];
      vyp = x[ar[oyp]];
      vzm = x[ar[ozm]];
      vzp = x[ar[ozp]];
    } else if (PACKED && !TABLE && (reinterpret_cast<uintptr_t>(x) & (2 * sizeof(T) - 1)) == 0) {
      // a regular-run row has both x-neighbours: x[row - 1 .. row + 1] as one aligned pair and
      // one single element (two loads for the same three values)
      using T2 = typename std::conditional<sizeof(T) == 8, double2, float2>::type;
      const T2 v = *reinterpret_cast<const T2*>(x + (row & ~1));
      const bool odd = (row & 1) != 0;
      const T v1 = x[odd ? row + 1 : row - 1];
      vxm = odd ? v.x : v1;
      xc = odd ? v.y : v.x;
      vxp = odd ? v1 : v.y;
      const T* xr = x + row;
      vym = xr[oym];
      vyp = xr[oyp];
      vzm = xr[ozm];
      vzp = xr[ozp];
    } else {
      const T* xr = x + row;
      xc = xr[0];
      vxm = xr[oxm];
      vxp = xr[oxp];
      vym = xr[oym];
      vyp = xr[oyp];
      vzm = xr[ozm];
      vzp = xr[ozp];
    }
    // SPMV modes accumulate A x; RESID / CHEB accumulate r = b - A x directly (one FMA per
    // term: FP64 issue slots bound this kernel in double precision)
    constexpr bool kResid = (MODE == ST_RESID || MODE == ST_CHEB || MODE == ST_CHEB1);
    T acc;
    if (kResid) {
      acc = fma(-a0, xc, b[row]);
      acc = fma(-axm, vxm, acc);
      acc = fma(-axp, vxp, acc);
      acc = fma(-aym, vym, acc);
      acc = fma(-ayp, vyp, acc);
      acc = fma(-azm, vzm, acc);
      acc = fma(-azp, vzp, acc);
    } else {
      acc = a0 * xc;
      acc = fma(axm, vxm, acc);
      acc = fma(axp, vxp, acc);
      acc = fma(aym, vym, acc);
      acc = fma(ayp, vyp, acc);
      acc = fma(azm, vzm, acc);
      acc = fma(azp, vzp, acc);
    }
    if (MODE == ST_DINV_DOT) {  // c2 carries the scale of x: w = c2 D^-1 A x
      const T w = c2i * acc;
      y[row] = w;
      dacc = fma(to_d(w), to_d(w), dacc);
    } else if (MODE == ST_SPMV || MODE == ST_SPMV_DOT) {
      y[row] = acc;
      if (MODE == ST_SPMV_DOT) dacc = fma(to_d(xc), to_d(acc), dacc);
    } else if (MODE == ST_RESID) {
      y[row] = acc;
    } else if (MODE == ST_PROLONG) {  // c2 = omega: y += (T v)_i - omega invd_i (A T v)_i
      y[row] = y[row] + fma(-c2i, acc, xc);
    } else {  // ST_CHEB / ST_CHEB1: d = c1 d + c2 D^-1 r; x_out = x + d
      const T dv = (MODE == ST_CHEB1) ? acc * c2i : fma(c1, d[row], acc * c2i);
      d[row] = dv;
      y[row] = xc + dv;
    }
}

// The FP64 passes are bound by FP64 issue, where an idle lane costs as much as a busy one: they
// take 32 regular-run rows per warp across line ends (one more 8-byte load per row: the row
// and its line), and the table rows 32 at a time in a second phase, so that no lane idles and
// no warp issues the table rows' extra multiply for a few lanes; the latency-bound FP32
// passes keep the line chunks.
template <class T>
__host__ __device__ constexpr bool packed_rows() {
  return sizeof(T) == 8;
}

// K chunks per warp iteration: the unrolled copies let the read-only loads of the next chunk
// be issued before the stores of the current one (more bytes in flight per warp).
template <class T, int MODE, int K, bool PACKED>
__global__ void __launch_bounds__(256) stencil_k(StencilDev<T> S, const T* __restrict__ x,
                                                 T* __restrict__ y, const T* __restrict__ b,
                                                 T* __restrict__ d, T c1, T c2, T c2invd0,
                                                 double* __restrict__ partials,
                                                 const double* __restrict__ xscale,
                                                 const int* __restrict__ agg) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const int nw = gridDim.x * wpb;
  if (MODE == ST_DINV_DOT) {
    c2 = xscale ? (T)*xscale : T(1);
    c2invd0 = c2 * S.invd0;
  }
  double dacc = 0.0;
  constexpr bool kPacked = PACKED;
  // packed: the regular-run chunks, then the table chunks (the branch is uniform per warp)
  const int nreg = kPacked ? (S.nrun + 31) / 32 : S.nchunks;
  const int nch = kPacked ? nreg + (S.ntable + 31) / 32 : nreg;
  // the reductions' fixed grid holds half the warps an SM can: there a step takes two grid
  // strides (the chunks and their order per lane are those of one stride per step)
  constexpr int U = (MODE == ST_SPMV_DOT || MODE == ST_DINV_DOT) ? 2 : 1;
  for (int cs = (blockIdx.x * wpb + (threadIdx.x >> 5)) * K; cs < nch; cs += U * nw * K) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int c0 = cs + u * nw * K;
#pragma unroll
      for (int k = 0; k < K; ++k)
        if (c0 + k < nch) {
          if (kPacked && c0 + k >= nreg)
            stencil_row<T, MODE, true, true>(S, c0 + k - nreg, lane, x, y, b, d, c1, c2,
                                             c2invd0, dacc, agg);
          else
            stencil_row<T, MODE, kPacked>(S, c0 + k, lane, x, y, b, d, c1, c2, c2invd0, dacc,
                                          agg);
        }
    }
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
__host__ __device__ constexpr int kChunks() {
  return sizeof(T) == 4 ? 2 : 1;
}

// Batched form: a block takes one work block (task, first chunk, end chunk) at a time and
// copies the task into shared memory; its warps take two chunks at a time, as the one-solve
// FP32 launch does, and apply each exactly as the one-solve launch applies it.
template <class T>
__device__ __forceinline__ void load_task(const StTask<T>* __restrict__ tasks, int t,
                                          StTask<T>& sk) {
  const int* src = reinterpret_cast<const int*>(tasks + t);
  int* dst = reinterpret_cast<int*>(&sk);
  for (int i = threadIdx.x; i < (int)(sizeof(StTask<T>) / 4); i += blockDim.x) dst[i] = src[i];
}

template <class T, int MODE>
__global__ void __launch_bounds__(256, 4) bstencil_k(const StTask<T>* __restrict__ tasks,
                                                  const int4* __restrict__ wbs, int nwb) {
  __shared__ StTask<T> sk;
  const int lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  constexpr int K = kChunks<T>();
  double dacc = 0.0;
  for (int wb = blockIdx.x; wb < nwb; wb += gridDim.x) {
    const int4 B = wbs[wb];
    __syncthreads();  // the previous work block is done with sk
    load_task<T>(tasks, B.x, sk);
    __syncthreads();
    if (!*sk.go) continue;  // uniform across the block
    const int nreg = packed_rows<T>() ? (sk.S.nrun + 31) / 32 : sk.S.nchunks;
    for (int c0 = B.y + (threadIdx.x >> 5) * K; c0 < B.z; c0 += wpb * K) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int c = c0 + k;
        if (c >= B.z) continue;
        if (packed_rows<T>()) {
          if (c >= nreg)
            stencil_row<T, MODE, true, true>(sk.S, c - nreg, lane, sk.x, sk.y, sk.b, sk.d, sk.c1,
                                             sk.c2, sk.c2i0, dacc, sk.agg);
          else
            stencil_row<T, MODE, true>(sk.S, c, lane, sk.x, sk.y, sk.b, sk.d, sk.c1, sk.c2,
                                       sk.c2i0, dacc, sk.agg);
        } else {
          stencil_row<T, MODE, false>(sk.S, c, lane, sk.x, sk.y, sk.b, sk.d, sk.c1, sk.c2,
                                      sk.c2i0, dacc, sk.agg);
        }
      }
    }
  }
}

// q = A p with p'q partials, FP64: every (task t, block b) pair computes block b of the
// one-solve launch (kRedBlocks blocks of 8 warps, one chunk per warp step) for task t,
// emulated by one warp: lane l runs the rows of lane l of the block's warps w = 0..7 in turn,
// each warp's sum of its own accumulator by the xor tree, the eight added in warp order --
// the bits of the one-solve partial.  A pair without chunks stores 0.
__global__ void __launch_bounds__(256) bstencil_dot_k(const StTask<double>* __restrict__ tasks,
                                                      int ntasks) {
  const int lane = threadIdx.x & 31;
  constexpr int wpb = 8;
  const int nw = kRedBlocks * wpb;
  const long long npairs = (long long)ntasks * kRedBlocks;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long pr = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; pr < npairs;
       pr += nwarps) {
    const StTask<double>& k = tasks[pr / kRedBlocks];
    const int b = (int)(pr % kRedBlocks);
    if (!*k.go) continue;
    const int nreg = (k.S.nrun + 31) / 32;
    const int nch = nreg + (k.S.ntable + 31) / 32;
    if (b * wpb >= nch) {
      if (lane == 0) k.part[b] = 0.0;
      continue;
    }
    double t = 0.0;
    for (int w = 0; w < wpb; ++w) {
      double dacc = 0.0;
      for (int c = b * wpb + w; c < nch; c += nw) {
        if (c >= nreg)
          stencil_row<double, ST_SPMV_DOT, true, true>(k.S, c - nreg, lane, k.x, k.y, k.b, k.d,
                                                       k.c1, k.c2, k.c2i0, dacc, k.agg);
        else
          stencil_row<double, ST_SPMV_DOT, true>(k.S, c, lane, k.x, k.y, k.b, k.d, k.c1, k.c2,
                                                 k.c2i0, dacc, k.agg);
      }
      t += rows::warp_tree(dacc);
    }
    if (lane == 0) k.part[b] = t;
  }
}

}  // namespace

template <class T>
int stencil_units(const StencilDev<T>& S) {
  if (S.nchunks == 0) return 0;
  return packed_rows<T>() ? (S.nrun + 31) / 32 + (S.ntable + 31) / 32 : S.nchunks;
}
template int stencil_units<float>(const StencilDev<float>&);
template int stencil_units<double>(const StencilDev<double>&);

template <class T>
void batched_stencil(int mode, const StTask<T>* tasks, const int4* wbs, int nwb, cudaStream_t s) {
  if (nwb <= 0) return;
  // one wave of resident blocks, each taking work blocks in turn
  auto grid = [&](const void* k) {
    int nb = 0;
    SAAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 256, 0));
    return std::max(1, std::min(nwb, sm_count() * std::max(nb, 1)));
  };
#define SAAMG_BST(M)                                                                  \
  bstencil_k<T, M><<<grid(reinterpret_cast<const void*>(bstencil_k<T, M>)), 256, 0, s>>>( \
      tasks, wbs, nwb)
  switch (mode) {
    case ST_CHEB0:
      SAAMG_BST(ST_CHEB0);
      break;
    case ST_CHEB:
      SAAMG_BST(ST_CHEB);
      break;
    case ST_CHEB1:
      SAAMG_BST(ST_CHEB1);
      break;
    case ST_RESID:
      SAAMG_BST(ST_RESID);
      break;
    case ST_PROLONG:
      SAAMG_BST(ST_PROLONG);
      break;
    default:
      fail(SAAMG_EINVAL, "bad batched stencil mode");
  }
#undef SAAMG_BST
  SAAMG_LAUNCH();
}
template void batched_stencil<float>(int, const StTask<float>*, const int4*, int, cudaStream_t);
template void batched_stencil<double>(int, const StTask<double>*, const int4*, int, cudaStream_t);

void batched_stencil_dot(const StTask<double>* tasks, int ntasks, cudaStream_t s) {
  if (ntasks <= 0) return;
  const long long pairs = (long long)ntasks * kRedBlocks;
  int nb = 0;
  SAAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &nb, reinterpret_cast<const void*>(bstencil_dot_k), 256, 0));
  const int blocks =
      (int)std::min<long long>((pairs + 7) / 8, (long long)sm_count() * std::max(nb, 1));
  bstencil_dot_k<<<blocks, 256, 0, s>>>(tasks, ntasks);
  SAAMG_LAUNCH();
}

// Launches MODE with the shape of cfg (K and packed from the instantiated set).
template <class T, int MODE>
void launch_shaped(const StencilCfg& cfg, long long units, int blocks_cap, const StencilDev<T>& S,
                   const T* x, T* y, const T* b, T* d, T c1, T c2, T c2i0, double* partials,
                   const double* xscale, const int* agg, cudaStream_t s) {
  const int wpb = cfg.block / 32;
  const long long need = (units + (long long)wpb * cfg.k - 1) / ((long long)wpb * cfg.k);
  const int blocks = (int)std::max<long long>(1, std::min<long long>(need, blocks_cap));
#define SAAMG_SHAPE(KK, PP)                                                                  \
  if (cfg.k == KK && (cfg.packed != 0) == PP) {                                              \
    launch_pdl(stencil_k<T, MODE, KK, PP>, blocks, cfg.block, 0, s, S, x, y, b, d, c1, c2,   \
               c2i0, partials, xscale, agg);                                                 \
    return;                                                                                  \
  }
  SAAMG_SHAPE(1, false)
  SAAMG_SHAPE(2, false)
  SAAMG_SHAPE(4, false)
  SAAMG_SHAPE(1, true)
  SAAMG_SHAPE(2, true)
  SAAMG_SHAPE(4, true)
#undef SAAMG_SHAPE
  fail(SAAMG_EINVAL, "unsupported stencil launch shape");
}

// Chunks of 32 rows a launch of the shape processes (packed: regular-run then table chunks).
template <class T>
long long shaped_units(const StencilDev<T>& S, bool packed) {
  return packed ? ((long long)S.nrun + 31) / 32 + (S.ntable + 31) / 32 : S.nchunks;
}

template <class T>
void stencil_apply(const StencilDev<T>& S, int mode, const T* x, T* y, const T* b, T* d, T c1,
                   T c2, double* partials, cudaStream_t s, const double* xscale) {
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
  // c2 / diag of the regular rows, formed here: a kernel that forms it from c2 lets the
  // compiler merge it with the table rows' c2 * (1/diag) into one multiply on every row
  const T c2i0 = c2 * S.invd0;
  if (mode == ST_SPMV_DOT || mode == ST_DINV_DOT) {
    // reductions: the fixed grid and the default shape, so that partial sums are always
    // taken the same way
    constexpr bool P = packed_rows<T>();
    const int* no_agg = nullptr;
    if (mode == ST_SPMV_DOT)
      launch_pdl(stencil_k<T, ST_SPMV_DOT, kChunks<T>(), P>, kRedBlocks, kRedThreads, 0, s, S, x,
                 y, b, d, c1, c2, c2i0, partials, xscale, no_agg);
    else
      launch_pdl(stencil_k<T, ST_DINV_DOT, kChunks<T>(), P>, kRedBlocks, kRedThreads, 0, s, S, x,
                 y, b, d, c1, c2, c2i0, partials, xscale, no_agg);
    SAAMG_LAUNCH();
    return;
  }
  const StencilCfg& cfg = S.cfg;
  const long long units = shaped_units(S, cfg.packed != 0);
  const int cap = sm_count() * cfg.per_sm;
  switch (mode) {
    case ST_SPMV:
      launch_shaped<T, ST_SPMV>(cfg, units, cap, S, x, y, b, d, c1, c2, c2i0, partials, xscale,
                                nullptr, s);
      break;
    case ST_RESID:
      launch_shaped<T, ST_RESID>(cfg, units, cap, S, x, y, b, d, c1, c2, c2i0, partials, xscale,
                                 nullptr, s);
      break;
    case ST_CHEB:
      launch_shaped<T, ST_CHEB>(cfg, units, cap, S, x, y, b, d, c1, c2, c2i0, partials, xscale,
                                nullptr, s);
      break;
    case ST_CHEB0:
      launch_shaped<T, ST_CHEB0>(cfg, units, cap, S, x, y, b, d, c1, c2, c2i0, partials, xscale,
                                 nullptr, s);
      break;
    case ST_CHEB1:
      launch_shaped<T, ST_CHEB1>(cfg, units, cap, S, x, y, b, d, c1, c2, c2i0, partials, xscale,
                                 nullptr, s);
      break;
    default:
      fail(SAAMG_EINVAL, "bad stencil mode");
  }
  SAAMG_LAUNCH();
}

template <class T>
void stencil_prolong(const StencilDev<T>& S, const int* agg, T omega, const T* v, T* y,
                     cudaStream_t s) {
  if (S.nchunks == 0) return;
  KernelTimer kt(SAAMG_KT_PROLONG0, S.n, s);
  const StencilCfg& cfg = S.cfg;
  launch_shaped<T, ST_PROLONG>(cfg, shaped_units(S, cfg.packed != 0), sm_count() * cfg.per_sm, S,
                               v, y, nullptr, nullptr, T(0), omega, T(omega * S.invd0), nullptr,
                               nullptr, agg, s);
  SAAMG_LAUNCH();
}

// Times the Chebyshev step of every launch shape on scratch vectors and returns the fastest
// (median of three launches after one untimed).
template <class T>
StencilCfg stencil_autotune(const StencilDev<T>& S0, cudaStream_t s, double* best_us) {
  StencilDev<T> S = S0;
  const size_t n = (size_t)(S.n > 0 ? S.n : 1);
  Buf<T> x, y, b, d;
  x.alloc(n, s);
  y.alloc(n, s);
  b.alloc(n, s);
  d.alloc(n, s);
  SAAMG_CUDA(cudaMemsetAsync(x.p, 0, n * sizeof(T), s));
  SAAMG_CUDA(cudaMemsetAsync(b.p, 0, n * sizeof(T), s));
  SAAMG_CUDA(cudaMemsetAsync(d.p, 0, n * sizeof(T), s));
  cudaEvent_t e[4];
  for (auto& ev : e) SAAMG_CUDA(cudaEventCreate(&ev));
  StencilCfg best = S0.cfg;
  float best_ms = -1.f;
  try {
    for (int k : {1, 2, 4})
      for (int packed : {0, 1})
        for (int block : {128, 256})
          for (int per_sm : {8, 16, 32}) {
            S.cfg = StencilCfg{k, packed, block, per_sm};
            stencil_apply<T>(S, ST_CHEB, x.p, y.p, b.p, d.p, T(0.5), T(0.25), nullptr, s);
            float t[3];
            for (int r = 0; r < 3; ++r) {
              SAAMG_CUDA(cudaEventRecord(e[0], s));
              stencil_apply<T>(S, ST_CHEB, x.p, y.p, b.p, d.p, T(0.5), T(0.25), nullptr, s);
              SAAMG_CUDA(cudaEventRecord(e[1], s));
              SAAMG_CUDA(cudaEventSynchronize(e[1]));
              SAAMG_CUDA(cudaEventElapsedTime(&t[r], e[0], e[1]));
            }
            std::sort(t, t + 3);
            if (best_ms < 0.f || t[1] < best_ms) {
              best_ms = t[1];
              best = S.cfg;
            }
          }
  } catch (...) {
    for (auto& ev : e) cudaEventDestroy(ev);
    throw;
  }
  for (auto& ev : e) cudaEventDestroy(ev);
  if (best_us) *best_us = 1e3 * best_ms;
  return best;
}

template StencilCfg stencil_autotune<float>(const StencilDev<float>&, cudaStream_t, double*);
template StencilCfg stencil_autotune<double>(const StencilDev<double>&, cudaStream_t, double*);

template void stencil_prolong<float>(const StencilDev<float>&, const int*, float, const float*,
                                     float*, cudaStream_t);
template void stencil_prolong<double>(const StencilDev<double>&, const int*, double,
                                      const double*, double*, cudaStream_t);

template void stencil_apply<double>(const StencilDev<double>&, int, const double*, double*,
                                    const double*, double*, double, double, double*,
                                    cudaStream_t, const double*);
template void stencil_apply<float>(const StencilDev<float>&, int, const float*, float*,
                                   const float*, float*, float, float, double*, cudaStream_t,
                                   const double*);

}  // namespace saamg
