// Hierarchy construction (Sec. 3.2): power iteration for the spectral bound, smoothed
// prolongator P = (I - omega D^-1 A) T, R = P^T and the Galerkin product R A P.
//
// Sparse products run one warp per output row with an open-addressing hash table of the
// row's columns in shared memory (global scratch for very long rows).  The row's values are
// accumulated in a fixed order -- X's entries one after the other, the lanes spread over
// the (distinct) columns of the matching row of Y -- so every entry is summed in the same
// order on every run, and the output columns are written in ascending order.
#include <algorithm>
#include <vector>

#include "csr.cuh"
#include "galerkin.cuh"
#include "operator.cuh"

namespace saamg {

namespace {

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__global__ void power_init_k(int n, const unsigned* __restrict__ ids, double* __restrict__ v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t id = ids ? ids[i] : (uint32_t)i;
  v[i] = 0.5 + (double)fmix32(id ^ 0xA5A5A5A5u) / 4294967296.0;
}

// --- sparse product --------------------------------------------------------
struct CsrView {
  const int* rowptr;
  const int* col;
  const double* val;
};

__device__ __forceinline__ int hash_slot(int key, int logcap) {
  return (int)(((uint32_t)key * 0x9E3779B1u) >> (32 - logcap));
}

// Inserts key; returns 1 if it was new, 0 if present, -1 if the table is full.
__device__ __forceinline__ int hash_insert(int* keys, int logcap, int key) {
  const int cap = 1 << logcap;
  int slot = hash_slot(key, logcap);
  for (int probe = 0; probe < cap; ++probe) {
    int old = atomicCAS(&keys[slot], -1, key);
    if (old == -1) return 1;
    if (old == key) return 0;
    slot = (slot + 1) & (cap - 1);
  }
  return -1;
}

__device__ __forceinline__ int hash_find(const int* keys, int logcap, int key) {
  const int cap = 1 << logcap;
  int slot = hash_slot(key, logcap);
  for (int probe = 0; probe < cap; ++probe) {
    if (keys[slot] == key) return slot;
    slot = (slot + 1) & (cap - 1);
  }
  return -1;
}

// Warp-wide exclusive prefix of v; *total gets the sum over the warp.
__device__ __forceinline__ int warp_excl_scan(int v, int lane, int* total) {
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  *total = __shfl_sync(0xffffffffu, inc, 31);
  return inc - v;
}

// Hash path, symbolic: distinct columns of each listed row (-1 and an overflow count when a
// row does not fit half of the table).  Lanes take 32 entries of X's row at a time and
// insert the columns of their Y rows; insertion order does not matter for the count.
__global__ void __launch_bounds__(128) spgemm_hash_symbolic_k(const int* __restrict__ list,
                                                              int nlist, int logcap, CsrView X,
                                                              CsrView Y, int* __restrict__ count,
                                                              int* __restrict__ overflow) {
  extern __shared__ int smem_i[];
  const int lane = threadIdx.x & 31;
  const int cap = 1 << logcap;
  int* keys = smem_i + (threadIdx.x >> 5) * cap;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int t = gw; t < nlist; t += nw) {
    const int i = list[t];
    for (int q = lane; q < cap; q += 32) keys[q] = -1;
    __syncwarp();
    int cnt = 0, full = 0;
    const int p1 = X.rowptr[i + 1];
    for (int pb = X.rowptr[i]; pb < p1; pb += 32) {
      const int p = pb + lane;
      if (p < p1) {
        const int k = X.col[p];
        for (int q = Y.rowptr[k]; q < Y.rowptr[k + 1]; ++q) {
          const int r = hash_insert(keys, logcap, Y.col[q]);
          cnt += r > 0;
          full |= r < 0;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      full |= __shfl_xor_sync(0xffffffffu, full, o);
    }
    if (lane == 0) {
      const bool over = full || 2 * cnt > cap;
      count[i] = over ? -1 : cnt;
      if (over) atomicAdd(overflow, 1);
    }
    __syncwarp();
  }
}

// Hash path, numeric.  1) insert every column (lane-parallel); 2) compact the distinct
// columns and give each its rank in ascending order; 3) accumulate the products: the warp
// splits into NG groups of 32/NG lanes, group g takes X's entries g, g + NG, ... in order and
// its lanes the distinct columns of that entry's Y row, adding into the group's own copy of
// the value table (no two lanes of a group share a slot, no two groups share a copy), which
// fixes the summation order; 4) the copies are added in group order and the row is written
// in ascending column order.  Per warp: cap keys, cap ranks, cap/2 compacted keys (ints)
// and NG x cap values (doubles).
template <int NG>
__global__ void __launch_bounds__(128) spgemm_hash_numeric_k(const int* __restrict__ list,
                                                             int nlist, int logcap, CsrView X,
                                                             CsrView Y,
                                                             const int* __restrict__ crowptr,
                                                             int* __restrict__ ccol,
                                                             double* __restrict__ cval) {
  extern __shared__ double smem_d[];
  constexpr int GL = 32 / NG;
  const int lane = threadIdx.x & 31;
  const int grp = lane / GL, gl = lane % GL;
  const int wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int cap = 1 << logcap;
  // copy g starts at g (cap + 1): the same slot of two groups falls in different banks
  const int cstride = cap + (NG > 1 ? 1 : 0);
  double* vals = smem_d + (size_t)wib * cstride * NG;
  int* ibase = reinterpret_cast<int*>(smem_d + (size_t)wpb * cstride * NG) + (size_t)wib * (cap * 5 / 2);
  int* keys = ibase;
  int* rank = ibase + cap;
  int* uniq = ibase + 2 * cap;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int t = gw; t < nlist; t += nw) {
    const int i = list[t];
    for (int q = lane; q < cap; q += 32) keys[q] = -1;
    for (int q = lane; q < cstride * NG; q += 32) vals[q] = 0.0;
    __syncwarp();
    const int p0 = X.rowptr[i], p1 = X.rowptr[i + 1];
    for (int pb = p0; pb < p1; pb += 32) {
      const int p = pb + lane;
      if (p < p1) {
        const int k = X.col[p];
        for (int q = Y.rowptr[k]; q < Y.rowptr[k + 1]; ++q) hash_insert(keys, logcap, Y.col[q]);
      }
    }
    __syncwarp();
    // compact the distinct columns
    int nu = 0;
    for (int q0 = 0; q0 < cap; q0 += 32) {
      const int key = keys[q0 + lane];
      const unsigned bm = __ballot_sync(0xffffffffu, key >= 0);
      if (key >= 0) uniq[nu + __popc(bm & ((1u << lane) - 1u))] = key;
      nu += __popc(bm);
    }
    __syncwarp();
    for (int q = lane; q < cap; q += 32) {
      const int key = keys[q];
      if (key < 0) continue;
      int r = 0;
      for (int u = 0; u < nu; ++u) r += uniq[u] < key;
      rank[q] = r;
    }
    __syncwarp();
    double* mine = vals + (size_t)grp * cstride;
    for (int pb = p0; pb < p1; pb += NG) {
      const int p = pb + grp;
      if (p < p1) {
        const int k = X.col[p];
        const double xv = X.val[p];
        for (int q = Y.rowptr[k] + gl; q < Y.rowptr[k + 1]; q += GL) {
          const int slot = hash_find(keys, logcap, Y.col[q]);
          if (slot >= 0) mine[slot] += xv * Y.val[q];
        }
      }
      __syncwarp();
    }
    const int base = crowptr[i];
    for (int q = lane; q < cap; q += 32) {
      const int key = keys[q];
      if (key < 0) continue;
      double v = vals[q];
#pragma unroll
      for (int g = 1; g < NG; ++g) v += vals[(size_t)g * cstride + q];
      ccol[base + rank[q]] = key;
      cval[base + rank[q]] = v;
    }
    __syncwarp();
  }
}

// Expand-sort-compress for rows with at most CAP products (one warp per row).
// Products are keyed (column << 32 | product index) with the product index running over
// X's row, then Y's row, so after sorting every column's products appear in that order and
// are summed in it -- the accumulation order of the plain row-by-row product.
template <int CAP, bool NUMERIC>
__global__ void __launch_bounds__(128) spgemm_esc_k(const int* __restrict__ list, int nlist,
                                                    CsrView X, CsrView Y,
                                                    const int* __restrict__ crowptr,
                                                    int* __restrict__ count,
                                                    int* __restrict__ ccol,
                                                    double* __restrict__ cval) {
  extern __shared__ unsigned long long esc_smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  unsigned long long* keys = esc_smem + (size_t)wib * CAP * (NUMERIC ? 2 : 1);
  double* vals = reinterpret_cast<double*>(keys + CAP);
  for (int t = gw; t < nlist; t += nw) {
    const int i = list[t];
    const int p1 = X.rowptr[i + 1];
    int nprod = 0;
    for (int pb = X.rowptr[i]; pb < p1; pb += 32) {
      const int p = pb + lane;
      const bool ok = p < p1;
      const int k = ok ? X.col[p] : 0;
      const double xv = (NUMERIC && ok) ? X.val[p] : 0.0;
      const int q0 = ok ? Y.rowptr[k] : 0;
      const int len = ok ? Y.rowptr[k + 1] - q0 : 0;
      int total;
      const int off = warp_excl_scan(len, lane, &total);
      for (int q = 0; q < len; ++q) {
        const int idx = nprod + off + q;
        keys[idx] = ((unsigned long long)(uint32_t)Y.col[q0 + q] << 32) | (uint32_t)idx;
        if (NUMERIC) vals[idx] = xv * Y.val[q0 + q];
      }
      nprod += total;
    }
    int m = 2;
    while (m < nprod) m <<= 1;
    for (int idx = nprod + lane; idx < m; idx += 32) keys[idx] = ~0ull;
    __syncwarp();
    // bitonic sort, ascending; pairs (lo, lo + stride) with bit `stride` of lo clear
    for (int size = 2; size <= m; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int e = lane; e < (m >> 1); e += 32) {
          const int lo = e + (e & ~(stride - 1));
          const int hi = lo + stride;
          const bool asc = (lo & size) == 0;
          const unsigned long long ka = keys[lo], kb = keys[hi];
          if ((ka > kb) == asc) {
            keys[lo] = kb;
            keys[hi] = ka;
            if (NUMERIC) {
              const double va = vals[lo];
              vals[lo] = vals[hi];
              vals[hi] = va;
            }
          }
        }
        __syncwarp();
      }
    }
    const int outbase = NUMERIC ? crowptr[i] : 0;
    int run = 0;
    for (int c0 = 0; c0 < nprod; c0 += 32) {
      const int idx = c0 + lane;
      const bool valid = idx < nprod;
      const uint32_t c = valid ? (uint32_t)(keys[idx] >> 32) : 0u;
      const bool head = valid && (idx == 0 || (uint32_t)(keys[idx - 1] >> 32) != c);
      const unsigned hm = __ballot_sync(0xffffffffu, head);
      if (NUMERIC && head) {
        const int r = run + __popc(hm & ((1u << lane) - 1u));
        double sum = 0.0;
        for (int j = idx; j < nprod && (uint32_t)(keys[j] >> 32) == c; ++j) sum += vals[j];
        ccol[outbase + r] = (int)c;
        cval[outbase + r] = sum;
      }
      run += __popc(hm);
    }
    if (!NUMERIC && lane == 0) count[i] = run;
    __syncwarp();
  }
}

// One thread per row for rows whose X row has at most kMergeWays entries: a k-way merge of
// the (sorted) Y rows that X's row selects.  Every output column is produced once, in
// ascending order, and its products are summed in X's entry order -- the accumulation
// order of the plain row-by-row product.  The lists' cursors stay in registers.
constexpr int kMergeWays = 8;

template <bool NUMERIC>
__global__ void __launch_bounds__(128) spgemm_merge_k(const int* __restrict__ list, int nlist,
                                                      CsrView X, CsrView Y,
                                                      const int* __restrict__ crowptr,
                                                      int* __restrict__ count,
                                                      int* __restrict__ ccol,
                                                      double* __restrict__ cval) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nlist; t += gridDim.x * blockDim.x) {
    const int i = list[t];
    const int p0 = X.rowptr[i], nxr = X.rowptr[i + 1] - p0;
    int cur[kMergeWays], end[kMergeWays], head[kMergeWays];
    double xv[kMergeWays];
#pragma unroll
    for (int w = 0; w < kMergeWays; ++w) {
      cur[w] = 0;
      end[w] = 0;
      xv[w] = 0.0;
      if (w < nxr) {
        const int k = X.col[p0 + w];
        cur[w] = Y.rowptr[k];
        end[w] = Y.rowptr[k + 1];
        if (NUMERIC) xv[w] = X.val[p0 + w];
      }
      head[w] = cur[w] < end[w] ? Y.col[cur[w]] : INT_MAX;
    }
    const int base = NUMERIC ? crowptr[i] : 0;
    int out = 0;
    for (;;) {
      int m = head[0];
#pragma unroll
      for (int w = 1; w < kMergeWays; ++w) m = min(m, head[w]);
      if (m == INT_MAX) break;
      double sum = 0.0;
#pragma unroll
      for (int w = 0; w < kMergeWays; ++w) {
        if (head[w] == m) {
          if (NUMERIC) sum += xv[w] * Y.val[cur[w]];
          ++cur[w];
          head[w] = cur[w] < end[w] ? Y.col[cur[w]] : INT_MAX;
        }
      }
      if (NUMERIC) {
        ccol[base + out] = m;
        cval[base + out] = sum;
      }
      ++out;
    }
    if (!NUMERIC) count[i] = out;
  }
}

// Row classes.  0: X row of <= kMergeWays entries (thread per row, merge); 1: <= 64 products
// (warp ESC);
// 2 + (log2(table) - kHashMinLog): hash table of 2^log2 slots, log2 in [kHashMinLog, kHashMaxLog].
constexpr int kHashMinLog = 6;
constexpr int kHashMaxLog = 12;
constexpr int kClasses = 2 + (kHashMaxLog - kHashMinLog + 1);

__global__ void row_products_k(int n, CsrView X, CsrView Y, int* __restrict__ nprod) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long t = 0;
  for (int p = X.rowptr[i]; p < X.rowptr[i + 1]; ++p) {
    int k = X.col[p];
    t += Y.rowptr[k + 1] - Y.rowptr[k];
  }
  nprod[i] = (int)(t < 0x7fffffffLL ? t : 0x7fffffffLL);
}

// Class of every row (symbolic: table sized from min(products, m); numeric: from the exact
// count); block-aggregated histogram.
__global__ void classify_rows_k(int n, const int* __restrict__ xrowptr,
                                const int* __restrict__ nprod, const int* __restrict__ cnt,
                                int m, int* __restrict__ cls, int* __restrict__ hist) {
  __shared__ int sh[kClasses];
  if (threadIdx.x < kClasses) sh[threadIdx.x] = 0;
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int np = nprod[i];
    int c;
    if (xrowptr[i + 1] - xrowptr[i] <= kMergeWays) {
      c = 0;
    } else if (np <= 64) {
      c = 1;
    } else {
      long long need = cnt ? cnt[i] : (np < m ? np : m);
      int lg = kHashMinLog;
      while (lg < kHashMaxLog && (1LL << lg) < 2 * need) ++lg;
      c = 2 + lg - kHashMinLog;
    }
    cls[i] = c;
    atomicAdd(&sh[c], 1);
  }
  __syncthreads();
  if (threadIdx.x < kClasses && sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

// Rows into per-class lists (order inside a class is irrelevant: rows are independent).
__global__ void scatter_rows_k(int n, const int* __restrict__ cls, int* __restrict__ cursor,
                               int* __restrict__ list) {
  __shared__ int cnt[kClasses], base[kClasses];
  if (threadIdx.x < kClasses) cnt[threadIdx.x] = 0;
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = -1, local = 0;
  if (i < n) {
    c = cls[i];
    local = atomicAdd(&cnt[c], 1);
  }
  __syncthreads();
  if (threadIdx.x < kClasses && cnt[threadIdx.x])
    base[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], cnt[threadIdx.x]);
  __syncthreads();
  if (c >= 0) list[base[c] + local] = i;
}

// P_iJ = [J == agg(i)] - (omega * invd_i) * (AT)_iJ
__global__ void prolong_values_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                 double* __restrict__ val, const int* __restrict__ agg,
                                 const double* __restrict__ invd, double omega) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double w = omega * invd[i];
  int a = agg[i];
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
    double tij = (col[p] == a) ? 1.0 : 0.0;
    val[p] = tij - w * val[p];
  }
}

__global__ void tentative_k(int n, const int* __restrict__ agg, int* __restrict__ rowptr,
                            int* __restrict__ col, double* __restrict__ val) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    rowptr[i] = i;
    col[i] = agg[i];
    val[i] = 1.0;
  }
  if (i == n) rowptr[n] = n;
}

__global__ void col_count_k(long long nnz, const int* __restrict__ col, int* __restrict__ cnt) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < nnz;
       p += (long long)gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[p]], 1);
}

__global__ void transpose_fill_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                 const double* __restrict__ val, int* __restrict__ fill,
                                 int* __restrict__ tcol, double* __restrict__ tval) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
    int q = atomicAdd(&fill[col[p]], 1);
    tcol[q] = i;
    tval[q] = val[p];
  }
}

// Warp per row: every entry's rank among the row's (distinct) columns gives its place.
__global__ void rank_rows_k(int n, const int* __restrict__ rowptr, const int* __restrict__ tcol,
                            const double* __restrict__ tval, int* __restrict__ col,
                            double* __restrict__ val) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < n; i += nw) {
    const int p0 = rowptr[i], p1 = rowptr[i + 1];
    for (int p = p0 + lane; p < p1; p += 32) {
      const int c = tcol[p];
      int rank = 0;
      for (int q = p0; q < p1; ++q) rank += tcol[q] < c;
      col[p0 + rank] = c;
      val[p0 + rank] = tval[p];
    }
  }
}

inline int blocks_for(long long n, int t = 256) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

constexpr int kSpgemmWarps = 4;

CsrView view(const DevCsr& a) { return CsrView{a.rowptr.p, a.col.p, a.val.p}; }

}  // namespace

double power_lambda(const DevCsr& A, const double* invd, const unsigned* ids, int iters,
                    cudaStream_t s, const StencilDev<double>* S) {
  int n = A.n;
  if (n == 0) return 1.0;
  // v_{k+1} = D^-1 A v_k / |D^-1 A v_k|: the pass that forms D^-1 A v_{k+1} applies the
  // division by the previous norm to its output (one multiply per row, no separate sweep)
  Buf<double> v, w, part, nrm2;
  v.alloc(n, s);
  w.alloc(n, s);
  part.alloc(kRedBlocks, s);
  nrm2.alloc(2, s);  // |w|^2 and 1 / |w|
  power_init_k<<<blocks_for(n), 256, 0, s>>>(n, ids, v.p);
  SAAMG_LAUNCH();
  double avg = (double)A.nnz / n;
  for (int it = 0; it <= iters; ++it) {
    const double* xscale = it > 0 ? nrm2.p + 1 : nullptr;
    if (S)
      stencil_apply<double>(*S, ST_DINV_DOT, v.p, w.p, nullptr, nullptr, 0.0, 0.0, part.p, s,
                            xscale);
    else
      csr_apply<double, double>(CSR_SPMV_DINV_DOT, n, A.rowptr.p, A.col.p, A.val.p, avg, v.p,
                                w.p, nullptr, nullptr, invd, 0.0, 0.0, part.p, s, -1, xscale);
    sum_partials(part.p, kRedBlocks, nrm2.p, s, nrm2.p + 1);
    v.swap(w);
  }
  double h = 0;
  d2h_sync(&h, nrm2.p, sizeof(double), s);
  return sqrt(h);
}

void tentative(const int* agg, int n, int nagg, DevCsr& T, cudaStream_t s) {
  T.n = n;
  T.m = nagg;
  T.nnz = n;
  T.rowptr.alloc(n + 1, s);
  T.col.alloc(n, s);
  T.val.alloc(n, s);
  tentative_k<<<blocks_for(n + 1), 256, 0, s>>>(n, agg, T.rowptr.p, T.col.p, T.val.p);
  SAAMG_LAUNCH();
}

namespace {

// Bins rows into per-class lists; returns the per-class counts and list offsets.
void bin_rows(int n, const int* xrowptr, const int* nprod, const int* cnt, int m, int* cls,
              int* list, int* ctl, int hist[kClasses], int start[kClasses + 1], cudaStream_t s) {
  SAAMG_CUDA(cudaMemsetAsync(ctl, 0, sizeof(int) * 2 * kClasses, s));
  classify_rows_k<<<blocks_for(n), 256, 0, s>>>(n, xrowptr, nprod, cnt, m, cls, ctl);
  SAAMG_LAUNCH();
  d2h_sync(hist, ctl, sizeof(int) * kClasses, s);
  start[0] = 0;
  for (int c = 0; c < kClasses; ++c) start[c + 1] = start[c] + hist[c];
  SAAMG_CUDA(cudaMemcpyAsync(ctl + kClasses, start, sizeof(int) * kClasses, cudaMemcpyHostToDevice, s));
  scatter_rows_k<<<blocks_for(n), 256, 0, s>>>(n, cls, ctl + kClasses, list);
  SAAMG_LAUNCH();
  SAAMG_CUDA(cudaStreamSynchronize(s));  // `start` lives on this frame
}

template <bool NUMERIC>
void run_class(int c, const int* list, int nl, CsrView X, CsrView Y, double yavg,
               const int* crowptr, int* count, int* overflow, int* ccol, double* cval,
               cudaStream_t s) {
  if (nl == 0) return;
  KernelTimer kt(SAAMG_KT_SPGEMM, nl, s);
  const int threads = 32 * kSpgemmWarps;
  if (c == 0) {
    const int blocks = std::max(1, std::min((nl + 127) / 128, 152 * 16));
    spgemm_merge_k<NUMERIC><<<blocks, 128, 0, s>>>(list, nl, X, Y, crowptr, count, ccol, cval);
    SAAMG_LAUNCH();
    return;
  }
  const int blocks = std::max(1, std::min((nl + kSpgemmWarps - 1) / kSpgemmWarps, 152 * 16));
  if (c == 1) {
    const size_t sm = (size_t)kSpgemmWarps * 64 * (NUMERIC ? 16 : 8);
    spgemm_esc_k<64, NUMERIC><<<blocks, threads, sm, s>>>(list, nl, X, Y, crowptr, count, ccol, cval);
    SAAMG_LAUNCH();
    return;
  }
  const int lg = kHashMinLog + (c - 2);
  const int cap = 1 << lg;
  if (!NUMERIC) {
    const size_t sm = (size_t)kSpgemmWarps * cap * sizeof(int);
    if (sm > 48 * 1024)
      SAAMG_CUDA(cudaFuncSetAttribute(spgemm_hash_symbolic_k,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    spgemm_hash_symbolic_k<<<blocks, threads, sm, s>>>(list, nl, lg, X, Y, count, overflow);
  } else {
    // lane groups sized to Y's rows (one group covers a typical row in one pass)
    const int ng = yavg <= 7.0 ? 4 : (yavg <= 14.0 ? 2 : 1);
    // 8 NG + 10 bytes per slot and warp; as many warps per block as fit in 200 KB
    const size_t per_warp = (size_t)(cap + (ng > 1 ? 1 : 0)) * sizeof(double) * ng +
                            (size_t)cap * sizeof(int) * 5 / 2;
    const int wpb =
        (int)std::max<size_t>(1, std::min<size_t>(kSpgemmWarps, (size_t)(200 << 10) / per_warp));
    const size_t sm = (size_t)wpb * per_warp;
    const int nb = std::max(1, std::min((nl + wpb - 1) / wpb, 152 * 16));
    auto launch = [&](auto kernel) {
      if (sm > 48 * 1024)
        SAAMG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sm));
      kernel<<<nb, 32 * wpb, sm, s>>>(list, nl, lg, X, Y, crowptr, ccol, cval);
    };
    if (ng == 4) launch(spgemm_hash_numeric_k<4>);
    else if (ng == 2) launch(spgemm_hash_numeric_k<2>);
    else launch(spgemm_hash_numeric_k<1>);
  }
  SAAMG_LAUNCH();
}

}  // namespace

void spgemm(const DevCsr& X, const DevCsr& Y, DevCsr& C, cudaStream_t s) {
  const int n = X.n;
  C.n = n;
  C.m = Y.m;
  C.rowptr.alloc(n + 1, s);
  if (n == 0) {
    fill_int(C.rowptr.p, 0, 1, s);
    C.nnz = 0;
    C.col.alloc(0, s);
    C.val.alloc(0, s);
    return;
  }
  const double yavg = Y.n > 0 ? (double)Y.nnz / Y.n : 0.0;
  Buf<int> nprod, cls, list, cnt, ctl;
  nprod.alloc(n, s);
  cls.alloc(n, s);
  list.alloc(n, s);
  cnt.alloc(n + 1, s);
  ctl.alloc(2 * kClasses + 1, s);
  int* overflow = ctl.p + 2 * kClasses;
  SAAMG_CUDA(cudaMemsetAsync(overflow, 0, sizeof(int), s));
  row_products_k<<<blocks_for(n), 256, 0, s>>>(n, view(X), view(Y), nprod.p);
  SAAMG_LAUNCH();
  int hist[kClasses], start[kClasses + 1];
  // symbolic: distinct columns per row
  bin_rows(n, X.rowptr.p, nprod.p, nullptr, Y.m, cls.p, list.p, ctl.p, hist, start, s);
  for (int c = 0; c < kClasses; ++c)
    run_class<false>(c, list.p + start[c], hist[c], view(X), view(Y), yavg, nullptr, cnt.p, overflow,
                     nullptr, nullptr, s);
  int nover = 0;
  d2h_sync(&nover, overflow, sizeof(int), s);
  if (nover) fail(SAAMG_UNIMPLEMENTED, "sparse product row with more than 2048 distinct columns");
  fill_int(cnt.p + n, 0, 1, s);
  long long nnz = exclusive_scan(cnt.p, C.rowptr.p, n + 1, s);
  if (nnz > 0x7fffffffLL) fail(SAAMG_EINVAL, "more than 2^31 nonzeros in a coarse operator");
  C.nnz = nnz;
  C.col.alloc(nnz, s);
  C.val.alloc(nnz, s);
  // numeric: tables sized from the exact counts
  bin_rows(n, X.rowptr.p, nprod.p, cnt.p, Y.m, cls.p, list.p, ctl.p, hist, start, s);
  for (int c = 0; c < kClasses; ++c)
    run_class<true>(c, list.p + start[c], hist[c], view(X), view(Y), yavg, C.rowptr.p, nullptr, nullptr,
                    C.col.p, C.val.p, s);
}

void smoothed_prolongator(DevCsr& AT, const int* agg, const double* invd, double omega,
                          DevCsr& P, cudaStream_t s) {
  prolong_values_k<<<blocks_for(AT.n), 256, 0, s>>>(AT.n, AT.rowptr.p, AT.col.p, AT.val.p, agg,
                                                     invd, omega);
  SAAMG_LAUNCH();
  P = std::move(AT);
}

void transpose(const DevCsr& P, DevCsr& R, cudaStream_t s) {
  R.n = P.m;
  R.m = P.n;
  R.nnz = P.nnz;
  Buf<int> cnt, fill;
  cnt.alloc(P.m + 1, s);
  fill.alloc(P.m + 1, s);
  fill_int(cnt.p, 0, P.m + 1, s);
  if (P.nnz > 0) {
    col_count_k<<<std::min(blocks_for(P.nnz), 4096), 256, 0, s>>>(P.nnz, P.col.p, cnt.p);
    SAAMG_LAUNCH();
  }
  R.rowptr.alloc(P.m + 1, s);
  exclusive_scan(cnt.p, R.rowptr.p, P.m + 1, s);
  SAAMG_CUDA(cudaMemcpyAsync(fill.p, R.rowptr.p, sizeof(int) * (P.m + 1), cudaMemcpyDeviceToDevice, s));
  R.col.alloc(P.nnz, s);
  R.val.alloc(P.nnz, s);
  Buf<int> tcol;
  Buf<double> tval;
  tcol.alloc(P.nnz, s);
  tval.alloc(P.nnz, s);
  if (P.n > 0) {
    transpose_fill_k<<<blocks_for(P.n), 256, 0, s>>>(P.n, P.rowptr.p, P.col.p, P.val.p, fill.p,
                                                     tcol.p, tval.p);
    SAAMG_LAUNCH();
  }
  if (R.n > 0) {
    long long warps = R.n;
    int blocks = (int)std::min<long long>((warps * 32 + 255) / 256, 152 * 32);
    rank_rows_k<<<blocks, 256, 0, s>>>(R.n, R.rowptr.p, tcol.p, tval.p, R.col.p, R.val.p);
    SAAMG_LAUNCH();
  }
}

}  // namespace saamg
