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

__global__ void power_normalize_k(int n, const double* __restrict__ w,
                                  const double* __restrict__ nrm2, double* __restrict__ v) {
  double nrm = sqrt(*nrm2);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v[i] = w[i] / nrm;
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

// Symbolic pass: number of distinct columns of each listed row (-1 on overflow).
__global__ void spgemm_symbolic_k(const int* __restrict__ list, int nlist, int logcap,
                                  int* __restrict__ gkeys, CsrView X, CsrView Y,
                                  int* __restrict__ count, int* __restrict__ overflow) {
  extern __shared__ int smem_i[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int cap = 1 << logcap;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  int* keys = gkeys ? gkeys + (size_t)gw * cap : smem_i + wib * cap;
  for (int t = gw; t < nlist; t += nw) {
    const int i = list[t];
    for (int q = lane; q < cap; q += 32) keys[q] = -1;
    __syncwarp();
    int cnt = 0, full = 0;
    for (int p = X.rowptr[i]; p < X.rowptr[i + 1]; ++p) {
      const int k = X.col[p];
      for (int q = Y.rowptr[k] + lane; q < Y.rowptr[k + 1]; q += 32) {
        int r = hash_insert(keys, logcap, Y.col[q]);
        if (r > 0) ++cnt;
        if (r < 0) full = 1;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      full |= __shfl_xor_sync(0xffffffffu, full, o);
    }
    if (lane == 0) {
      bool over = full || 2 * cnt > cap;
      count[i] = over ? -1 : cnt;
      if (over) atomicAdd(overflow, 1);
    }
    __syncwarp();
  }
}

// Numeric pass: fixed-order accumulation, then rank-sort of the distinct columns.
__global__ void spgemm_numeric_k(const int* __restrict__ list, int nlist, int logcap,
                                 int* __restrict__ gkeys, double* __restrict__ gvals, CsrView X,
                                 CsrView Y, const int* __restrict__ crowptr,
                                 int* __restrict__ ccol, double* __restrict__ cval) {
  extern __shared__ double smem_d[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const int cap = 1 << logcap;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  double* vals;
  int* keys;
  if (gkeys) {
    vals = gvals + (size_t)gw * cap;
    keys = gkeys + (size_t)gw * cap;
  } else {
    vals = smem_d + (size_t)wib * cap;
    keys = reinterpret_cast<int*>(smem_d + (size_t)wpb * cap) + wib * cap;
  }
  for (int t = gw; t < nlist; t += nw) {
    const int i = list[t];
    for (int q = lane; q < cap; q += 32) {
      keys[q] = -1;
      vals[q] = 0.0;
    }
    __syncwarp();
    const int p0 = X.rowptr[i], p1 = X.rowptr[i + 1];
    for (int p = p0; p < p1; ++p) {
      const int k = X.col[p];
      for (int q = Y.rowptr[k] + lane; q < Y.rowptr[k + 1]; q += 32) hash_insert(keys, logcap, Y.col[q]);
    }
    __syncwarp();
    for (int p = p0; p < p1; ++p) {
      const int k = X.col[p];
      const double xv = X.val[p];
      // the columns of one Y row are distinct: every lane owns a different slot
      for (int q = Y.rowptr[k] + lane; q < Y.rowptr[k + 1]; q += 32) {
        int slot = hash_find(keys, logcap, Y.col[q]);
        if (slot >= 0) vals[slot] += xv * Y.val[q];
      }
      __syncwarp();
    }
    const int base = crowptr[i];
    for (int q = lane; q < cap; q += 32) {
      int key = keys[q];
      if (key < 0) continue;
      int rank = 0;
      for (int u = 0; u < cap; ++u) {
        int ku = keys[u];
        rank += (ku >= 0 && ku < key);
      }
      ccol[base + rank] = key;
      cval[base + rank] = vals[q];
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
    // lanes take 32 entries of X's row at a time; a warp scan of the Y-row lengths gives
    // every product its index (X entry order, then Y entry order)
    for (int pb = X.rowptr[i]; pb < p1; pb += 32) {
      const int p = pb + lane;
      const bool ok = p < p1;
      const int k = ok ? X.col[p] : 0;
      const double xv = (NUMERIC && ok) ? X.val[p] : 0.0;
      const int q0 = ok ? Y.rowptr[k] : 0;
      const int len = ok ? Y.rowptr[k + 1] - q0 : 0;
      int off = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, off, o);
        if (lane >= o) off += v;
      }
      const int total = __shfl_sync(0xffffffffu, off, 31);
      off -= len;
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
    // bitonic sort, ascending
    for (int size = 2; size <= m; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int e = lane; e < (m >> 1); e += 32) {
          const int lo = (e / stride) * 2 * stride + (e % stride);
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
    // compress: one output entry per run of equal columns
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

// One thread per row for rows with at most 32 products: expand into a local list, stable
// insertion sort by column (equal columns keep their product order), sum the runs.
template <bool NUMERIC>
__global__ void __launch_bounds__(128) spgemm_row_k(const int* __restrict__ list, int nlist,
                                                    CsrView X, CsrView Y,
                                                    const int* __restrict__ crowptr,
                                                    int* __restrict__ count,
                                                    int* __restrict__ ccol,
                                                    double* __restrict__ cval) {
  int c[32];
  double v[32];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nlist; t += gridDim.x * blockDim.x) {
    const int i = list[t];
    int np = 0;
    for (int p = X.rowptr[i]; p < X.rowptr[i + 1]; ++p) {
      const int k = X.col[p];
      const double xv = NUMERIC ? X.val[p] : 0.0;
      for (int q = Y.rowptr[k]; q < Y.rowptr[k + 1]; ++q) {
        c[np] = Y.col[q];
        if (NUMERIC) v[np] = xv * Y.val[q];
        ++np;
      }
    }
    for (int a = 1; a < np; ++a) {
      const int ca = c[a];
      const double va = NUMERIC ? v[a] : 0.0;
      int j = a - 1;
      while (j >= 0 && c[j] > ca) {
        c[j + 1] = c[j];
        if (NUMERIC) v[j + 1] = v[j];
        --j;
      }
      c[j + 1] = ca;
      if (NUMERIC) v[j + 1] = va;
    }
    int out = 0;
    const int base = NUMERIC ? crowptr[i] : 0;
    for (int a = 0; a < np;) {
      const int ca = c[a];
      double sum = 0.0;
      while (a < np && c[a] == ca) {
        if (NUMERIC) sum += v[a];
        ++a;
      }
      if (NUMERIC) {
        ccol[base + out] = ca;
        cval[base + out] = sum;
      }
      ++out;
    }
    if (!NUMERIC) count[i] = out;
  }
}

// Row classes: 0..5 = ESC with 32 << class product slots, 6 = hash table.
constexpr int kEscClasses = 6;
constexpr int kClasses = kEscClasses + 1;

// Class of every row from its number of products; per-block counts in shared memory,
// one global atomic per class and block.
__global__ void classify_rows_k(int n, CsrView X, CsrView Y, int* __restrict__ cls,
                                int* __restrict__ hist) {
  __shared__ int sh[kClasses];
  if (threadIdx.x < kClasses) sh[threadIdx.x] = 0;
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    long long t = 0;
    for (int p = X.rowptr[i]; p < X.rowptr[i + 1]; ++p) {
      int k = X.col[p];
      t += Y.rowptr[k + 1] - Y.rowptr[k];
    }
    int c = 0;
    while (c < kEscClasses && (32LL << c) < t) ++c;
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

constexpr int kMinLog = 5;    // 32 slots
constexpr int kMaxSmemLog = 11;  // 2048 slots in shared memory
constexpr int kSpgemmWarps = 4;

CsrView view(const DevCsr& a) { return CsrView{a.rowptr.p, a.col.p, a.val.p}; }

}  // namespace

double power_lambda(const DevCsr& A, const double* invd, const unsigned* ids, int iters,
                    cudaStream_t s) {
  int n = A.n;
  if (n == 0) return 1.0;
  Buf<double> v, w, part, nrm2;
  v.alloc(n, s);
  w.alloc(n, s);
  part.alloc(kRedBlocks, s);
  nrm2.alloc(1, s);
  power_init_k<<<blocks_for(n), 256, 0, s>>>(n, ids, v.p);
  SAAMG_LAUNCH();
  double avg = (double)A.nnz / n;
  for (int it = 0; it <= iters; ++it) {
    csr_apply<double, double>(CSR_SPMV_DINV_DOT, n, A.rowptr.p, A.col.p, A.val.p, avg, v.p, w.p,
                              nullptr, nullptr, invd, 0.0, 0.0, part.p, s);
    sum_partials(part.p, kRedBlocks, nrm2.p, s);
    if (it == iters) break;
    power_normalize_k<<<std::min(blocks_for(n), 4096), 256, 0, s>>>(n, w.p, nrm2.p, v.p);
    SAAMG_LAUNCH();
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

template <int CAP, bool NUMERIC>
static void launch_esc(const int* list, int nl, CsrView X, CsrView Y, const int* crowptr,
                       int* count, int* ccol, double* cval, cudaStream_t s) {
  const int warps = 4;
  const size_t sm = (size_t)warps * CAP * (NUMERIC ? 16 : 8);
  if (sm > 48 * 1024)
    SAAMG_CUDA(cudaFuncSetAttribute(spgemm_esc_k<CAP, NUMERIC>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  const int blocks = std::min((nl + warps - 1) / warps, 152 * 16);
  spgemm_esc_k<CAP, NUMERIC><<<blocks, 32 * warps, sm, s>>>(list, nl, X, Y, crowptr, count, ccol,
                                                             cval);
  SAAMG_LAUNCH();
}

template <bool NUMERIC>
static void esc_class(int c, const int* list, int nl, CsrView X, CsrView Y, const int* crowptr,
                      int* count, int* ccol, double* cval, cudaStream_t s) {
  switch (c) {
    case 0: {
      const int blocks = std::max(1, std::min((nl + 127) / 128, 152 * 16));
      spgemm_row_k<NUMERIC><<<blocks, 128, 0, s>>>(list, nl, X, Y, crowptr, count, ccol, cval);
      SAAMG_LAUNCH();
      break;
    }
    case 1: launch_esc<64, NUMERIC>(list, nl, X, Y, crowptr, count, ccol, cval, s); break;
    case 2: launch_esc<128, NUMERIC>(list, nl, X, Y, crowptr, count, ccol, cval, s); break;
    case 3: launch_esc<256, NUMERIC>(list, nl, X, Y, crowptr, count, ccol, cval, s); break;
    case 4: launch_esc<512, NUMERIC>(list, nl, X, Y, crowptr, count, ccol, cval, s); break;
    case 5: launch_esc<1024, NUMERIC>(list, nl, X, Y, crowptr, count, ccol, cval, s); break;
    default: fail(SAAMG_EINVAL, "bad product class");
  }
}

void spgemm(const DevCsr& X, const DevCsr& Y, DevCsr& C, cudaStream_t s) {
  const int n = X.n;
  KernelTimer kt(SAAMG_KT_SPGEMM, n, s);
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
  // classify rows by their number of products; one list per class
  Buf<int> cls, list, cnt, ctl;
  cls.alloc(n, s);
  list.alloc(n, s);
  cnt.alloc(n + 1, s);
  ctl.alloc(2 * kClasses + 1, s);  // histogram, cursors, overflow flag
  SAAMG_CUDA(cudaMemsetAsync(ctl.p, 0, sizeof(int) * (2 * kClasses + 1), s));
  classify_rows_k<<<blocks_for(n), 256, 0, s>>>(n, view(X), view(Y), cls.p, ctl.p);
  SAAMG_LAUNCH();
  int hist[kClasses];
  d2h_sync(hist, ctl.p, sizeof(hist), s);
  int start[kClasses + 1];
  start[0] = 0;
  for (int c = 0; c < kClasses; ++c) start[c + 1] = start[c] + hist[c];
  SAAMG_CUDA(cudaMemcpyAsync(ctl.p + kClasses, start, sizeof(int) * kClasses,
                             cudaMemcpyHostToDevice, s));
  scatter_rows_k<<<blocks_for(n), 256, 0, s>>>(n, cls.p, ctl.p + kClasses, list.p);
  SAAMG_LAUNCH();
  int* overflow = ctl.p + 2 * kClasses;
  const int threads = 32 * kSpgemmWarps;
  const int lc_hash = kMaxSmemLog;
  // symbolic: distinct columns per row
  for (int c = 0; c < kClasses; ++c) {
    if (hist[c] == 0) continue;
    const int* lp = list.p + start[c];
    if (c < kEscClasses) {
      esc_class<false>(c, lp, hist[c], view(X), view(Y), nullptr, cnt.p, nullptr, nullptr, s);
    } else {
      size_t sm = (size_t)kSpgemmWarps * (1u << lc_hash) * sizeof(int);
      int blocks = std::min((hist[c] + kSpgemmWarps - 1) / kSpgemmWarps, 152 * 8);
      spgemm_symbolic_k<<<blocks, threads, sm, s>>>(lp, hist[c], lc_hash, nullptr, view(X),
                                                    view(Y), cnt.p, overflow);
      SAAMG_LAUNCH();
    }
  }
  if (hist[kEscClasses] > 0) {
    int nover = 0;
    d2h_sync(&nover, overflow, sizeof(int), s);
    if (nover) fail(SAAMG_UNIMPLEMENTED, "sparse product row longer than 1024 distinct columns");
  }
  fill_int(cnt.p + n, 0, 1, s);
  long long nnz = exclusive_scan(cnt.p, C.rowptr.p, n + 1, s);
  if (nnz > 0x7fffffffLL) fail(SAAMG_EINVAL, "more than 2^31 nonzeros in a coarse operator");
  C.nnz = nnz;
  C.col.alloc(nnz, s);
  C.val.alloc(nnz, s);
  for (int c = 0; c < kClasses; ++c) {
    if (hist[c] == 0) continue;
    const int* lp = list.p + start[c];
    if (c < kEscClasses) {
      esc_class<true>(c, lp, hist[c], view(X), view(Y), C.rowptr.p, nullptr, C.col.p, C.val.p, s);
    } else {
      size_t sm = (size_t)kSpgemmWarps * (1u << lc_hash) * (sizeof(int) + sizeof(double));
      if (sm > 48 * 1024)
        SAAMG_CUDA(cudaFuncSetAttribute(spgemm_numeric_k,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      int blocks = std::min((hist[c] + kSpgemmWarps - 1) / kSpgemmWarps, 152 * 8);
      spgemm_numeric_k<<<blocks, threads, sm, s>>>(lp, hist[c], lc_hash, nullptr, nullptr,
                                                   view(X), view(Y), C.rowptr.p, C.col.p, C.val.p);
      SAAMG_LAUNCH();
    }
  }
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
