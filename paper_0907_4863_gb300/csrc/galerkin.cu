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
#include "sell.cuh"
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

// Inserts key (absent from the table); returns its slot, -1 if the table is full.
__device__ __forceinline__ int hash_insert_slot(int* keys, int logcap, int key) {
  const int cap = 1 << logcap;
  int slot = hash_slot(key, logcap);
  for (int probe = 0; probe < cap; ++probe) {
    const int old = atomicCAS(&keys[slot], -1, key);
    if (old == -1 || old == key) return slot;
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

// Ascending bitonic sort of 64 values held two per lane (element lane in x0, lane + 32 in x1).
template <class T>
__device__ __forceinline__ void bitonic64(T& x0, T& x1, int lane) {
#pragma unroll
  for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j == 32) {  // partners in the same lane (k = 64: ascending everywhere)
        const T lo = min(x0, x1), hi = max(x0, x1);
        x0 = lo;
        x1 = hi;
        continue;
      }
      const T y0 = __shfl_xor_sync(0xffffffffu, x0, j);
      const T y1 = __shfl_xor_sync(0xffffffffu, x1, j);
      const bool lower = (lane & j) == 0;
      const bool asc0 = (lane & k) == 0, asc1 = ((lane + 32) & k) == 0;
      x0 = lower == asc0 ? min(x0, y0) : max(x0, y0);
      x1 = lower == asc1 ? min(x1, y1) : max(x1, y1);
    }
  }
}

// Adds x_p * Y(k_p, :) into the group's value copy for X's entries p = e0 + grp, e0 + grp + NG,
// ... < e1 (k_p = X.col[p], x_p = X.val[p]); lane gl of a group takes the entries gl, gl + GL,
// ... of each Y row, so no two lanes of a group add into the same slot at once and every slot
// receives its products in the group's entry order.  Warp-collective (the whole warp calls it
// with the same range).  The X entries, their Y row bounds and x_p are loaded 32 at a time, one
// per lane, and handed to the groups by shuffles; the first Y entry of a group's next X entry
// is loaded while the current one is added, so a step waits on one global load, not three.
template <int NG>
__device__ __forceinline__ void accumulate_entries(int e0, int e1, const CsrView& X,
                                                   const CsrView& Y, const int* keys, int logcap,
                                                   double* mine, int lane) {
  constexpr int GL = 32 / NG;
  const int grp = lane / GL, gl = lane % GL;
  for (int cb = e0; cb < e1; cb += 32) {
    const int cn = min(32, e1 - cb);
    int rs = 0, re = 0;
    double xs = 0.0;
    if (lane < cn) {
      const int k = X.col[cb + lane];
      xs = X.val[cb + lane];
      rs = Y.rowptr[k];
      re = Y.rowptr[k + 1];
    }
    // the group's first entry of the chunk
    int e = grp;
    int ys = __shfl_sync(0xffffffffu, rs, e & 31), ye = __shfl_sync(0xffffffffu, re, e & 31);
    double xv = __shfl_sync(0xffffffffu, xs, e & 31);
    if (e >= cn) ye = ys;
    int q = ys + gl;
    int yc = q < ye ? Y.col[q] : -1;
    double yv = q < ye ? Y.val[q] : 0.0;
    for (int eb = 0; eb < cn; eb += NG) {
      const int en = eb + NG + grp;
      int nys = __shfl_sync(0xffffffffu, rs, en & 31), nye = __shfl_sync(0xffffffffu, re, en & 31);
      const double nxv = __shfl_sync(0xffffffffu, xs, en & 31);
      if (en >= cn) nye = nys;
      const int nq = nys + gl;
      const int nyc = nq < nye ? Y.col[nq] : -1;
      const double nyv = nq < nye ? Y.val[nq] : 0.0;
      if (yc >= 0) {
        const int slot = hash_find(keys, logcap, yc);
        if (slot >= 0) mine[slot] += xv * yv;
      }
      for (int qq = q + GL; qq < ye; qq += GL) {
        const int slot = hash_find(keys, logcap, Y.col[qq]);
        if (slot >= 0) mine[slot] += xv * Y.val[qq];
      }
      __syncwarp();
      ye = nye;
      xv = nxv;
      q = nq;
      yc = nyc;
      yv = nyv;
    }
  }
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
                                                              int* __restrict__ overflow,
                                                              int* __restrict__ skeys,
                                                              const int* __restrict__ soff) {
  extern __shared__ int smem_i[];
  const int lane = threadIdx.x & 31;
  const int cap = 1 << logcap;
  // per warp: the table, then (skeys given) cap / 2 compacted keys
  int* keys = smem_i + (threadIdx.x >> 5) * (skeys ? cap + cap / 2 : cap);
  int* uniq = keys + cap;
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
        const int q1 = Y.rowptr[k + 1];
        // four independent column loads in flight, then their inserts
        for (int q = Y.rowptr[k]; q < q1; q += 4) {
          int c[4];
#pragma unroll
          for (int b = 0; b < 4; ++b) c[b] = q + b < q1 ? Y.col[q + b] : -1;
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            if (c[b] < 0) continue;
            const int r = hash_insert(keys, logcap, c[b]);
            cnt += r > 0;
            full |= r < 0;
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      full |= __shfl_xor_sync(0xffffffffu, full, o);
    }
    const bool over = full || 2 * cnt > cap;
    if (lane == 0) {
      count[i] = over ? -1 : cnt;
      if (over) atomicAdd(overflow, 1);
    }
    if (skeys && !over) {
      // the distinct columns in ascending order, for the numeric pass (no second insertion
      // of every product there)
      __syncwarp();
      int nu = 0;
      for (int q0 = 0; q0 < cap; q0 += 32) {
        const int key = keys[q0 + lane];
        const unsigned bm = __ballot_sync(0xffffffffu, key >= 0);
        if (key >= 0) uniq[nu + __popc(bm & ((1u << lane) - 1u))] = key;
        nu += __popc(bm);
      }
      __syncwarp();
      int* out = skeys + soff[i];
      for (int u = lane; u < nu; u += 32) {
        const int key = uniq[u];
        int r = 0;
        for (int v = 0; v < nu; ++v) r += uniq[v] < key;
        out[r] = key;
      }
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
// (16 blocks of 128 threads per SM: the pass is latency-bound and wants every warp slot)
template <int NG>
__global__ void __launch_bounds__(128, 16) spgemm_hash_numeric_k(const int* __restrict__ list,
                                                             int nlist, int logcap, CsrView X,
                                                             CsrView Y,
                                                             const int* __restrict__ crowptr,
                                                             int* __restrict__ ccol,
                                                             double* __restrict__ cval,
                                                             const int* __restrict__ skeys,
                                                             const int* __restrict__ soff) {
  extern __shared__ double smem_d[];
  constexpr int GL = 32 / NG;
  const int lane = threadIdx.x & 31;
  const int grp = lane / GL;
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
    if (skeys && soff[i + 1] > soff[i]) {
      // the symbolic pass left the row's columns in ascending order: each one's place is its rank
      const int* in = skeys + soff[i];
      const int cnt = crowptr[i + 1] - crowptr[i];
      for (int u = lane; u < cnt; u += 32) {
        const int slot = hash_insert_slot(keys, logcap, in[u]);  // never full: cap >= 2 cnt
        if (slot >= 0) rank[slot] = u;
      }
      __syncwarp();
    } else {
      for (int pb = p0; pb < p1; pb += 32) {
        const int p = pb + lane;
        if (p < p1) {
          const int k = X.col[p];
          const int q1 = Y.rowptr[k + 1];
          for (int q = Y.rowptr[k]; q < q1; q += 4) {
            int c[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) c[b] = q + b < q1 ? Y.col[q + b] : -1;
#pragma unroll
            for (int b = 0; b < 4; ++b)
              if (c[b] >= 0) hash_insert(keys, logcap, c[b]);
          }
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
    }
    accumulate_entries<NG>(p0, p1, X, Y, keys, logcap, vals + (size_t)grp * cstride, lane);
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

// Block-per-row forms of the hash passes for classes of few rows (the long rows of the
// smallest levels): the block's threads share one key table; in the numeric pass warp w
// accumulates the w-th contiguous share of X's entries into its own NG value copies, and the
// copies are added in (warp, group) order, so the sums are fixed for a given launch shape.
__global__ void __launch_bounds__(256) spgemm_hash_symbolic_blk_k(const int* __restrict__ list,
                                                                  int nlist, int logcap,
                                                                  CsrView X, CsrView Y,
                                                                  int* __restrict__ count,
                                                                  int* __restrict__ overflow) {
  extern __shared__ int smem_b[];
  __shared__ int tot[2];
  const int cap = 1 << logcap;
  int* keys = smem_b;
  for (int t = blockIdx.x; t < nlist; t += gridDim.x) {
    const int i = list[t];
    for (int q = threadIdx.x; q < cap; q += blockDim.x) keys[q] = -1;
    if (threadIdx.x < 2) tot[threadIdx.x] = 0;
    __syncthreads();
    int cnt = 0, full = 0;
    const int p1 = X.rowptr[i + 1];
    for (int p = X.rowptr[i] + threadIdx.x; p < p1; p += blockDim.x) {
      const int k = X.col[p];
      for (int q = Y.rowptr[k]; q < Y.rowptr[k + 1]; ++q) {
        const int r = hash_insert(keys, logcap, Y.col[q]);
        cnt += r > 0;
        full |= r < 0;
      }
    }
    if (cnt) atomicAdd(&tot[0], cnt);
    if (full) atomicOr(&tot[1], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      const bool over = tot[1] || 2 * tot[0] > cap;
      count[i] = over ? -1 : tot[0];
      if (over) atomicAdd(overflow, 1);
    }
    __syncthreads();
  }
}

template <int NG>
__global__ void __launch_bounds__(256) spgemm_hash_numeric_blk_k(const int* __restrict__ list,
                                                                 int nlist, int logcap, CsrView X,
                                                                 CsrView Y,
                                                                 const int* __restrict__ crowptr,
                                                                 int* __restrict__ ccol,
                                                                 double* __restrict__ cval) {
  extern __shared__ double smem_bd[];
  __shared__ int nus;
  constexpr int GL = 32 / NG;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int grp = lane / GL;
  const int cap = 1 << logcap;
  const int cstride = cap + 1;
  double* vals = smem_bd;
  int* keys = reinterpret_cast<int*>(vals + (size_t)cstride * NG * nwarps);
  int* rank = keys + cap;
  int* uniq = keys + 2 * cap;
  double* mine = vals + (size_t)(warp * NG + grp) * cstride;
  for (int t = blockIdx.x; t < nlist; t += gridDim.x) {
    const int i = list[t];
    for (int q = threadIdx.x; q < cap; q += blockDim.x) keys[q] = -1;
    for (int q = threadIdx.x; q < cstride * NG * nwarps; q += blockDim.x) vals[q] = 0.0;
    __syncthreads();
    const int p0 = X.rowptr[i], p1 = X.rowptr[i + 1];
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
      const int k = X.col[p];
      for (int q = Y.rowptr[k]; q < Y.rowptr[k + 1]; ++q) hash_insert(keys, logcap, Y.col[q]);
    }
    __syncthreads();
    if (warp == 0) {  // compact the distinct columns
      int nu = 0;
      for (int q0 = 0; q0 < cap; q0 += 32) {
        const int key = keys[q0 + lane];
        const unsigned bm = __ballot_sync(0xffffffffu, key >= 0);
        if (key >= 0) uniq[nu + __popc(bm & ((1u << lane) - 1u))] = key;
        nu += __popc(bm);
      }
      if (lane == 0) nus = nu;
    }
    __syncthreads();
    const int nu = nus;
    for (int q = threadIdx.x; q < cap; q += blockDim.x) {
      const int key = keys[q];
      if (key < 0) continue;
      int r = 0;
      for (int u = 0; u < nu; ++u) r += uniq[u] < key;
      rank[q] = r;
    }
    // warp w: entries [p0 + w * share, p0 + (w + 1) * share), its groups in turn
    const int share = (p1 - p0 + nwarps - 1) / nwarps;
    const int w0 = p0 + warp * share, w1 = min(p1, w0 + share);
    accumulate_entries<NG>(w0, w1, X, Y, keys, logcap, mine, lane);
    __syncthreads();
    const int base = crowptr[i];
    for (int q = threadIdx.x; q < cap; q += blockDim.x) {
      const int key = keys[q];
      if (key < 0) continue;
      double v = vals[q];
      for (int c = 1; c < NG * nwarps; ++c) v += vals[(size_t)c * cstride + q];
      ccol[base + rank[q]] = key;
      cval[base + rank[q]] = v;
    }
    __syncthreads();
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

// Warp per row, for a few long X rows (the small coarse levels).
__global__ void row_products_warp_k(int n, CsrView X, CsrView Y, int* __restrict__ nprod) {
  const int lane = threadIdx.x & 31;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    long long t = 0;
    for (int p = X.rowptr[i] + lane; p < X.rowptr[i + 1]; p += 32) {
      const int k = X.col[p];
      t += Y.rowptr[k + 1] - Y.rowptr[k];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) nprod[i] = (int)(t < 0x7fffffffLL ? t : 0x7fffffffLL);
  }
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

// Room for the sorted columns a symbolic hash pass leaves for the numeric one:
// min(products, columns) for the rows of the warp hash classes, 0 for the others.
__global__ void hash_caps_k(int n, const int* __restrict__ cls, const int* __restrict__ nprod,
                            int m, unsigned warp_classes, int* __restrict__ caps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) caps[i] = ((warp_classes >> cls[i]) & 1u) ? min(nprod[i], m) : 0;
  if (i == n) caps[n] = 0;
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

__global__ void row_lengths_k(int n, const int* __restrict__ rowptr, int* __restrict__ len) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) len[i] = rowptr[i + 1] - rowptr[i];
}

// Thread per row i of P: entry (i, J) goes to the place of column i in row J of R (columns
// ascending: a binary search).
__global__ void transpose_known_k(int n, const int* __restrict__ prow, const int* __restrict__ pcol,
                                  const double* __restrict__ pval, const int* __restrict__ rrow,
                                  const int* __restrict__ rcol, double* __restrict__ rval) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = prow[i]; p < prow[i + 1]; ++p) {
    const int J = pcol[p];
    int lo = rrow[J], hi = rrow[J + 1];
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (rcol[mid] < i) lo = mid + 1;
      else hi = mid;
    }
    if (lo < rrow[J + 1] && rcol[lo] == i) rval[lo] = pval[p];
  }
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

// Row i of A T for the level-0 operator (rows of at most 8 entries, the 7-point star): the
// distinct aggregates of the row's columns in ascending order, each with the sum of its
// entries in entry order starting from 0 -- the sums of the merge product A T, whose products
// a_ij * 1 are exact -- a lane per row.  A warp takes 32 consecutive rows: their entries
// (contiguous in A) come into shared memory by coalesced loads, with each column's aggregate,
// and the rows' outputs (contiguous in the result) go back the same way.  COUNT: the number of
// distinct aggregates only.  FINAL: P's values [J == agg(i)] - (omega invd_i) (A T)_iJ instead
// of (A T)_iJ (the expression of prolong_values_k).  A longer row sets *err.
constexpr int kAtWarps = 4;
template <bool COUNT, bool FINAL>
__global__ void __launch_bounds__(32 * kAtWarps) at_stencil_k(
    int n, const int* __restrict__ rowptr, const int* __restrict__ col,
    const double* __restrict__ val, const int* __restrict__ agg, const double* __restrict__ invd,
    double omega, int* __restrict__ cnt, const int* __restrict__ out_rowptr,
    int* __restrict__ out_col, double* __restrict__ out_val, int* __restrict__ err) {
  __shared__ int skey[kAtWarps][256];
  __shared__ double sval[kAtWarps][256];
  __shared__ int ocol[kAtWarps][256];
  __shared__ double oval[kAtWarps][256];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int r0 = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; r0 < n; r0 += nw * 32) {
    const int rend = min(n, r0 + 32);
    const int e0 = rowptr[r0], ne = rowptr[rend] - e0;
    if (ne > 256) {  // some row has more than 8 entries (uniform across the warp)
      if (lane == 0) *err = 1;
      continue;
    }
    for (int q = lane; q < ne; q += 32) {
      skey[wib][q] = agg[col[e0 + q]];
      if (!COUNT) sval[wib][q] = val[e0 + q];
    }
    __syncwarp();
    const int i = r0 + lane;
    const int o0 = COUNT ? 0 : out_rowptr[r0];
    if (i < n) {
      const int p0 = rowptr[i] - e0, len = rowptr[i + 1] - rowptr[i];
      if (len > 8) *err = 1;
      int key[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) key[q] = q < len ? skey[wib][p0 + q] : INT_MAX;
      if (COUNT) {
        int m = 0, last = -1;
        for (;;) {
          int next = INT_MAX;
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (key[q] > last && key[q] < next) next = key[q];
          if (next == INT_MAX) break;
          ++m;
          last = next;
        }
        cnt[i] = m;
      } else {
        // the output place of each entry: the number of distinct smaller aggregates (integer
        // work only); then each entry is added into its place in entry order, from 0 -- one
        // FP64 add per entry instead of one per (aggregate, entry) pair under a predicate
        const int oi = out_rowptr[i] - o0, m = min(8, out_rowptr[i + 1] - out_rowptr[i]);
        bool first[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          first[q] = key[q] != INT_MAX;
#pragma unroll
          for (int q2 = 0; q2 < q; ++q2) first[q] = first[q] && key[q2] != key[q];
        }
        int dk[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          dk[q] = 0;
#pragma unroll
          for (int q2 = 0; q2 < 8; ++q2) dk[q] += (first[q2] && key[q2] < key[q]) ? 1 : 0;
        }
        for (int o = 0; o < m; ++o) oval[wib][oi + o] = 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (q < len) {
            ocol[wib][oi + dk[q]] = key[q];
            oval[wib][oi + dk[q]] += sval[wib][p0 + q];
          }
        }
        if (FINAL) {
          const double w = omega * invd[i];
          const int a = agg[i];
          for (int o = 0; o < m; ++o) {
            const double tij = (ocol[wib][oi + o] == a) ? 1.0 : 0.0;
            oval[wib][oi + o] = tij - w * oval[wib][oi + o];
          }
        }
      }
    }
    __syncwarp();
    if (!COUNT) {
      const int no = out_rowptr[rend] - o0;
      for (int q = lane; q < no; q += 32) {
        out_col[o0 + q] = ocol[wib][q];
        out_val[o0 + q] = oval[wib][q];
      }
    }
    __syncwarp();
  }
}

// --- A T and the smoothed prolongator ------------------------------------------
// The list of row i (G lanes of group `sub`; warp-collective) by lane matches, chunk by chunk.
template <int G>
__device__ __forceinline__ void at_list_general(int i, bool act, int p0, int len, int maxlen,
                                                int lane, int sub, int gl, unsigned gmask,
                                                const int* __restrict__ col,
                                                const double* __restrict__ val,
                                                const int* __restrict__ agg,
                                                int* __restrict__ lcol, double* __restrict__ lval,
                                                int* __restrict__ cnt) {
  int m = 0;  // the group's list length
  for (int cb = 0; cb < maxlen; cb += G) {
    const bool ok = cb + gl < len;
    const int p = p0 + cb + gl;
    const int key = ok ? agg[col[p]] : -1;
    const double v = ok ? val[p] : 0.0;
    // the lanes of this group holding the same aggregate
    const unsigned long long k64 = ((unsigned long long)(unsigned)sub << 32) | (unsigned)key;
    const unsigned mt = __match_any_sync(0xffffffffu, k64);
    int cmax = __popc(mt);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cmax = max(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
    double sum = 0.0;
    unsigned rem = mt;
    for (int t = 0; t < cmax; ++t) {
      const int src = rem ? __ffs(rem) - 1 : lane;
      const double sv = __shfl_sync(0xffffffffu, v, src);
      if (rem) {
        sum = t == 0 ? sv : sum + sv;
        rem &= rem - 1u;
      }
    }
    const bool lead = ok && lane == __ffs(mt) - 1;
    int pos = -1;
    if (lead)
      for (int u = 0; u < m; ++u)
        if (lcol[p0 + u] == key) {
          pos = u;
          break;
        }
    const bool fresh = lead && pos < 0;
    const unsigned fm = __ballot_sync(0xffffffffu, fresh) & gmask;
    if (fresh) {
      pos = m + __popc(fm & ((1u << lane) - 1u));
      lcol[p0 + pos] = key;
      lval[p0 + pos] = sum;
    } else if (lead) {
      lval[p0 + pos] += sum;
    }
    m += __popc(fm);
    __syncwarp();
  }
  if (act && gl == 0) cnt[i] = m;
}

// Row i of A T (T(j, agg(j)) = 1) holds the distinct aggregates agg(j) of A's row i, each with
// the sum of the row's a_ij over it.  A group of G lanes takes one row, G entries at a time:
// equal aggregates inside a chunk are found by a match and summed by their lowest lane in
// lane (= entry) order, and the chunk sums are merged into the row's list, kept in scratch
// arrays laid out like A (a row never has more aggregates than entries), in order of first
// appearance.  A row of at most G entries is therefore summed strictly in entry order.  (Rows
// of a 32-lane class whose aggregates sort in 32 bits go to at_lists_sorted_k instead.)
template <int G>
__global__ void __launch_bounds__(256) at_lists_k(int n, const int* __restrict__ rowptr,
                                                  const int* __restrict__ col,
                                                  const double* __restrict__ val,
                                                  const int* __restrict__ agg,
                                                  int* __restrict__ lcol,
                                                  double* __restrict__ lval,
                                                  int* __restrict__ cnt) {
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int sub = lane / G, gl = lane % G;
  const unsigned gmask = G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (sub * G);
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int wb = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW; wb < n; wb += nw * RPW) {
    const int i = wb + sub;
    const bool act = i < n;
    const int p0 = act ? rowptr[i] : 0;
    const int len = act ? rowptr[i + 1] - p0 : 0;
    int maxlen = len;
#pragma unroll
    for (int o = G; o < 32; o <<= 1) maxlen = max(maxlen, __shfl_xor_sync(0xffffffffu, maxlen, o));
    at_list_general<G>(i, act, p0, len, maxlen, lane, sub, gl, gmask, col, val, agg, lcol, lval,
                       cnt);
  }
}

// Rows of at most 64 entries (one row per warp, aggregate numbers below 2^25): the row's
// (aggregate, entry) pairs are sorted in registers, so that equal aggregates become neighbours
// in entry order and the list comes out in ascending order -- as in at_lists_k -- but a warp
// sorts kAtBatch rows into shared memory and then sums all of their runs at once, a lane per
// run, each run from its first entry in order.  On the coarse levels a row's entries fall in
// few aggregates (runs of about ten), and one run summed at a time by its head lane issued a
// warp-wide FP64 add per entry with only the heads of one row active.  Longer rows take the
// general path.
constexpr int kAtBatch = 4;

__global__ void __launch_bounds__(256) at_lists_sorted_k(int n, const int* __restrict__ rowptr,
                                                         const int* __restrict__ col,
                                                         const double* __restrict__ val,
                                                         const int* __restrict__ agg,
                                                         int* __restrict__ lcol,
                                                         double* __restrict__ lval,
                                                         int* __restrict__ cnt) {
  __shared__ int skey[8][kAtBatch * 64];      // aggregate of each sorted entry, -1 past the row
  __shared__ double sval[8][kAtBatch * 64];   // its value
  __shared__ short shead[8][kAtBatch * 64];   // batch positions of the runs' first entries
  __shared__ int sinfo[8][3 * kAtBatch + 1];  // rows, their first entries, first runs (+ total)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  int* srow = sinfo[w];
  int* sp0 = srow + kAtBatch;
  int* srun = sp0 + kAtBatch;
  int nb = 0;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;; i += nw) {
    const bool have = i < n;
    const int p0 = have ? rowptr[i] : 0;
    const int len = have ? rowptr[i + 1] - p0 : 0;
    const bool sorted = have && len <= 64;
    if (sorted) {
      unsigned x0 = 0xffffffffu, x1 = 0xffffffffu;
      if (lane < len) x0 = ((unsigned)agg[col[p0 + lane]] << 6) | (unsigned)lane;
      if (lane + 32 < len) x1 = ((unsigned)agg[col[p0 + lane + 32]] << 6) | (unsigned)(lane + 32);
      bitonic64(x0, x1, lane);
      const int q = nb * 64 + lane;
      skey[w][q] = lane < len ? (int)(x0 >> 6) : -1;
      skey[w][q + 32] = lane + 32 < len ? (int)(x1 >> 6) : -1;
      sval[w][q] = lane < len ? val[p0 + (x0 & 63u)] : 0.0;
      sval[w][q + 32] = lane + 32 < len ? val[p0 + (x1 & 63u)] : 0.0;
      if (lane == 0) {
        srow[nb] = i;
        sp0[nb] = p0;
      }
      ++nb;
      if (nb < kAtBatch) continue;
    }
    if (nb > 0) {
      __syncwarp();
      int nrun = 0;
      for (int q0 = 0; q0 < nb * 64; q0 += 32) {
        if ((q0 & 63) == 0 && lane == 0) srun[q0 >> 6] = nrun;
        const int q = q0 + lane;
        const int k = skey[w][q];
        const bool head = k >= 0 && ((q & 63) == 0 || skey[w][q - 1] != k);
        const unsigned hm = __ballot_sync(0xffffffffu, head);
        if (head) shead[w][nrun + __popc(hm & ((1u << lane) - 1u))] = (short)q;
        nrun += __popc(hm);
      }
      if (lane == 0) srun[nb] = nrun;
      __syncwarp();
      for (int r = lane; r < nrun; r += 32) {
        const int q = shead[w][r];
        const int b = q >> 6, k = skey[w][q];
        double sum = sval[w][q];
        for (int t = q + 1; (t & 63) != 0 && skey[w][t] == k; ++t) sum += sval[w][t];
        const int pos = sp0[b] + (r - srun[b]);
        lcol[pos] = k;
        lval[pos] = sum;
      }
      if (lane < nb) cnt[srow[lane]] = srun[lane + 1] - srun[lane];
      __syncwarp();
      nb = 0;
    }
    if (!have) break;
    if (!sorted)
      at_list_general<32>(i, true, p0, len, len, lane, 0, lane, 0xffffffffu, col, val, agg, lcol,
                          lval, cnt);
  }
}

// P's row i from the list: P_iJ = [J == agg(i)] - (omega invd_i) (A T)_iJ, columns ascending
// (each entry's rank among the row's aggregates gives its place).
template <int G>
__global__ void __launch_bounds__(256) at_prolong_k(int n, const int* __restrict__ arowptr,
                                                    const int* __restrict__ lcol,
                                                    const double* __restrict__ lval,
                                                    const int* __restrict__ prowptr,
                                                    const int* __restrict__ agg,
                                                    const double* __restrict__ invd,
                                                    double omega, int* __restrict__ pcol,
                                                    double* __restrict__ pval) {
  constexpr int RPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int sub = lane / G, gl = lane % G;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int wb = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * RPW; wb < n; wb += nw * RPW) {
    const int i = wb + sub;
    if (i >= n) continue;  // no collective operation below
    const int a0 = arowptr[i], b0 = prowptr[i], m = prowptr[i + 1] - b0;
    const double w = omega * invd[i];
    const int a = agg[i];
    for (int u = gl; u < m; u += G) {
      const int key = lcol[a0 + u];
      int r = 0;
      for (int q = 0; q < m; ++q) r += lcol[a0 + q] < key;
      const double tij = key == a ? 1.0 : 0.0;
      pcol[b0 + r] = key;
      pval[b0 + r] = tij - w * lval[a0 + u];
    }
  }
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

// Warp per row: every entry's rank among the row's (distinct) columns gives its place.  Rows of
// at most 64 entries whose columns fit 26 bits are sorted in registers instead, (column, entry)
// pairs by a bitonic network: the same order, without a pass over the row per entry.
__global__ void rank_rows_k(int n, const int* __restrict__ rowptr, const int* __restrict__ tcol,
                            const double* __restrict__ tval, int* __restrict__ col,
                            double* __restrict__ val, bool sortable) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = warp; i < n; i += nw) {
    const int p0 = rowptr[i], p1 = rowptr[i + 1];
    const int len = p1 - p0;
    if (sortable && len <= 64) {  // uniform across the warp
      unsigned x0 = 0xffffffffu, x1 = 0xffffffffu;
      if (lane < len) x0 = ((unsigned)tcol[p0 + lane] << 6) | (unsigned)lane;
      if (lane + 32 < len) x1 = ((unsigned)tcol[p0 + lane + 32] << 6) | (unsigned)(lane + 32);
      bitonic64(x0, x1, lane);
      if (lane < len) {
        col[p0 + lane] = (int)(x0 >> 6);
        val[p0 + lane] = tval[p0 + (x0 & 63u)];
      }
      if (lane + 32 < len) {
        col[p0 + lane + 32] = (int)(x1 >> 6);
        val[p0 + lane + 32] = tval[p0 + (x1 & 63u)];
      }
      continue;
    }
    for (int p = p0 + lane; p < p1; p += 32) {
      const int c = tcol[p];
      int rank = 0;
      for (int q = p0; q < p1; ++q) rank += tcol[q] < c;
      col[p0 + rank] = c;
      val[p0 + rank] = tval[p];
    }
  }
}

// Block per row for the long rows of small levels: the row's columns are staged in shared
// memory and every entry counts the smaller ones there.
constexpr int kRankStage = 8192;
__global__ void __launch_bounds__(256) rank_rows_block_k(int n, const int* __restrict__ rowptr,
                                                         const int* __restrict__ tcol,
                                                         const double* __restrict__ tval,
                                                         int* __restrict__ col,
                                                         double* __restrict__ val) {
  __shared__ int sc[kRankStage];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const int p0 = rowptr[i], len = rowptr[i + 1] - p0;
    const bool staged = len <= kRankStage;
    if (staged)
      for (int u = threadIdx.x; u < len; u += blockDim.x) sc[u] = tcol[p0 + u];
    __syncthreads();
    const int* cs = staged ? sc : tcol + p0;
    for (int u = threadIdx.x; u < len; u += blockDim.x) {
      const int c = cs[u];
      int rank = 0;
      for (int q = 0; q < len; ++q) rank += cs[q] < c;
      col[p0 + rank] = c;
      val[p0 + rank] = tval[p0 + u];
    }
    __syncthreads();
  }
}

inline int blocks_for(long long n, int t = 256) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }
// blocks of at_stencil_k: a warp per 32 rows, every warp of the grid resident at once
inline int at_blocks(int n) {
  const long long warps = (n + 31) / 32;
  return (int)std::max<long long>(1, std::min<long long>((warps + kAtWarps - 1) / kAtWarps,
                                                        (long long)sm_count() * 16));
}

constexpr int kSpgemmWarps = 4;
// a hash class of at most this many rows runs a block per row
constexpr int kFewRows = 2048;

CsrView view(const DevCsr& a) { return CsrView{a.rowptr.p, a.col.p, a.val.p}; }

}  // namespace

void power_lambda_start(const DevCsr& A, const double* invd, const unsigned* ids, int iters,
                        cudaStream_t s, PowerRun& run, const StencilDev<double>* S,
                        const DevSell* As) {
  const int n = A.n;
  run.n = n;
  if (n == 0) return;
  // v_{k+1} = D^-1 A v_k / |D^-1 A v_k|: the pass that forms D^-1 A v_{k+1} applies the
  // division by the previous norm to its output (one multiply per row, no separate sweep)
  run.v.alloc(n, s);
  run.w.alloc(n, s);
  run.part.alloc(kRedBlocks, s);
  run.nrm2.alloc(2, s);  // |w|^2 and 1 / |w|
  power_init_k<<<blocks_for(n), 256, 0, s>>>(n, ids, run.v.p);
  SAAMG_LAUNCH();
  const double avg = (double)A.nnz / n;
  for (int it = 0; it <= iters; ++it) {
    const double* xscale = it > 0 ? run.nrm2.p + 1 : nullptr;
    if (S)
      stencil_apply<double>(*S, ST_DINV_DOT, run.v.p, run.w.p, nullptr, nullptr, 0.0, 0.0,
                            run.part.p, s, xscale);
    else if (As && As->val.p)
      sell_apply<double, double>(CSR_SPMV_DINV_DOT, *As, As->val.p, run.v.p, run.w.p, nullptr,
                                 nullptr, invd, 0.0, 0.0, s, -1, run.part.p, xscale);
    else
      csr_apply<double, double>(CSR_SPMV_DINV_DOT, n, A.rowptr.p, A.col.p, A.val.p, avg,
                                run.v.p, run.w.p, nullptr, nullptr, invd, 0.0, 0.0, run.part.p,
                                s, -1, xscale);
    sum_partials(run.part.p, kRedBlocks, run.nrm2.p, s, run.nrm2.p + 1);
    run.v.swap(run.w);
  }
}

double power_lambda_finish(PowerRun& run, cudaStream_t s) {
  if (run.n == 0) return 1.0;
  double h = 0;
  d2h_sync(&h, run.nrm2.p, sizeof(double), s);
  run.v.release();
  run.w.release();
  run.part.release();
  run.nrm2.release();
  return sqrt(h);
}

double power_lambda(const DevCsr& A, const double* invd, const unsigned* ids, int iters,
                    cudaStream_t s, const StencilDev<double>* S, const DevSell* As) {
  PowerRun run;
  power_lambda_start(A, invd, ids, iters, s, run, S, As);
  return power_lambda_finish(run, s);
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
               int* skeys, const int* soff, cudaStream_t s) {
  if (nl == 0) return;
  KernelTimer kt(SAAMG_KT_SPGEMM, nl, s);
  const int threads = 32 * kSpgemmWarps;
  if (c == 0) {
    const int blocks = std::max(1, std::min((nl + 127) / 128, sm_count() * 16));
    spgemm_merge_k<NUMERIC><<<blocks, 128, 0, s>>>(list, nl, X, Y, crowptr, count, ccol, cval);
    SAAMG_LAUNCH();
    return;
  }
  const int blocks = std::max(1, std::min((nl + kSpgemmWarps - 1) / kSpgemmWarps, sm_count() * 16));
  if (c == 1) {
    const size_t sm = (size_t)kSpgemmWarps * 64 * (NUMERIC ? 16 : 8);
    spgemm_esc_k<64, NUMERIC><<<blocks, threads, sm, s>>>(list, nl, X, Y, crowptr, count, ccol, cval);
    SAAMG_LAUNCH();
    return;
  }
  const int lg = kHashMinLog + (c - 2);
  const int cap = 1 << lg;
  if (nl <= kFewRows) {  // few rows: a block per row
    const int nb = std::min(nl, sm_count() * 4);
    if (!NUMERIC) {
      const size_t sm = (size_t)cap * sizeof(int);
      if (sm > 48 * 1024)
        SAAMG_CUDA(cudaFuncSetAttribute(spgemm_hash_symbolic_blk_k,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      spgemm_hash_symbolic_blk_k<<<nb, 256, sm, s>>>(list, nl, lg, X, Y, count, overflow);
    } else {
      const int ng = yavg <= 7.0 ? 4 : (yavg <= 14.0 ? 2 : 1);
      // 8 warps when their value copies fit 160 KB, else fewer
      int wpb = 8;
      auto bytes = [&](int w) {
        return (size_t)(cap + 1) * sizeof(double) * ng * w + (size_t)cap * sizeof(int) * 5 / 2;
      };
      while (wpb > 1 && bytes(wpb) > (160u << 10)) wpb >>= 1;
      const size_t sm = bytes(wpb);
      auto launch = [&](auto kernel) {
        if (sm > 48 * 1024)
          SAAMG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sm));
        kernel<<<nb, 32 * wpb, sm, s>>>(list, nl, lg, X, Y, crowptr, ccol, cval);
      };
      if (ng == 4) launch(spgemm_hash_numeric_blk_k<4>);
      else if (ng == 2) launch(spgemm_hash_numeric_blk_k<2>);
      else launch(spgemm_hash_numeric_blk_k<1>);
    }
    SAAMG_LAUNCH();
    return;
  }
  if (!NUMERIC) {
    const size_t sm = (size_t)kSpgemmWarps * (skeys ? cap + cap / 2 : cap) * sizeof(int);
    if (sm > 48 * 1024)
      SAAMG_CUDA(cudaFuncSetAttribute(spgemm_hash_symbolic_k,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    spgemm_hash_symbolic_k<<<blocks, threads, sm, s>>>(list, nl, lg, X, Y, count, overflow,
                                                       skeys, soff);
  } else {
    // lane groups sized to Y's rows (one group covers a typical row in one pass)
    const int ng = yavg <= 7.0 ? 4 : (yavg <= 14.0 ? 2 : 1);
    // 8 NG + 10 bytes per slot and warp; as many warps per block as fit in 200 KB
    const size_t per_warp = (size_t)(cap + (ng > 1 ? 1 : 0)) * sizeof(double) * ng +
                            (size_t)cap * sizeof(int) * 5 / 2;
    const int wpb =
        (int)std::max<size_t>(1, std::min<size_t>(kSpgemmWarps, (size_t)(200 << 10) / per_warp));
    const size_t sm = (size_t)wpb * per_warp;
    const int nb = std::max(1, std::min((nl + wpb - 1) / wpb, sm_count() * 16));
    auto launch = [&](auto kernel) {
      if (sm > 48 * 1024)
        SAAMG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sm));
      kernel<<<nb, 32 * wpb, sm, s>>>(list, nl, lg, X, Y, crowptr, ccol, cval, skeys, soff);
    };
    if (ng == 4) launch(spgemm_hash_numeric_k<4>);
    else if (ng == 2) launch(spgemm_hash_numeric_k<2>);
    else launch(spgemm_hash_numeric_k<1>);
  }
  SAAMG_LAUNCH();
}

}  // namespace

void spgemm_symbolic(const DevCsr& X, const DevCsr& Y, SpgemmPlan& plan, cudaStream_t s,
                     const DevCsr* known) {
  const int n = X.n;
  plan.n = n;
  plan.m = Y.m;
  plan.rowptr.alloc(n + 1, s);
  plan.hist.assign(kClasses, 0);
  plan.start.assign(kClasses + 1, 0);
  plan.keys = plan.koff = nullptr;
  if (n == 0) {
    fill_int(plan.rowptr.p, 0, 1, s);
    plan.nnz = 0;
    return;
  }
  plan.yavg = Y.n > 0 ? (double)Y.nnz / Y.n : 0.0;
  plan.nprod.alloc(n, s);
  plan.cls.alloc(n, s);
  plan.list.alloc(n, s);
  plan.ctl.alloc(2 * kClasses + 1, s);
  int* nprod = plan.nprod.p;
  int* ctl = plan.ctl.p;
  if (n < 32768 && (double)X.nnz > 32.0 * n) {
    row_products_warp_k<<<(n * 32 + 255) / 256, 256, 0, s>>>(n, view(X), view(Y), nprod);
  } else {
    row_products_k<<<blocks_for(n), 256, 0, s>>>(n, view(X), view(Y), nprod);
  }
  SAAMG_LAUNCH();
  Buf<int> cnt;
  cnt.alloc(n + 1, s);
  if (known) {
    // C's pattern is known: its row lengths bin the rows, its columns are the sorted keys
    if (known->n != n || known->m != Y.m) fail(SAAMG_EINVAL, "known product pattern has other sizes");
    SAAMG_CUDA(cudaMemcpyAsync(plan.rowptr.p, known->rowptr.p, sizeof(int) * (n + 1),
                               cudaMemcpyDeviceToDevice, s));
    row_lengths_k<<<blocks_for(n), 256, 0, s>>>(n, known->rowptr.p, cnt.p);
    SAAMG_LAUNCH();
    plan.nnz = known->nnz;
    plan.keys = known->col.p;
    plan.koff = known->rowptr.p;
  } else {
    int* overflow = ctl + 2 * kClasses;
    SAAMG_CUDA(cudaMemsetAsync(overflow, 0, sizeof(int), s));
    int hist[kClasses], start[kClasses + 1];
    // symbolic: distinct columns per row
    bin_rows(n, X.rowptr.p, nprod, nullptr, Y.m, plan.cls.p, plan.list.p, ctl, hist, start, s);
    // the warp hash passes leave each row's sorted columns for the numeric pass (room
    // min(products, columns) per row) when the total fits 32-bit offsets
    unsigned warp_classes = 0;
    for (int c = 2; c < kClasses; ++c)
      if (hist[c] > kFewRows) warp_classes |= 1u << c;
    if (warp_classes) {
      Buf<int> caps;
      caps.alloc(n + 1, s);
      hash_caps_k<<<blocks_for(n + 1), 256, 0, s>>>(n, plan.cls.p, nprod, Y.m, warp_classes, caps.p);
      SAAMG_LAUNCH();
      plan.soff.alloc(n + 1, s);
      const long long total = exclusive_scan(caps.p, plan.soff.p, n + 1, s);
      if (total > 0 && total < 0x7fffffffLL) plan.skeys.alloc(total, s);
      else plan.soff.release();
    }
    for (int c = 0; c < kClasses; ++c)
      run_class<false>(c, plan.list.p + start[c], hist[c], view(X), view(Y), plan.yavg, nullptr,
                       cnt.p, overflow, nullptr, nullptr, plan.skeys.p, plan.soff.p, s);
    int nover = 0;
    d2h_sync(&nover, overflow, sizeof(int), s);
    if (nover) fail(SAAMG_UNIMPLEMENTED, "sparse product row with more than 2048 distinct columns");
    fill_int(cnt.p + n, 0, 1, s);
    const long long nnz = exclusive_scan(cnt.p, plan.rowptr.p, n + 1, s);
    if (nnz > 0x7fffffffLL) fail(SAAMG_EINVAL, "more than 2^31 nonzeros in a coarse operator");
    plan.nnz = nnz;
    plan.keys = plan.skeys.p;
    plan.koff = plan.soff.p;
  }
  // numeric classes: tables sized from the exact counts
  bin_rows(n, X.rowptr.p, nprod, cnt.p, Y.m, plan.cls.p, plan.list.p, ctl, plan.hist.data(),
           plan.start.data(), s);
}

void spgemm_numeric(const DevCsr& X, const DevCsr& Y, SpgemmPlan& plan, DevCsr& C, cudaStream_t s) {
  const int n = plan.n;
  C.n = n;
  C.m = plan.m;
  C.nnz = plan.nnz;
  C.rowptr = std::move(plan.rowptr);
  C.col.alloc(plan.nnz, s);
  C.val.alloc(plan.nnz, s);
  if (n == 0) return;
  for (int c = 0; c < kClasses; ++c)
    run_class<true>(c, plan.list.p + plan.start[c], plan.hist[c], view(X), view(Y), plan.yavg,
                    C.rowptr.p, nullptr, nullptr, C.col.p, C.val.p, const_cast<int*>(plan.keys), plan.koff, s);
}

void spgemm(const DevCsr& X, const DevCsr& Y, DevCsr& C, cudaStream_t s) {
  SpgemmPlan plan;
  spgemm_symbolic(X, Y, plan, s);
  spgemm_numeric(X, Y, plan, C, s);
}

void smoothed_prolongator(DevCsr& AT, const int* agg, const double* invd, double omega,
                          DevCsr& P, cudaStream_t s);

void prolongator_start(const DevCsr& A, const int* agg, int nagg, ProlongState& st,
                       cudaStream_t s, const DevCsr* known, bool stencil_rows) {
  const int n = A.n;
  st.n = n;
  st.nagg = nagg;
  st.A = &A;
  st.agg = agg;
  const double avg = n > 0 ? (double)A.nnz / n : 0.0;
  st.lists = avg > 8.0;
  if (!st.lists && stencil_rows) {  // the 7-point operator: A T a row at a time
    DevCsr& AT = st.AT;
    AT.n = n;
    AT.m = nagg;
    AT.rowptr.alloc(n + 1, s);
    Buf<int> err;
    err.alloc(1, s);
    fill_int(err.p, 0, 1, s);
    if (known) {
      SAAMG_CUDA(cudaMemcpyAsync(AT.rowptr.p, known->rowptr.p, sizeof(int) * (n + 1),
                                 cudaMemcpyDeviceToDevice, s));
      AT.nnz = known->nnz;
    } else {
      Buf<int> cnt;
      cnt.alloc(n + 1, s);
      {
        KernelTimer kt(SAAMG_KT_SPGEMM, n, s);
        at_stencil_k<true, false><<<at_blocks(n), 32 * kAtWarps, 0, s>>>(
            n, A.rowptr.p, A.col.p, A.val.p, agg, nullptr, 0.0, cnt.p, nullptr, nullptr, nullptr,
            err.p);
        SAAMG_LAUNCH();
      }
      fill_int(cnt.p + n, 0, 1, s);
      AT.nnz = exclusive_scan(cnt.p, AT.rowptr.p, n + 1, s);
    }
    AT.col.alloc(AT.nnz, s);
    AT.val.alloc(AT.nnz, s);
    {
      KernelTimer kt(SAAMG_KT_SPGEMM, n, s);
      if (st.invd)
        at_stencil_k<false, true><<<at_blocks(n), 32 * kAtWarps, 0, s>>>(
            n, A.rowptr.p, A.col.p, A.val.p, agg, st.invd, st.omega, nullptr, AT.rowptr.p,
            AT.col.p, AT.val.p, err.p);
      else
        at_stencil_k<false, false><<<at_blocks(n), 32 * kAtWarps, 0, s>>>(
            n, A.rowptr.p, A.col.p, A.val.p, agg, nullptr, 0.0, nullptr, AT.rowptr.p, AT.col.p,
            AT.val.p, err.p);
      SAAMG_LAUNCH();
    }
    int herr = 0;
    d2h_sync(&herr, err.p, sizeof(int), s);
    if (herr) fail(SAAMG_ECUDA, "level-0 operator row with more than 8 entries");
    st.final_values = st.invd != nullptr;
    return;
  }
  if (!st.lists) {  // short rows: T and the register k-way merge product
    DevCsr T;
    tentative(agg, n, nagg, T, s);
    SpgemmPlan plan;
    spgemm_symbolic(A, T, plan, s, known);
    spgemm_numeric(A, T, plan, st.AT, s);
    return;
  }
  DevCsr& P = st.AT;  // P's row pointers and size
  P.n = n;
  P.m = nagg;
  P.rowptr.alloc(n + 1, s);
  Buf<int> cnt;
  st.lcol.alloc(A.nnz, s);
  st.lval.alloc(A.nnz, s);
  cnt.alloc(n + 1, s);
  st.G = avg <= 16.0 ? 16 : 32;
  const bool sortable = nagg < (1 << 25);  // (aggregate << 6 | entry) stays below 0xffffffff
  const int blocks = (int)std::min<long long>(((long long)n * st.G + 255) / 256, sm_count() * 32);
  {
    KernelTimer kt(SAAMG_KT_SPGEMM, n, s);
    if (st.G == 16)
      at_lists_k<16><<<blocks, 256, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, agg, st.lcol.p,
                                            st.lval.p, cnt.p);
    else if (sortable)
      at_lists_sorted_k<<<blocks, 256, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, agg, st.lcol.p,
                                               st.lval.p, cnt.p);
    else
      at_lists_k<32><<<blocks, 256, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, agg, st.lcol.p,
                                            st.lval.p, cnt.p);
    SAAMG_LAUNCH();
  }
  fill_int(cnt.p + n, 0, 1, s);
  P.nnz = exclusive_scan(cnt.p, P.rowptr.p, n + 1, s);
}

void prolongator_finish(ProlongState& st, const double* invd, double omega, DevCsr& P,
                        cudaStream_t s) {
  if (st.final_values) {  // formed with omega already
    P = std::move(st.AT);
    return;
  }
  if (!st.lists) {
    smoothed_prolongator(st.AT, st.agg, invd, omega, P, s);
    return;
  }
  const int n = st.n;
  const DevCsr& A = *st.A;
  P.n = n;
  P.m = st.nagg;
  P.nnz = st.AT.nnz;
  P.rowptr = std::move(st.AT.rowptr);
  P.col.alloc(P.nnz, s);
  P.val.alloc(P.nnz, s);
  const int blocks = (int)std::min<long long>(((long long)n * st.G + 255) / 256, sm_count() * 32);
  KernelTimer kt(SAAMG_KT_SPGEMM, n, s);
  if (st.G == 16)
    at_prolong_k<16><<<blocks, 256, 0, s>>>(n, A.rowptr.p, st.lcol.p, st.lval.p, P.rowptr.p,
                                            st.agg, invd, omega, P.col.p, P.val.p);
  else
    at_prolong_k<32><<<blocks, 256, 0, s>>>(n, A.rowptr.p, st.lcol.p, st.lval.p, P.rowptr.p,
                                            st.agg, invd, omega, P.col.p, P.val.p);
  SAAMG_LAUNCH();
}

void prolongator(const DevCsr& A, const int* agg, int nagg, const double* invd, double omega,
                 DevCsr& P, cudaStream_t s) {
  ProlongState st;
  prolongator_start(A, agg, nagg, st, s);
  prolongator_finish(st, invd, omega, P, s);
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
  exclusive_scan_async(cnt.p, R.rowptr.p, P.m + 1, s);  // the total is P.nnz
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
  if (R.n > 0 && R.n < 65536 && P.nnz > 64LL * R.n) {  // few long rows
    rank_rows_block_k<<<std::min(R.n, sm_count() * 8), 256, 0, s>>>(R.n, R.rowptr.p, tcol.p, tval.p,
                                                            R.col.p, R.val.p);
    SAAMG_LAUNCH();
  } else if (R.n > 0) {
    long long warps = R.n;
    int blocks = (int)std::min<long long>((warps * 32 + 255) / 256, sm_count() * 32);
    rank_rows_k<<<blocks, 256, 0, s>>>(R.n, R.rowptr.p, tcol.p, tval.p, R.col.p, R.val.p,
                                       P.n < (1 << 26));
    SAAMG_LAUNCH();
  }
}

void transpose_known(const DevCsr& P, const DevCsr& known, DevCsr& R, cudaStream_t s) {
  if (known.n != P.m || known.m != P.n || known.nnz != P.nnz)
    fail(SAAMG_EINVAL, "known transpose pattern has other sizes");
  R.n = P.m;
  R.m = P.n;
  R.nnz = P.nnz;
  R.rowptr.alloc(R.n + 1, s);
  R.col.alloc(R.nnz, s);
  R.val.alloc(R.nnz, s);
  SAAMG_CUDA(cudaMemcpyAsync(R.rowptr.p, known.rowptr.p, sizeof(int) * (R.n + 1),
                             cudaMemcpyDeviceToDevice, s));
  if (R.nnz == 0) return;
  SAAMG_CUDA(cudaMemcpyAsync(R.col.p, known.col.p, sizeof(int) * R.nnz, cudaMemcpyDeviceToDevice, s));
  transpose_known_k<<<blocks_for(P.n), 256, 0, s>>>(P.n, P.rowptr.p, P.col.p, P.val.p,
                                                    known.rowptr.p, known.col.p, R.val.p);
  SAAMG_LAUNCH();
}

}  // namespace saamg
