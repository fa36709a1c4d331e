// Coarsest-level direct solver (Sec. 3.2, "Coarse level solver"; Algorithm 1,
// DirectSolve).  The paper factors A_L with KLU; here A_L is small (<= max_coarse) and its
// inverse is formed once, densely in FP64, by Gauss-Jordan elimination with the pivoting of
// an LU with partial pivoting (largest |a_ik|, lowest row on ties), so that every V-cycle
// applies x = A_L^-1 b as one dense product.
// The elimination works on column-major arrays, a(i, j) at [j * n + i]; the finished inverse
// is stored by rows, A_L^-1(i, j) at [i * n + j], for the per-cycle product.
#include "coarse.cuh"
#include "rows.cuh"

namespace saamg {

namespace {

__global__ void densify_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                          const double* __restrict__ val, double* __restrict__ a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) a[(size_t)col[p] * n + i] = val[p];
}

// --- explicit inverse by Gauss-Jordan elimination ------------------------------------
// Partial pivoting as in the LU: at step k the pivot is the row i >= k of largest |a_ik|
// (lowest row on ties); rows k and p are exchanged and column k is eliminated from every
// other row, which leaves (P A)^-1 in place; the columns are unscrambled at the end.
// One launch per step: each block owns a range of columns, so all writes of a step stay in
// the writer's own columns.  Column k is read from a copy (made in the previous step by the
// owner of that column, together with its pivot row), so no block reads a column that
// another block is writing.

// Block argmax of |col[i]| over i in [lo, n), lowest index on ties.
__device__ void block_argmax(const double* __restrict__ col, int lo, int n, double* sv, int* si,
                             double& best_out, int& idx_out) {
  double best = -1.0;
  int bi = n;
  for (int i = lo + threadIdx.x; i < n; i += blockDim.x) {
    const double v = fabs(col[i]);
    if (v > best) {
      best = v;
      bi = i;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double v = sv[threadIdx.x + w];
      const int i = si[threadIdx.x + w];
      if (v > sv[threadIdx.x] || (v == sv[threadIdx.x] && i < si[threadIdx.x])) {
        sv[threadIdx.x] = v;
        si[threadIdx.x] = i;
      }
    }
    __syncthreads();
  }
  best_out = sv[0];
  idx_out = si[0];
}

constexpr int kGjThreads = 256;
constexpr int kGjMaxCols = 64;  // columns per block

// step 0: pivot of column 0 and its copy
__global__ void __launch_bounds__(kGjThreads) gj_first_k(int n, const double* __restrict__ a,
                                                         double* __restrict__ colk,
                                                         int* __restrict__ pivrow,
                                                         int* __restrict__ err) {
  __shared__ double sv[kGjThreads];
  __shared__ int si[kGjThreads];
  double best;
  int p;
  block_argmax(a, 0, n, sv, si, best, p);
  if (threadIdx.x == 0) {
    // a zero or NaN column: flagged, and the pivot index stays a valid row
    if (!(best > 0.0)) {
      atomicOr(err, 1);
      p = 0;
    }
    pivrow[0] = p;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) colk[i] = a[i];
}

__global__ void __launch_bounds__(kGjThreads) gj_step_k(int n, int k, int cpb,
                                                        double* __restrict__ a,
                                                        const double* __restrict__ colk,
                                                        double* __restrict__ colk_next,
                                                        int* __restrict__ pivrow,
                                                        int* __restrict__ err) {
  __shared__ double rk[kGjMaxCols], rp[kGjMaxCols];
  __shared__ double sv[kGjThreads / 32];
  __shared__ int si[kGjThreads / 32];
  const int p = pivrow[k];
  const double piv = colk[p];  // a_kk after the exchange
  const double ip = 1.0 / piv;
  const int c0 = blockIdx.x * cpb, c1 = min(n, c0 + cpb);
  for (int t = threadIdx.x; t < c1 - c0; t += blockDim.x) {
    const size_t o = (size_t)(c0 + t) * n;
    rk[t] = a[o + k];
    rp[t] = a[o + p];
  }
  __syncthreads();
  // the owner of column k + 1 updates it first, copies it for the next step and finds its
  // pivot on the way (largest |a_i,k+1| over i > k, lowest row on ties)
  const int kn = k + 1;
  const bool owner = kn < n && kn >= c0 && kn < c1;
  double best = -1.0;
  int bi = n;
  for (int tt = 0; tt < c1 - c0; ++tt) {
    const int t = owner ? (tt == 0 ? kn - c0 : (tt <= kn - c0 ? tt - 1 : tt)) : tt;
    const int j = c0 + t;
    const double r = rp[t] * ip;  // the new row k (row p before the exchange)
    double* col = a + (size_t)j * n;
    const bool next = j == kn;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double ci = i == k ? colk[p] : (i == p ? colk[k] : colk[i]);  // column k, exchanged
      double v;
      if (j == k) v = i == k ? ip : -ci * ip;
      else if (i == k) v = r;
      else v = (i == p ? rk[t] : col[i]) - ci * r;
      col[i] = v;
      if (next) {
        colk_next[i] = v;
        const double av = fabs(v);
        if (i > k && av > best) {  // ascending i per thread: the first maximum is kept
          best = av;
          bi = i;
        }
      }
    }
  }
  if (owner) {
    // block argmax of (best, bi), lowest index on ties
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if ((threadIdx.x & 31) == 0) {
      sv[threadIdx.x >> 5] = best;
      si[threadIdx.x >> 5] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double bb = sv[0];
      int ii = si[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (sv[w] > bb || (sv[w] == bb && si[w] < ii)) {
          bb = sv[w];
          ii = si[w];
        }
      if (!(bb > 0.0)) {  // a zero or NaN column: flagged, the pivot stays a valid row
        atomicOr(err, 1);
        ii = kn;
      }
      pivrow[kn] = ii;
    }
  }
}

// Panel form with the panel factored in every block (no exchange between blocks inside a
// launch).  A launch takes b pivot steps k0 .. k0 + b - 1.  Each block loads those b columns
// and runs the b steps on them in shared memory: pivot search, exchanged column c_s, and the
// step on the panel columns not yet pivoted.  It then moves its own columns through the b
// steps (a panel column from its own step on, where it becomes 1 / pivot in row k and
// -c_s(i) / pivot elsewhere).  For one column only the rows k_s and p_s follow special
// formulas; one warp walks those rows (one per lane) through the steps, which gives
// r_s = x_{p_s} / pivot_s of every step, and every other row takes x <- x - c_s(i) r_s.
// Every element sees the operations of the one-launch-per-step form in the same order.  A
// launch reads src and writes every column to dst, so no block overwrites a column that
// another block of the same launch may still be loading.  The own columns are copied to
// shared memory asynchronously while the panel is factored.
constexpr int kGjRpThreads = 256;

// Pivot keys: the bits of |v| as an integer, which order like |v| for every non-NaN v; a NaN
// gets -1 and is never chosen, as with a floating-point comparison.  The search then runs
// on the integer units instead of the FP64 pipe.
__device__ __forceinline__ long long pivot_key(double v) {
  const long long b = __double_as_longlong(v) & 0x7fffffffffffffffLL;
  return b > 0x7ff0000000000000LL ? -1LL : b;
}

// (key, index) maximum over a warp, lowest index on ties; every lane holds the result
__device__ __forceinline__ void rp_warp_argmax(long long& best, int& bi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) {
      best = ob;
      bi = oi;
    }
  }
}

// the same over the block; after the barrier inside, every lane of warp 0 holds the result
__device__ __forceinline__ void rp_block_argmax(long long& best, int& bi, long long* sv, int* si) {
  rp_warp_argmax(best, bi);
  if ((threadIdx.x & 31) == 0) {
    sv[threadIdx.x >> 5] = best;
    si[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    best = threadIdx.x < nw ? sv[threadIdx.x] : -1LL;
    bi = threadIdx.x < nw ? si[threadIdx.x] : 0x7fffffff;
    rp_warp_argmax(best, bi);
  }
}

template <int B, int NT, bool STAGE>
__global__ void __launch_bounds__(NT) gj_rp_k(int n, int k0, int cpb,
                                                        const double* __restrict__ src,
                                                        double* __restrict__ dst,
                                                        int* __restrict__ pivrow,
                                                        int* __restrict__ err) {
  extern __shared__ double rp_smem[];
  double* pan = rp_smem;                      // B columns of n
  double* cs = rp_smem + (size_t)B * n;       // c_s of every step, B x n
  // the block's own columns: a shared copy, or (too large for it) src itself
  const double* own;
  __shared__ long long sv[NT / 32];
  __shared__ int si[NT / 32];
  __shared__ int sp[B];
  __shared__ double sip[B], s_xk[B], s_r[B];
  __shared__ double s_ck, s_cp;
  __shared__ int srow[2 * B];
  __shared__ int nspec;
  __shared__ double rr[kGjMaxCols][B];        // r_s of each own column
  __shared__ double fin[kGjMaxCols][2 * B];  // final values of its special rows
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int bw = min(B, n - k0);
  const int c0 = blockIdx.x * cpb, c1 = min(n, c0 + cpb);
  const int ncols = max(0, c1 - c0), nown = ncols * n;
  if constexpr (STAGE) {
    double* own_s = rp_smem + (size_t)2 * B * n;
    for (int e = tid; e < nown; e += nt) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(own_s + e);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d),
                   "l"(src + (size_t)c0 * n + e)
                   : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    own = own_s;
  } else {
    own = src + (size_t)c0 * n;
  }
  for (int e = tid; e < bw * n; e += nt) pan[e] = src[(size_t)k0 * n + e];
  __syncthreads();
  // pivot search of the first panel column (rows k0 .. n - 1; ascending i per thread keeps
  // the first maximum)
  long long best = -1;
  int bi = n;
  for (int i = k0 + tid; i < n; i += nt) {
    const long long v = pivot_key(pan[i]);
    if (v > best) {
      best = v;
      bi = i;
    }
  }
  for (int s = 0; s < bw; ++s) {
    const int k = k0 + s;
    rp_block_argmax(best, bi, sv, si);
    if (tid < 32) {
      if (best <= 0) {  // a zero or NaN column: flagged, the pivot stays a valid row
        if (blockIdx.x == 0 && tid == 0) atomicOr(err, 1);
        bi = k;
      }
      const double* col = pan + (size_t)s * n;
      const double ip = 1.0 / col[bi];
      if (tid == 0) {
        sp[s] = bi;
        sip[s] = ip;
        s_ck = col[k];
        s_cp = col[bi];
      }
      if (tid < bw) {
        s_xk[tid] = pan[(size_t)tid * n + k];
        s_r[tid] = pan[(size_t)tid * n + bi] * ip;  // the new row k (row p before the exchange)
      }
    }
    __syncthreads();
    const int p = sp[s];
    const double ip = sip[s], ck = s_ck, cpv = s_cp;
    double* c = cs + (size_t)s * n;
    // c_s (column k with rows k and p exchanged), the step on the panel columns still to be
    // pivoted and the pivot search of the next one (rows > k), row by row
    best = -1;
    bi = n;
    for (int i = tid; i < n; i += nt) {
      const double ci = i == k ? cpv : (i == p ? ck : pan[(size_t)s * n + i]);
      c[i] = ci;
#pragma unroll
      for (int j = 0; j < B; ++j) {
        if (j >= bw) break;
        if (j <= s) continue;  // pivoted panel columns are finished by their owner
        const double v =
            i == k ? s_r[j] : (i == p ? s_xk[j] : pan[(size_t)j * n + i]) - ci * s_r[j];
        pan[(size_t)j * n + i] = v;
        if (j == s + 1 && i > k) {
          const long long av = pivot_key(v);
          if (av > best) {
            best = av;
            bi = i;
          }
        }
      }
    }
  }
  // the special rows: k0 .. k0 + bw - 1 and the pivot rows, each once
  if (tid == 0) {
    int m = 0;
    for (int s = 0; s < bw; ++s) srow[m++] = k0 + s;
    for (int s = 0; s < bw; ++s) {
      bool seen = false;
      for (int u = 0; u < m; ++u) seen |= srow[u] == sp[s];
      if (!seen) srow[m++] = sp[s];
    }
    nspec = m;
    if (blockIdx.x == 0)
      for (int s = 0; s < bw; ++s) pivrow[k0 + s] = sp[s];
  }
  if constexpr (STAGE) asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  const int m = nspec;
  // one warp per own column walks its special rows (one per lane) through the b steps
  for (int t = warp; t < ncols; t += nw) {
    const int j = c0 + t;
    // a panel column starts after its own step s0: the inverse's column, 1 / pivot in row
    // k_s0 and -c_s0(i) / pivot elsewhere
    const int s0 = j >= k0 && j < k0 + bw ? j - k0 : -1;
    const int row = lane < m ? srow[lane] : -1;
    double x = 0.0;
    if (lane < m) {
      if (s0 < 0) x = own[(size_t)t * n + row];
      else x = row == k0 + s0 ? sip[s0] : -cs[(size_t)s0 * n + row] * sip[s0];
    }
    for (int s = s0 + 1; s < bw; ++s) {
      const int k = k0 + s, p = sp[s];
      const int uk = __ffs(__ballot_sync(0xffffffffu, row == k)) - 1;
      const int up = __ffs(__ballot_sync(0xffffffffu, row == p)) - 1;
      const double r = __shfl_sync(0xffffffffu, x, up) * sip[s];  // the new row k
      const double xk = __shfl_sync(0xffffffffu, x, uk);
      if (lane == 0) rr[t][s] = r;
      if (lane < m) {
        const double ci = cs[(size_t)s * n + row];
        x = row == k ? r : (row == p ? xk : x) - ci * r;
      }
    }
    if (lane < m) fin[t][lane] = x;
  }
  __syncthreads();
  // every row of the own columns: x <- x - c_s(i) r_s over the steps s > s0 (the special
  // rows are rewritten below)
  {
    int t = tid / max(n, 1), i = tid - t * n;
    for (int e = tid; e < nown; e += nt) {
      const int j = c0 + t;
      const int s0 = j >= k0 && j < k0 + bw ? j - k0 : -1;
      double x;
      if (s0 < 0) x = own[e];
      else x = i == k0 + s0 ? sip[s0] : -cs[(size_t)s0 * n + i] * sip[s0];
#pragma unroll
      for (int s = 0; s < B; ++s)
        if (s > s0 && s < bw) x = x - cs[(size_t)s * n + i] * rr[t][s];
      dst[(size_t)c0 * n + e] = x;
      i += nt;
      while (i >= n) {
        i -= n;
        ++t;
      }
    }
  }
  __syncthreads();
  for (int e = tid; e < ncols * m; e += nt) {
    const int t = e / m, u = e - t * m;
    dst[(size_t)(c0 + t) * n + srow[u]] = fin[t][u];
  }
}

// inverse(:, j) = work(:, q_j), q: the exchanges undone in reverse order (one thread)
__global__ void gj_perm_k(int n, const int* __restrict__ pivrow, int* __restrict__ q) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int j = 0; j < n; ++j) q[j] = j;
  for (int k = n - 1; k >= 0; --k) {
    const int p = pivrow[k];
    const int t = q[k];
    q[k] = q[p];
    q[p] = t;
  }
}

// inverse(i, j) = work(i, q_j), stored by rows: a 32 x 32 tile read along the work's columns
// and written along the inverse's rows through shared memory (q = NULL: a plain transpose)
__global__ void __launch_bounds__(256) gj_gather_k(int n, const double* __restrict__ w,
                                                   const int* __restrict__ q,
                                                   double* __restrict__ inv) {
  __shared__ double tile[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int jj = ty; jj < 32; jj += 8) {
    const int j = j0 + jj, i = i0 + tx;
    if (j < n && i < n) tile[jj][tx] = w[(size_t)(q ? q[j] : j) * n + i];
  }
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, j = j0 + tx;
    if (i < n && j < n) inv[(size_t)i * n + j] = tile[tx][ii];
  }
}

// x_i = sum_c inv(i, c) b_c, FP64 accumulation: one warp per row (the row is contiguous, so
// every load is coalesced), lane l summing the columns c = l mod 32, the lanes' partial sums
// added by a fixed butterfly
constexpr int kGemvWarps = 8;

template <class TV>
__global__ void __launch_bounds__(32 * kGemvWarps) coarse_apply_k(int n,
                                                                  const double* __restrict__ inv,
                                                                  const TV* __restrict__ b,
                                                                  TV* __restrict__ x) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kGemvWarps + (threadIdx.x >> 5);
  if (i >= n) return;  // whole warps leave together
  rows::gemv_row<TV>(i, n, lane, inv, b, x);
}

// --- Gauss-Seidel (one CTA) ---------------------------------------------------------
constexpr int kGsThreads = 1024;
constexpr int kGsMaxColours = 256;

__device__ __forceinline__ uint32_t fmix32_gs(uint32_t h) {  // MurmurHash3 finaliser
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ unsigned long long gs_key(const unsigned* ids, int v) {
  const uint32_t id = ids ? ids[v] : (uint32_t)v;
  return ((unsigned long long)fmix32_gs(id ^ 0x2545F491u) << 32) | id;
}

// Colouring by synchronous rounds, then a stable sort of the rows by colour (order, coff).
// pick: n bytes of scratch.  err: set when more than kGsMaxColours colours are needed.
__global__ void __launch_bounds__(kGsThreads) gs_colour_k(int n, const int* __restrict__ rowptr,
                                                          const int* __restrict__ col,
                                                          const unsigned* __restrict__ ids,
                                                          int* __restrict__ colour,
                                                          unsigned char* __restrict__ pick,
                                                          int* __restrict__ order,
                                                          int* __restrict__ coff,
                                                          int* __restrict__ ncol_out) {
  __shared__ int left, wcount[kGsThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < n; i += blockDim.x) colour[i] = -1;
  if (tid == 0) left = n;
  __syncthreads();
  int c = 0;
  while (left > 0 && c < kGsMaxColours) {
    for (int i = tid; i < n; i += blockDim.x) {
      unsigned char pk = 0;
      if (colour[i] < 0) {
        const unsigned long long ki = gs_key(ids, i);
        pk = 1;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
          const int j = col[p];
          if (j != i && colour[j] < 0 && gs_key(ids, j) > ki) pk = 0;
        }
      }
      pick[i] = pk;
    }
    __syncthreads();
    int got = 0;
    for (int i = tid; i < n; i += blockDim.x)
      if (pick[i]) {
        colour[i] = c;
        ++got;
      }
    got = __reduce_add_sync(0xffffffffu, got);
    if (lane == 0 && got) atomicSub(&left, got);
    ++c;
    __syncthreads();
  }
  const int ncol = left > 0 ? -1 : c;
  if (tid == 0) *ncol_out = ncol;
  if (ncol < 0) return;
  // stable partition by colour: for each colour, rows in ascending order
  int base = 0;
  for (int cc = 0; cc < ncol; ++cc) {
    if (tid == 0) coff[cc] = base;
    for (int b0 = 0; b0 < n; b0 += blockDim.x) {
      const int i = b0 + tid;
      const bool f = i < n && colour[i] == cc;
      const unsigned bal = __ballot_sync(0xffffffffu, f);
      if (lane == 0) wcount[warp] = __popc(bal);
      __syncthreads();
      int before = 0, total = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        before += w < warp ? wcount[w] : 0;
        total += wcount[w];
      }
      if (f) order[base + before + __popc(bal & ((1u << lane) - 1u))] = i;
      base += total;
      __syncthreads();
    }
  }
  if (tid == 0) coff[ncol] = base;
}

// `steps` symmetric sweeps from x = 0; x and b in shared memory (FP64); warp per row,
// lanes over the row's entries, shuffle reduction in a fixed order.
template <class TV>
__global__ void __launch_bounds__(kGsThreads) gs_apply_k(int n, const int* __restrict__ rowptr,
                                                         const int* __restrict__ col,
                                                         const double* __restrict__ val,
                                                         const double* __restrict__ invd,
                                                         const int* __restrict__ order,
                                                         const int* __restrict__ coff, int ncol,
                                                         int steps, const TV* __restrict__ b,
                                                         TV* __restrict__ x) {
  extern __shared__ double gs_sm[];
  double* xs = gs_sm;
  double* bs = gs_sm + n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  for (int i = tid; i < n; i += blockDim.x) {
    xs[i] = 0.0;
    bs[i] = (double)b[i];
  }
  __syncthreads();
  for (int st = 0; st < steps; ++st)
    for (int half = 0; half < 2; ++half)
      for (int cc = 0; cc < ncol; ++cc) {
        const int c = half == 0 ? cc : ncol - 1 - cc;
        for (int k = coff[c] + warp; k < coff[c + 1]; k += nwarp) {
          const int i = order[k];
          double acc = 0.0;
          for (int p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
            const int j = col[p];
            if (j != i) acc += val[p] * xs[j];
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) xs[i] = (bs[i] - acc) * invd[i];
        }
        __syncthreads();
      }
  for (int i = tid; i < n; i += blockDim.x) x[i] = (TV)xs[i];
}

}  // namespace

void coarse_gs_setup(const DevCsr& A, const double* invd, const unsigned* ids, int steps,
                     CoarseSolver& cs, cudaStream_t s) {
  const int n = A.n;
  if (n > kCoarseGsMax) fail(SAAMG_UNIMPLEMENTED, "Gauss-Seidel coarse level above 12288 rows");
  cs.kind = SAAMG_COARSE_GS;
  cs.n = n;
  cs.steps = steps;
  cs.rowptr = A.rowptr.p;
  cs.col = A.col.p;
  cs.val = A.val.p;
  cs.invd = invd;
  // shared-memory opt-in for the largest coarse level (set outside any stream capture)
  const int smax = (int)(2 * kCoarseGsMax * sizeof(double));
  SAAMG_CUDA(cudaFuncSetAttribute(gs_apply_k<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smax));
  SAAMG_CUDA(cudaFuncSetAttribute(gs_apply_k<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  smax));
  cs.colour.alloc(n, s);
  cs.order.alloc(n, s);
  cs.coff.alloc(kGsMaxColours + 1, s);
  if (n == 0) return;
  Buf<unsigned char> pick;
  Buf<int> ncol;
  pick.alloc(n, s);
  ncol.alloc(1, s);
  gs_colour_k<<<1, kGsThreads, 0, s>>>(n, A.rowptr.p, A.col.p, ids, cs.colour.p, pick.p,
                                       cs.order.p, cs.coff.p, ncol.p);
  SAAMG_LAUNCH();
  int h = 0;
  d2h_sync(&h, ncol.p, sizeof(int), s);
  if (h <= 0) fail(SAAMG_NUMERICAL, "coarse-level colouring needs more than 256 colours");
  cs.ncolours = h;
}

// A^-1 by Gauss-Jordan elimination of the column-major n x n work array w (overwritten),
// written by rows to inv; synchronises to read the zero-pivot flag
static void gauss_jordan_inverse(int n, Buf<double>& w, double* inv, cudaStream_t s) {
  Buf<double> w2, colk;
  Buf<int> pivrow, q, err;
  colk.alloc(2 * (size_t)n, s);
  pivrow.alloc(n, s);
  q.alloc(n, s);
  err.alloc(1, s);
  fill_int(err.p, 0, 1, s);
  // b pivot steps per launch with the panel factored in every block (one block per SM, its
  // own columns in a contiguous range); the panel and the b exchanged columns must fit
  // shared memory, else one launch per step
  const int nsm = sm_count();
  const int rcpb = (n + nsm - 1) / nsm;
  // the widest panel (5 .. 2 steps) whose shared arrays fit, with the own columns staged if
  // possible
  constexpr size_t kRpSmem = 212u << 10;
  int B = 0;
  bool stage = false;
  for (int b = 5; b >= 2 && !B; --b)
    if ((size_t)(2 * b + rcpb) * n * sizeof(double) <= kRpSmem) B = b, stage = true;
  for (int b = 5; b >= 2 && !B; --b)
    if ((size_t)(2 * b) * n * sizeof(double) <= kRpSmem) B = b;
  if (B && rcpb <= kGjMaxCols) {
    const size_t rsm = (size_t)(2 * B + (stage ? rcpb : 0)) * n * sizeof(double);
    const int rblocks = (n + rcpb - 1) / rcpb;
    w2.alloc((size_t)n * n, s);
    auto run = [&](auto kern) {
      SAAMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
      for (int k0 = 0; k0 < n; k0 += B) {
        kern<<<rblocks, kGjRpThreads, rsm, s>>>(n, k0, rcpb, w.p, w2.p, pivrow.p, err.p);
        SAAMG_LAUNCH();
        w.swap(w2);
      }
    };
    switch (B * 2 + (stage ? 1 : 0)) {
      case 11: run(gj_rp_k<5, kGjRpThreads, true>); break;
      case 10: run(gj_rp_k<5, kGjRpThreads, false>); break;
      case 9: run(gj_rp_k<4, kGjRpThreads, true>); break;
      case 8: run(gj_rp_k<4, kGjRpThreads, false>); break;
      case 7: run(gj_rp_k<3, kGjRpThreads, true>); break;
      case 6: run(gj_rp_k<3, kGjRpThreads, false>); break;
      case 5: run(gj_rp_k<2, kGjRpThreads, true>); break;
      default: run(gj_rp_k<2, kGjRpThreads, false>); break;
    }
  } else {
    gj_first_k<<<1, kGjThreads, 0, s>>>(n, w.p, colk.p, pivrow.p, err.p);
    SAAMG_LAUNCH();
    // about two blocks per SM, at most kGjMaxCols columns each
    const int cpb = std::min(kGjMaxCols, std::max(1, (n + 303) / 304));
    const int blocks = (n + cpb - 1) / cpb;
    for (int k = 0; k < n; ++k) {
      gj_step_k<<<blocks, kGjThreads, 0, s>>>(n, k, cpb, w.p, colk.p + (size_t)(k & 1) * n,
                                              colk.p + (size_t)((k + 1) & 1) * n, pivrow.p,
                                              err.p);
      SAAMG_LAUNCH();
    }
  }
  gj_perm_k<<<1, 32, 0, s>>>(n, pivrow.p, q.p);
  SAAMG_LAUNCH();
  const dim3 tiles((n + 31) / 32, (n + 31) / 32);
  gj_gather_k<<<tiles, 256, 0, s>>>(n, w.p, q.p, inv);
  SAAMG_LAUNCH();
  int herr = 0;
  d2h_sync(&herr, err.p, sizeof(int), s);
  if (herr) fail(SAAMG_NUMERICAL, "zero pivot in the coarse factorisation");
}

void coarse_factor(const DevCsr& A, CoarseSolver& cs, cudaStream_t s) {
  const int n = A.n;
  cs.n = n;
  cs.inv.alloc((size_t)n * n, s);
  if (n == 0) return;
  Buf<double> w;
  w.alloc((size_t)n * n, s);
  SAAMG_CUDA(cudaMemsetAsync(w.p, 0, sizeof(double) * (size_t)n * n, s));
  densify_k<<<(n + 255) / 256, 256, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, w.p);
  SAAMG_LAUNCH();
  gauss_jordan_inverse(n, w, cs.inv.p, s);
}

void dense_inverse(int n, const double* a, double* inv, cudaStream_t s) {
  if (n == 0) return;
  Buf<double> w;
  w.alloc((size_t)n * n, s);
  const dim3 tiles((n + 31) / 32, (n + 31) / 32);
  gj_gather_k<<<tiles, 256, 0, s>>>(n, a, nullptr, w.p);  // rows of a -> columns of w
  SAAMG_LAUNCH();
  gauss_jordan_inverse(n, w, inv, s);
}

template <class TV>
void coarse_apply(const CoarseSolver& cs, const TV* b, TV* x, cudaStream_t s) {
  if (cs.n == 0) return;
  if (cs.kind == SAAMG_COARSE_GS) {
    const size_t sm = 2 * (size_t)cs.n * sizeof(double);
    gs_apply_k<TV><<<1, kGsThreads, sm, s>>>(cs.n, cs.rowptr, cs.col, cs.val, cs.invd,
                                             cs.order.p, cs.coff.p, cs.ncolours, cs.steps, b, x);
    SAAMG_LAUNCH();
    return;
  }
  launch_pdl(coarse_apply_k<TV>, (cs.n + kGemvWarps - 1) / kGemvWarps, 32 * kGemvWarps, 0, s,
             cs.n, cs.inv.p, b, x);
  SAAMG_LAUNCH();
}

template void coarse_apply<double>(const CoarseSolver&, const double*, double*, cudaStream_t);
template void coarse_apply<float>(const CoarseSolver&, const float*, float*, cudaStream_t);

}  // namespace saamg
