// Coarsest-level direct solver (Sec. 3.2, "Coarse level solver"; Algorithm 1,
// DirectSolve).  The paper factors A_L with KLU; here A_L is small (<= max_coarse) and
// is factored densely in FP64 with partial pivoting (largest |a_ik|, lowest row on ties),
// then inverted once so that every V-cycle applies x = A_L^-1 b as one dense product.
// All dense arrays are column-major: a(i, j) at [j * n + i].
#include "coarse.cuh"

namespace saamg {

namespace {

__global__ void densify_k(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                          const double* __restrict__ val, double* __restrict__ a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) a[(size_t)col[p] * n + i] = val[p];
}

// Step k, one block: pivot search in column k, row swap k <-> p over all columns,
// multipliers l_ik = a_ik / a_kk stored below the diagonal.
__global__ void lu_pivot_k(int n, int k, double* __restrict__ a, int* __restrict__ perm,
                           int* __restrict__ err) {
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  double best = -1.0;
  int bidx = n;
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    double v = fabs(a[(size_t)k * n + i]);
    if (v > best || (v == best && i < bidx)) {
      best = v;
      bidx = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double v = bv[threadIdx.x + w];
      int i = bi[threadIdx.x + w];
      if (v > bv[threadIdx.x] || (v == bv[threadIdx.x] && i < bi[threadIdx.x])) {
        bv[threadIdx.x] = v;
        bi[threadIdx.x] = i;
      }
    }
    __syncthreads();
  }
  const int p = bi[0];
  if (!(bv[0] > 0.0)) {
    if (threadIdx.x == 0) atomicOr(err, 1);
    return;
  }
  if (p != k) {
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      double t = a[(size_t)j * n + k];
      a[(size_t)j * n + k] = a[(size_t)j * n + p];
      a[(size_t)j * n + p] = t;
    }
    if (threadIdx.x == 0) {
      int t = perm[k];
      perm[k] = perm[p];
      perm[p] = t;
    }
  }
  __syncthreads();
  const double piv = a[(size_t)k * n + k];
  for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) a[(size_t)k * n + i] /= piv;
}

// Step k: trailing update a_ij -= l_ik a_kj for i, j > k.
__global__ void lu_update_k(int n, int k, double* __restrict__ a) {
  const int m = n - k - 1;
  const int i = k + 1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double lik = a[(size_t)k * n + i];
  for (int j = k + 1 + blockIdx.y; j < n; j += gridDim.y) a[(size_t)j * n + i] -= lik * a[(size_t)j * n + k];
  (void)m;
}

__global__ void perm_init_k(int n, int* perm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) perm[i] = i;
}

// Warp per column c of A^-1: solve L U x = P e_c (forward then backward substitution,
// column-oriented, lanes over rows).  Output column-major.
__global__ void lu_inverse_k(int n, const double* __restrict__ lu, const int* __restrict__ perm,
                             double* __restrict__ inv) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= n) return;
  double* x = inv + (size_t)c * n;
  for (int i = lane; i < n; i += 32) x[i] = (perm[i] == c) ? 1.0 : 0.0;
  __syncwarp();
  for (int j = 0; j < n; ++j) {
    const double xj = x[j];
    __syncwarp();
    if (xj != 0.0)
      for (int i = j + 1 + lane; i < n; i += 32) x[i] -= lu[(size_t)j * n + i] * xj;
    __syncwarp();
  }
  for (int j = n - 1; j >= 0; --j) {
    double xj = 0.0;
    if (lane == 0) {
      xj = x[j] / lu[(size_t)j * n + j];
      x[j] = xj;
    }
    xj = __shfl_sync(0xffffffffu, xj, 0);
    __syncwarp();
    if (xj != 0.0)
      for (int i = lane; i < j; i += 32) x[i] -= lu[(size_t)j * n + i] * xj;
    __syncwarp();
  }
}

// x_i = sum_c inv(i, c) b_c, FP64 accumulation.
template <class TV>
__global__ void coarse_apply_k(int n, const double* __restrict__ inv, const TV* __restrict__ b,
                               TV* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int c = 0; c < n; ++c) acc += inv[(size_t)c * n + i] * (double)b[c];
  x[i] = (TV)acc;
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

void coarse_factor(const DevCsr& A, CoarseSolver& cs, cudaStream_t s) {
  const int n = A.n;
  cs.n = n;
  cs.inv.alloc((size_t)n * n, s);
  if (n == 0) return;
  Buf<double> lu;
  Buf<int> perm, err;
  lu.alloc((size_t)n * n, s);
  perm.alloc(n, s);
  err.alloc(1, s);
  SAAMG_CUDA(cudaMemsetAsync(lu.p, 0, sizeof(double) * (size_t)n * n, s));
  fill_int(err.p, 0, 1, s);
  densify_k<<<(n + 255) / 256, 256, 0, s>>>(n, A.rowptr.p, A.col.p, A.val.p, lu.p);
  SAAMG_LAUNCH();
  perm_init_k<<<(n + 255) / 256, 256, 0, s>>>(n, perm.p);
  SAAMG_LAUNCH();
  for (int k = 0; k < n; ++k) {
    lu_pivot_k<<<1, 1024, 0, s>>>(n, k, lu.p, perm.p, err.p);
    SAAMG_LAUNCH();
    int m = n - k - 1;
    if (m > 0) {
      dim3 grid((m + 127) / 128, m < 64 ? m : 64);
      lu_update_k<<<grid, 128, 0, s>>>(n, k, lu.p);
      SAAMG_LAUNCH();
    }
  }
  int herr = 0;
  d2h_sync(&herr, err.p, sizeof(int), s);
  if (herr) fail(SAAMG_NUMERICAL, "zero pivot in the coarse LU");
  lu_inverse_k<<<(n * 32 + 255) / 256, 256, 0, s>>>(n, lu.p, perm.p, cs.inv.p);
  SAAMG_LAUNCH();
  SAAMG_CUDA(cudaStreamSynchronize(s));
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
  coarse_apply_k<TV><<<(cs.n + 127) / 128, 128, 0, s>>>(cs.n, cs.inv.p, b, x);
  SAAMG_LAUNCH();
}

template void coarse_apply<double>(const CoarseSolver&, const double*, double*, cudaStream_t);
template void coarse_apply<float>(const CoarseSolver&, const float*, float*, cudaStream_t);

}  // namespace saamg
