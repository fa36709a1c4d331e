// Device-wide exclusive prefix sums and small utilities.
#include "common.cuh"

namespace saamg {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 2;  // per thread
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive sum over the block (blockDim.x == kScanThreads); *agg receives the total.
__device__ long long block_exclusive_sum(long long v, long long* agg) {
  __shared__ long long warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    long long w = warp_tot[lane];
    long long winc = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long t = __shfl_up_sync(0xffffffffu, winc, o);
      if (lane >= o) winc += t;
    }
    warp_tot[lane] = winc - w;  // exclusive prefix of the warp totals
  }
  __syncthreads();
  long long excl = inc - v + warp_tot[wid];
  __shared__ long long total;
  if (threadIdx.x == kScanThreads - 1) total = excl + v;  // inclusive sum of the last thread
  __syncthreads();
  *agg = total;
  __syncthreads();
  return excl;
}

// Phase 1: each block scans one tile, writes tile-local exclusive sums and its total.
template <class TIn>
__global__ void scan_tiles(const TIn* __restrict__ in, int* __restrict__ out,
                           long long* __restrict__ tile_sum, int n) {
  long long v[kScanItems];
  long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  long long mine = 0;
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    v[t] = (base + t < n) ? (long long)in[base + t] : 0;
    mine += v[t];
  }
  long long agg;
  long long run = block_exclusive_sum(mine, &agg);
#pragma unroll
  for (int t = 0; t < kScanItems; ++t) {
    if (base + t < n) out[base + t] = (int)run;
    run += v[t];
  }
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = agg;
}

// Phase 2: one block scans the tile totals sequentially by chunks (carry in a register).
__global__ void scan_tile_sums(long long* __restrict__ tile_sum, int ntiles,
                               long long* __restrict__ total) {
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += kScanThreads) {
    int i = base + threadIdx.x;
    long long v = (i < ntiles) ? tile_sum[i] : 0, agg;
    v = block_exclusive_sum(v, &agg);
    if (i < ntiles) tile_sum[i] = v + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += agg;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Phase 3: add the tile offsets.
__global__ void scan_add(int* __restrict__ out, const long long* __restrict__ tile_sum, int n) {
  long long off = tile_sum[blockIdx.x];
  long long base = (long long)blockIdx.x * kScanTile;
  for (int t = threadIdx.x; t < kScanTile; t += blockDim.x) {
    long long i = base + t;
    if (i < n) out[i] = (int)((long long)out[i] + off);
  }
}

template <class TIn>
long long scan_impl(const TIn* in, int* out, int n, cudaStream_t s, bool readback = true) {
  if (n <= 0) return 0;
  int ntiles = (n + kScanTile - 1) / kScanTile;
  Buf<long long> tiles;
  tiles.alloc((size_t)ntiles + 1, s);
  scan_tiles<TIn><<<ntiles, kScanThreads, 0, s>>>(in, out, tiles.p, n);
  SAAMG_LAUNCH();
  scan_tile_sums<<<1, kScanThreads, 0, s>>>(tiles.p, ntiles, tiles.p + ntiles);
  SAAMG_LAUNCH();
  scan_add<<<ntiles, 256, 0, s>>>(out, tiles.p, n);
  SAAMG_LAUNCH();
  if (!readback) return -1;
  long long total = 0;
  d2h_sync(&total, tiles.p + ntiles, sizeof(long long), s);
  return total;
}

__global__ void fill_int_k(int* p, int v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void fill_double_k(double* p, double v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// Sums `count` partials in index order (one block, fixed tree), deterministic.
// With `inv_sqrt`, also writes 1 / sqrt(sum) (the power iteration's normalisation).
__global__ void sum_partials_k(const double* __restrict__ part, int count, double* out,
                               double* inv_sqrt) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) acc += part[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out = sh[0];
    if (inv_sqrt) *inv_sqrt = 1.0 / sqrt(sh[0]);
  }
}

}  // namespace

long long scan_u8_tiles_needed(int n) { return n > 0 ? (n + kScanTile - 1) / kScanTile + 1 : 1; }

long long exclusive_scan_u8_into(const unsigned char* in, int* out, int n, long long* tiles,
                                 cudaStream_t s) {
  if (n <= 0) return 0;
  int ntiles = (n + kScanTile - 1) / kScanTile;
  scan_tiles<unsigned char><<<ntiles, kScanThreads, 0, s>>>(in, out, tiles, n);
  SAAMG_LAUNCH();
  scan_tile_sums<<<1, kScanThreads, 0, s>>>(tiles, ntiles, tiles + ntiles);
  SAAMG_LAUNCH();
  scan_add<<<ntiles, 256, 0, s>>>(out, tiles, n);
  SAAMG_LAUNCH();
  long long total = 0;
  d2h_sync(&total, tiles + ntiles, sizeof(long long), s);
  return total;
}

long long exclusive_scan(const int* in, int* out, int n, cudaStream_t s) {
  return scan_impl<int>(in, out, n, s);
}

void exclusive_scan_async(const int* in, int* out, int n, cudaStream_t s) {
  scan_impl<int>(in, out, n, s, false);
}

long long exclusive_scan_u8(const unsigned char* in, int* out, int n, cudaStream_t s) {
  return scan_impl<unsigned char>(in, out, n, s);
}

void fill_int(int* p, int v, size_t n, cudaStream_t s) {
  if (n == 0) return;
  int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  fill_int_k<<<blocks, 256, 0, s>>>(p, v, n);
  SAAMG_LAUNCH();
}

void fill_double(double* p, double v, size_t n, cudaStream_t s) {
  if (n == 0) return;
  int blocks = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  fill_double_k<<<blocks, 256, 0, s>>>(p, v, n);
  SAAMG_LAUNCH();
}

void sum_partials(const double* partials, int count, double* out, cudaStream_t s,
                  double* inv_sqrt) {
  sum_partials_k<<<1, kRedThreads, 0, s>>>(partials, count, out, inv_sqrt);
  SAAMG_LAUNCH();
}

}  // namespace saamg
