// C ABI of libsaamg: handles, the setup of the SA-AMG hierarchy (Sec. 3.2), the V-cycle
// (Algorithm 1) and the PCG driver (Sec. 3.1).  Host code here only orchestrates; every
// arithmetic step runs in the kernels of the other translation units.
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "aggregate.cuh"
#include "batch.cuh"
#include "hier.cuh"
#include "coarse.cuh"
#include "csr.cuh"
#include "galerkin.cuh"
#include "operator.cuh"
#include "pcg.cuh"
#include "pic.cuh"
#include "sell.cuh"

namespace saamg {

// ---------------------------------------------------------------------------
// errors and allocation
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

void fail(saamg_status st, const std::string& msg) { throw Error{st, msg}; }

void set_last_error(const std::string& msg) { g_last_error = msg; }

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e) + " (" + file + ":" +
                  std::to_string(line) + ")";
  if (e == cudaErrorMemoryAllocation) throw Error{SAAMG_ENOMEM, m};
  throw Error{SAAMG_ECUDA, m};
}

static AllocHook g_alloc;

AllocHook current_allocator() { return g_alloc; }

namespace {

struct CachedBlock {
  void* p;
  cudaStream_t s;
  AllocHook hook;
};

constexpr size_t kPoolMaxBlock = 64ull << 20;
constexpr size_t kPoolMaxBytes = 1ull << 30;

std::mutex g_pool_mu;
std::multimap<size_t, CachedBlock> g_pool;  // rounded size -> free block
size_t g_pool_bytes = 0;

bool same_hook(const AllocHook& a, const AllocHook& b) {
  return a.alloc == b.alloc && a.free == b.free && a.ctx == b.ctx;
}

// size classes: multiples of 512 B up to 64 KB, then eight steps per power of two
size_t pool_class(size_t bytes) {
  if (bytes <= (64u << 10)) return (bytes + 511) & ~size_t(511);
  size_t top = size_t(1) << (63 - __builtin_clzll(bytes - 1));
  const size_t step = top >> 3;
  return (bytes + step - 1) / step * step;
}

void* raw_alloc(const AllocHook& h, size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  if (h.alloc) {
    p = h.alloc(bytes, (void*)s, h.ctx);
    if (!p) fail(SAAMG_ENOMEM, "allocator hook returned NULL for " + std::to_string(bytes) + " bytes");
    return p;
  }
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(e == cudaErrorMemoryAllocation ? SAAMG_ENOMEM : SAAMG_ECUDA,
         std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  return p;
}

void raw_free(const AllocHook& h, void* p, cudaStream_t s) {
  if (h.free) {
    h.free(p, (void*)s, h.ctx);
    return;
  }
  // cudaFree synchronises the device: pending work that reads p finishes first
  cudaFree(p);
}

// Returns every cached block to its hook (the caller holds no lock).
void pool_drain() {
  std::multimap<size_t, CachedBlock> blocks;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    blocks.swap(g_pool);
    g_pool_bytes = 0;
  }
  for (auto& kv : blocks) raw_free(kv.second.hook, kv.second.p, kv.second.s);
}

}  // namespace

void* dev_alloc(const AllocHook& h, size_t bytes, cudaStream_t s) {
  const size_t c = pool_class(bytes);
  if (c <= kPoolMaxBlock) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    auto range = g_pool.equal_range(c);
    for (auto it = range.first; it != range.second; ++it) {
      if (it->second.s == s && same_hook(it->second.hook, h)) {
        void* p = it->second.p;
        g_pool.erase(it);
        g_pool_bytes -= c;
        return p;
      }
    }
  }
  try {
    return raw_alloc(h, c, s);
  } catch (const Error& e) {
    if (e.status != SAAMG_ENOMEM) throw;
    pool_drain();  // give the cached blocks back and try once more
    return raw_alloc(h, c, s);
  }
}

void dev_free(const AllocHook& h, void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  const size_t c = pool_class(bytes);
  if (c <= kPoolMaxBlock) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (g_pool_bytes + c <= kPoolMaxBytes && same_hook(h, g_alloc)) {
      g_pool.emplace(c, CachedBlock{p, s, h});
      g_pool_bytes += c;
      return;
    }
  }
  raw_free(h, p, s);
}

HostScratch::~HostScratch() {
  if (p) cudaFreeHost(p);
}

void* HostScratch::need(size_t b) {
  if (b > bytes) {
    if (p) cudaFreeHost(p);
    p = nullptr;
    SAAMG_CUDA(cudaMallocHost(&p, b));
    bytes = b;
  }
  return p;
}

int sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  SAAMG_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int n = 0;
  SAAMG_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  if (n < 1) n = 1;
  if (dev >= 0 && dev < 64) cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

void d2h_sync(void* host, const void* dev, size_t bytes, cudaStream_t s) {
  SAAMG_CUDA(cudaMemcpyAsync(host, dev, bytes, cudaMemcpyDeviceToHost, s));
  SAAMG_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------
// optional phase timing (SAAMG_PROFILE=1): synchronises at phase ends, prints to stderr
// ---------------------------------------------------------------------------
struct PhaseTimer {
  bool on = false;
  cudaStream_t s = nullptr;
  std::chrono::steady_clock::time_point t;
  std::string out;
  explicit PhaseTimer(cudaStream_t st) : s(st) {
    const char* e = std::getenv("SAAMG_PROFILE");
    on = e && e[0] == '1';
    t = std::chrono::steady_clock::now();
  }
  void mark(const std::string& name) {
    if (!on) return;
    cudaStreamSynchronize(s);
    auto now = std::chrono::steady_clock::now();
    char buf[96];
    std::snprintf(buf, sizeof(buf), " %s=%.2f", name.c_str(),
                  std::chrono::duration<double, std::milli>(now - t).count());
    out += buf;
    t = now;
  }
  void flush(const char* what) {
    if (on) std::fprintf(stderr, "[saamg %s ms]%s\n", what, out.c_str());
  }
};

// ---------------------------------------------------------------------------
// hierarchy
// ---------------------------------------------------------------------------

// Chebyshev steps on [hi/ratio, hi], hi = safety * lambda (Saad, Alg. 12.1 on D^-1 A):
// step 0: c1 = 0, c2 = 1/theta; step k: rho_k = 1/(2 sigma - rho_{k-1}),
// c1 = rho_k rho_{k-1}, c2 = 2 rho_k / delta.
static ChebCoef cheb_coefficients(double lambda, double ratio, double safety, int degree) {
  ChebCoef c;
  const double hi = safety * lambda;
  const double lo = hi / ratio;
  const double theta = 0.5 * (hi + lo);
  const double delta = 0.5 * (hi - lo);
  const double sigma = theta / delta;
  double rho_prev = 1.0 / sigma;
  for (int k = 0; k < degree; ++k) {
    if (k == 0) {
      c.c1.push_back(0.0);
      c.c2.push_back(1.0 / theta);
    } else {
      const double rho = 1.0 / (2.0 * sigma - rho_prev);
      c.c1.push_back(rho * rho_prev);
      c.c2.push_back((2.0 * rho) / delta);
      rho_prev = rho;
    }
  }
  return c;
}

}  // namespace saamg

using namespace saamg;

namespace saamg {

static int status_of(const Error& e, const char* where) {
  g_last_error = std::string(where) + ": " + e.msg;
  return e.status;
}

template <class F>
static saamg_status guard(const char* where, F&& f) {
  try {
    f();
    return SAAMG_OK;
  } catch (const Error& e) {
    return (saamg_status)status_of(e, where);
  } catch (const std::bad_alloc&) {
    g_last_error = std::string(where) + ": host allocation failed";
    return SAAMG_ENOMEM;
  } catch (...) {
    g_last_error = std::string(where) + ": unexpected exception";
    return SAAMG_ECUDA;
  }
}

static bool mixed(const saamg_hierarchy* h) { return h->prm.precision != SAAMG_PREC_FP64; }

static void check_params_ext(const saamg_params& p) {
  if (p.aggregation != SAAMG_AGG_MIS2 && p.aggregation != SAAMG_AGG_CUBES)
    fail(SAAMG_EINVAL, "unknown aggregation");
  if (p.coarse_solver != SAAMG_COARSE_LU && p.coarse_solver != SAAMG_COARSE_GS)
    fail(SAAMG_EINVAL, "unknown coarse solver");
  if (p.coarse_sweeps < 1 || p.coarse_sweeps > 64) fail(SAAMG_EINVAL, "coarse_sweeps must be in 1..64");
  if (p.device_loop != 0 && p.device_loop != 1) fail(SAAMG_EINVAL, "device_loop must be 0 or 1");
}

// Matrix of level l (level 0 = the operator's CSR)
static const DevCsr& level_matrix(const saamg_hierarchy* h, int l) {
  return l == 0 ? h->op->d.A : h->lev[l]->A;
}

static void alloc_level_vectors(saamg_hierarchy* h, Level& L, bool is0, cudaStream_t s) {
  if (!mixed(h)) {
    L.x0.alloc(L.n, s);
    if (!is0) L.x1.alloc(L.n, s);
    L.b.alloc(L.n, s);
    L.d.alloc(L.n, s);
    L.r.alloc(L.n, s);
  } else {
    L.fx0.alloc(L.n, s);
    if (!is0) L.fx1.alloc(L.n, s);
    L.fb.alloc(L.n, s);
    L.fd.alloc(L.n, s);
    L.fr.alloc(L.n, s);
  }
}

__global__ void pattern_diff_k(int n, const int* __restrict__ rp1, const int* __restrict__ c1,
                               const int* __restrict__ rp2, const int* __restrict__ c2,
                               int* __restrict__ diff) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (rp1[i] != rp2[i] || rp1[i + 1] != rp2[i + 1]) {
      *diff = 1;
      continue;
    }
    for (int p = rp1[i]; p < rp1[i + 1]; ++p)
      if (c1[p] != c2[p]) *diff = 1;
  }
}

static bool same_pattern(const DevCsr& a, const DevCsr& b, cudaStream_t s) {
  if (a.n != b.n || a.nnz != b.nnz) return false;
  if (a.n == 0) return true;
  Buf<int> diff;
  diff.alloc(1, s);
  SAAMG_CUDA(cudaMemsetAsync(diff.p, 0, sizeof(int), s));
  pattern_diff_k<<<std::min((a.n + 255) / 256, sm_count() * 8), 256, 0, s>>>(a.n, a.rowptr.p, a.col.p,
                                                                      b.rowptr.p, b.col.p, diff.p);
  SAAMG_LAUNCH();
  int h = 0;
  d2h_sync(&h, diff.p, sizeof(int), s);
  return h == 0;
}

// PCG vectors of level 0, reduction partials and the loop's control block.
static void alloc_pcg_vectors(saamg_hierarchy* h, int n, cudaStream_t s) {
  h->bhat.alloc(n, s);
  h->xhat.alloc(n, s);
  h->r.alloc(n, s);
  h->z.alloc(n, s);
  h->p.alloc(n, s);
  h->q.alloc(n, s);
  if (mixed(h)) {
    h->z32.alloc(n, s);
    h->r32.alloc(n, s);
  }
  h->part0.alloc(kRedBlocks, s);
  h->part1.alloc(kRedBlocks, s);
  h->part2.alloc(kRedBlocks, s);
  h->ctl.alloc(1, s);
}

// Device bytes of the V-cycle and PCG vectors of h.
static long long vector_bytes(const saamg_hierarchy* h) {
  long long bytes = 0;
  for (auto& L : h->lev)
    bytes += L->x0.bytes() + L->x1.bytes() + L->b.bytes() + L->d.bytes() + L->r.bytes() +
             L->fx0.bytes() + L->fx1.bytes() + L->fb.bytes() + L->fd.bytes() + L->fr.bytes();
  const long long n = h->op->d.n;
  return bytes + 6LL * n * 8 + (mixed(h) ? 8LL * n : 0);
}

// prev != NULL: the aggregates of every level are copied from prev (whose level-0 pattern
// must equal op's) instead of being recomputed; everything numeric is rebuilt.
// A second stream for setup work that overlaps the work on the caller's stream (created once).
static cudaStream_t aux_stream() {
  static std::mutex mu;
  static cudaStream_t st = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!st) SAAMG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  return st;
}

// SELL copy of a coarse level's operator with the value arrays of the V-cycle's precision.
// like: the same level of a reused hierarchy (same pattern), whose SELL layout is copied
static void build_level_sell(saamg_hierarchy* h, Level& L, cudaStream_t s,
                             const Level* like = nullptr) {
  const bool f64 = !mixed(h), f32 = h->prm.precision == SAAMG_PREC_FP32;
  const bool bf16 = h->prm.precision == SAAMG_PREC_FP32_BF16;
  if (like && like->As.n == L.n && like->As.nnz == L.A.nnz && like->As.nslices > 0)
    sell_like(L.A, like->As, L.As, f64, f32, bf16, s);
  else
    sell_from_csr(L.A, L.As, f64, f32, bf16, s);
}

static void setup_levels(const saamg_operator* op, const saamg_params& prm, cudaStream_t s,
                         saamg_hierarchy* h, const saamg_hierarchy* prev);

// A failed setup waits for both of its streams before the hierarchy's arrays are released (the
// second stream may still be reading them).
static void setup_impl(const saamg_operator* op, const saamg_params& prm, cudaStream_t s,
                       saamg_hierarchy* h, const saamg_hierarchy* prev = nullptr) {
  try {
    setup_levels(op, prm, s, h, prev);
  } catch (...) {
    cudaStreamSynchronize(aux_stream());
    cudaStreamSynchronize(s);
    throw;
  }
}

static void setup_levels(const saamg_operator* op, const saamg_params& prm, cudaStream_t s,
                         saamg_hierarchy* h, const saamg_hierarchy* prev) {
  auto t0 = std::chrono::steady_clock::now();
  PhaseTimer pt(s);
  h->op = op;
  h->prm = prm;
  const OperatorData& od = op->d;
  {
    auto L0 = std::make_unique<Level>();
    L0->n = od.n;
    L0->nnz = od.nnz;
    L0->avg = od.n ? (double)od.nnz / od.n : 0.0;
    L0->invd.alloc(od.n, s);
    L0->invd32.alloc(od.n, s);
    stencil_diag_inverse(od, L0->invd.p, L0->invd32.p, s);
    h->lev.push_back(std::move(L0));
  }
  int l = 0;
  AggScratchBufs agg_scratch;
  if (!prev) agg_scratch.alloc(od.n > 0 ? od.n : 1, s);
  for (;;) {
    Level& L = *h->lev[l];
    const DevCsr& A = level_matrix(h, l);
    // node ids: level 0 the box index; coarse levels the cube lattice index (cube
    // aggregation) or the row itself (MIS-2)
    const unsigned* ids = (l == 0) ? od.ids.p : L.ids.p;
    if (l == 0) {
      L.dims[0] = od.g.nx;
      L.dims[1] = od.g.ny;
      L.dims[2] = od.g.nz;
    }
    int nagg = 0;
    Buf<unsigned> next_ids;
    int next_dims[3] = {0, 0, 0};
    // The spectral bound of a level that will be coarsened only reads A_l (or the level-0
    // stencil, or the SELL copy): it runs on a second stream while the aggregation (latency-
    // bound, where the power iteration is FP64-bound) runs on s.
    const bool coarsen = prev ? l + 1 < (int)prev->lev.size()
                              : !(L.n <= prm.max_coarse || l == prm.max_levels - 1 ||
                                  l == SAAMG_MAX_LEVELS - 1);
    PowerRun power;
    cudaStream_t s2 = aux_stream();
    if (coarsen) {
      // a smoothed level >= 1 large enough for SELL gets its SELL copy now (it is not the
      // coarsest), so that in the FP64 V-cycle the power iteration runs on it too
      if (l >= 1 && L.n >= kSellMinRows && L.As.n == 0)
        build_level_sell(h, L, s, prev ? prev->lev[l].get() : nullptr);
      const StencilDev<double> S0 = od.view<double>();
      cudaEvent_t fork;
      SAAMG_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
      SAAMG_CUDA(cudaEventRecord(fork, s));
      SAAMG_CUDA(cudaStreamWaitEvent(s2, fork, 0));
      cudaEventDestroy(fork);
      power_lambda_start(A, L.invd.p, ids, prm.power_iters, s2, power, l == 0 ? &S0 : nullptr,
                         l >= 1 && L.As.n > 0 ? &L.As : nullptr);
    }
    if (prev) {
      // reuse: the previous hierarchy decides the levels and the aggregates
      if (l + 1 >= (int)prev->lev.size()) break;
      const Level& PL = *prev->lev[l];
      if (PL.n != L.n) fail(SAAMG_EINVAL, "level sizes differ from the reused hierarchy");
      L.root.alloc(L.n, s);
      L.agg.alloc(L.n, s);
      SAAMG_CUDA(cudaMemcpyAsync(L.root.p, PL.root.p, L.n, cudaMemcpyDeviceToDevice, s));
      SAAMG_CUDA(cudaMemcpyAsync(L.agg.p, PL.agg.p, sizeof(int) * L.n, cudaMemcpyDeviceToDevice, s));
      nagg = prev->lev[l + 1]->n;
      const Level& PN = *prev->lev[l + 1];
      if (PN.ids.p) {
        next_ids.alloc(nagg, s);
        SAAMG_CUDA(cudaMemcpyAsync(next_ids.p, PN.ids.p, sizeof(unsigned) * nagg,
                                   cudaMemcpyDeviceToDevice, s));
        std::memcpy(next_dims, PN.dims, sizeof(next_dims));
      }
      pt.mark("L" + std::to_string(l) + ".reuse");
    } else {
      if (L.n <= prm.max_coarse || l == prm.max_levels - 1 || l == SAAMG_MAX_LEVELS - 1) break;
      const unsigned seed = 0x9E3779B9u * (unsigned)(l + 1);
      L.root.alloc(L.n, s);
      L.agg.alloc(L.n, s);
      pt.mark("L" + std::to_string(l) + ".pre");
      if (prm.aggregation == SAAMG_AGG_CUBES) {
        nagg = cube_aggregate(L.n, ids, L.dims, L.agg.p, L.root.p, next_ids, next_dims, s);
      } else if (l == 0) {
        // level 0: the graph of the 7-point star, walked on the line structure
        GridGraph gg{od.lines.p, od.nbr.p, od.chunks.p, od.nchunks, od.nbmask.p,
                     (unsigned)od.g.nx, (unsigned)od.g.nx * (unsigned)od.g.ny, od.rline.p};
        nagg = mis2_aggregate_grid(L.n, gg, ids, seed, L.root.p, L.agg.p, agg_scratch.view(), s);
      } else {
        nagg = mis2_aggregate(L.n, A.rowptr.p, A.col.p, A.nnz, ids, seed, L.root.p, L.agg.p,
                              agg_scratch.view(), s);
      }
      pt.mark("L" + std::to_string(l) + ".agg");
      if (10LL * nagg > 9LL * L.n) {  // coarsening stalled
        power_lambda_finish(power, s2);
        L.root.release();
        L.agg.release();
        L.As = DevSell();  // the coarsest level keeps CSR
        break;
      }
    }
    // Reuse: the patterns of P, R, A P and A_{l+1} are prev's, so A T and the symbolic part
    // of A P (neither depends on lambda_hat) run while the power iteration does, and R and
    // R (A P) take their patterns from prev.
    const Level* PL = prev ? prev->lev[l].get() : nullptr;
    ProlongState pst;
    SpgemmPlan ap_plan;
    if (PL) {
      prolongator_start(A, L.agg.p, nagg, pst, s, &PL->P, l == 0);
      spgemm_symbolic(A, PL->P, ap_plan, s, PL->APpat.n > 0 ? &PL->APpat : nullptr);
      pt.mark("L" + std::to_string(l) + ".early");
    }
    L.lambda = power_lambda_finish(power, s2);
    L.omega = 4.0 / (3.0 * L.lambda);
    pt.mark("L" + std::to_string(l) + ".lambda");
    if (!PL) {
      pst.invd = L.invd.p;
      pst.omega = L.omega;
      prolongator_start(A, L.agg.p, nagg, pst, s, nullptr, l == 0);
    }
    prolongator_finish(pst, L.invd.p, L.omega, L.P, s);
    pt.mark("L" + std::to_string(l) + ".P");
    // R = P^T on the second stream (it waits on the host for nothing) while A P runs on s
    {
      cudaEvent_t ev;
      SAAMG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      SAAMG_CUDA(cudaEventRecord(ev, s));
      SAAMG_CUDA(cudaStreamWaitEvent(s2, ev, 0));
      cudaEventDestroy(ev);
    }
    if (PL) transpose_known(L.P, PL->R, L.R, s2);
    else transpose(L.P, L.R, s2);
    if (!PL) spgemm_symbolic(A, L.P, ap_plan, s);
    DevCsr AP;
    spgemm_numeric(A, L.P, ap_plan, AP, s);
    pt.mark("L" + std::to_string(l) + ".AP");
    {
      cudaEvent_t ev;
      SAAMG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      SAAMG_CUDA(cudaEventRecord(ev, s2));
      SAAMG_CUDA(cudaStreamWaitEvent(s, ev, 0));
      cudaEventDestroy(ev);
    }
    pt.mark("L" + std::to_string(l) + ".R");
    auto N = std::make_unique<Level>();
    {
      SpgemmPlan rap_plan;
      spgemm_symbolic(L.R, AP, rap_plan, s, PL ? &prev->lev[l + 1]->A : nullptr);
      spgemm_numeric(L.R, AP, rap_plan, N->A, s);
    }
    {  // keep the pattern of A P: a reuse of this hierarchy skips its symbolic pass
      L.APpat.n = AP.n;
      L.APpat.m = AP.m;
      L.APpat.nnz = AP.nnz;
      L.APpat.rowptr = std::move(AP.rowptr);
      L.APpat.col = std::move(AP.col);
    }
    pt.mark("L" + std::to_string(l) + ".RAP");
    N->n = N->A.n;
    N->nnz = N->A.nnz;
    N->ids = std::move(next_ids);
    std::memcpy(N->dims, next_dims, sizeof(next_dims));
    N->avg = N->n ? (double)N->nnz / N->n : 0.0;
    N->invd.alloc(N->n, s);
    N->invd32.alloc(N->n, s);
    csr_diag_inverse(N->A, N->invd.p, N->invd32.p, s);
    h->lev.push_back(std::move(N));
    ++l;
  }
  const int nl = (int)h->lev.size();
  Level& C = *h->lev[nl - 1];
  pt.mark("levels");
  if (prm.coarse_solver == SAAMG_COARSE_GS) {
    const unsigned* cids = (nl == 1) ? od.ids.p : C.ids.p;  // key ids of the colouring
    coarse_gs_setup(level_matrix(h, nl - 1), C.invd.p, cids, prm.coarse_sweeps, h->coarse, s);
  } else {
    if (C.n > 16384) fail(SAAMG_NUMERICAL, "coarsest level has more than 16384 unknowns");
    coarse_factor(level_matrix(h, nl - 1), h->coarse, s);
  }
  pt.mark("coarse");
  for (int q = 0; q < nl; ++q) {
    Level& L = *h->lev[q];
    if (q < nl - 1) L.cheb = cheb_coefficients(L.lambda, prm.cheb_ratio, prm.cheb_safety, prm.cheb_degree);
    alloc_level_vectors(h, L, q == 0, s);
    const bool f64 = !mixed(h), f32 = prm.precision == SAAMG_PREC_FP32;
    const bool bf16 = prm.precision == SAAMG_PREC_FP32_BF16;
    // SELL for the large smoothed levels (built before their spectral bound); a small level
    // runs on CSR with wide row groups
    if (q >= 1 && q < nl - 1 && L.n >= kSellMinRows) {
      if (L.As.n == 0)
        build_level_sell(h, L, s,
                         prev && q < (int)prev->lev.size() ? prev->lev[q].get() : nullptr);
    } else if (q >= 1 && q < nl - 1) {
      if (f32) {
        L.A.val32.alloc(L.A.nnz, s);
        to_float(L.A.val.p, L.A.val32.p, L.A.nnz, s);
      } else if (bf16) {
        L.A.val16.alloc(L.A.nnz, s);
        to_bf16(L.A.val.p, L.A.val16.p, L.A.nnz, s);
      }
    }
    if (!f64 && q < nl - 1) {
      L.P32.alloc(L.P.nnz, s);
      to_float(L.P.val.p, L.P32.p, L.P.nnz, s);
      L.R32.alloc(L.R.nnz, s);
      to_float(L.R.val.p, L.R32.p, L.R.nnz, s);
    }
  }
  alloc_pcg_vectors(h, od.n, s);
  SAAMG_CUDA(cudaStreamSynchronize(s));
  pt.mark("finish");
  pt.flush("setup");
  long long bytes = 0;
  for (auto& L : h->lev) {
    bytes += L->A.bytes() + L->P.bytes() + L->R.bytes() + L->APpat.bytes() + L->invd.bytes() +
             L->invd32.bytes() +
             L->agg.bytes() + L->root.bytes() + L->ids.bytes() + L->As.bytes() + L->P32.bytes() +
             L->R32.bytes();
  }
  h->bytes = bytes + h->coarse.bytes() + vector_bytes(h);
  h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

static void borrow_csr(DevCsr& d, const DevCsr& o) {
  d.n = o.n;
  d.m = o.m;
  d.nnz = o.nnz;
  d.rowptr.borrow(o.rowptr);
  d.col.borrow(o.col);
  d.val.borrow(o.val);
  d.val32.borrow(o.val32);
  d.val16.borrow(o.val16);
}

static void borrow_sell(DevSell& d, const DevSell& o) {
  d.n = o.n;
  d.m = o.m;
  d.nslices = o.nslices;
  d.nnz = o.nnz;
  d.nent = o.nent;
  d.perm.borrow(o.perm);
  d.soff.borrow(o.soff);
  d.col.borrow(o.col);
  d.dcol.borrow(o.dcol);
  d.index_bytes = o.index_bytes;
  d.val.borrow(o.val);
  d.val32.borrow(o.val32);
  d.val16.borrow(o.val16);
}

// h = a work set of src: every level's matrices, transfers, aggregates and the coarse solver
// are borrowed from the hierarchy that owns them (src, or the one src borrows from), the
// smoother coefficients are src's, and the vectors are h's own.
static void work_set_impl(const saamg_hierarchy* src, cudaStream_t s, saamg_hierarchy* h) {
  auto t0 = std::chrono::steady_clock::now();
  h->op = src->op;
  h->prm = src->prm;
  for (const auto& S : src->lev) {
    auto L = std::make_unique<Level>();
    L->n = S->n;
    L->nnz = S->nnz;
    L->avg = S->avg;
    borrow_csr(L->A, S->A);
    L->invd.borrow(S->invd);
    L->invd32.borrow(S->invd32);
    L->agg.borrow(S->agg);
    L->root.borrow(S->root);
    L->ids.borrow(S->ids);
    for (int k = 0; k < 3; ++k) L->dims[k] = S->dims[k];
    borrow_csr(L->P, S->P);
    borrow_csr(L->R, S->R);
    borrow_csr(L->APpat, S->APpat);
    L->lambda = S->lambda;
    L->omega = S->omega;
    L->cheb = S->cheb;
    borrow_sell(L->As, S->As);
    L->P32.borrow(S->P32);
    L->R32.borrow(S->R32);
    h->lev.push_back(std::move(L));
  }
  for (size_t q = 0; q < h->lev.size(); ++q) alloc_level_vectors(h, *h->lev[q], q == 0, s);
  const CoarseSolver& c = src->coarse;
  h->coarse.n = c.n;
  h->coarse.kind = c.kind;
  h->coarse.inv.borrow(c.inv);
  h->coarse.rowptr = c.rowptr;
  h->coarse.col = c.col;
  h->coarse.val = c.val;
  h->coarse.invd = c.invd;
  h->coarse.colour.borrow(c.colour);
  h->coarse.order.borrow(c.order);
  h->coarse.coff.borrow(c.coff);
  h->coarse.ncolours = c.ncolours;
  h->coarse.steps = c.steps;
  alloc_pcg_vectors(h, h->op->d.n, s);
  SAAMG_CUDA(cudaStreamSynchronize(s));
  h->bytes = vector_bytes(h);
  h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Drops one reference to h (the handle's own or a work set's); the last one deletes it.
static void release_hierarchy(saamg_hierarchy* h) {
  if (h->refs.fetch_sub(1) == 1) {
    h->magic = 0;
    delete h;
  }
}

// --- V-cycle (Algorithm 1) -------------------------------------------------
// Level l smooths b_l -> x_l; the final iterate lands in `out` (length n_l).  The
// Chebyshev steps ping-pong between two buffers: with nu pre- and nu post-steps there are
// 2 nu - 1 swaps after the first step, so starting in `tmp` ends in `out`.
template <class T>
struct LevelVecs;

template <>
struct LevelVecs<double> {
  static double* x0(Level& L) { return L.x0.p; }
  static double* x1(Level& L) { return L.x1.p; }
  static double* b(Level& L) { return L.b.p; }
  static double* d(Level& L) { return L.d.p; }
  static double* r(Level& L) { return L.r.p; }
};
template <>
struct LevelVecs<float> {
  static float* x0(Level& L) { return L.fx0.p; }
  static float* x1(Level& L) { return L.fx1.p; }
  static float* b(Level& L) { return L.fb.p; }
  static float* d(Level& L) { return L.fd.p; }
  static float* r(Level& L) { return L.fr.p; }
};

// y (+)= M x for a coarse matrix in the working precision
template <class T>
static void level_csr(saamg_hierarchy* h, int l, int mode, const T* x, T* y, const T* b, T* d,
                      T c1, T c2, cudaStream_t s);

template <>
void level_csr<double>(saamg_hierarchy* h, int l, int mode, const double* x, double* y,
                       const double* b, double* d, double c1, double c2, cudaStream_t s) {
  Level& L = *h->lev[l];
  const int kc = l == 1 ? SAAMG_KT_COARSE : SAAMG_KT_COARSE_DEEP;
  if (L.As.n > 0)
    sell_apply<double, double>(mode, L.As, L.As.val.p, x, y, b, d, L.invd.p, c1, c2, s, kc);
  else
    csr_apply<double, double>(mode, L.n, L.A.rowptr.p, L.A.col.p, L.A.val.p, L.avg, x, y, b, d,
                              L.invd.p, c1, c2, nullptr, s, kc);
}

template <>
void level_csr<float>(saamg_hierarchy* h, int l, int mode, const float* x, float* y,
                      const float* b, float* d, float c1, float c2, cudaStream_t s) {
  Level& L = *h->lev[l];
  const int kc = l == 1 ? SAAMG_KT_COARSE : SAAMG_KT_COARSE_DEEP;
  const bool fp32 = h->prm.precision == SAAMG_PREC_FP32;
  if (L.As.n > 0) {
    if (fp32)
      sell_apply<float, float>(mode, L.As, L.As.val32.p, x, y, b, d, L.invd32.p, c1, c2, s, kc);
    else
      sell_apply<float, __nv_bfloat16>(mode, L.As, L.As.val16.p, x, y, b, d, L.invd32.p, c1, c2,
                                       s, kc);
  } else if (fp32) {
    csr_apply<float, float>(mode, L.n, L.A.rowptr.p, L.A.col.p, L.A.val32.p, L.avg, x, y, b, d,
                            L.invd32.p, c1, c2, nullptr, s, kc);
  } else {
    csr_apply<float, __nv_bfloat16>(mode, L.n, L.A.rowptr.p, L.A.col.p, L.A.val16.p, L.avg, x,
                                    y, b, d, L.invd32.p, c1, c2, nullptr, s, kc);
  }
}

template <class T>
static void transfer(saamg_hierarchy* h, int l, bool restrict_, const T* x, T* y, cudaStream_t s);

template <>
void transfer<double>(saamg_hierarchy* h, int l, bool restrict_, const double* x, double* y,
                      cudaStream_t s) {
  Level& L = *h->lev[l];
  const DevCsr& M = restrict_ ? L.R : L.P;
  csr_apply<double, double>(restrict_ ? CSR_SPMV : CSR_ADD, M.n, M.rowptr.p, M.col.p, M.val.p,
                            M.n ? (double)M.nnz / M.n : 0.0, x, y, nullptr, nullptr, nullptr, 0.0,
                            0.0, nullptr, s, l == 0 ? SAAMG_KT_TRANSFER : SAAMG_KT_TRANSFER_DEEP);
}

template <>
void transfer<float>(saamg_hierarchy* h, int l, bool restrict_, const float* x, float* y,
                     cudaStream_t s) {
  Level& L = *h->lev[l];
  if (l == 0 && !restrict_) {
    // level 0, FP32: the prolongation from the stencil and the aggregates (about 12 bytes per
    // row instead of the 39 of the CSR matrix); FP64 keeps the CSR, which needs fewer FP64
    // operations per row
    stencil_prolong<float>(h->op->d.template view<float>(), L.agg.p, (float)L.omega, x, y, s);
    return;
  }
  const DevCsr& M = restrict_ ? L.R : L.P;
  const float* v = restrict_ ? L.R32.p : L.P32.p;
  csr_apply<float, float>(restrict_ ? CSR_SPMV : CSR_ADD, M.n, M.rowptr.p, M.col.p, v,
                          M.n ? (double)M.nnz / M.n : 0.0, x, y, nullptr, nullptr, nullptr, 0.0f,
                          0.0f, nullptr, s, l == 0 ? SAAMG_KT_TRANSFER : SAAMG_KT_TRANSFER_DEEP);
}

template <class T>
static void smooth_step(saamg_hierarchy* h, int l, int mode0, const T* x, T* y, const T* b, T* d,
                        T c1, T c2, cudaStream_t s) {
  if (l == 0) {
    StencilDev<T> S = h->op->d.template view<T>();
    const int m = mode0 == CSR_CHEB0   ? ST_CHEB0
                  : mode0 == CSR_RESID ? ST_RESID
                  : (c1 == T(0))       ? ST_CHEB1
                                       : ST_CHEB;
    stencil_apply<T>(S, m, x, y, b, d, c1, c2, nullptr, s);
  } else {
    level_csr<T>(h, l, mode0, x, y, b, d, c1, c2, s);
  }
}

template <class T>
static void vcycle_level(saamg_hierarchy* h, int l, const T* b, T* out, cudaStream_t s) {
  const int nl = (int)h->lev.size();
  Level& L = *h->lev[l];
  if (l == nl - 1) {
    coarse_apply<T>(h->coarse, b, out, s);
    return;
  }
  const int nu = (int)L.cheb.c1.size();
  T* bufs[2] = {LevelVecs<T>::x0(L), out};
  T* d = LevelVecs<T>::d(L);
  int cur = 0;
  // presmoothing from x = 0
  smooth_step<T>(h, l, CSR_CHEB0, nullptr, bufs[cur], b, d, T(0), (T)L.cheb.c2[0], s);
  for (int k = 1; k < nu; ++k) {
    smooth_step<T>(h, l, CSR_CHEB, bufs[cur], bufs[1 - cur], b, d, (T)L.cheb.c1[k],
                   (T)L.cheb.c2[k], s);
    cur = 1 - cur;
  }
  // residual, restriction, coarse correction
  T* r = LevelVecs<T>::r(L);
  smooth_step<T>(h, l, CSR_RESID, bufs[cur], r, b, nullptr, T(0), T(0), s);
  Level& N = *h->lev[l + 1];
  T* bc = LevelVecs<T>::b(N);
  T* vc = (l + 1 == nl - 1) ? LevelVecs<T>::x0(N) : LevelVecs<T>::x1(N);
  transfer<T>(h, l, true, r, bc, s);
  vcycle_level<T>(h, l + 1, bc, vc, s);
  transfer<T>(h, l, false, vc, bufs[cur], s);
  // postsmoothing with the same polynomial
  for (int k = 0; k < nu; ++k) {
    smooth_step<T>(h, l, CSR_CHEB, bufs[cur], bufs[1 - cur], b, d, (T)L.cheb.c1[k],
                   (T)L.cheb.c2[k], s);
    cur = 1 - cur;
  }
  if (bufs[cur] != out) {
    SAAMG_CUDA(cudaMemcpyAsync(out, bufs[cur], sizeof(T) * L.n, cudaMemcpyDeviceToDevice, s));
  }
}

// z = M r on level 0, FP64 in and out (FP32 inside in mixed mode)
// r32_current: the FP32 copy h->r32 of r is already up to date (written by the update)
static void apply_preconditioner(saamg_hierarchy* h, const double* r, double* z, float* z32,
                                 cudaStream_t s, bool r32_current = false) {
  const int n = h->op->d.n;
  if (!mixed(h)) {
    vcycle_level<double>(h, 0, r, z, s);
  } else {
    if (!r32_current) to_float(r, h->r32.p, n, s);
    vcycle_level<float>(h, 0, h->r32.p, z32, s);
  }
}

// r'z (and z'q for the Polak-Ribiere rule) of the new preconditioned residual
static void rz_partials(saamg_hierarchy* h, const double* r, const double* z, const double* q,
                        cudaStream_t s) {
  const int n = h->op->d.n;
  const bool pr = h->prm.beta_rule == 1;
  if (mixed(h)) {
    if (pr) dot2_partials<float>(n, r, h->z32.p, q, h->part0.p, h->part2.p, s);
    else dot_partials<double, float>(n, r, h->z32.p, h->part0.p, s);
  } else {
    if (pr) dot2_partials<double>(n, r, z, q, h->part0.p, h->part2.p, s);
    else dot_partials<double, double>(n, r, z, h->part0.p, s);
  }
}

// --- PCG --------------------------------------------------------------------
static int pcg_impl(saamg_hierarchy* h, double rtol, cudaStream_t s, saamg_solve_info* info) {
  const OperatorData& od = h->op->d;
  const int n = od.n;
  const bool mx = mixed(h);
  double* x = h->xhat.p;
  double* r = h->r.p;
  double* p = h->p.p;
  double* q = h->q.p;
  double* z = h->z.p;
  PcgCtl* ctl = h->ctl.p;
  PcgCtl* hc = static_cast<PcgCtl*>(h->host.need(sizeof(PcgCtl)));
  const StencilDev<double> S = od.view<double>();
  info->iters = 0;
  info->converged = 0;
  info->relres = 0;
  info->relres_true = 0;
  if (n == 0) {
    info->converged = 1;
    return SAAMG_OK;
  }
  // ||b||
  dot_partials<double, double>(n, h->bhat.p, h->bhat.p, h->part0.p, s);
  Buf<double>& sc = h->scratch;
  if (!sc.p) sc.alloc(4, s);
  sum_partials(h->part0.p, kRedBlocks, sc.p, s);
  double bb = 0;
  d2h_sync(&bb, sc.p, sizeof(double), s);
  if (!std::isfinite(bb)) fail(SAAMG_NUMERICAL, "right-hand side holds NaN or Inf");
  if (bb == 0.0) {
    SAAMG_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, s));
    info->converged = 1;
    return SAAMG_OK;
  }
  const double bnorm = std::sqrt(bb);
  // r = b - A x
  stencil_apply<double>(S, ST_RESID, x, r, h->bhat.p, nullptr, 0.0, 0.0, nullptr, s);
  PcgCtl init{};
  init.tol2 = (rtol * bnorm) * (rtol * bnorm);
  SAAMG_CUDA(cudaMemcpyAsync(ctl, &init, sizeof(PcgCtl), cudaMemcpyHostToDevice, s));
  dot_partials<double, double>(n, r, r, h->part0.p, s);
  pcg_check(h->part0.p, ctl, s);  // counts one; reset below
  d2h_sync(hc, ctl, sizeof(PcgCtl), s);
  double rr = hc->rr;
  if (!std::isfinite(rr)) fail(SAAMG_NUMERICAL, "initial residual holds NaN or Inf");
  init.rr = rr;
  init.iters = 0;
  SAAMG_CUDA(cudaMemcpyAsync(ctl, &init, sizeof(PcgCtl), cudaMemcpyHostToDevice, s));
  int status = SAAMG_NOT_CONVERGED;
  if (rr <= init.tol2) {
    status = SAAMG_OK;
    info->converged = 1;
  } else {
    apply_preconditioner(h, r, z, h->z32.p, s);
    if (mx) {
      vec_copy_to_double<float>(n, h->z32.p, p, s);
      dot_partials<double, float>(n, r, h->z32.p, h->part0.p, s);
    } else {
      vec_copy_to_double<double>(n, z, p, s);
      dot_partials<double, double>(n, r, z, h->part0.p, s);
    }
    pcg_beta(h->part0.p, nullptr, -1, ctl, s);  // rz of the first direction
    for (int it = 1; it <= h->prm.maxit; ++it) {
      stencil_apply<double>(S, ST_SPMV_DOT, p, q, nullptr, nullptr, 0.0, 0.0, h->part0.p, s);
      pcg_alpha(h->part0.p, ctl, s);
      pcg_update(n, x, r, p, q, ctl, h->part1.p, s, mx ? h->r32.p : nullptr);
      pcg_check(h->part1.p, ctl, s);
      d2h_sync(hc, ctl, sizeof(PcgCtl), s);
      info->iters = hc->iters;
      if (hc->breakdown) {
        status = SAAMG_NUMERICAL;
        break;
      }
      if (hc->converged) {
        status = SAAMG_OK;
        info->converged = 1;
        break;
      }
      apply_preconditioner(h, r, z, h->z32.p, s, true);
      rz_partials(h, r, z, q, s);
      pcg_beta(h->part0.p, h->prm.beta_rule == 1 ? h->part2.p : nullptr, h->prm.beta_rule, ctl, s);
      if (mx) pcg_direction<float>(n, h->z32.p, p, ctl, s);
      else pcg_direction<double>(n, z, p, ctl, s);
    }
  }
  d2h_sync(hc, ctl, sizeof(PcgCtl), s);
  info->relres = std::sqrt(hc->rr) / bnorm;
  // true residual of the scaled system
  stencil_apply<double>(S, ST_RESID, x, q, h->bhat.p, nullptr, 0.0, 0.0, nullptr, s);
  dot_partials<double, double>(n, q, q, h->part0.p, s);
  sum_partials(h->part0.p, kRedBlocks, sc.p, s);
  double tr = 0;
  d2h_sync(&tr, sc.p, sizeof(double), s);
  info->relres_true = std::sqrt(tr) / bnorm;
  if (status == SAAMG_NUMERICAL) g_last_error = "saamg_solve: breakdown (NaN/Inf or p'Ap = 0)";
  return status;
}

// --- device-loop PCG ------------------------------------------------------------
// The whole solve of Sec. 3.1 as one CUDA graph: a prologue (||b||, r = b - A x, the loop
// condition), a conditional while node whose body is one PCG pass (V-cycle, beta,
// direction, A p, alpha, update, convergence test that clears the condition), and an
// epilogue (true residual).  Pointers and Chebyshev coefficients are fixed at capture, the
// tolerance is read from the device scalars, so one capture serves every right-hand side.
__global__ void set_rtol_k(PcgCtl* ctl, double rtol) { ctl->rtol = rtol; }

static void pcg_pass(saamg_hierarchy* h, cudaGraphConditionalHandle cond, cudaStream_t s) {
  const OperatorData& od = h->op->d;
  const int n = od.n;
  const StencilDev<double> S = od.view<double>();
  const int rule = h->prm.beta_rule;
  double* r = h->r.p;
  double* p = h->p.p;
  double* q = h->q.p;
  PcgCtl* ctl = h->ctl.p;
  apply_preconditioner(h, r, h->z.p, h->z32.p, s, true);
  rz_partials(h, r, h->z.p, q, s);
  pcg_graph_beta(h->part0.p, rule == 1 ? h->part2.p : nullptr, rule, ctl, s);
  if (mixed(h)) pcg_direction<float>(n, h->z32.p, p, ctl, s);
  else pcg_direction<double>(n, h->z.p, p, ctl, s);
  stencil_apply<double>(S, ST_SPMV_DOT, p, q, nullptr, nullptr, 0.0, 0.0, h->part0.p, s);
  pcg_alpha(h->part0.p, ctl, s);
  pcg_update(n, h->xhat.p, r, p, q, ctl, h->part1.p, s, mixed(h) ? h->r32.p : nullptr);
  pcg_graph_check(h->part1.p, ctl, cond, h->prm.maxit, s);
}

// Kernels of a captured solve: `fixed` run once per graph launch, `body` once per PCG pass.
struct GraphKernels {
  long long fixed = 0, body = 0;
};

// Capture needs a stream that can be captured (not the legacy default stream): the graph is
// recorded on private streams (nothing executes during capture) and launched on the caller's
// stream.  Stream 0 records the graph, stream 1 the body of a conditional node, the others
// the parallel branches of a batch.
static std::mutex g_capture_mu;  // one capture at a time on the private streams

static cudaStream_t capture_stream(int k) {
  static std::mutex mu;
  static std::vector<cudaStream_t> cs;
  std::lock_guard<std::mutex> lock(mu);
  while ((int)cs.size() <= k) {
    cudaStream_t st;
    SAAMG_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    cs.push_back(st);
  }
  return cs[k];
}

static unsigned long long next_version() {
  static std::atomic<unsigned long long> v{0};
  return ++v;
}

// One whole PCG solve into the graph that stream s is capturing: prologue (||b||, r = b - A x,
// the loop condition), a conditional while node whose body (captured on body_s) is one PCG
// pass, and the epilogue (true residual).  cond belongs to the graph being captured.
static GraphKernels capture_pcg(saamg_hierarchy* h, cudaGraphConditionalHandle cond,
                                cudaStream_t s, cudaStream_t body_s) {
  CaptureCount counting;
  const long long k0 = captured();
  const OperatorData& od = h->op->d;
  const int n = od.n;
  const StencilDev<double> S = od.view<double>();
  dot_partials<double, double>(n, h->bhat.p, h->bhat.p, h->part2.p, s);
  stencil_apply<double>(S, ST_RESID, h->xhat.p, h->r.p, h->bhat.p, nullptr, 0.0, 0.0, nullptr, s);
  if (mixed(h)) to_float(h->r.p, h->r32.p, n, s);  // the first pass's V-cycle input
  dot_partials<double, double>(n, h->r.p, h->r.p, h->part1.p, s);
  SAAMG_CUDA(cudaMemsetAsync(h->p.p, 0, sizeof(double) * n, s));
  pcg_graph_init(h->part2.p, h->part1.p, h->ctl.p, cond, h->prm.maxit, h->xhat.p, n, s);
  cudaStreamCaptureStatus st;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  SAAMG_CUDA(cudaStreamGetCaptureInfo(s, &st, nullptr, &cg, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  SAAMG_CUDA(cudaGraphAddNode(&cnode, cg, deps, nullptr, nd, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  SAAMG_CUDA(cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  stencil_apply<double>(S, ST_RESID, h->xhat.p, h->q.p, h->bhat.p, nullptr, 0.0, 0.0, nullptr, s);
  dot_partials<double, double>(n, h->q.p, h->q.p, h->part0.p, s);
  pcg_store_true(h->part0.p, h->ctl.p, s);
  const long long k1 = captured();
  SAAMG_CUDA(cudaStreamBeginCaptureToGraph(body_s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  try {
    pcg_pass(h, cond, body_s);
  } catch (...) {
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(body_s, &junk);
    throw;
  }
  SAAMG_CUDA(cudaStreamEndCapture(body_s, &body));
  return GraphKernels{k1 - k0, captured() - k1};
}

static void build_solve_graph(saamg_hierarchy* h) {
  std::lock_guard<std::mutex> lock(g_capture_mu);
  cudaStream_t s = capture_stream(0);
  cudaGraph_t g = nullptr;
  SAAMG_CUDA(cudaGraphCreate(&g, 0));
  bool capturing = false;
  try {
    cudaGraphConditionalHandle cond;
    SAAMG_CUDA(cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault));
    SAAMG_CUDA(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capturing = true;
    const GraphKernels gk = capture_pcg(h, cond, s, capture_stream(1));
    h->gk_fixed = gk.fixed;
    h->gk_body = gk.body;
    capturing = false;
    SAAMG_CUDA(cudaStreamEndCapture(s, &g));
    SAAMG_CUDA(cudaGraphInstantiate(&h->gexec, g, 0));
    h->graph = g;
  } catch (...) {
    if (capturing) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(s, &junk);
      if (junk && junk != g) cudaGraphDestroy(junk);
    }
    cudaGraphDestroy(g);
    throw;
  }
}

static void drop_solve_graph(saamg_hierarchy* h) {
  if (h->done) cudaEventSynchronize(h->done);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->gexec = nullptr;
  h->graph = nullptr;
}

// Enqueues gather -> graph -> result copy -> scatter -> completion event; returns at once.
static void solve_async_impl(saamg_hierarchy* h, const double* rho, double* phi, double rtol,
                             cudaStream_t s, PcgCtl* host_out) {
  const OperatorData& od = h->op->d;
  if (!h->done) SAAMG_CUDA(cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming));
  if (od.n == 0) {
    PcgCtl z{};
    z.converged = 1;
    *host_out = z;
    scatter_solution(od, h->xhat.p, phi, s);
    SAAMG_CUDA(cudaEventRecord(h->done, s));
    return;
  }
  if (!h->gexec) build_solve_graph(h);
  gather_rhs(od, rho, phi, h->bhat.p, h->xhat.p, s);
  set_rtol_k<<<1, 1, 0, s>>>(h->ctl.p, rtol);
  SAAMG_LAUNCH();
  SAAMG_CUDA(cudaGraphLaunch(h->gexec, s));
  SAAMG_CUDA(cudaMemcpyAsync(host_out, h->ctl.p, sizeof(PcgCtl), cudaMemcpyDeviceToHost, s));
  scatter_solution(od, h->xhat.p, phi, s);
  SAAMG_CUDA(cudaEventRecord(h->done, s));
}

static saamg_status info_from_ctl(const PcgCtl& c, saamg_solve_info* info) {
  const double bn = std::sqrt(c.bb);
  info->iters = c.iters;
  info->converged = (c.converged && !c.breakdown) ? 1 : 0;
  info->relres = bn > 0 ? std::sqrt(c.rr) / bn : 0.0;
  info->relres_true = bn > 0 ? std::sqrt(c.rr_true) / bn : 0.0;
  if (c.breakdown) return SAAMG_NUMERICAL;
  return info->converged ? SAAMG_OK : SAAMG_NOT_CONVERGED;
}

static void recompute_cheb(saamg_hierarchy* h, int degree) {
  const int nl = (int)h->lev.size();
  for (int q = 0; q + 1 < nl; ++q) {
    Level& L = *h->lev[q];
    L.cheb = cheb_coefficients(L.lambda, h->prm.cheb_ratio, h->prm.cheb_safety, degree);
  }
  h->prm.cheb_degree = degree;
  drop_solve_graph(h);
  h->version = next_version();
}

}  // namespace saamg

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

saamg_status saamg_params_default(saamg_params* p) {
  if (!p) return SAAMG_EINVAL;
  p->cheb_degree = 2;
  p->cheb_ratio = 30.0;
  p->cheb_safety = 1.1;
  p->max_coarse = 1000;
  p->max_levels = 10;
  p->power_iters = 10;
  p->precision = SAAMG_PREC_FP64;
  p->beta_rule = 0;
  p->maxit = 1000;
  p->aggregation = SAAMG_AGG_MIS2;
  p->coarse_solver = SAAMG_COARSE_LU;
  p->coarse_sweeps = 3;
  p->device_loop = 1;
  return SAAMG_OK;
}

saamg_status saamg_set_allocator(saamg_alloc_fn alloc, saamg_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) {
    g_last_error = "saamg_set_allocator: alloc and free must both be set or both be NULL";
    return SAAMG_EINVAL;
  }
  try {
    pool_drain();  // cached blocks belong to the allocator being replaced
  } catch (...) {
  }
  g_alloc.alloc = alloc;
  g_alloc.free = free_fn;
  g_alloc.ctx = ctx;
  return SAAMG_OK;
}

const char* saamg_last_error(void) { return g_last_error.c_str(); }

saamg_status saamg_build_operator(const saamg_domain* domain, const saamg_grid* grid, int mode,
                                  void* stream, saamg_operator** out) {
  return guard("saamg_build_operator", [&] {
    if (!domain || !grid || !out) fail(SAAMG_EINVAL, "NULL argument");
    *out = nullptr;
    GeomParams g{};
    g.nx = grid->n[0];
    g.ny = grid->n[1];
    g.nz = grid->n[2];
    for (int d = 0; d < 3; ++d) {
      g.h[d] = grid->h[d];
      g.o[d] = grid->origin[d];
      if (!(grid->h[d] > 0.0) || !std::isfinite(grid->h[d]) || !std::isfinite(grid->origin[d]))
        fail(SAAMG_EINVAL, "grid spacing must be positive and finite");
    }
    if (g.nx < 1 || g.ny < 1 || g.nz < 2) fail(SAAMG_EINVAL, "grid needs n >= 1 and nz >= 2");
    if (domain->zbc != SAAMG_Z_ROBIN && domain->zbc != SAAMG_Z_DIRICHLET)
      fail(SAAMG_EINVAL, "unknown z boundary");
    if (domain->zbc == SAAMG_Z_DIRICHLET && g.nz < 3) fail(SAAMG_EINVAL, "Dirichlet ends need nz >= 3");
    if (!(domain->a > 0) || !(domain->b > 0) || !(domain->taper > 0) || !std::isfinite(domain->a) ||
        !std::isfinite(domain->b) || !std::isfinite(domain->taper) || !std::isfinite(domain->cx) ||
        !std::isfinite(domain->cy))
      fail(SAAMG_EINVAL, "domain semi-axes and taper must be positive and finite");
    if (mode < SAAMG_BC_CONSTANT || mode > SAAMG_BC_QUADRATIC) fail(SAAMG_EINVAL, "unknown boundary mode");
    if ((long long)g.nx * g.ny * g.nz > (1LL << 31) - 1) fail(SAAMG_EINVAL, "box larger than 2^31 nodes");
    g.a = domain->a;
    g.b = domain->b;
    g.taper = domain->taper;
    g.cx = domain->cx;
    g.cy = domain->cy;
    g.zbc = domain->zbc;
    g.sym = domain->symmetrize_gamma2 ? 1 : 0;
    g.mode = mode;
    for (int d = 0; d < 3; ++d) g.cdir[d] = 1.0 / (g.h[d] * g.h[d]);
    const double dist = 0.5 * ((double)(g.nz - 1) * g.h[2]);  // Robin distance d
    g.robin = (2.0 * g.h[2]) / dist;
    auto op = std::make_unique<saamg_operator>();
    op->stream = (cudaStream_t)stream;
    build_operator_data(g, (cudaStream_t)stream, op->d);
    *out = op.release();
  });
}

saamg_status saamg_operator_size(const saamg_operator* op, int* n, long long* nnz) {
  return guard("saamg_operator_size", [&] {
    if (!op || op->magic != kOpMagic) fail(SAAMG_EINVAL, "not an operator handle");
    if (n) *n = op->d.n;
    if (nnz) *nnz = op->d.nnz;
  });
}

saamg_status saamg_operator_copy(const saamg_operator* op, int* node_of_row, double* scale,
                                 int* rowptr, int* col, double* val, unsigned char* is_regular,
                                 void* stream) {
  return guard("saamg_operator_copy", [&] {
    if (!op || op->magic != kOpMagic) fail(SAAMG_EINVAL, "not an operator handle");
    cudaStream_t s = (cudaStream_t)stream;
    const OperatorData& d = op->d;
    auto cp = [&](void* dst, const void* src, size_t b) {
      if (dst && b) SAAMG_CUDA(cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, s));
    };
    cp(node_of_row, d.ids.p, sizeof(int) * d.n);
    cp(scale, d.scale.p, sizeof(double) * d.n);
    cp(rowptr, d.A.rowptr.p, sizeof(int) * (d.n + 1));
    cp(col, d.A.col.p, sizeof(int) * d.nnz);
    cp(val, d.A.val.p, sizeof(double) * d.nnz);
    cp(is_regular, d.regular.p, d.n);
    SAAMG_CUDA(cudaStreamSynchronize(s));
  });
}

saamg_status saamg_operator_apply(const saamg_operator* op, const double* x, double* y,
                                  void* stream) {
  return guard("saamg_operator_apply", [&] {
    if (!op || op->magic != kOpMagic) fail(SAAMG_EINVAL, "not an operator handle");
    if (op->d.n > 0 && (!x || !y)) fail(SAAMG_EINVAL, "NULL vector");
    stencil_apply<double>(op->d.view<double>(), ST_SPMV, x, y, nullptr, nullptr, 0.0, 0.0, nullptr,
                          (cudaStream_t)stream);
  });
}

saamg_status saamg_dense_inverse(int n, const double* a, double* inv, void* stream) {
  return guard("saamg_dense_inverse", [&] {
    if (n < 0 || n > 16384) fail(SAAMG_EINVAL, "n out of range");
    if (n > 0 && (!a || !inv)) fail(SAAMG_EINVAL, "NULL array");
    const uintptr_t a0 = (uintptr_t)a, i0 = (uintptr_t)inv, len = (uintptr_t)n * n * 8;
    if (n > 0 && a0 < i0 + len && i0 < a0 + len) fail(SAAMG_EINVAL, "inv overlaps a");
    dense_inverse(n, a, inv, (cudaStream_t)stream);
  });
}

static void check_grid(const saamg_grid* g) {
  if (!g) fail(SAAMG_EINVAL, "NULL grid");
  for (int d = 0; d < 3; ++d)
    if (g->n[d] < 1 || !(g->h[d] > 0.0) || !std::isfinite(g->origin[d]))
      fail(SAAMG_EINVAL, "bad grid");
  if ((double)g->n[0] * g->n[1] * g->n[2] > 4.0e9) fail(SAAMG_EINVAL, "grid too large");
}

saamg_status saamg_deposit_cic(const saamg_grid* grid, int np, const double* x, const double* y,
                               const double* z, const double* q, double* rho, void* stream) {
  return guard("saamg_deposit_cic", [&] {
    check_grid(grid);
    if (np < 0 || !rho || (np > 0 && (!x || !y || !z || !q))) fail(SAAMG_EINVAL, "bad arrays");
    deposit_cic(*grid, np, x, y, z, q, rho, (cudaStream_t)stream);
  });
}

saamg_status saamg_field_gradient(const saamg_operator* op, const double* phi, double* ex,
                                  double* ey, double* ez, void* stream) {
  return guard("saamg_field_gradient", [&] {
    if (!op || op->magic != kOpMagic) fail(SAAMG_EINVAL, "not an operator handle");
    if (!phi || !ex || !ey || !ez) fail(SAAMG_EINVAL, "NULL array");
    field_gradient(op->d, phi, ex, ey, ez, (cudaStream_t)stream);
  });
}

saamg_status saamg_gather_cic(const saamg_grid* grid, const double* ex, const double* ey,
                              const double* ez, int np, const double* x, const double* y,
                              const double* z, double* epx, double* epy, double* epz,
                              void* stream) {
  return guard("saamg_gather_cic", [&] {
    check_grid(grid);
    if (np < 0 || (np > 0 && (!ex || !ey || !ez || !x || !y || !z || !epx || !epy || !epz)))
      fail(SAAMG_EINVAL, "bad arrays");
    gather_cic(*grid, ex, ey, ez, np, x, y, z, epx, epy, epz, (cudaStream_t)stream);
  });
}

saamg_status saamg_setup(const saamg_operator* op, const saamg_params* params, void* stream,
                         saamg_hierarchy** out) {
  return guard("saamg_setup", [&] {
    if (!op || op->magic != kOpMagic || !out) fail(SAAMG_EINVAL, "NULL or invalid argument");
    *out = nullptr;
    saamg_params prm;
    saamg_params_default(&prm);
    if (params) prm = *params;
    if (prm.cheb_degree < 1 || prm.cheb_degree > 16) fail(SAAMG_EINVAL, "cheb_degree must be in 1..16");
    if (!(prm.cheb_ratio > 1.0) || !(prm.cheb_safety > 0.0)) fail(SAAMG_EINVAL, "bad Chebyshev interval");
    if (prm.max_coarse < 1 || prm.max_levels < 1 || prm.power_iters < 1 || prm.maxit < 0)
      fail(SAAMG_EINVAL, "max_coarse, max_levels, power_iters must be >= 1");
    if (prm.precision < SAAMG_PREC_FP64 || prm.precision > SAAMG_PREC_FP32_BF16)
      fail(SAAMG_EINVAL, "unknown precision");
    if (prm.beta_rule != 0 && prm.beta_rule != 1) fail(SAAMG_EINVAL, "beta_rule must be 0 or 1");
    check_params_ext(prm);
    auto h = std::make_unique<saamg_hierarchy>();
    setup_impl(op, prm, (cudaStream_t)stream, h.get());
    h->version = next_version();
    SAAMG_CUDA(cudaMallocHost(&h->result, sizeof(PcgCtl)));
    *out = h.release();
  });
}

saamg_status saamg_setup_reuse(const saamg_operator* op, const saamg_hierarchy* prev,
                               const saamg_params* params, void* stream, saamg_hierarchy** out) {
  return guard("saamg_setup_reuse", [&] {
    if (!op || op->magic != kOpMagic || !prev || prev->magic != kHierMagic || !out)
      fail(SAAMG_EINVAL, "NULL or invalid argument");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (!same_pattern(op->d.A, prev->op->d.A, s))
      fail(SAAMG_EINVAL, "the operator's pattern differs from the one the hierarchy was built on");
    saamg_params prm = prev->prm;
    if (params) prm = *params;
    prm.aggregation = prev->prm.aggregation;  // the aggregates come from `prev`
    if (prm.cheb_degree < 1 || prm.cheb_degree > 16) fail(SAAMG_EINVAL, "cheb_degree must be in 1..16");
    if (prm.precision < SAAMG_PREC_FP64 || prm.precision > SAAMG_PREC_FP32_BF16)
      fail(SAAMG_EINVAL, "unknown precision");
    check_params_ext(prm);
    auto h = std::make_unique<saamg_hierarchy>();
    setup_impl(op, prm, s, h.get(), prev);
    h->version = next_version();
    SAAMG_CUDA(cudaMallocHost(&h->result, sizeof(PcgCtl)));
    *out = h.release();
  });
}

saamg_status saamg_hierarchy_work_set(const saamg_hierarchy* h, void* stream, saamg_hierarchy** out) {
  return guard("saamg_hierarchy_work_set", [&] {
    if (!h || h->magic != kHierMagic || !out) fail(SAAMG_EINVAL, "NULL or invalid argument");
    *out = nullptr;
    saamg_hierarchy* owner = h->base ? h->base : const_cast<saamg_hierarchy*>(h);
    auto w = std::make_unique<saamg_hierarchy>();
    work_set_impl(h, (cudaStream_t)stream, w.get());
    w->version = next_version();
    SAAMG_CUDA(cudaMallocHost(&w->result, sizeof(PcgCtl)));
    owner->refs.fetch_add(1);
    w->base = owner;
    *out = w.release();
  });
}

saamg_status saamg_hierarchy_get_info(const saamg_hierarchy* h, saamg_hierarchy_info* info) {
  return guard("saamg_hierarchy_get_info", [&] {
    if (!h || h->magic != kHierMagic || !info) fail(SAAMG_EINVAL, "NULL or invalid argument");
    std::memset(info, 0, sizeof(*info));
    info->levels = (int)h->lev.size();
    for (int l = 0; l < info->levels; ++l) {
      info->n[l] = h->lev[l]->n;
      info->nnz[l] = h->lev[l]->nnz;
      info->nnz_p[l] = h->lev[l]->P.nnz;
      info->lambda[l] = h->lev[l]->lambda;
      info->sell_index_bytes[l] = h->lev[l]->As.n > 0 ? h->lev[l]->As.index_bytes : 0;
    }
    info->device_bytes = h->bytes;
    info->setup_ms = h->setup_ms;
  });
}

saamg_status saamg_hierarchy_copy_level(const saamg_hierarchy* h, int l, int* rowptr, int* col,
                                        double* val, int* agg, unsigned char* root, int* p_rowptr,
                                        int* p_col, double* p_val, int* r_rowptr, int* r_col,
                                        double* r_val, void* stream) {
  return guard("saamg_hierarchy_copy_level", [&] {
    if (!h || h->magic != kHierMagic) fail(SAAMG_EINVAL, "not a hierarchy handle");
    if (l < 0 || l >= (int)h->lev.size()) fail(SAAMG_EINVAL, "level out of range");
    cudaStream_t s = (cudaStream_t)stream;
    const Level& L = *h->lev[l];
    const DevCsr& A = level_matrix(h, l);
    auto cp = [&](void* dst, const void* src, size_t b) {
      if (dst && src && b) SAAMG_CUDA(cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToHost, s));
    };
    cp(rowptr, A.rowptr.p, sizeof(int) * (A.n + 1));
    cp(col, A.col.p, sizeof(int) * A.nnz);
    cp(val, A.val.p, sizeof(double) * A.nnz);
    cp(agg, L.agg.p, sizeof(int) * (L.agg.p ? L.n : 0));
    cp(root, L.root.p, L.root.p ? L.n : 0);
    if (L.P.rowptr.p) {
      cp(p_rowptr, L.P.rowptr.p, sizeof(int) * (L.P.n + 1));
      cp(p_col, L.P.col.p, sizeof(int) * L.P.nnz);
      cp(p_val, L.P.val.p, sizeof(double) * L.P.nnz);
      cp(r_rowptr, L.R.rowptr.p, sizeof(int) * (L.R.n + 1));
      cp(r_col, L.R.col.p, sizeof(int) * L.R.nnz);
      cp(r_val, L.R.val.p, sizeof(double) * L.R.nnz);
    }
    SAAMG_CUDA(cudaStreamSynchronize(s));
  });
}

saamg_status saamg_vcycle(const saamg_hierarchy* hc, const double* r, double* z, void* stream) {
  return guard("saamg_vcycle", [&] {
    if (!hc || hc->magic != kHierMagic) fail(SAAMG_EINVAL, "not a hierarchy handle");
    saamg_hierarchy* h = const_cast<saamg_hierarchy*>(hc);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->op->d.n;
    if (n == 0) return;
    if (!r || !z) fail(SAAMG_EINVAL, "NULL vector");
    if (!mixed(h)) {
      vcycle_level<double>(h, 0, r, z, s);
    } else {
      apply_preconditioner(h, r, nullptr, h->z32.p, s);
      to_double(h->z32.p, z, n, s);
    }
    if (!h->done) SAAMG_CUDA(cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming));
    SAAMG_CUDA(cudaEventRecord(h->done, s));
  });
}

// The device-loop solve (the graph of saamg_solve_async), waited for; the breakdown status
// carries a message like the host loop's.
static int solve_device(saamg_hierarchy* h, const double* rho, double* phi, double rtol,
                        cudaStream_t s, saamg_solve_info* info) {
  solve_async_impl(h, rho, phi, rtol, s, h->result);
  SAAMG_CUDA(cudaEventSynchronize(h->done));
  if (h->op->d.n > 0) count_launches(h->gk_fixed + h->result->iters * h->gk_body);
  const saamg_status st = info_from_ctl(*h->result, info);
  if (st == SAAMG_NUMERICAL)
    set_last_error("saamg_solve: breakdown (NaN/Inf in the right-hand side or p'Ap = 0)");
  return st;
}

saamg_status saamg_solve(saamg_hierarchy* h, const double* rho, double* phi, double rtol,
                         void* stream, saamg_solve_info* info) {
  saamg_solve_info local{};
  if (!info) info = &local;
  int st = SAAMG_OK;
  auto t0 = std::chrono::steady_clock::now();
  saamg_status g = guard("saamg_solve", [&] {
    if (!h || h->magic != kHierMagic) fail(SAAMG_EINVAL, "not a hierarchy handle");
    if (!rho || !phi) fail(SAAMG_EINVAL, "NULL rho or phi");
    if (!(rtol > 0.0) || !std::isfinite(rtol)) fail(SAAMG_EINVAL, "rtol must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    const OperatorData& od = h->op->d;
    if (h->prm.device_loop) {
      st = solve_device(h, rho, phi, rtol, s, info);
      return;
    }
    gather_rhs(od, rho, phi, h->bhat.p, h->xhat.p, s);
    st = pcg_impl(h, rtol, s, info);
    scatter_solution(od, h->xhat.p, phi, s);
    SAAMG_CUDA(cudaStreamSynchronize(s));
  });
  info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return g != SAAMG_OK ? g : (saamg_status)st;
}

// The device address of page-locked host memory mapped into the device's address space, or
// NULL for other memory.
static void* mapped_host(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

saamg_status saamg_solve_host(saamg_hierarchy* h, const double* rho_host, double* phi_host,
                              double rtol, void* stream, saamg_solve_info* info) {
  saamg_solve_info local{};
  if (!info) info = &local;
  int st = SAAMG_OK;
  auto t0 = std::chrono::steady_clock::now();
  saamg_status g = guard("saamg_solve_host", [&] {
    if (!h || h->magic != kHierMagic) fail(SAAMG_EINVAL, "not a hierarchy handle");
    if (!rho_host || !phi_host) fail(SAAMG_EINVAL, "NULL rho or phi");
    if (!(rtol > 0.0) || !std::isfinite(rtol)) fail(SAAMG_EINVAL, "rtol must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    const OperatorData& od = h->op->d;
    size_t nbox = (size_t)od.g.nx * od.g.ny * od.g.nz;
    // Pinned (page-locked, mapped) host arrays are read by the gather and written by the
    // scatter directly, through their device addresses: the values cross the host link once,
    // with no staging copy.  Other host memory is staged through device box arrays.
    const double* rho_dev = static_cast<const double*>(mapped_host(rho_host));
    double* phi_dev = static_cast<double*>(mapped_host(phi_host));
    Buf<double> rho, phi;
    if (!rho_dev || !phi_dev) {
      rho.alloc(nbox, s);
      phi.alloc(nbox, s);
      SAAMG_CUDA(cudaMemcpyAsync(rho.p, rho_host, nbox * 8, cudaMemcpyHostToDevice, s));
      SAAMG_CUDA(cudaMemcpyAsync(phi.p, phi_host, nbox * 8, cudaMemcpyHostToDevice, s));
      rho_dev = rho.p;
      phi_dev = phi.p;
    }
    if (h->prm.device_loop) {
      st = solve_device(h, rho_dev, phi_dev, rtol, s, info);
    } else {
      gather_rhs(od, rho_dev, phi_dev, h->bhat.p, h->xhat.p, s);
      st = pcg_impl(h, rtol, s, info);
      scatter_solution(od, h->xhat.p, phi_dev, s);
    }
    if (phi.p) SAAMG_CUDA(cudaMemcpyAsync(phi_host, phi.p, nbox * 8, cudaMemcpyDeviceToHost, s));
    SAAMG_CUDA(cudaStreamSynchronize(s));
  });
  info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return g != SAAMG_OK ? g : (saamg_status)st;
}

saamg_status saamg_solve_async(saamg_hierarchy* h, const double* rho, double* phi, double rtol,
                               void* stream) {
  return guard("saamg_solve_async", [&] {
    if (!h || h->magic != kHierMagic) fail(SAAMG_EINVAL, "not a hierarchy handle");
    if (!rho || !phi) fail(SAAMG_EINVAL, "NULL rho or phi");
    if (!(rtol > 0.0) || !std::isfinite(rtol)) fail(SAAMG_EINVAL, "rtol must be positive");
    solve_async_impl(h, rho, phi, rtol, (cudaStream_t)stream, h->result);
  });
}

saamg_status saamg_solve_test(const saamg_hierarchy* h) {
  if (!h || h->magic != kHierMagic) return SAAMG_EINVAL;
  if (!h->done) return SAAMG_OK;
  cudaError_t e = cudaEventQuery(h->done);
  if (e == cudaSuccess) return SAAMG_OK;
  if (e == cudaErrorNotReady) return SAAMG_NOT_READY;
  cudaGetLastError();
  set_last_error(std::string("saamg_solve_test: ") + cudaGetErrorString(e));
  return SAAMG_ECUDA;
}

saamg_status saamg_solve_wait(saamg_hierarchy* h, saamg_solve_info* info) {
  saamg_solve_info local{};
  if (!info) info = &local;
  saamg_status st = SAAMG_OK;
  saamg_status g = guard("saamg_solve_wait", [&] {
    if (!h || h->magic != kHierMagic) fail(SAAMG_EINVAL, "not a hierarchy handle");
    if (h->done) SAAMG_CUDA(cudaEventSynchronize(h->done));
    if (h->gexec && h->op->d.n > 0) count_launches(h->gk_fixed + h->result->iters * h->gk_body);
    st = info_from_ctl(*h->result, info);
    if (st == SAAMG_NUMERICAL) set_last_error("saamg_solve_wait: breakdown (NaN/Inf or p'Ap = 0)");
  });
  return g != SAAMG_OK ? g : st;
}

// --- batched solves as one graph -----------------------------------------------------
// The whole batch is captured once into one graph: one branch per group of hierarchies (the
// solves of one hierarchy share its work vectors and run in order on their branch), every
// solve inline as gather -> prologue -> conditional while (PCG pass) -> epilogue -> result
// copy -> scatter.  A call whose hierarchies (by version), arrays and tolerance match a
// cached graph is one graph launch.
struct BatchGraph {
  std::vector<const saamg_hierarchy*> hs;
  std::vector<unsigned long long> versions;
  std::vector<const double*> rho;
  std::vector<double*> phi;
  double rtol = 0.0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  PcgCtl* res = nullptr;  // pinned, one per solve
  std::vector<long long> kfixed, kbody;  // kernels of each solve: once, and per PCG pass
  BatchEngine* eng = nullptr;            // the merged form (one launch per operation)
  // wall time of the first run of each form (-1: not run yet); later runs take the faster
  double ms_merged = -1.0, ms_graphs = -1.0;
  ~BatchGraph() {
    if (eng) batch_engine_free(eng);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (res) cudaFreeHost(res);
  }
  bool matches(saamg_hierarchy* const* h, const double* const* r, double* const* x, int count,
               double tol) const {
    if ((int)hs.size() != count || tol != rtol) return false;
    for (int j = 0; j < count; ++j)
      if (hs[j] != h[j] || versions[j] != h[j]->version || rho[j] != r[j] || phi[j] != x[j])
        return false;
    return true;
  }
};

static std::mutex g_batch_mu;  // batched calls run one at a time
struct BatchLast {
  int merged = 0;
  double ms_merged = -1.0, ms_graphs = -1.0;
};
static BatchLast g_batch_last;  // the most recent batched call (under g_batch_mu)
// Most recent last.  Never destroyed at process exit: an entry's work vectors go back through
// the allocator hook that gave them out, which may no longer be callable then (a Python
// callback during interpreter shutdown); saamg_release_batch_cache empties it while it is.
static std::vector<std::unique_ptr<BatchGraph>>& g_batch_cache =
    *new std::vector<std::unique_ptr<BatchGraph>>();
constexpr size_t kBatchCache = 2;

// The per-solve form of a batch: one device-loop graph per solve inside one graph, solves of
// one hierarchy in order on a branch, up to 32 branches.
static void build_batch_graph(BatchGraph* bg, saamg_hierarchy* const* hs,
                              const double* const* rho, double* const* phi, int count,
                              double rtol, const std::vector<saamg_hierarchy*>& order,
                              std::map<saamg_hierarchy*, std::vector<int>>& groups) {
  SAAMG_CUDA(cudaMallocHost(&bg->res, sizeof(PcgCtl) * count));
  std::lock_guard<std::mutex> lock(g_capture_mu);
  cudaStream_t cs = capture_stream(0), body = capture_stream(1);
  const int nbr = (int)std::min<size_t>(order.size(), 32);
  std::vector<cudaEvent_t> evs;
  cudaGraph_t g = nullptr;
  SAAMG_CUDA(cudaGraphCreate(&g, 0));
  bool capturing = false;
  try {
    std::vector<cudaGraphConditionalHandle> conds(count);
    for (int j = 0; j < count; ++j)  // a handle that no conditional node uses fails instantiation
      if (hs[j]->op->d.n > 0)
        SAAMG_CUDA(cudaGraphConditionalHandleCreate(&conds[j], g, 0, cudaGraphCondAssignDefault));
    SAAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capturing = true;
    CaptureCount counting;  // the graph's kernels are counted when it runs
    bg->kfixed.assign(count, 0);
    bg->kbody.assign(count, 0);
    cudaEvent_t fork;
    SAAMG_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    evs.push_back(fork);
    SAAMG_CUDA(cudaEventRecord(fork, cs));
    for (int k = 0; k < nbr; ++k) SAAMG_CUDA(cudaStreamWaitEvent(capture_stream(2 + k), fork, 0));
    for (size_t gi = 0; gi < order.size(); ++gi) {
      saamg_hierarchy* h = order[gi];
      const OperatorData& od = h->op->d;
      cudaStream_t ps = capture_stream(2 + (int)(gi % nbr));
      for (int j : groups[h]) {
        const long long c0 = captured();
        if (od.n == 0) {  // no unknowns: phi = 0, converged at once
          bg->res[j] = PcgCtl{};
          bg->res[j].converged = 1;
          scatter_solution(od, h->xhat.p, phi[j], ps);
          continue;
        }
        gather_rhs(od, rho[j], phi[j], h->bhat.p, h->xhat.p, ps);
        set_rtol_k<<<1, 1, 0, ps>>>(h->ctl.p, rtol);
        SAAMG_LAUNCH();
        const GraphKernels gk = capture_pcg(h, conds[j], ps, body);
        SAAMG_CUDA(cudaMemcpyAsync(&bg->res[j], h->ctl.p, sizeof(PcgCtl), cudaMemcpyDeviceToHost, ps));
        scatter_solution(od, h->xhat.p, phi[j], ps);
        bg->kfixed[j] = captured() - c0 - gk.body;
        bg->kbody[j] = gk.body;
      }
    }
    for (int k = 0; k < nbr; ++k) {
      cudaEvent_t e;
      SAAMG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      evs.push_back(e);
      SAAMG_CUDA(cudaEventRecord(e, capture_stream(2 + k)));
      SAAMG_CUDA(cudaStreamWaitEvent(cs, e, 0));
    }
    capturing = false;
    SAAMG_CUDA(cudaStreamEndCapture(cs, &g));
    SAAMG_CUDA(cudaGraphInstantiate(&bg->exec, g, 0));
    bg->graph = g;
    SAAMG_CUDA(cudaGraphUpload(bg->exec, cs));  // the first run does not pay for the upload
    SAAMG_CUDA(cudaStreamSynchronize(cs));
  } catch (...) {
    if (capturing) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(cs, &junk);
      if (junk && junk != g) cudaGraphDestroy(junk);
    }
    cudaGraphDestroy(g);
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
    throw;
  }
  for (cudaEvent_t e : evs) cudaEventDestroy(e);
}

saamg_status saamg_solve_batched(saamg_hierarchy* const* hs, const double* const* rho,
                                 double* const* phi, int count, double rtol, void* stream,
                                 saamg_solve_info* infos) {
  saamg_status worst = SAAMG_OK;
  auto t0 = std::chrono::steady_clock::now();
  saamg_status g = guard("saamg_solve_batched", [&] {
    if (count < 0 || (count > 0 && (!hs || !rho || !phi || !infos)))
      fail(SAAMG_EINVAL, "bad count or NULL arrays");
    if (!(rtol > 0.0) || !std::isfinite(rtol)) fail(SAAMG_EINVAL, "rtol must be positive");
    if (count == 0) return;
    for (int j = 0; j < count; ++j) {
      if (!hs[j] || hs[j]->magic != kHierMagic) fail(SAAMG_EINVAL, "not a hierarchy handle");
      if (!rho[j] || !phi[j]) fail(SAAMG_EINVAL, "NULL rho or phi");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // solves of one hierarchy share its work vectors: they run in order on one stream;
    // different hierarchies run on different streams and overlap on the device
    std::vector<saamg_hierarchy*> order;
    std::map<saamg_hierarchy*, std::vector<int>> groups;
    for (int j = 0; j < count; ++j) {
      if (!groups.count(hs[j])) order.push_back(hs[j]);
      groups[hs[j]].push_back(j);
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchGraph* bg = nullptr;
    for (size_t e = 0; e < g_batch_cache.size(); ++e)
      if (g_batch_cache[e]->matches(hs, rho, phi, count, rtol)) {
        // most recent last
        std::unique_ptr<BatchGraph> hit = std::move(g_batch_cache[e]);
        g_batch_cache.erase(g_batch_cache.begin() + e);
        g_batch_cache.push_back(std::move(hit));
        bg = g_batch_cache.back().get();
        break;
      }
    if (!bg) {
      auto built = std::make_unique<BatchGraph>();
      for (int j = 0; j < count; ++j) {
        built->hs.push_back(hs[j]);
        built->versions.push_back(hs[j]->version);
        built->rho.push_back(rho[j]);
        built->phi.push_back(phi[j]);
      }
      built->rtol = rtol;
      if (g_batch_cache.size() >= kBatchCache) g_batch_cache.erase(g_batch_cache.begin());
      g_batch_cache.push_back(std::move(built));
      bg = g_batch_cache.back().get();
    }
    // Two forms give the same bits: one launch per operation across all solves (merged), or
    // one device-loop graph per solve on concurrent branches.  The first run of a batch takes
    // the merged form, the second the per-solve form, and later runs the faster of the two.
    const bool can_merge = batch_engine_supports(hs, count);
    bool merged;
    if (!can_merge) merged = false;
    else if (bg->ms_merged < 0) merged = true;
    else if (bg->ms_graphs < 0) merged = false;
    else merged = bg->ms_merged <= bg->ms_graphs;
    if (merged && !bg->eng) {
      std::lock_guard<std::mutex> lock(g_capture_mu);
      bg->eng = batch_engine_build(hs, rho, phi, count, rtol, capture_stream);
    }
    if (!merged && !bg->exec) build_batch_graph(bg, hs, rho, phi, count, rtol, order, groups);
    const auto l0 = std::chrono::steady_clock::now();
    if (merged) batch_engine_launch(bg->eng, s);
    else SAAMG_CUDA(cudaGraphLaunch(bg->exec, s));
    for (saamg_hierarchy* h : order) {
      if (!h->done) SAAMG_CUDA(cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming));
      SAAMG_CUDA(cudaEventRecord(h->done, s));
    }
    SAAMG_CUDA(cudaStreamSynchronize(s));
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - l0).count();
    double& slot = merged ? bg->ms_merged : bg->ms_graphs;
    if (slot < 0) slot = ms;
    g_batch_last = {merged ? 1 : 0, bg->ms_merged, bg->ms_graphs};
    const PcgCtl* res = merged ? batch_engine_results(bg->eng) : bg->res;
    long long kernels = 0;
    if (merged) kernels = batch_engine_kernels(bg->eng);
    else
      for (int j = 0; j < count; ++j) kernels += bg->kfixed[j] + bg->res[j].iters * bg->kbody[j];
    count_launches(kernels);
    for (int j = 0; j < count; ++j) {
      saamg_status st = info_from_ctl(res[j], &infos[j]);
      if (st < 0 && worst >= 0) worst = st;
      else if (st == SAAMG_NOT_CONVERGED && worst == SAAMG_OK) worst = st;
    }
  });
  if (count > 0 && infos) {
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int j = 0; j < count; ++j) infos[j].solve_ms = ms;
  }
  return g != SAAMG_OK ? g : worst;
}

saamg_status saamg_batch_last(int* merged, double* ms_merged, double* ms_graphs) {
  return guard("saamg_batch_last", [&] {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    if (merged) *merged = g_batch_last.merged;
    if (ms_merged) *ms_merged = g_batch_last.ms_merged;
    if (ms_graphs) *ms_graphs = g_batch_last.ms_graphs;
  });
}

saamg_status saamg_release_batch_cache(void) {
  return guard("saamg_release_batch_cache", [&] {
    std::lock_guard<std::mutex> lock(g_batch_mu);
    g_batch_cache.clear();
  });
}

static void check_stencil_cfg(const saamg_stencil_config& c) {
  const bool ok = (c.chunks_per_step == 1 || c.chunks_per_step == 2 || c.chunks_per_step == 4) &&
                  (c.packed == 0 || c.packed == 1) && (c.block == 128 || c.block == 256) &&
                  (c.blocks_per_sm == 8 || c.blocks_per_sm == 16 || c.blocks_per_sm == 32);
  if (!ok) fail(SAAMG_EINVAL, "stencil launch shape outside the supported sets");
}

saamg_status saamg_stencil_config_get(const saamg_operator* op, int precision,
                                      saamg_stencil_config* cfg) {
  return guard("saamg_stencil_config_get", [&] {
    if (!op || op->magic != kOpMagic || !cfg) fail(SAAMG_EINVAL, "NULL or invalid argument");
    if (precision != 0 && precision != 1) fail(SAAMG_EINVAL, "precision must be 0 or 1");
    const StencilCfg& c = op->d.cfg[precision];
    *cfg = saamg_stencil_config{c.k, c.packed, c.block, c.per_sm};
  });
}

saamg_status saamg_stencil_config_set(saamg_operator* op, int precision,
                                      const saamg_stencil_config* cfg) {
  return guard("saamg_stencil_config_set", [&] {
    if (!op || op->magic != kOpMagic) fail(SAAMG_EINVAL, "NULL or invalid argument");
    if (precision != 0 && precision != 1) fail(SAAMG_EINVAL, "precision must be 0 or 1");
    if (!cfg) {
      op->d.cfg[precision] = OperatorData{}.cfg[precision];
      return;
    }
    check_stencil_cfg(*cfg);
    op->d.cfg[precision] = StencilCfg{cfg->chunks_per_step, cfg->packed, cfg->block,
                                      cfg->blocks_per_sm};
  });
}

saamg_status saamg_autotune_stencil(saamg_operator* op, int precision, void* stream,
                                    saamg_stencil_config* best, double* best_us) {
  return guard("saamg_autotune_stencil", [&] {
    if (!op || op->magic != kOpMagic) fail(SAAMG_EINVAL, "NULL or invalid argument");
    if (precision != 0 && precision != 1) fail(SAAMG_EINVAL, "precision must be 0 or 1");
    cudaStream_t s = (cudaStream_t)stream;
    double us = 0;
    const StencilCfg c = precision == 0 ? stencil_autotune<double>(op->d.view<double>(), s, &us)
                                        : stencil_autotune<float>(op->d.view<float>(), s, &us);
    op->d.cfg[precision] = c;
    if (best) *best = saamg_stencil_config{c.k, c.packed, c.block, c.per_sm};
    if (best_us) *best_us = us;
  });
}

saamg_status saamg_set_cheb_degree(saamg_hierarchy* h, int degree) {
  return guard("saamg_set_cheb_degree", [&] {
    if (!h || h->magic != kHierMagic) fail(SAAMG_EINVAL, "not a hierarchy handle");
    if (degree < 1 || degree > 16) fail(SAAMG_EINVAL, "degree must be in 1..16");
    if (h->done) SAAMG_CUDA(cudaEventSynchronize(h->done));
    recompute_cheb(h, degree);
  });
}

saamg_status saamg_autotune_cheb_degree(saamg_hierarchy* h, const double* rho, int lo, int hi,
                                        double rtol, void* stream, int* best_degree,
                                        double* best_ms) {
  return guard("saamg_autotune_cheb_degree", [&] {
    if (!h || h->magic != kHierMagic || !rho) fail(SAAMG_EINVAL, "NULL or invalid argument");
    if (lo < 1 || hi > 16 || lo > hi) fail(SAAMG_EINVAL, "degree range must satisfy 1 <= lo <= hi <= 16");
    if (!(rtol > 0.0)) fail(SAAMG_EINVAL, "rtol must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    const OperatorData& od = h->op->d;
    Buf<double> phi;
    phi.alloc((size_t)od.g.nx * od.g.ny * od.g.nz, s);
    cudaEvent_t e0, e1;
    SAAMG_CUDA(cudaEventCreate(&e0));
    SAAMG_CUDA(cudaEventCreate(&e1));
    int best = h->prm.cheb_degree;
    float best_t = -1.f;
    try {
      for (int d = lo; d <= hi; ++d) {
        recompute_cheb(h, d);
        for (int rep = 0; rep < 2; ++rep) {  // the first pass captures the graph
          SAAMG_CUDA(cudaMemsetAsync(phi.p, 0, phi.bytes(), s));
          SAAMG_CUDA(cudaEventRecord(e0, s));
          solve_async_impl(h, rho, phi.p, rtol, s, h->result);
          SAAMG_CUDA(cudaEventRecord(e1, s));
          SAAMG_CUDA(cudaEventSynchronize(e1));
        }
        float ms = 0.f;
        SAAMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (h->result->converged && (best_t < 0.f || ms < best_t)) {
          best_t = ms;
          best = d;
        }
      }
    } catch (...) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    recompute_cheb(h, best);
    if (best_degree) *best_degree = best;
    if (best_ms) *best_ms = best_t;
  });
}

saamg_status saamg_mis2_aggregate(int n, const int* rowptr, const int* col, const uint32_t* ids,
                                  uint32_t seed, unsigned char* root, int* agg, int* n_agg,
                                  void* stream) {
  return guard("saamg_mis2_aggregate", [&] {
    if (n < 0 || !n_agg) fail(SAAMG_EINVAL, "bad size or NULL n_agg");
    *n_agg = 0;
    if (n == 0) return;
    if (!rowptr || !col || !root || !agg) fail(SAAMG_EINVAL, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    int nnz = 0;
    d2h_sync(&nnz, rowptr + n, sizeof(int), s);
    AggScratchBufs w;
    w.alloc(n, s);
    *n_agg = mis2_aggregate(n, rowptr, col, nnz, ids, seed, root, agg, w.view(), s);
    SAAMG_CUDA(cudaStreamSynchronize(s));
  });
}

void saamg_free(void* handle) {
  if (!handle) return;
  uint32_t magic = *static_cast<uint32_t*>(handle);
  try {
    if (magic == kOpMagic) {
      saamg_operator* op = static_cast<saamg_operator*>(handle);
      cudaStreamSynchronize(op->stream);
      op->magic = 0;
      delete op;
    } else if (magic == kHierMagic) {
      saamg_hierarchy* h = static_cast<saamg_hierarchy*>(handle);
      // asynchronous calls record `done`; the synchronous ones end with a stream sync
      if (h->done) cudaEventSynchronize(h->done);
      saamg_hierarchy* base = h->base;
      release_hierarchy(h);
      if (base) release_hierarchy(base);
    }
  } catch (...) {
  }
}

}  // extern "C"
