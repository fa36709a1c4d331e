// Batched PCG: many right-hand sides on many hierarchies (Sec. 3.1 with one V-cycle of
// Algorithm 1 per iteration) advanced together, so that every operation of a PCG iteration
// is ONE launch across all solves instead of one launch per solve.
//
// Each solve gets its own work vectors (every level of its V-cycle, the CG vectors, its
// scalars), so solves that share a hierarchy run side by side.  The V-cycle of every solve
// is planned on the host as the one-solve code would run it (same kernels, same arguments,
// same order); the operations are then merged across solves by their place in the cycle
// (level, phase, Chebyshev step) and by kernel form, and each merged group is one launch over
// a table of tasks (one per solve).  Each task's work units (chunks, slices, row groups, rows)
// are cut into work blocks of a few units, listed with their task, so a block of threads
// reads its task once.  Every unit runs exactly the per-row arithmetic of the one-solve kernel (shared
// device functions), and reductions keep the one-solve grid per task, so a solve gives the
// same bits here as alone.
//
// The PCG loop is one CUDA graph: a prologue per solve, a conditional while node whose body
// is one PCG pass over all solves, and an epilogue per solve.  A solve that has converged,
// broken down or reached its iteration limit clears its flag, after which every task of that
// solve does nothing; the loop ends when no flag is left.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "batch.cuh"
#include "hier.cuh"
#include "rows.cuh"

namespace saamg {

namespace {

constexpr int kWarps = 8;         // warps per block of the batched kernels
constexpr int kWarpUnits = 4;     // warp-sized units per warp and work block
constexpr int kBlockUnits = 4;    // 256-element units per work block (vector kernels)
constexpr int kMaxLanes = 8;      // concurrent sub-batches of a batch
constexpr int kLaneSolves = 32;   // solves per lane (about)

// --- tasks ----------------------------------------------------------------------------------
struct MTask {  // a sparse-matrix, coarse-solve or copy operation of one solve
  const int* go;
  int n;        // rows (CSR, SELL, coarse inverse) or elements (copy)
  int nslices;  // SELL
  const int* rowptr;
  const int* col;
  const void* val;  // CSR / SELL values, or the coarse inverse (double)
  const int* perm;
  const int* soff;
  const short* dcol;
  const void* x;
  void* y;
  const void* b;
  void* d;
  const void* invd;
  double c1, c2;
};

struct VTask {  // the CG recursion of one solve
  int* go;
  int n;
  PcgCtl* ctl;
  double* x;
  double* r;
  double* p;
  double* q;
  const void* z;  // z (FP64 V-cycle) or z32 (mixed)
  float* r32;     // mixed: FP32 copy of r
  double* part0;
  double* part1;
  double* part2;
  int rule, maxit;
  double rtol;
};

// Copies task t into shared memory (the whole block takes part).
template <class Task>
__device__ __forceinline__ void load_task(const Task* __restrict__ tasks, int t, Task& sk) {
  const int* src = reinterpret_cast<const int*>(tasks + t);
  int* dst = reinterpret_cast<int*>(&sk);
  for (int i = threadIdx.x; i < (int)(sizeof(Task) / 4); i += blockDim.x) dst[i] = src[i];
}

// Every work-block kernel starts a work block the same way: the task into shared memory, and
// nothing to do when its solve has ended.
#define SAAMG_WORK_BLOCK(TaskT)            \
  const int4 B = wbs[wb];                  \
  __syncthreads();                         \
  load_task<TaskT>(tasks, B.x, sk);        \
  __syncthreads();                         \
  if (!*sk.go) continue;                   \
  const TaskT& k = sk;

// --- sparse-matrix kernels --------------------------------------------------------------------
template <class TV, class TM, int G, int MODE>
__global__ void __launch_bounds__(256, 5) bcsr_k(const MTask* __restrict__ tasks,
                                              const int4* __restrict__ wbs, int nwb) {
  __shared__ MTask sk;
  const int lane = threadIdx.x & 31, gl = lane % G, warp = threadIdx.x >> 5;
  constexpr int kRows = 32 / G;
  double dacc = 0.0;
  for (int wb = blockIdx.x; wb < nwb; wb += gridDim.x) {
    SAAMG_WORK_BLOCK(MTask)
    for (int u = B.y + warp; u < B.z; u += kWarps) {
    const int row = u * kRows + lane / G;
    rows::csr_group_row<TV, TM, G, MODE>(row, row < k.n, gl, k.rowptr, k.col,
                                         (const TM*)k.val, (const TV*)k.x, (TV*)k.y,
                                         (const TV*)k.b, (TV*)k.d, (const TV*)k.invd, (TV)k.c1,
                                         (TV)k.c2, dacc);
    }
  }
}

template <class TV, class TM, int MODE>
__global__ void __launch_bounds__(256, 5) bshort_k(const MTask* __restrict__ tasks,
                                                const int4* __restrict__ wbs, int nwb) {
  __shared__ MTask sk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int wb = blockIdx.x; wb < nwb; wb += gridDim.x) {
    SAAMG_WORK_BLOCK(MTask)
    for (int u = B.y + warp; u < B.z; u += kWarps) {
      const int row = u * 32 + lane;
      if (row < k.n)
        rows::csr_short_row<TV, TM, MODE>(row, k.rowptr, k.col, (const TM*)k.val,
                                          (const TV*)k.x, (TV*)k.y);
    }
  }
}

template <class TV, class TM, int MODE, bool REL>
__global__ void __launch_bounds__(256, 5) bsell_k(const MTask* __restrict__ tasks,
                                               const int4* __restrict__ wbs, int nwb) {
  __shared__ MTask sk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double dacc = 0.0;
  for (int wb = blockIdx.x; wb < nwb; wb += gridDim.x) {
    SAAMG_WORK_BLOCK(MTask)
    for (int u = B.y + warp; u < B.z; u += kWarps)
      rows::sell_row<TV, TM, MODE, REL>(u, lane, k.n, k.perm, k.soff, k.col, k.dcol,
                                        (const TM*)k.val, (const TV*)k.x, (TV*)k.y,
                                        (const TV*)k.b, (TV*)k.d, (const TV*)k.invd, (TV)k.c1,
                                        (TV)k.c2, dacc);
  }
}

template <class TV>
__global__ void __launch_bounds__(256, 5) bgemv_k(const MTask* __restrict__ tasks,
                                               const int4* __restrict__ wbs, int nwb) {
  __shared__ MTask sk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int wb = blockIdx.x; wb < nwb; wb += gridDim.x) {
    SAAMG_WORK_BLOCK(MTask)
    for (int u = B.y + warp; u < B.z; u += kWarps)
      rows::gemv_row<TV>(u, k.n, lane, (const double*)k.val, (const TV*)k.b, (TV*)k.y);
  }
}

template <class T>
__global__ void __launch_bounds__(256, 5) bcopy_k(const MTask* __restrict__ tasks,
                                               const int4* __restrict__ wbs, int nwb) {
  __shared__ MTask sk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int wb = blockIdx.x; wb < nwb; wb += gridDim.x) {
    SAAMG_WORK_BLOCK(MTask)
    for (int u = B.y + warp; u < B.z; u += kWarps) {
      const int i = u * 32 + lane;
      if (i < k.n) ((T*)k.y)[i] = ((const T*)k.x)[i];
    }
  }
}

// --- CG vector kernels ----------------------------------------------------------------------
// Every (task t, block b) pair computes block b of the one-solve grid (kRedBlocks blocks of
// kRedThreads) for task t, emulated by one warp (rows::*_block_warp), so each partial has the
// one-solve bits; warps take pairs in turn.  A pair past the vector's end only stores its
// partial, 0 (what the one-solve block sums).
#define SAAMG_WARP_PAIRS                                                          \
  const int lane = threadIdx.x & 31;                                              \
  const long long npairs = (long long)ntasks * kRedBlocks;                        \
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);              \
  for (long long pr = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;    \
       pr < npairs; pr += nwarps) {                                               \
    const VTask& k = tasks[pr / kRedBlocks];                                      \
    const int b = (int)(pr % kRedBlocks);                                         \
    if (!*k.go) continue;

template <class TZ>
__global__ void __launch_bounds__(256) bdot_rz_k(const VTask* __restrict__ tasks, int ntasks) {
  SAAMG_WARP_PAIRS
    if (b * kRedThreads >= k.n) {
      if (lane == 0) k.part0[b] = 0.0;
      continue;
    }
    const double t = rows::dot_block_warp<double, TZ>(b, k.n, k.r, (const TZ*)k.z, lane);
    if (lane == 0) k.part0[b] = t;
  }
}

template <class TZ>
__global__ void __launch_bounds__(256) bdot2_k(const VTask* __restrict__ tasks, int ntasks) {
  SAAMG_WARP_PAIRS
    if (b * kRedThreads >= k.n) {
      if (lane == 0) {
        k.part0[b] = 0.0;
        k.part2[b] = 0.0;
      }
      continue;
    }
    double t1, t2;
    rows::dot2_block_warp<TZ>(b, k.n, k.r, (const TZ*)k.z, k.q, lane, t1, t2);
    if (lane == 0) {
      k.part0[b] = t1;
      k.part2[b] = t2;
    }
  }
}

__global__ void __launch_bounds__(256) bupdate_k(const VTask* __restrict__ tasks, int ntasks) {
  SAAMG_WARP_PAIRS
    if (b * kRedThreads >= k.n) {
      if (lane == 0) k.part1[b] = 0.0;
      continue;
    }
    const double t =
        rows::update_block_warp(b, k.n, k.ctl->alpha, k.x, k.r, k.p, k.q, k.r32, lane);
    if (lane == 0) k.part1[b] = t;
  }
}

int resident_blocks(const void* kernel);

inline int grid_pairs(int ntasks, const void* kernel) {  // blocks of 8 warps, a warp per pair
  return (int)std::max<long long>(
      1, std::min<long long>(((long long)ntasks * kRedBlocks + 7) / 8,
                             (long long)sm_count() * resident_blocks(kernel)));
}

// p = z + beta p; a unit is 256 elements
template <class TZ>
__global__ void __launch_bounds__(256, 5) bdirection_k(const VTask* __restrict__ tasks,
                                                    const int4* __restrict__ wbs, int nwb) {
  for (int wb = blockIdx.x; wb < nwb; wb += gridDim.x) {
    const int4 B = wbs[wb];
    const VTask& k = tasks[B.x];
    if (!*k.go) continue;  // uniform across the block
    const double beta = k.ctl->beta;
    const TZ* z = (const TZ*)k.z;
    for (int u = B.y; u < B.z; ++u) {
      const int i = u * 256 + threadIdx.x;
      if (i < k.n) k.p[i] = (double)z[i] + beta * k.p[i];
    }
  }
}

// x = 0 where ||b|| = 0 (the prologue); a unit is 256 elements
__global__ void __launch_bounds__(256, 5) bzero_k(const VTask* __restrict__ tasks,
                                               const int4* __restrict__ wbs, int nwb) {
  for (int wb = blockIdx.x; wb < nwb; wb += gridDim.x) {
    const int4 B = wbs[wb];
    const VTask& k = tasks[B.x];
    if (k.ctl->bb != 0.0) continue;
    for (int u = B.y; u < B.z; ++u) {
      const int i = u * 256 + threadIdx.x;
      if (i < k.n) k.x[i] = 0.0;
    }
  }
}

// --- CG scalars: a block per task -------------------------------------------------------------
__global__ void __launch_bounds__(kRedThreads) binit_k(const VTask* __restrict__ tasks) {
  const VTask& k = tasks[blockIdx.x];
  PcgCtl* ctl = k.ctl;
  const double bb = rows::sum_fixed(k.part2);
  const double rr = rows::sum_fixed(k.part1);
  if (threadIdx.x == 0) {
    ctl->rtol = k.rtol;
    ctl->bb = bb;
    ctl->rr = rr;
    ctl->tol2 = (ctl->rtol * ctl->rtol) * bb;
    ctl->iters = 0;
    ctl->breakdown = !(isfinite(bb) && isfinite(rr));
    ctl->converged = (bb == 0.0) || rr <= ctl->tol2;
    ctl->rz = 0.0;
    ctl->alpha = 0.0;
    ctl->beta = 0.0;
    *k.go = !ctl->converged && !ctl->breakdown && k.maxit > 0;
  }
}

__global__ void __launch_bounds__(kRedThreads) bbeta_k(const VTask* __restrict__ tasks) {
  const VTask& k = tasks[blockIdx.x];
  if (!*k.go) return;
  PcgCtl* ctl = k.ctl;
  const double rz = rows::sum_fixed(k.part0);
  const double zq = k.rule == 1 ? rows::sum_fixed(k.part2) : 0.0;
  if (threadIdx.x == 0) {
    double b = 0.0;
    if (ctl->iters > 0) b = (k.rule == 1) ? (-ctl->alpha * zq) / ctl->rz : rz / ctl->rz;
    if (!isfinite(b) || !isfinite(rz)) {
      ctl->breakdown = 1;
      b = 0.0;
    }
    ctl->rz_new = rz;
    ctl->zq = zq;
    ctl->beta = b;
    ctl->rz = rz;
  }
}

__global__ void __launch_bounds__(kRedThreads) balpha_k(const VTask* __restrict__ tasks) {
  const VTask& k = tasks[blockIdx.x];
  if (!*k.go) return;
  PcgCtl* ctl = k.ctl;
  const double pq = rows::sum_fixed(k.part0);
  if (threadIdx.x == 0) {
    ctl->pq = pq;
    double a = ctl->rz / pq;
    if (!(pq != 0.0) || !isfinite(a)) {
      ctl->breakdown = 1;
      a = 0.0;
    }
    ctl->alpha = a;
  }
}

__global__ void __launch_bounds__(kRedThreads) bcheck_k(const VTask* __restrict__ tasks) {
  const VTask& k = tasks[blockIdx.x];
  if (!*k.go) return;
  PcgCtl* ctl = k.ctl;
  const double rr = rows::sum_fixed(k.part1);
  if (threadIdx.x == 0) {
    ctl->rr = rr;
    ctl->iters += 1;
    if (!isfinite(rr)) ctl->breakdown = 1;
    ctl->converged = rr <= ctl->tol2;
    *k.go = !ctl->converged && !ctl->breakdown && ctl->iters < k.maxit;
  }
}

// The loop goes on while any solve goes on.
__global__ void bany_k(const int* __restrict__ go, int count, cudaGraphConditionalHandle cond) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int mine = 0;
  for (int j = threadIdx.x; j < count; j += blockDim.x) mine |= go[j];
  if (mine) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(cond, any ? 1u : 0u);
}

// --- operation keys -------------------------------------------------------------------------
enum Family { F_ST32, F_ST64, F_CSR, F_SHORT, F_SELL, F_GEMV, F_COPY };
// value types: TV 0 double / 1 float; TM 0 double / 1 float / 2 bf16
struct Key {
  int fam = 0, tv = 0, tm = 0, g = 0, mode = 0, rel = 0;
  bool operator<(const Key& o) const {
    return std::tie(fam, tv, tm, g, mode, rel) < std::tie(o.fam, o.tv, o.tm, o.g, o.mode, o.rel);
  }
  bool operator==(const Key& o) const {
    return !(*this < o) && !(o < *this);
  }
};

// Blocks of 256 threads of `kernel` that are resident on one SM at a time (cached).
int resident_blocks(const void* kernel) {
  static std::mutex mu;
  static std::map<const void*, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(kernel);
  if (it != cache.end()) return it->second;
  int nb = 0;
  SAAMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, 256, 0));
  nb = std::max(nb, 1);
  cache[kernel] = nb;
  return nb;
}

// A grid of work-block kernels: one wave of resident blocks, each taking work blocks in turn
// (a second, partial wave would start late and finish last).
inline int grid_wb(int nwb, const void* kernel) {
  return std::max(1, std::min(nwb, sm_count() * resident_blocks(kernel)));
}

#define SAAMG_WB_LAUNCH(KERNEL)                                                        \
  KERNEL<<<grid_wb(nwb, reinterpret_cast<const void*>(KERNEL)), 256, 0, s>>>(t, wbs, nwb)

template <class TV, class TM, int G>
void launch_csr_g(int mode, const MTask* t, const int4* wbs, int nwb, cudaStream_t s) {
  switch (mode) {
    case CSR_SPMV: SAAMG_WB_LAUNCH((bcsr_k<TV, TM, G, CSR_SPMV>)); break;
    case CSR_RESID: SAAMG_WB_LAUNCH((bcsr_k<TV, TM, G, CSR_RESID>)); break;
    case CSR_CHEB: SAAMG_WB_LAUNCH((bcsr_k<TV, TM, G, CSR_CHEB>)); break;
    case CSR_CHEB0: SAAMG_WB_LAUNCH((bcsr_k<TV, TM, G, CSR_CHEB0>)); break;
    case CSR_ADD: SAAMG_WB_LAUNCH((bcsr_k<TV, TM, G, CSR_ADD>)); break;
    default: fail(SAAMG_EINVAL, "batched CSR mode");
  }
  SAAMG_LAUNCH();
}

template <class TV, class TM>
void launch_csr(int g, int mode, const MTask* t, const int4* wbs, int nwb, cudaStream_t s) {
  switch (g) {
    case 2: launch_csr_g<TV, TM, 2>(mode, t, wbs, nwb, s); break;
    case 4: launch_csr_g<TV, TM, 4>(mode, t, wbs, nwb, s); break;
    case 8: launch_csr_g<TV, TM, 8>(mode, t, wbs, nwb, s); break;
    case 16: launch_csr_g<TV, TM, 16>(mode, t, wbs, nwb, s); break;
    default: launch_csr_g<TV, TM, 32>(mode, t, wbs, nwb, s); break;
  }
}

template <class TV, class TM, bool REL>
void launch_sell_r(int mode, const MTask* t, const int4* wbs, int nwb, cudaStream_t s) {
  switch (mode) {
    case CSR_RESID: SAAMG_WB_LAUNCH((bsell_k<TV, TM, CSR_RESID, REL>)); break;
    case CSR_CHEB: SAAMG_WB_LAUNCH((bsell_k<TV, TM, CSR_CHEB, REL>)); break;
    case CSR_CHEB0: SAAMG_WB_LAUNCH((bsell_k<TV, TM, CSR_CHEB0, REL>)); break;
    case rows::kSellCheb1: SAAMG_WB_LAUNCH((bsell_k<TV, TM, rows::kSellCheb1, REL>)); break;
    default: fail(SAAMG_EINVAL, "batched SELL mode");
  }
  SAAMG_LAUNCH();
}

template <class TV, class TM>
void launch_sell(int rel, int mode, const MTask* t, const int4* wbs, int nwb, cudaStream_t s) {
  if (rel) launch_sell_r<TV, TM, true>(mode, t, wbs, nwb, s);
  else launch_sell_r<TV, TM, false>(mode, t, wbs, nwb, s);
}

template <class TV, class TM>
void launch_short(int mode, const MTask* t, const int4* wbs, int nwb, cudaStream_t s) {
  if (mode == CSR_ADD) SAAMG_WB_LAUNCH((bshort_k<TV, TM, CSR_ADD>));
  else SAAMG_WB_LAUNCH((bshort_k<TV, TM, CSR_SPMV>));
  SAAMG_LAUNCH();
}

// One merged group: a launch of the family and form of `k` over its work blocks.
void launch_group(const Key& k, const void* tasks, const int4* wbs, int nwb, cudaStream_t s) {
  if (nwb <= 0) return;
  const MTask* mt = static_cast<const MTask*>(tasks);
  switch (k.fam) {
    case F_ST32:
      batched_stencil<float>(k.mode, static_cast<const StTask<float>*>(tasks), wbs, nwb, s);
      return;
    case F_ST64:
      batched_stencil<double>(k.mode, static_cast<const StTask<double>*>(tasks), wbs, nwb, s);
      return;
    case F_CSR:
      if (k.tv == 0) launch_csr<double, double>(k.g, k.mode, mt, wbs, nwb, s);
      else if (k.tm == 1) launch_csr<float, float>(k.g, k.mode, mt, wbs, nwb, s);
      else launch_csr<float, __nv_bfloat16>(k.g, k.mode, mt, wbs, nwb, s);
      return;
    case F_SHORT:
      if (k.tv == 0) launch_short<double, double>(k.mode, mt, wbs, nwb, s);
      else launch_short<float, float>(k.mode, mt, wbs, nwb, s);
      return;
    case F_SELL:
      if (k.tv == 0) launch_sell<double, double>(k.rel, k.mode, mt, wbs, nwb, s);
      else if (k.tm == 1) launch_sell<float, float>(k.rel, k.mode, mt, wbs, nwb, s);
      else launch_sell<float, __nv_bfloat16>(k.rel, k.mode, mt, wbs, nwb, s);
      return;
    case F_GEMV: {
      const MTask* t = mt;
      if (k.tv == 0) SAAMG_WB_LAUNCH(bgemv_k<double>);
      else SAAMG_WB_LAUNCH(bgemv_k<float>);
      SAAMG_LAUNCH();
      return;
    }
    default: {
      const MTask* t = mt;
      if (k.tv == 0) SAAMG_WB_LAUNCH(bcopy_k<double>);
      else SAAMG_WB_LAUNCH(bcopy_k<float>);
      SAAMG_LAUNCH();
      return;
    }
  }
}

// Work blocks of a launch: each task's units cut into blocks of `per` units.
void work_blocks(const std::vector<int>& units, int per, std::vector<int4>& out) {
  for (size_t t = 0; t < units.size(); ++t)
    for (int u = 0; u < units[t]; u += per)
      out.push_back(make_int4((int)t, u, std::min(units[t], u + per), 0));
}

// --- planning ---------------------------------------------------------------------------------
enum Phase { P_PRE = 0, P_RESID, P_RESTRICT, P_COARSE, P_PROLONG, P_POST, P_COPY };

struct Op {
  int phase, level, step;
  Key key;
  int units;
  MTask m;
  StTask<float> sf;
  StTask<double> sd;
};

// Work vectors of one solve (every level of its V-cycle and the CG vectors).
struct SolveWork {
  saamg_hierarchy* h = nullptr;
  Buf<double> bhat, xhat, r, z, p, q;
  Buf<float> z32, r32;
  Buf<double> part0, part1, part2;
  Buf<PcgCtl> ctl;
  std::vector<Buf<double>> dx0, dx1, db, dd, dr;
  std::vector<Buf<float>> fx0, fx1, fb, fd, fr;
};

template <class T>
struct WV;
template <>
struct WV<double> {
  static double* x0(SolveWork& w, int l) { return w.dx0[l].p; }
  static double* x1(SolveWork& w, int l) { return w.dx1[l].p; }
  static double* b(SolveWork& w, int l) { return w.db[l].p; }
  static double* d(SolveWork& w, int l) { return w.dd[l].p; }
  static double* r(SolveWork& w, int l) { return w.dr[l].p; }
};
template <>
struct WV<float> {
  static float* x0(SolveWork& w, int l) { return w.fx0[l].p; }
  static float* x1(SolveWork& w, int l) { return w.fx1[l].p; }
  static float* b(SolveWork& w, int l) { return w.fb[l].p; }
  static float* d(SolveWork& w, int l) { return w.fd[l].p; }
  static float* r(SolveWork& w, int l) { return w.fr[l].p; }
};

struct Planner {
  std::vector<Op>& ops;
  const int* go;
  SolveWork& w;

  bool fp32() const { return w.h->prm.precision == SAAMG_PREC_FP32; }

  void add(Op o) { ops.push_back(o); }

  Op base(int phase, int level, int step) {
    Op o{};
    o.phase = phase;
    o.level = level;
    o.step = step;
    o.m.go = go;
    o.sf.go = go;
    o.sd.go = go;
    return o;
  }

  // smooth_step of the one-solve V-cycle
  template <class T>
  void smooth(int phase, int l, int step, int mode0, const T* x, T* y, const T* b, T* d, T c1,
              T c2) {
    saamg_hierarchy* h = w.h;
    Op o = base(phase, l, step);
    if (l == 0) {
      StencilDev<T> S = h->op->d.template view<T>();
      const int m = mode0 == CSR_CHEB0   ? ST_CHEB0
                    : mode0 == CSR_RESID ? ST_RESID
                    : (c1 == T(0))       ? ST_CHEB1
                                         : ST_CHEB;
      StTask<T> t{};
      t.S = S;
      t.go = go;
      t.x = x;
      t.y = y;
      t.b = b;
      t.d = d;
      t.c1 = c1;
      t.c2 = c2;
      t.c2i0 = c2 * S.invd0;
      t.agg = nullptr;
      t.part = nullptr;
      o.key.fam = sizeof(T) == 4 ? F_ST32 : F_ST64;
      o.key.mode = m;
      o.units = stencil_units<T>(S);
      set_st(o, t);
      add(o);
      return;
    }
    Level& L = *h->lev[l];
    const bool dbl = sizeof(T) == 8;
    o.key.tv = dbl ? 0 : 1;
    o.key.tm = dbl ? 0 : (fp32() ? 1 : 2);
    o.m.x = x;
    o.m.y = y;
    o.m.b = b;
    o.m.d = d;
    o.m.c1 = (double)c1;
    o.m.c2 = (double)c2;
    if (L.As.n > 0) {
      o.key.fam = F_SELL;
      o.key.mode = (mode0 == CSR_CHEB && c1 == T(0)) ? rows::kSellCheb1 : mode0;
      o.key.rel = L.As.index_bytes == 2;
      o.m.n = L.As.n;
      o.m.nslices = L.As.nslices;
      o.m.perm = L.As.perm.p;
      o.m.soff = L.As.soff.p;
      o.m.col = L.As.col.p;
      o.m.dcol = L.As.dcol.p;
      o.m.val = dbl ? (const void*)L.As.val.p
                    : (fp32() ? (const void*)L.As.val32.p : (const void*)L.As.val16.p);
      o.m.invd = dbl ? (const void*)L.invd.p : (const void*)L.invd32.p;
      o.units = L.As.nslices;
    } else {
      const int g = csr_plan(mode0, L.n, L.avg, dbl);
      o.key.fam = F_CSR;
      o.key.mode = mode0;
      o.key.g = g;
      o.m.n = L.n;
      o.m.rowptr = L.A.rowptr.p;
      o.m.col = L.A.col.p;
      o.m.val = dbl ? (const void*)L.A.val.p
                    : (fp32() ? (const void*)L.A.val32.p : (const void*)L.A.val16.p);
      o.m.invd = dbl ? (const void*)L.invd.p : (const void*)L.invd32.p;
      o.units = (L.n + 32 / g - 1) / (32 / g);
    }
    add(o);
  }

  void set_st(Op& o, const StTask<float>& t) { o.sf = t; }
  void set_st(Op& o, const StTask<double>& t) { o.sd = t; }

  // transfer of the one-solve V-cycle
  template <class T>
  void transfer(int phase, int l, bool restrict_, const T* x, T* y) {
    saamg_hierarchy* h = w.h;
    Level& L = *h->lev[l];
    Op o = base(phase, l, 0);
    const bool dbl = sizeof(T) == 8;
    if (!dbl && l == 0 && !restrict_) {  // matrix-free level-0 prolongation (FP32)
      StencilDev<T> S = h->op->d.template view<T>();
      const T omega = (T)L.omega;
      StTask<T> t{};
      t.S = S;
      t.go = go;
      t.x = x;
      t.y = y;
      t.c1 = T(0);
      t.c2 = omega;
      t.c2i0 = T(omega * S.invd0);
      t.agg = L.agg.p;
      o.key.fam = F_ST32;
      o.key.mode = ST_PROLONG;
      o.units = stencil_units<T>(S);
      set_st(o, t);
      add(o);
      return;
    }
    const DevCsr& M = restrict_ ? L.R : L.P;
    if (M.n == 0) return;
    const int mode = restrict_ ? CSR_SPMV : CSR_ADD;
    const double avg = M.n ? (double)M.nnz / M.n : 0.0;
    const int g = csr_plan(mode, M.n, avg, dbl);
    o.key.tv = dbl ? 0 : 1;
    o.key.tm = dbl ? 0 : 1;
    o.key.mode = mode;
    o.m.n = M.n;
    o.m.rowptr = M.rowptr.p;
    o.m.col = M.col.p;
    o.m.val = dbl ? (const void*)M.val.p : (const void*)(restrict_ ? L.R32.p : L.P32.p);
    o.m.x = x;
    o.m.y = y;
    if (g == 0) {
      o.key.fam = F_SHORT;
      o.units = (M.n + 31) / 32;
    } else {
      o.key.fam = F_CSR;
      o.key.g = g;
      o.units = (M.n + 32 / g - 1) / (32 / g);
    }
    add(o);
  }

  // vcycle_level of the one-solve V-cycle
  template <class T>
  void vcycle(int l, const T* b, T* out) {
    saamg_hierarchy* h = w.h;
    const int nl = (int)h->lev.size();
    Level& L = *h->lev[l];
    if (l == nl - 1) {
      Op o = base(P_COARSE, l, 0);
      o.key.fam = F_GEMV;
      o.key.tv = sizeof(T) == 8 ? 0 : 1;
      o.m.n = h->coarse.n;
      o.m.val = h->coarse.inv.p;
      o.m.b = b;
      o.m.y = out;
      o.units = h->coarse.n;
      add(o);
      return;
    }
    const int nu = (int)L.cheb.c1.size();
    T* bufs[2] = {WV<T>::x0(w, l), out};
    T* d = WV<T>::d(w, l);
    int cur = 0;
    smooth<T>(P_PRE, l, 0, CSR_CHEB0, nullptr, bufs[cur], b, d, T(0), (T)L.cheb.c2[0]);
    for (int k = 1; k < nu; ++k) {
      smooth<T>(P_PRE, l, k, CSR_CHEB, bufs[cur], bufs[1 - cur], b, d, (T)L.cheb.c1[k],
                (T)L.cheb.c2[k]);
      cur = 1 - cur;
    }
    T* r = WV<T>::r(w, l);
    smooth<T>(P_RESID, l, 0, CSR_RESID, bufs[cur], r, b, nullptr, T(0), T(0));
    T* bc = WV<T>::b(w, l + 1);
    T* vc = (l + 1 == nl - 1) ? WV<T>::x0(w, l + 1) : WV<T>::x1(w, l + 1);
    transfer<T>(P_RESTRICT, l, true, r, bc);
    vcycle<T>(l + 1, bc, vc);
    transfer<T>(P_PROLONG, l, false, vc, bufs[cur]);
    for (int k = 0; k < nu; ++k) {
      smooth<T>(P_POST, l, k, CSR_CHEB, bufs[cur], bufs[1 - cur], b, d, (T)L.cheb.c1[k],
                (T)L.cheb.c2[k]);
      cur = 1 - cur;
    }
    if (bufs[cur] != out) {
      Op o = base(P_COPY, l, 0);
      o.key.fam = F_COPY;
      o.key.tv = sizeof(T) == 8 ? 0 : 1;
      o.m.n = L.n;
      o.m.x = bufs[cur];
      o.m.y = out;
      o.units = (L.n + 31) / 32;
      add(o);
    }
  }
};

// A merged launch: tasks and offsets in device memory.
struct Group {
  Key key;
  int ntasks = 0, nwb = 0;
  size_t task_off = 0;  // byte offset of the task array in the task buffer
  size_t wb_off = 0;    // byte offset of the work blocks in the task buffer
};

}  // namespace

// A lane: a sub-batch with its own loop (the lanes of a batch run side by side in one graph,
// so that one lane's short, latency-bound launches overlap another's).
struct Lane {
  std::vector<int> sol;       // global indices of its solves
  Buf<int> go;                // loop flags, one per solve of the lane
  Buf<unsigned char> tasks;   // every task table and work-block list of the loop body
  Buf<VTask> vtasks;
  std::vector<Group> groups;            // the V-cycle launches, in order
  std::vector<std::vector<int>> vsets;  // CG task subsets by (V-cycle type, rule): lane indices
  std::vector<Buf<VTask>> vsub;
  std::vector<int> vsub_kind;  // 0: FP64, rule 0 / 1: FP64, rule 1 / 2: mixed, rule 0 / 3: mixed, rule 1
  Buf<int4> vsub_off;          // per subset: work blocks of 256-element units (direction)
  std::vector<int> vsub_units; // work blocks of each subset
  std::vector<size_t> vsub_offpos;  // first work block of each subset
  Buf<int4> vall_off;          // all solves of the lane: work blocks (zero)
  int vall_units = 0;
  Buf<StTask<double>> dot_tasks;  // A p with p'Ap partials
  long long k_body = 0;
};

struct BatchEngine {
  std::vector<std::unique_ptr<SolveWork>> work;
  std::vector<std::unique_ptr<Lane>> lanes;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  PcgCtl* res = nullptr;  // pinned host copies of every solve's scalars after a run
  long long k_fixed = 0;
  ~BatchEngine() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (res) cudaFreeHost(res);
  }
};

bool batch_engine_supports(saamg_hierarchy* const* hs, int count) {
  if (count < 2) return false;
  for (int j = 0; j < count; ++j) {
    const saamg_hierarchy* h = hs[j];
    if (h->op->d.n == 0 || h->prm.coarse_solver != SAAMG_COARSE_LU || h->lev.size() < 1)
      return false;
  }
  return true;
}

namespace {

void alloc_work(SolveWork& w, cudaStream_t s) {
  saamg_hierarchy* h = w.h;
  const int n = h->op->d.n;
  const bool mx = h->prm.precision != SAAMG_PREC_FP64;
  w.bhat.alloc(n, s);
  w.xhat.alloc(n, s);
  w.r.alloc(n, s);
  w.p.alloc(n, s);
  w.q.alloc(n, s);
  if (mx) {
    w.z32.alloc(n, s);
    w.r32.alloc(n, s);
  } else {
    w.z.alloc(n, s);
  }
  w.part0.alloc(kRedBlocks, s);
  w.part1.alloc(kRedBlocks, s);
  w.part2.alloc(kRedBlocks, s);
  w.ctl.alloc(1, s);
  const int nl = (int)h->lev.size();
  if (mx) {
    w.fx0.resize(nl);
    w.fx1.resize(nl);
    w.fb.resize(nl);
    w.fd.resize(nl);
    w.fr.resize(nl);
  } else {
    w.dx0.resize(nl);
    w.dx1.resize(nl);
    w.db.resize(nl);
    w.dd.resize(nl);
    w.dr.resize(nl);
  }
  for (int l = 0; l < nl; ++l) {
    const int m = h->lev[l]->n;
    if (mx) {
      w.fx0[l].alloc(m, s);
      w.fx1[l].alloc(m, s);
      w.fb[l].alloc(m, s);
      w.fd[l].alloc(m, s);
      w.fr[l].alloc(m, s);
    } else {
      w.dx0[l].alloc(m, s);
      w.dx1[l].alloc(m, s);
      w.db[l].alloc(m, s);
      w.dd[l].alloc(m, s);
      w.dr[l].alloc(m, s);
    }
  }
}

// Slot of an operation in the merged cycle: the down-going phases level by level, then the
// up-going ones from the second-coarsest level up; inside a level the order of the one-solve
// V-cycle.
long long slot_of(const Op& o, int lmax, int numax) {
  const int down = numax + 3;  // PRE 0..numax-1, RESID, RESTRICT, COARSE
  const int up = numax + 2;    // PROLONG, POST 0..numax-1, COPY
  switch (o.phase) {
    case P_PRE: return (long long)o.level * down + o.step;
    case P_RESID: return (long long)o.level * down + numax;
    case P_RESTRICT: return (long long)o.level * down + numax + 1;
    case P_COARSE: return (long long)o.level * down + numax + 2;
    case P_PROLONG: return (long long)lmax * down + (long long)(lmax - 1 - o.level) * up;
    case P_POST: return (long long)lmax * down + (long long)(lmax - 1 - o.level) * up + 1 + o.step;
    default: return (long long)lmax * down + (long long)(lmax - 1 - o.level) * up + 1 + numax;
  }
}

}  // namespace

namespace {

// Plans the lane's V-cycles, merges their operations and uploads every task table.
void build_lane(Lane& L, std::vector<std::unique_ptr<SolveWork>>& work, double rtol,
                cudaStream_t s) {
  const int m = (int)L.sol.size();
  L.go.alloc(m, s);
  std::vector<Op> ops;
  int lmax = 0, numax = 0;
  for (int i = 0; i < m; ++i) {
    SolveWork& w = *work[L.sol[i]];
    saamg_hierarchy* h = w.h;
    lmax = std::max(lmax, (int)h->lev.size());
    for (size_t l = 0; l + 1 < h->lev.size(); ++l)
      numax = std::max(numax, (int)h->lev[l]->cheb.c1.size());
    Planner pl{ops, L.go.p + i, w};
    if (h->prm.precision != SAAMG_PREC_FP64) pl.vcycle<float>(0, w.r32.p, w.z32.p);
    else pl.vcycle<double>(0, w.r.p, w.z.p);
  }
  // stable order: slot, then kernel form, then solve (ops of one solve keep their order)
  std::vector<int> idx(ops.size());
  for (size_t i = 0; i < ops.size(); ++i) idx[i] = (int)i;
  std::vector<long long> slot(ops.size());
  for (size_t i = 0; i < ops.size(); ++i) slot[i] = slot_of(ops[i], lmax, numax);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
    if (slot[a] != slot[b]) return slot[a] < slot[b];
    return ops[a].key < ops[b].key;
  });
  // task buffer layout: per group its task array (aligned) and its work blocks
  std::vector<unsigned char> host;
  auto align = [&](size_t a) {
    while (host.size() % a) host.push_back(0);
  };
  auto append = [&](const void* p, size_t b) {
    const unsigned char* q = static_cast<const unsigned char*>(p);
    host.insert(host.end(), q, q + b);
  };
  for (size_t i = 0; i < idx.size();) {
    size_t k = i;
    const Op& first = ops[idx[i]];
    while (k < idx.size() && slot[idx[k]] == slot[idx[i]] && ops[idx[k]].key == first.key) ++k;
    Group g;
    g.key = first.key;
    g.ntasks = (int)(k - i);
    align(64);
    g.task_off = host.size();
    std::vector<int> units;
    for (size_t q = i; q < k; ++q) {
      const Op& o = ops[idx[q]];
      if (o.key.fam == F_ST32) append(&o.sf, sizeof(o.sf));
      else if (o.key.fam == F_ST64) append(&o.sd, sizeof(o.sd));
      else append(&o.m, sizeof(o.m));
      units.push_back(o.units);
    }
    std::vector<int4> wb;
    work_blocks(units, kWarps * kWarpUnits, wb);
    g.nwb = (int)wb.size();
    align(16);
    g.wb_off = host.size();
    append(wb.data(), wb.size() * sizeof(int4));
    L.groups.push_back(g);
    i = k;
  }
  L.tasks.alloc(std::max<size_t>(host.size(), 1), s);
  if (!host.empty())
    SAAMG_CUDA(cudaMemcpyAsync(L.tasks.p, host.data(), host.size(), cudaMemcpyHostToDevice, s));
  // --- CG tasks
  std::vector<VTask> vt(m);
  for (int i = 0; i < m; ++i) {
    SolveWork& w = *work[L.sol[i]];
    saamg_hierarchy* h = w.h;
    const bool mx = h->prm.precision != SAAMG_PREC_FP64;
    VTask& t = vt[i];
    t.go = L.go.p + i;
    t.n = h->op->d.n;
    t.ctl = w.ctl.p;
    t.x = w.xhat.p;
    t.r = w.r.p;
    t.p = w.p.p;
    t.q = w.q.p;
    t.z = mx ? (const void*)w.z32.p : (const void*)w.z.p;
    t.r32 = mx ? w.r32.p : nullptr;
    t.part0 = w.part0.p;
    t.part1 = w.part1.p;
    t.part2 = w.part2.p;
    t.rule = h->prm.beta_rule;
    t.maxit = h->prm.maxit;
    t.rtol = rtol;
  }
  L.vtasks.alloc(m, s);
  SAAMG_CUDA(cudaMemcpyAsync(L.vtasks.p, vt.data(), sizeof(VTask) * m, cudaMemcpyHostToDevice, s));
  // subsets by V-cycle type and beta rule (different kernels)
  L.vsets.assign(4, {});
  for (int i = 0; i < m; ++i) {
    const bool mx = work[L.sol[i]]->h->prm.precision != SAAMG_PREC_FP64;
    L.vsets[(mx ? 2 : 0) + (vt[i].rule == 1 ? 1 : 0)].push_back(i);
  }
  std::vector<int4> wbs;
  for (int k = 0; k < 4; ++k) {
    if (L.vsets[k].empty()) continue;
    std::vector<VTask> sub;
    std::vector<int> units;
    for (int i : L.vsets[k]) {
      sub.push_back(vt[i]);
      units.push_back((vt[i].n + 255) / 256);
    }
    L.vsub_offpos.push_back(wbs.size());
    const size_t before = wbs.size();
    work_blocks(units, kBlockUnits, wbs);
    L.vsub_units.push_back((int)(wbs.size() - before));
    L.vsub_kind.push_back(k);
    L.vsub.emplace_back();
    L.vsub.back().alloc(sub.size(), s);
    SAAMG_CUDA(cudaMemcpyAsync(L.vsub.back().p, sub.data(), sizeof(VTask) * sub.size(),
                               cudaMemcpyHostToDevice, s));
  }
  L.vsub_off.alloc(std::max<size_t>(wbs.size(), 1), s);
  if (!wbs.empty())
    SAAMG_CUDA(cudaMemcpyAsync(L.vsub_off.p, wbs.data(), sizeof(int4) * wbs.size(),
                               cudaMemcpyHostToDevice, s));
  {
    std::vector<int> units;
    for (int i = 0; i < m; ++i) units.push_back((vt[i].n + 255) / 256);
    std::vector<int4> all;
    work_blocks(units, kBlockUnits, all);
    L.vall_units = (int)all.size();
    L.vall_off.alloc(std::max<size_t>(all.size(), 1), s);
    SAAMG_CUDA(cudaMemcpyAsync(L.vall_off.p, all.data(), sizeof(int4) * all.size(),
                               cudaMemcpyHostToDevice, s));
  }
  {
    std::vector<StTask<double>> dt(m);
    for (int i = 0; i < m; ++i) {
      SolveWork& w = *work[L.sol[i]];
      StTask<double> t{};
      t.S = w.h->op->d.view<double>();
      t.go = L.go.p + i;
      t.x = w.p.p;
      t.y = w.q.p;
      t.part = w.part0.p;
      dt[i] = t;
    }
    L.dot_tasks.alloc(m, s);
    SAAMG_CUDA(cudaMemcpyAsync(L.dot_tasks.p, dt.data(), sizeof(StTask<double>) * m,
                               cudaMemcpyHostToDevice, s));
  }
}

// One pass of the lane's loop body on stream s.
void lane_body(Lane& L, cudaGraphConditionalHandle cond, cudaStream_t s) {
  const int m = (int)L.sol.size();
  for (const Group& gr : L.groups)
    launch_group(gr.key, L.tasks.p + gr.task_off,
                 reinterpret_cast<const int4*>(L.tasks.p + gr.wb_off), gr.nwb, s);
  for (size_t q = 0; q < L.vsub.size(); ++q) {
    const int kind = L.vsub_kind[q];
    const int nt = (int)L.vsets[kind].size();
    const VTask* t = L.vsub[q].p;
    if (kind == 0)
      bdot_rz_k<double><<<grid_pairs(nt, reinterpret_cast<const void*>(bdot_rz_k<double>)), 256, 0,
                          s>>>(t, nt);
    else if (kind == 1)
      bdot2_k<double><<<grid_pairs(nt, reinterpret_cast<const void*>(bdot2_k<double>)), 256, 0,
                        s>>>(t, nt);
    else if (kind == 2)
      bdot_rz_k<float><<<grid_pairs(nt, reinterpret_cast<const void*>(bdot_rz_k<float>)), 256, 0,
                         s>>>(t, nt);
    else
      bdot2_k<float><<<grid_pairs(nt, reinterpret_cast<const void*>(bdot2_k<float>)), 256, 0,
                       s>>>(t, nt);
    SAAMG_LAUNCH();
  }
  bbeta_k<<<m, kRedThreads, 0, s>>>(L.vtasks.p);
  SAAMG_LAUNCH();
  for (size_t q = 0; q < L.vsub.size(); ++q) {
    const int kind = L.vsub_kind[q];
    const int4* wb = L.vsub_off.p + L.vsub_offpos[q];
    const int nwb = L.vsub_units[q];
    if (kind < 2)
      bdirection_k<double><<<grid_wb(nwb, reinterpret_cast<const void*>(bdirection_k<double>)),
                             256, 0, s>>>(L.vsub[q].p, wb, nwb);
    else
      bdirection_k<float><<<grid_wb(nwb, reinterpret_cast<const void*>(bdirection_k<float>)),
                            256, 0, s>>>(L.vsub[q].p, wb, nwb);
    SAAMG_LAUNCH();
  }
  batched_stencil_dot(L.dot_tasks.p, m, s);
  balpha_k<<<m, kRedThreads, 0, s>>>(L.vtasks.p);
  SAAMG_LAUNCH();
  bupdate_k<<<grid_pairs(m, reinterpret_cast<const void*>(bupdate_k)), 256, 0, s>>>(L.vtasks.p, m);
  SAAMG_LAUNCH();
  bcheck_k<<<m, kRedThreads, 0, s>>>(L.vtasks.p);
  SAAMG_LAUNCH();
  bany_k<<<1, 256, 0, s>>>(L.go.p, m, cond);
  SAAMG_LAUNCH();
}

// Lanes of a batch: about 32 solves each, at most 8, sizes balanced (largest first onto the
// lightest lane).
std::vector<std::vector<int>> make_lanes(saamg_hierarchy* const* hs, int count, int nlanes) {
  std::vector<int> order(count);
  for (int j = 0; j < count; ++j) order[j] = j;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return hs[a]->op->d.n > hs[b]->op->d.n;
  });
  std::vector<std::vector<int>> lanes(nlanes);
  std::vector<long long> load(nlanes, 0);
  for (int j : order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    lanes[l].push_back(j);
    load[l] += hs[j]->op->d.n;
  }
  for (auto& l : lanes) std::sort(l.begin(), l.end());
  lanes.erase(std::remove_if(lanes.begin(), lanes.end(), [](const std::vector<int>& l) { return l.empty(); }),
              lanes.end());
  return lanes;
}

}  // namespace

BatchEngine* batch_engine_build(saamg_hierarchy* const* hs, const double* const* rho,
                                double* const* phi, int count, double rtol,
                                cudaStream_t (*stream_of)(int)) {
  std::unique_ptr<BatchEngine> e(new BatchEngine());
  cudaStream_t cs = stream_of(0);
  cudaStream_t s = cs;
  for (int j = 0; j < count; ++j) {
    e->work.emplace_back(new SolveWork());
    e->work[j]->h = hs[j];
    alloc_work(*e->work[j], s);
  }
  const int nlanes = std::max(1, std::min(kMaxLanes, (count + kLaneSolves - 1) / kLaneSolves));
  for (auto& sol : make_lanes(hs, count, nlanes)) {
    e->lanes.emplace_back(new Lane());
    e->lanes.back()->sol = sol;
    build_lane(*e->lanes.back(), e->work, rtol, s);
  }
  SAAMG_CUDA(cudaStreamSynchronize(s));
  SAAMG_CUDA(cudaMallocHost(&e->res, sizeof(PcgCtl) * count));

  // --- capture: per lane a prologue, a while node (one pass over the lane's solves) and an
  // epilogue, the lanes forked from one stream and joined back
  cudaGraph_t g = nullptr;
  SAAMG_CUDA(cudaGraphCreate(&g, 0));
  bool capturing = false;
  cudaStream_t body_cap = nullptr;
  std::vector<cudaEvent_t> evs;
  try {
    std::vector<cudaGraphConditionalHandle> conds(e->lanes.size());
    for (auto& c : conds)
      SAAMG_CUDA(cudaGraphConditionalHandleCreate(&c, g, 0, cudaGraphCondAssignDefault));
    SAAMG_CUDA(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    capturing = true;
    CaptureCount counting;
    const long long k0 = captured();
    cudaEvent_t fork;
    SAAMG_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    evs.push_back(fork);
    SAAMG_CUDA(cudaEventRecord(fork, cs));
    std::vector<cudaGraph_t> bodies(e->lanes.size());
    for (size_t li = 0; li < e->lanes.size(); ++li) {
      Lane& L = *e->lanes[li];
      cudaStream_t ls = stream_of(2 + 2 * (int)li);
      SAAMG_CUDA(cudaStreamWaitEvent(ls, fork, 0));
      const int m = (int)L.sol.size();
      // prologue of every solve (the one-solve graph's prologue, per solve)
      for (int j : L.sol) {
        SolveWork& w = *e->work[j];
        saamg_hierarchy* h = hs[j];
        const OperatorData& od = h->op->d;
        const int n = od.n;
        const StencilDev<double> S = od.view<double>();
        gather_rhs(od, rho[j], phi[j], w.bhat.p, w.xhat.p, ls);
        dot_partials<double, double>(n, w.bhat.p, w.bhat.p, w.part2.p, ls);
        stencil_apply<double>(S, ST_RESID, w.xhat.p, w.r.p, w.bhat.p, nullptr, 0.0, 0.0, nullptr, ls);
        if (h->prm.precision != SAAMG_PREC_FP64) to_float(w.r.p, w.r32.p, n, ls);
        dot_partials<double, double>(n, w.r.p, w.r.p, w.part1.p, ls);
        SAAMG_CUDA(cudaMemsetAsync(w.p.p, 0, sizeof(double) * n, ls));
      }
      binit_k<<<m, kRedThreads, 0, ls>>>(L.vtasks.p);
      SAAMG_LAUNCH();
      bzero_k<<<grid_wb(L.vall_units, reinterpret_cast<const void*>(bzero_k)), 256, 0, ls>>>(
          L.vtasks.p, L.vall_off.p, L.vall_units);
      SAAMG_LAUNCH();
      bany_k<<<1, 256, 0, ls>>>(L.go.p, m, conds[li]);
      SAAMG_LAUNCH();
      // the while node
      cudaStreamCaptureStatus st;
      cudaGraph_t cg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      SAAMG_CUDA(cudaStreamGetCaptureInfo(ls, &st, nullptr, &cg, &deps, nullptr, &nd));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = conds[li];
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t cnode;
      SAAMG_CUDA(cudaGraphAddNode(&cnode, cg, deps, nullptr, nd, &cp));
      bodies[li] = cp.conditional.phGraph_out[0];
      SAAMG_CUDA(cudaStreamUpdateCaptureDependencies(ls, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
      // epilogue of every solve: recomputed residual, result copy, scatter
      for (int j : L.sol) {
        SolveWork& w = *e->work[j];
        const OperatorData& od = hs[j]->op->d;
        const StencilDev<double> S = od.view<double>();
        stencil_apply<double>(S, ST_RESID, w.xhat.p, w.q.p, w.bhat.p, nullptr, 0.0, 0.0, nullptr, ls);
        dot_partials<double, double>(od.n, w.q.p, w.q.p, w.part0.p, ls);
        pcg_store_true(w.part0.p, w.ctl.p, ls);
        SAAMG_CUDA(cudaMemcpyAsync(&e->res[j], w.ctl.p, sizeof(PcgCtl), cudaMemcpyDeviceToHost, ls));
        scatter_solution(od, w.xhat.p, phi[j], ls);
      }
      cudaEvent_t join;
      SAAMG_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
      evs.push_back(join);
      SAAMG_CUDA(cudaEventRecord(join, ls));
      SAAMG_CUDA(cudaStreamWaitEvent(cs, join, 0));
    }
    e->k_fixed = captured() - k0;
    // the bodies: one pass of every solve of the lane that goes on
    for (size_t li = 0; li < e->lanes.size(); ++li) {
      Lane& L = *e->lanes[li];
      const long long kb = captured();
      body_cap = stream_of(3 + 2 * (int)li);
      SAAMG_CUDA(cudaStreamBeginCaptureToGraph(body_cap, bodies[li], nullptr, nullptr, 0,
                                               cudaStreamCaptureModeRelaxed));
      lane_body(L, conds[li], body_cap);
      SAAMG_CUDA(cudaStreamEndCapture(body_cap, &bodies[li]));
      body_cap = nullptr;
      L.k_body = captured() - kb;
    }
    capturing = false;
    SAAMG_CUDA(cudaStreamEndCapture(cs, &g));
    SAAMG_CUDA(cudaGraphInstantiate(&e->exec, g, 0));
    e->graph = g;
    SAAMG_CUDA(cudaGraphUpload(e->exec, cs));  // the first run does not pay for the upload
    SAAMG_CUDA(cudaStreamSynchronize(cs));
  } catch (...) {
    if (body_cap) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(body_cap, &junk);
    }
    if (capturing) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(cs, &junk);
      if (junk && junk != g) cudaGraphDestroy(junk);
    }
    cudaGraphDestroy(g);
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    throw;
  }
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  return e.release();
}

void batch_engine_launch(BatchEngine* e, cudaStream_t s) {
  SAAMG_CUDA(cudaGraphLaunch(e->exec, s));
}

const PcgCtl* batch_engine_results(const BatchEngine* e) { return e->res; }

long long batch_engine_kernels(const BatchEngine* e) {
  long long k = e->k_fixed;
  for (const auto& L : e->lanes) {
    int passes = 0;
    for (int j : L->sol) passes = std::max(passes, e->res[j].iters);
    k += (long long)passes * L->k_body;
  }
  return k;
}

long long batch_engine_bytes(const BatchEngine* e) {
  long long b = 0;
  for (const auto& L : e->lanes) b += L->tasks.bytes();
  for (const auto& w : e->work) {
    b += w->bhat.bytes() + w->xhat.bytes() + w->r.bytes() + w->z.bytes() + w->p.bytes() +
         w->q.bytes() + w->z32.bytes() + w->r32.bytes();
    for (auto& v : w->fx0) b += v.bytes() * 5;
    for (auto& v : w->dx0) b += v.bytes() * 5;
  }
  return b;
}

void batch_engine_free(BatchEngine* e) { delete e; }

}  // namespace saamg
