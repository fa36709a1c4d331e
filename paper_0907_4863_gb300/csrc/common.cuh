// Internal declarations shared by the translation units of libsaamg (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <utility>

#include "saamg.h"

namespace saamg {

// ---------------------------------------------------------------------------
// Errors: every internal failure throws Error; the C ABI converts it to a status.
// ---------------------------------------------------------------------------
struct Error {
  saamg_status status;
  std::string msg;
};

[[noreturn]] void fail(saamg_status st, const std::string& msg);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);

void count_launch();
// Launch accounting across graph capture: while a CaptureCount is alive on this thread, launches
// are not counted as executed but tallied in captured(); the graph's executions are counted
// afterwards with count_launches (the kernels a run of the graph executed).
void count_launches(long long k);
long long captured();
struct CaptureCount {
  CaptureCount();
  ~CaptureCount();
};
// Stores the message returned by saamg_last_error() for the calling thread.
void set_last_error(const std::string& msg);

#define SAAMG_CUDA(x) ::saamg::check_cuda((x), #x, __FILE__, __LINE__)

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  The solve's kernels are launched with launch_pdl, so the
// launch of a kernel is prepared while the kernel before it on the stream runs; its blocks wait
// at pdl_wait (their first statement, before any memory access) until that kernel has finished
// and its writes are visible.  No kernel signals its dependents early: measured at 256^3, an
// early signal (at kernel entry) made the solve 5-8 % slower, none 0.8-1.3 % faster than plain
// launches.  The order and the results of the work are those of plain launches; pdl_wait does
// nothing in a kernel launched without the attribute.  SAAMG_PDL=0 in the environment turns
// the attribute off.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
bool pdl_enabled();

template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  check_cuda(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...), "cudaLaunchKernelEx",
             __FILE__, __LINE__);
}
#define SAAMG_LAUNCH()                                                                  \
  do {                                                                                  \
    ::saamg::count_launch();                                                            \
    ::saamg::check_cuda(cudaGetLastError(), "kernel launch", __FILE__, __LINE__);       \
  } while (0)

// Opt-in timing of kernel classes with CUDA events recorded on the launching stream.
// KernelTimer t(cls, rows, stream); <launch>; -- records a start event on construction
// and a stop event on destruction when timing is enabled; otherwise does nothing.
struct KernelTimer {
  int cls;
  long long rows;
  cudaStream_t s;
  cudaEvent_t e0 = nullptr;
  KernelTimer(int kclass, long long nrows, cudaStream_t stream);
  ~KernelTimer();
};

// ---------------------------------------------------------------------------
// Device memory through the installed allocator hook.
// ---------------------------------------------------------------------------
struct AllocHook {
  saamg_alloc_fn alloc = nullptr;
  saamg_free_fn free = nullptr;
  void* ctx = nullptr;
};
AllocHook current_allocator();
// Blocks come from the hook (cudaMalloc without one).  Blocks of up to 64 MB that the library
// frees are kept, up to 1 GB in all, and handed out again for the same stream and hook (stream
// order makes that reuse safe without a synchronisation); they go back to the hook when the
// allocator changes.  `bytes` of dev_free is the size given to dev_alloc.
void* dev_alloc(const AllocHook& h, size_t bytes, cudaStream_t s);
void dev_free(const AllocHook& h, void* p, size_t bytes, cudaStream_t s);

// Owning device array (move-only).  Memory comes from the hook captured at allocation.
// A borrowed Buf views another Buf's array and frees nothing.
template <class T>
struct Buf {
  T* p = nullptr;
  size_t n = 0;
  AllocHook hook;
  cudaStream_t stream = nullptr;
  bool own = true;

  Buf() = default;
  Buf(const Buf&) = delete;
  Buf& operator=(const Buf&) = delete;
  Buf(Buf&& o) noexcept { swap(o); }
  Buf& operator=(Buf&& o) noexcept {
    if (this != &o) {
      release();
      swap(o);
    }
    return *this;
  }
  ~Buf() { release(); }
  void swap(Buf& o) noexcept {
    std::swap(p, o.p);
    std::swap(n, o.n);
    std::swap(hook, o.hook);
    std::swap(stream, o.stream);
    std::swap(own, o.own);
  }
  void alloc(size_t count, cudaStream_t s) {
    release();
    own = true;
    hook = current_allocator();
    stream = s;
    n = count;
    p = static_cast<T*>(dev_alloc(hook, (count > 0 ? count : 1) * sizeof(T), s));
  }
  // views o's array; o must outlive this Buf and keep its array
  void borrow(const Buf& o) {
    release();
    p = o.p;
    n = o.n;
    own = false;
  }
  void release() noexcept {
    if (p && own) {
      try {
        dev_free(hook, p, (n > 0 ? n : 1) * sizeof(T), stream);
      } catch (...) {
      }
    }
    p = nullptr;
    n = 0;
    own = true;
  }
  size_t bytes() const { return n * sizeof(T); }
  T* get() const { return p; }
};

// Pinned host scratch used to read small device results back.
struct HostScratch {
  void* p = nullptr;
  size_t bytes = 0;
  ~HostScratch();
  void* need(size_t b);
};

// ---------------------------------------------------------------------------
// Level-0 stencil description (matrix-free operator)
// ---------------------------------------------------------------------------
// One record per x-line (j,k), line index L = j + ny*k.  The unknowns of a line form
// the contiguous run i in [lo, hi] and occupy compact rows start .. start+hi-lo.  Rows
// with i in [rlo, rhi] are applied with the constant interior coefficients; the others
// read 7 scaled coefficients and 1/diag from the table at tstart + (their rank among
// the line's table rows).
struct __align__(32) LineInfo {
  int lo, hi, start, rlo, rhi, tstart, pad0, pad1;
};

// One record per chunk of <= 32 consecutive unknowns of one line, everything a warp needs to
// apply it in one 32-byte load: the chunk's first compact row, the table row of its lane 0
// (left of the regular run), the lanes [a, b] of the chunk inside the regular run (the table
// row of a lane j > b is tl + j + (a - b) - 1), the number of unknowns n, and the line's
// neighbour row offsets (as nbr).
struct __align__(32) ChunkRec {
  int row0, tl;
  short a, b;  // read as one int: a in the low half
  int n;
  int ym, yp, zm, zp;
};
static_assert(sizeof(ChunkRec) == 32, "ChunkRec is two 16-byte loads");

// Launch shape of the level-0 stencil passes without reductions (every row's arithmetic is the
// same under every shape, so the results are too): K chunks of 32 rows per warp step (1, 2,
// 4), packed (1: 32 regular-run rows per warp from the row list, then the table rows 32 at a
// time; 0: the line chunks), threads per block (128, 256) and blocks per SM (8, 16, 32).
struct StencilCfg {
  int k, packed, block, per_sm;
};

template <class T>
struct StencilDev {
  StencilCfg cfg;      // launch shape (host side)
  const LineInfo* lines;
  // per line: row offset from an unknown (i, L) to its neighbour (i, L') in the -y, +y, -z,
  // +z line (start' - lo') - (start - lo); 0 where that line does not exist or is empty
  const int4* nbr;
  const int2* chunks;  // (line, offset of the first of <= 32 consecutive unknowns)
  const ChunkRec* crec;  // the same chunks as applied by the FP32 passes
  int nchunks;
  const int* rline;    // line of every compact row (the FP64 passes take 32 consecutive rows)
  int n;               // unknowns
  int nx, ny, nz;
  const T* table;      // 8 per table row: self, -x, +x, -y, +y, -z, +z, 1/self
  const int* trow;     // compact row of every table row
  int ntable;
  const int2* rrow;    // (compact row, line) of the lines' regular-run rows, in order
  int nrun;
  T c0, cx, cy, cz, invd0;  // regular-row coefficients (scaled)
};

// ---------------------------------------------------------------------------
// CSR matrix on the device
// ---------------------------------------------------------------------------
struct DevCsr {
  int n = 0, m = 0;
  long long nnz = 0;
  Buf<int> rowptr, col;
  Buf<double> val;
  Buf<float> val32;           // FP32 copy (mixed precision)
  Buf<__nv_bfloat16> val16;   // BF16 copy (mixed precision, BF16 storage)
  size_t bytes() const {
    return rowptr.bytes() + col.bytes() + val.bytes() + val32.bytes() + val16.bytes();
  }
};

// Reduction partials: kernels that reduce write one double per block into a fixed
// array, and a single block adds them in index order, so results do not depend on
// scheduling.
// The count is fixed (4 per SM of a 152-SM GB300) and not taken from the device: it defines
// the summation tree, which must not change with the part the library runs on.
constexpr int kRedBlocks = 608;
constexpr int kRedThreads = 256;

// ---------------------------------------------------------------------------
// Host launchers (implemented in the .cu files; each file owns its kernels)
// ---------------------------------------------------------------------------
// scan.cu
long long exclusive_scan(const int* in, int* out, int n, cudaStream_t s);  // returns the total
void exclusive_scan_async(const int* in, int* out, int n, cudaStream_t s);  // no host wait
long long exclusive_scan_u8(const unsigned char* in, int* out, int n, cudaStream_t s);
// Same scan of bytes with caller-provided tile scratch (scan_u8_tiles_needed(n) entries);
// allocates nothing.
long long scan_u8_tiles_needed(int n);
long long exclusive_scan_u8_into(const unsigned char* in, int* out, int n, long long* tiles,
                                 cudaStream_t s);
void fill_int(int* p, int v, size_t n, cudaStream_t s);
void fill_double(double* p, double v, size_t n, cudaStream_t s);
void sum_partials(const double* partials, int count, double* out, cudaStream_t s,
                  double* inv_sqrt = nullptr);
// Number of SMs of the current device (cached per device); grids of grid-stride kernels are
// sized as multiples of it.
int sm_count();
// Copies `bytes` from device to host and waits.
void d2h_sync(void* host, const void* dev, size_t bytes, cudaStream_t s);

}  // namespace saamg
