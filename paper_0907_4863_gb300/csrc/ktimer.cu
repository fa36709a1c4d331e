// Kernel launch accounting and opt-in per-class kernel timing (CUDA events).
#include <cstdlib>
#include <atomic>
#include <vector>

#include "common.cuh"

namespace saamg {

namespace {
std::atomic<long long> g_launches{0};
bool g_timing = false;

struct Record {
  cudaEvent_t e0, e1;
  long long rows;
};
struct ClassLog {
  std::vector<Record> pending;
  double ms = 0.0;
  long long launches = 0, rows = 0;
};
ClassLog g_log[SAAMG_KT_COUNT];
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  SAAMG_CUDA(cudaEventCreate(&e));
  return e;
}

void drain(ClassLog& L) {
  for (Record& r : L.pending) {
    float ms = 0.f;
    SAAMG_CUDA(cudaEventSynchronize(r.e1));
    SAAMG_CUDA(cudaEventElapsedTime(&ms, r.e0, r.e1));
    L.ms += ms;
    L.launches += 1;
    L.rows += r.rows;
    g_pool.push_back(r.e0);
    g_pool.push_back(r.e1);
  }
  L.pending.clear();
}
}  // namespace

namespace {
thread_local int t_capturing = 0;
thread_local long long t_captured = 0;
}  // namespace

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("SAAMG_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

void count_launch() {
  if (t_capturing) ++t_captured;
  else g_launches.fetch_add(1, std::memory_order_relaxed);
}
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long captured() { return t_captured; }
CaptureCount::CaptureCount() { ++t_capturing; }
CaptureCount::~CaptureCount() { --t_capturing; }

KernelTimer::KernelTimer(int kclass, long long nrows, cudaStream_t stream)
    : cls(kclass), rows(nrows), s(stream) {
  if (!g_timing || cls < 0 || cls >= SAAMG_KT_COUNT) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  e0 = take_event();
  SAAMG_CUDA(cudaEventRecord(e0, s));
}

KernelTimer::~KernelTimer() {
  if (!e0) return;
  try {
    cudaEvent_t e1 = take_event();
    SAAMG_CUDA(cudaEventRecord(e1, s));
    g_log[cls].pending.push_back(Record{e0, e1, rows});
    if (g_log[cls].pending.size() > 4096) drain(g_log[cls]);  // bound outstanding events
  } catch (...) {
  }
}

}  // namespace saamg

using namespace saamg;

extern "C" {

long long saamg_kernel_launches(void) { return g_launches.load(); }

saamg_status saamg_kernel_timing(int enable) {
  g_timing = enable != 0;
  return SAAMG_OK;
}

saamg_status saamg_kernel_timing_read(int kclass, double* total_ms, long long* launches,
                                      long long* rows) {
  if (kclass < 0 || kclass >= SAAMG_KT_COUNT) return SAAMG_EINVAL;
  try {
    ClassLog& L = g_log[kclass];
    drain(L);
    if (total_ms) *total_ms = L.ms;
    if (launches) *launches = L.launches;
    if (rows) *rows = L.rows;
    L.ms = 0.0;
    L.launches = 0;
    L.rows = 0;
  } catch (const Error&) {
    return SAAMG_ECUDA;
  }
  return SAAMG_OK;
}

}  // extern "C"
