// The hierarchy and operator handles behind the C ABI, and the data of one AMG level
// (internal; shared by the C ABI and the batched solver).
#pragma once

#include <atomic>
#include <memory>
#include <vector>

#include "coarse.cuh"
#include "csr.cuh"
#include "operator.cuh"
#include "pcg.cuh"
#include "sell.cuh"

namespace saamg {

struct ChebCoef {
  std::vector<double> c1, c2;
};

struct Level {
  int n = 0;
  long long nnz = 0;
  double avg = 0;
  DevCsr A;                     // levels >= 1 (level 0 uses the operator's CSR / stencil)
  Buf<double> invd;
  Buf<float> invd32;
  Buf<int> agg;
  Buf<unsigned char> root;
  Buf<unsigned> ids;            // lattice ids of the nodes (cube aggregation, levels >= 1)
  int dims[3] = {0, 0, 0};      // lattice of the ids (cube aggregation)
  DevCsr P, R;                  // to the next level
  DevCsr APpat;                 // pattern of A_l P_l (levels >= 1): a reusing setup skips its
                                // symbolic pass
  double lambda = 0, omega = 0;
  ChebCoef cheb;
  // V-cycle work vectors (FP64 and FP32 sets; only the one for the precision is allocated)
  Buf<double> x0, x1, b, d, r;
  Buf<float> fx0, fx1, fb, fd, fr;
  // SELL-32 copy of A used by the V-cycle smoother (levels 1 .. L-2), with the values of
  // the working precision (FP64, FP32 or BF16); P and R stay CSR (a warp-wide row group
  // gathers neighbouring columns, which one-thread-per-row slices would scatter)
  DevSell As;
  Buf<float> P32, R32;          // FP32 values of P and R (mixed precision)
};

}  // namespace saamg

constexpr uint32_t kOpMagic = 0x5341504fu;    // "SAPO"
constexpr uint32_t kHierMagic = 0x53414852u;  // "SAHR"

struct saamg_operator {
  uint32_t magic = kOpMagic;
  saamg::OperatorData d;
  cudaStream_t stream = nullptr;
};

struct saamg_hierarchy {
  uint32_t magic = kHierMagic;
  const saamg_operator* op = nullptr;
  saamg_params prm{};
  std::vector<std::unique_ptr<saamg::Level>> lev;
  saamg::CoarseSolver coarse;
  double setup_ms = 0;
  // PCG state
  saamg::Buf<double> bhat, xhat, r, z, p, q;
  saamg::Buf<float> z32, r32;
  saamg::Buf<double> part0, part1, part2;
  saamg::Buf<saamg::PcgCtl> ctl;
  saamg::HostScratch host;
  saamg::Buf<double> scratch;
  long long bytes = 0;
  // identity for cached batch graphs: a new value at creation and whenever the V-cycle
  // changes (a cached graph never outlives the kernels and pointers it was captured with)
  unsigned long long version = 0;
  long long gk_fixed = 0, gk_body = 0;  // kernels of the device-loop graph (fixed, per pass)
  // device-loop solve: the whole PCG as one graph (conditional while node)
  cudaGraph_t graph = nullptr;      // owns the conditional handle: lives as long as gexec
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t done = nullptr;
  saamg::PcgCtl* result = nullptr;  // pinned host copy of the last device-loop solve's scalars
  // A work set reads the levels (matrices, transfers, aggregates, coarse inverse) of `base`
  // through borrowed arrays and owns only its vectors and graph.  refs counts the handle
  // itself and its live work sets; the last release deletes it.
  saamg_hierarchy* base = nullptr;
  std::atomic<int> refs{1};
  ~saamg_hierarchy() {
    if (done) cudaEventSynchronize(done);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (done) cudaEventDestroy(done);
    if (result) cudaFreeHost(result);
  }
};

