// Batched PCG solves (internal): many right-hand sides on many hierarchies advanced together,
// one launch per operation across all of them.
#pragma once

#include "common.cuh"

struct saamg_hierarchy;

namespace saamg {

struct BatchEngine;  // cached graph, work vectors and task tables of one batch

// One solve's part of a batched level-0 stencil pass (the arguments of the one-solve launch).
template <class T>
struct StTask {
  StencilDev<T> S;
  const int* go;  // the solve's loop flag: 0 = finished, the task does nothing
  const T* x;
  T* y;
  const T* b;
  T* d;
  T c1, c2, c2i0;
  const int* agg;
  double* part;
};

// Work units (warp-sized chunks) of one solve's level-0 pass.
template <class T>
int stencil_units(const StencilDev<T>& S);
// The stencil pass `mode` (StencilMode, not the dot-product modes) over work blocks
// (task, first unit, end unit): a block of threads takes one work block at a time, its warps
// the units.
template <class T>
void batched_stencil(int mode, const StTask<T>* tasks, const int4* wbs, int nwb, cudaStream_t s);
// q = A p with the partials of p'q (FP64 CG product): kRedBlocks blocks per task, the
// one-solve launch's grid, so every partial has the same bits.
void batched_stencil_dot(const StTask<double>* tasks, int ntasks, cudaStream_t s);

struct PcgCtl;

// Whether the engine can run this batch (at least two solves, every hierarchy with unknowns
// and a dense coarse solve); otherwise the caller falls back to one device-loop graph per
// solve.
bool batch_engine_supports(saamg_hierarchy* const* hs, int count);
// Plans the batch and captures its graph; stream_of(k) gives capture stream k (the caller
// holds the capture lock).  Allocates every solve's work vectors.
BatchEngine* batch_engine_build(saamg_hierarchy* const* hs, const double* const* rho,
                                double* const* phi, int count, double rtol,
                                cudaStream_t (*stream_of)(int));
// Enqueues one run of the batch on s (gather, PCG of every solve, scatter).
void batch_engine_launch(BatchEngine* e, cudaStream_t s);
// Every solve's CG scalars after the last run (pinned host memory; valid once s is idle).
const PcgCtl* batch_engine_results(const BatchEngine* e);
// Kernels the last run executed.
long long batch_engine_kernels(const BatchEngine* e);
long long batch_engine_bytes(const BatchEngine* e);
void batch_engine_free(BatchEngine* e);

}  // namespace saamg
