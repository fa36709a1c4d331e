// Conjugate-gradient recursion (Sec. 3.1) on the scaled system: fused axpy + norm,
// direction update, dot products.  Every reduction writes one partial per block of a
// fixed grid and a single block adds the partials in index order, so a run is
// reproducible bit for bit.  The CG scalars stay on the device.
#include "pcg.cuh"
#include "rows.cuh"

namespace saamg {

namespace {

using rows::block_sum;
using rows::sum_fixed;

// Loads of four grid strides are issued before their (in-order) multiply-adds: the sum is
// the same sequence of operations as the plain strided loop, with more bytes in flight.
template <class TA, class TB>
__global__ void dot_k(int n, const TA* __restrict__ a, const TB* __restrict__ b,
                      double* __restrict__ part) {
  pdl_wait();
  const double t = rows::dot_block<TA, TB>(blockIdx.x, n, a, b);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// r'z and z'q in one sweep; the same per-thread order and block tree as two dot_k calls
template <class TZ>
__global__ void dot2_k(int n, const double* __restrict__ r, const TZ* __restrict__ z,
                       const double* __restrict__ q, double* __restrict__ part_rz,
                       double* __restrict__ part_zq) {
  pdl_wait();
  double t1, t2;
  rows::dot2_block<TZ>(blockIdx.x, n, r, z, q, t1, t2);
  if (threadIdx.x == 0) {
    part_rz[blockIdx.x] = t1;
    part_zq[blockIdx.x] = t2;
  }
}

__global__ void alpha_k(const double* __restrict__ part, PcgCtl* ctl) {
  pdl_wait();
  double pq = sum_fixed(part);
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

// r32 (mixed precision): the FP32 copy of the new residual, the next V-cycle's input
__global__ void update_k(int n, double* __restrict__ x, double* __restrict__ r,
                         const double* __restrict__ p, const double* __restrict__ q,
                         const PcgCtl* __restrict__ ctl, double* __restrict__ part,
                         float* __restrict__ r32) {
  pdl_wait();
  const double t = rows::update_block(blockIdx.x, n, ctl->alpha, x, r, p, q, r32);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void check_k(const double* __restrict__ part, PcgCtl* ctl) {
  pdl_wait();
  double rr = sum_fixed(part);
  if (threadIdx.x == 0) {
    ctl->rr = rr;
    ctl->iters += 1;
    if (!isfinite(rr)) ctl->breakdown = 1;
    ctl->converged = rr <= ctl->tol2;
  }
}

__global__ void beta_k(const double* __restrict__ part_rz, const double* __restrict__ part_zq,
                       int rule, PcgCtl* ctl) {
  pdl_wait();
  double rz = sum_fixed(part_rz);
  double zq = part_zq ? sum_fixed(part_zq) : 0.0;
  if (threadIdx.x == 0 && rule < 0) {  // first direction: only r'z
    ctl->rz = rz;
    if (!isfinite(rz)) ctl->breakdown = 1;
    return;
  }
  if (threadIdx.x == 0) {
    double b = (rule == 1) ? (-ctl->alpha * zq) / ctl->rz : rz / ctl->rz;
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

template <class TZ>
__global__ void direction_k(int n, const TZ* __restrict__ z, double* __restrict__ p,
                            const PcgCtl* __restrict__ ctl) {
  pdl_wait();
  const double b = ctl->beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = (double)z[i] + b * p[i];
}

__global__ void sub_k(int n, const double* __restrict__ b, const double* __restrict__ q,
                      double* __restrict__ r) {
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    r[i] = b[i] - q[i];
}

template <class TZ>
__global__ void copy_k(int n, const TZ* __restrict__ z, double* __restrict__ p) {
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = (double)z[i];
}

__global__ void graph_init_k(const double* __restrict__ part_bb, const double* __restrict__ part_rr,
                             PcgCtl* ctl, cudaGraphConditionalHandle cond, int maxit) {
  pdl_wait();
  const double bb = sum_fixed(part_bb);
  const double rr = sum_fixed(part_rr);
  if (threadIdx.x == 0) {
    ctl->bb = bb;
    ctl->rr = rr;
    ctl->tol2 = (ctl->rtol * ctl->rtol) * bb;
    ctl->iters = 0;
    ctl->breakdown = !(isfinite(bb) && isfinite(rr));
    ctl->converged = (bb == 0.0) || rr <= ctl->tol2;
    ctl->rz = 0.0;
    ctl->alpha = 0.0;
    ctl->beta = 0.0;
    const int go = !ctl->converged && !ctl->breakdown && maxit > 0;
    cudaGraphSetConditional(cond, go ? 1u : 0u);
  }
}

__global__ void zero_if_rhs_zero_k(double* __restrict__ x, int n, const PcgCtl* __restrict__ ctl) {
  pdl_wait();
  if (ctl->bb != 0.0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = 0.0;
}

__global__ void graph_beta_k(const double* __restrict__ part_rz, const double* __restrict__ part_zq,
                             int rule, PcgCtl* ctl) {
  pdl_wait();
  const double rz = sum_fixed(part_rz);
  const double zq = part_zq ? sum_fixed(part_zq) : 0.0;
  if (threadIdx.x == 0) {
    double b = 0.0;
    if (ctl->iters > 0) b = (rule == 1) ? (-ctl->alpha * zq) / ctl->rz : rz / ctl->rz;
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

__global__ void graph_check_k(const double* __restrict__ part, PcgCtl* ctl,
                              cudaGraphConditionalHandle cond, int maxit) {
  pdl_wait();
  const double rr = sum_fixed(part);
  if (threadIdx.x == 0) {
    ctl->rr = rr;
    ctl->iters += 1;
    if (!isfinite(rr)) ctl->breakdown = 1;
    ctl->converged = rr <= ctl->tol2;
    const int go = !ctl->converged && !ctl->breakdown && ctl->iters < maxit;
    cudaGraphSetConditional(cond, go ? 1u : 0u);
  }
}

__global__ void store_true_k(const double* __restrict__ part, PcgCtl* ctl) {
  pdl_wait();
  const double rr = sum_fixed(part);
  if (threadIdx.x == 0) ctl->rr_true = rr;
}

inline int vec_blocks(int n) {
  int b = (n + 255) / 256;
  return b < sm_count() * 8 ? (b > 0 ? b : 1) : sm_count() * 8;
}

}  // namespace

template <class TA, class TB>
void dot_partials(int n, const TA* a, const TB* b, double* partials, cudaStream_t s) {
  launch_pdl(dot_k<TA, TB>, kRedBlocks, kRedThreads, 0, s, n, a, b, partials);
  SAAMG_LAUNCH();
}
template void dot_partials<double, double>(int, const double*, const double*, double*, cudaStream_t);
template void dot_partials<double, float>(int, const double*, const float*, double*, cudaStream_t);
template void dot_partials<float, double>(int, const float*, const double*, double*, cudaStream_t);

template <class TZ>
void dot2_partials(int n, const double* r, const TZ* z, const double* q, double* part_rz,
                   double* part_zq, cudaStream_t s) {
  launch_pdl(dot2_k<TZ>, kRedBlocks, kRedThreads, 0, s, n, r, z, q, part_rz, part_zq);
  SAAMG_LAUNCH();
}
template void dot2_partials<double>(int, const double*, const double*, const double*, double*,
                                    double*, cudaStream_t);
template void dot2_partials<float>(int, const double*, const float*, const double*, double*,
                                   double*, cudaStream_t);

void pcg_alpha(const double* partials, PcgCtl* ctl, cudaStream_t s) {
  launch_pdl(alpha_k, 1, kRedThreads, 0, s, partials, ctl);
  SAAMG_LAUNCH();
}

void pcg_update(int n, double* x, double* r, const double* p, const double* q, const PcgCtl* ctl,
                double* partials, cudaStream_t s, float* r32) {
  launch_pdl(update_k, kRedBlocks, kRedThreads, 0, s, n, x, r, p, q, ctl, partials, r32);
  SAAMG_LAUNCH();
}

void pcg_check(const double* partials, PcgCtl* ctl, cudaStream_t s) {
  launch_pdl(check_k, 1, kRedThreads, 0, s, partials, ctl);
  SAAMG_LAUNCH();
}

void pcg_beta(const double* part_rz, const double* part_zq, int rule, PcgCtl* ctl,
              cudaStream_t s) {
  launch_pdl(beta_k, 1, kRedThreads, 0, s, part_rz, part_zq, rule, ctl);
  SAAMG_LAUNCH();
}

template <class TZ>
void pcg_direction(int n, const TZ* z, double* p, const PcgCtl* ctl, cudaStream_t s) {
  launch_pdl(direction_k<TZ>, vec_blocks(n), 256, 0, s, n, z, p, ctl);
  SAAMG_LAUNCH();
}
template void pcg_direction<double>(int, const double*, double*, const PcgCtl*, cudaStream_t);
template void pcg_direction<float>(int, const float*, double*, const PcgCtl*, cudaStream_t);

void vec_sub(int n, const double* b, const double* q, double* r, cudaStream_t s) {
  launch_pdl(sub_k, vec_blocks(n), 256, 0, s, n, b, q, r);
  SAAMG_LAUNCH();
}

void pcg_graph_init(const double* part_bb, const double* part_rr, PcgCtl* ctl,
                    cudaGraphConditionalHandle cond, int maxit, double* x, int n, cudaStream_t s) {
  launch_pdl(graph_init_k, 1, kRedThreads, 0, s, part_bb, part_rr, ctl, cond, maxit);
  SAAMG_LAUNCH();
  launch_pdl(zero_if_rhs_zero_k, vec_blocks(n), 256, 0, s, x, n, ctl);
  SAAMG_LAUNCH();
}

void pcg_graph_beta(const double* part_rz, const double* part_zq, int rule, PcgCtl* ctl,
                    cudaStream_t s) {
  launch_pdl(graph_beta_k, 1, kRedThreads, 0, s, part_rz, part_zq, rule, ctl);
  SAAMG_LAUNCH();
}

void pcg_graph_check(const double* partials, PcgCtl* ctl, cudaGraphConditionalHandle cond,
                     int maxit, cudaStream_t s) {
  launch_pdl(graph_check_k, 1, kRedThreads, 0, s, partials, ctl, cond, maxit);
  SAAMG_LAUNCH();
}

void pcg_store_true(const double* partials, PcgCtl* ctl, cudaStream_t s) {
  launch_pdl(store_true_k, 1, kRedThreads, 0, s, partials, ctl);
  SAAMG_LAUNCH();
}

template <class TZ>
void vec_copy_to_double(int n, const TZ* z, double* p, cudaStream_t s) {
  launch_pdl(copy_k<TZ>, vec_blocks(n), 256, 0, s, n, z, p);
  SAAMG_LAUNCH();
}
template void vec_copy_to_double<double>(int, const double*, double*, cudaStream_t);
template void vec_copy_to_double<float>(int, const float*, double*, cudaStream_t);

}  // namespace saamg
