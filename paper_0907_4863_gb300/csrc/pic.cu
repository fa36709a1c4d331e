// The steps on either side of the solve in a PIC time step (Sec. 1: E = -grad phi of the
// Poisson solution; Sec. 4.1: cloud-in-cell deposition of the particle charges): CIC
// deposition onto the box lattice and the CIC gather of the nodal field at the particles.
//
// Deposition is deterministic: every contribution ((q / V) wx) wy) wz is rounded once to a
// 64-bit fixed-point number with a power-of-two scale chosen from sum |q| (no node can hold
// more), and the integer atomic additions commute.  The gather uses explicit round-to-
// nearest multiply and add in the reference's order, so it is bitwise the CPU result.
#include "pic.cuh"

namespace saamg {

namespace {

__device__ __forceinline__ void cic_axis(double x, double o, double h, long long& c, double& f) {
  const double u = (x - o) / h;
  const double fl = floor(u);
  c = (long long)fl;
  f = u - fl;
}

struct Lattice {
  int nx, ny, nz;
  double hx, hy, hz, ox, oy, oz;
};

__global__ void abs_sum_k(int n, const double* __restrict__ q, double* __restrict__ part) {
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    acc += fabs(q[i]);
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// scale exponent: sum|q| / V * 2^S < 2^61, so no node sum can overflow 64 bits;
// exp[1] = 1 when the charges are not finite
__global__ void scale_k(const double* __restrict__ part, int nparts, double vol,
                        int* __restrict__ exp) {
  if (threadIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < nparts; ++i) t += part[i];
  const double b = t / vol;
  exp[1] = isfinite(b) ? 0 : 1;
  exp[0] = (b > 0.0 && isfinite(b)) ? 60 - ilogb(b) : 0;
}

__global__ void cic_deposit_k(Lattice g, int np, const double* __restrict__ x,
                              const double* __restrict__ y, const double* __restrict__ z,
                              const double* __restrict__ q, double vol,
                              const int* __restrict__ exp, unsigned long long* __restrict__ acc) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np || exp[1]) return;
  const int S = exp[0];
  long long ci, cj, ck;
  double fx, fy, fz;
  cic_axis(x[p], g.ox, g.hx, ci, fx);
  cic_axis(y[p], g.oy, g.hy, cj, fy);
  cic_axis(z[p], g.oz, g.hz, ck, fz);
  const double qv = q[p] / vol;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const long long i = ci + a, j = cj + b, k = ck + c;
        if (i < 0 || j < 0 || k < 0 || i >= g.nx || j >= g.ny || k >= g.nz) continue;
        const double wx = a ? fx : 1.0 - fx, wy = b ? fy : 1.0 - fy, wz = c ? fz : 1.0 - fz;
        const double v = __dmul_rn(__dmul_rn(__dmul_rn(qv, wx), wy), wz);
        const long long iv = llrint(ldexp(v, S));
        atomicAdd(&acc[i + (long long)g.nx * (j + (long long)g.ny * k)], (unsigned long long)iv);
      }
}

__global__ void fixed_to_double_k(size_t n, const unsigned long long* __restrict__ acc,
                                  const int* __restrict__ exp, double* __restrict__ rho) {
  const int S = exp[0];
  const bool bad = exp[1] != 0;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n;
       v += (size_t)gridDim.x * blockDim.x)
    rho[v] = bad ? __longlong_as_double(0x7ff8000000000000ll)
                 : ldexp((double)(long long)acc[v], -S);
}

__global__ void cic_gather_k(Lattice g, const double* __restrict__ ex,
                             const double* __restrict__ ey, const double* __restrict__ ez,
                             int np, const double* __restrict__ x, const double* __restrict__ y,
                             const double* __restrict__ z, double* __restrict__ epx,
                             double* __restrict__ epy, double* __restrict__ epz) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  long long ci, cj, ck;
  double fx, fy, fz;
  cic_axis(x[p], g.ox, g.hx, ci, fx);
  cic_axis(y[p], g.oy, g.hy, cj, fy);
  cic_axis(z[p], g.oz, g.hz, ck, fz);
  double sx = 0.0, sy = 0.0, sz = 0.0;
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        const long long i = ci + a, j = cj + b, k = ck + c;
        if (i < 0 || j < 0 || k < 0 || i >= g.nx || j >= g.ny || k >= g.nz) continue;
        const double w = __dmul_rn(__dmul_rn(a ? fx : 1.0 - fx, b ? fy : 1.0 - fy),
                                   c ? fz : 1.0 - fz);
        const long long v = i + (long long)g.nx * (j + (long long)g.ny * k);
        sx = __dadd_rn(sx, __dmul_rn(w, ex[v]));
        sy = __dadd_rn(sy, __dmul_rn(w, ey[v]));
        sz = __dadd_rn(sz, __dmul_rn(w, ez[v]));
      }
  epx[p] = sx;
  epy[p] = sy;
  epz[p] = sz;
}

Lattice lattice(const saamg_grid& g) {
  return Lattice{g.n[0], g.n[1], g.n[2], g.h[0], g.h[1], g.h[2],
                 g.origin[0], g.origin[1], g.origin[2]};
}

}  // namespace

void deposit_cic(const saamg_grid& grid, int np, const double* x, const double* y,
                 const double* z, const double* q, double* rho, cudaStream_t s) {
  const Lattice g = lattice(grid);
  const size_t nbox = (size_t)g.nx * g.ny * g.nz;
  const double vol = (g.hx * g.hy) * g.hz;
  Buf<unsigned long long> acc;
  Buf<double> part;
  Buf<int> exp;
  acc.alloc(nbox, s);
  part.alloc(kRedBlocks, s);
  exp.alloc(2, s);
  SAAMG_CUDA(cudaMemsetAsync(acc.p, 0, nbox * sizeof(unsigned long long), s));
  abs_sum_k<<<kRedBlocks, 256, 0, s>>>(np, q, part.p);
  SAAMG_LAUNCH();
  scale_k<<<1, 32, 0, s>>>(part.p, kRedBlocks, vol, exp.p);
  SAAMG_LAUNCH();
  if (np > 0) {
    KernelTimer kt(SAAMG_KT_PIC, np, s);
    cic_deposit_k<<<(np + 255) / 256, 256, 0, s>>>(g, np, x, y, z, q, vol, exp.p, acc.p);
    SAAMG_LAUNCH();
  }
  const int blocks = (int)std::min<size_t>((nbox + 255) / 256, sm_count() * 16);
  fixed_to_double_k<<<blocks, 256, 0, s>>>(nbox, acc.p, exp.p, rho);
  SAAMG_LAUNCH();
}

void gather_cic(const saamg_grid& grid, const double* ex, const double* ey, const double* ez,
                int np, const double* x, const double* y, const double* z, double* epx,
                double* epy, double* epz, cudaStream_t s) {
  if (np <= 0) return;
  KernelTimer kt(SAAMG_KT_PIC, np, s);
  cic_gather_k<<<(np + 255) / 256, 256, 0, s>>>(lattice(grid), ex, ey, ez, np, x, y, z, epx,
                                                epy, epz);
  SAAMG_LAUNCH();
}

}  // namespace saamg
