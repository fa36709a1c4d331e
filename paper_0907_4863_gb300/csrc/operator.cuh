// Level-0 operator data and the launchers that build and apply it (internal).
#pragma once

#include "common.cuh"

namespace saamg {

struct GeomParams {
  int nx, ny, nz;
  double h[3], o[3];
  double a, b, taper, cx, cy;
  int zbc, sym, mode;
  // derived once on the host (plain IEEE multiply / divide, no rounding differences):
  double cdir[3];   // 1 / h_i^2
  double robin;     // 2 h_z / d with d = (nz - 1) h_z / 2
};

// Scaled operator Ahat = D^-1/2 A D^-1/2 on the unknowns of the box grid.
struct OperatorData {
  GeomParams g{};
  int n = 0;            // unknowns
  long long nnz = 0;    // nonzeros of the explicit CSR
  int nlines = 0;       // ny * nz
  Buf<LineInfo> lines;
  Buf<int4> nbr;        // per line: row offsets to the -y, +y, -z, +z neighbour lines
  Buf<int2> chunks;
  Buf<ChunkRec> crec;
  int nchunks = 0;
  Buf<int> rline;       // line of every compact row
  Buf<double> table;    // 8 doubles per table row
  Buf<float> table32;
  Buf<int> trow;        // compact row of every table row
  int ntable = 0;
  Buf<int2> rrow;       // (compact row, line) of the lines' regular-run rows, in order
  int nrun = 0;
  double c0 = 0, cx = 0, cy = 0, cz = 0, invd0 = 0;  // regular-row coefficients
  Buf<double> scale;    // s_i = a_ii^-1/2 (unscaled diagonal)
  Buf<unsigned> ids;    // box index of each unknown
  Buf<unsigned char> regular;
  Buf<unsigned char> nbmask;  // bit q: neighbour q (-x,+x,-y,+y,-z,+z) is an unknown
  DevCsr A;             // explicit scaled CSR (used by the AMG setup)
  // launch shapes of the FP64 [0] and FP32 [1] passes: FP64 is bound by FP64 issue and takes
  // packed rows, one chunk per step; FP32 is latency-bound and takes line chunks, two per step
  StencilCfg cfg[2] = {{1, 1, 256, 16}, {2, 0, 256, 16}};
  size_t bytes() const {
    return lines.bytes() + nbr.bytes() + chunks.bytes() + crec.bytes() + rline.bytes() + table.bytes() +
           table32.bytes() + trow.bytes() + rrow.bytes() + scale.bytes() +
           ids.bytes() + regular.bytes() + nbmask.bytes() + A.bytes();
  }
  template <class T>
  StencilDev<T> view() const;
};

template <>
StencilDev<double> OperatorData::view<double>() const;
template <>
StencilDev<float> OperatorData::view<float>() const;

// geometry.cu
void build_operator_data(const GeomParams& g, cudaStream_t s, OperatorData& op);
// rho (box) -> bhat (compact) = s_i * (bfac_i * rho); phi0 (box) -> xhat0 = phi0 / s_i (if given)
void gather_rhs(const OperatorData& op, const double* rho, const double* phi0, double* bhat,
                double* xhat, cudaStream_t s);
// invd = 1 / a_ii of the scaled operator (and its FP32 copy, if given) from the stencil data
void stencil_diag_inverse(const OperatorData& op, double* invd, float* invd32, cudaStream_t s);
// xhat (compact) -> phi (box) = s_i * xhat at unknowns, 0 elsewhere
void scatter_solution(const OperatorData& op, const double* xhat, double* phi, cudaStream_t s);

// E = -grad phi on the box (phi and E box arrays; E is 0 outside the unknowns)
void field_gradient(const OperatorData& op, const double* phi, double* ex, double* ey,
                    double* ez, cudaStream_t s);

// stencil.cu -- matrix-free level-0 kernels.  MODE selects the fused operation.
enum StencilMode {
  ST_SPMV = 0,      // y = A x
  ST_SPMV_DOT = 1,  // y = A x, partials of x.y
  ST_RESID = 2,     // y = b - A x
  ST_CHEB = 3,      // r = b - A x; d = c1 d + c2 D^-1 r; y = x + d
  ST_CHEB0 = 4,     // d = c2 D^-1 b; y = d   (Chebyshev step 0 from x = 0)
  ST_DINV_DOT = 5,  // y = s D^-1 A x, partials of y.y (power iteration; s = *xscale or 1)
  ST_CHEB1 = 6,     // ST_CHEB with c1 = 0 (first step from a nonzero x): d is not read
  ST_PROLONG = 7    // y += P v with P = (I - omega D^-1 A) T, T from the aggregates
};
template <class T>
void stencil_apply(const StencilDev<T>& S, int mode, const T* x, T* y, const T* b, T* d, T c1,
                   T c2, double* partials, cudaStream_t s, const double* xscale = nullptr);
// Level-0 prolongation without the matrix P (Sec. 3.2: P = (I - omega D^-1 A) T):
// y_i += v_agg(i) - omega invd_i sum_j a_ij v_agg(j), agg = level-0 aggregate of each row
template <class T>
void stencil_prolong(const StencilDev<T>& S, const int* agg, T omega, const T* v, T* y,
                     cudaStream_t s);
// Times the level-0 Chebyshev step under every launch shape (K 1/2/4, packed or line chunks,
// 128/256 threads, 8/16/32 blocks per SM) on scratch vectors and returns the fastest; its
// time (median of three launches) in *best_us.
template <class T>
StencilCfg stencil_autotune(const StencilDev<T>& S, cudaStream_t s, double* best_us);

}  // namespace saamg
