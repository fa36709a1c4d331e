// Domain classification and operator assembly on the device (Sec. 2 of the paper).
//
// This file is compiled with --fmad=false: the inside test F < 0 and the boundary
// fractions s, t decide which lattice nodes are unknowns and how rows are formed, so
// they are evaluated with the plain IEEE multiply/add/divide/sqrt sequence written
// below and never with fused multiply-adds.
#include <climits>

#include "operator.cuh"

namespace saamg {

namespace {

__device__ __forceinline__ double node_coord(double o, int i, double h) { return o + (double)i * h; }

__device__ __forceinline__ double zlo(const GeomParams& g) { return g.o[2]; }
__device__ __forceinline__ double zhi(const GeomParams& g) {
  return g.o[2] + (double)(g.nz - 1) * g.h[2];
}

// Cross-section scale: 1 at the first z-plane, `taper` at the last, linear in z.
__device__ double taper_sigma(const GeomParams& g, double z) {
  if (g.taper == 1.0 || g.nz < 2) return 1.0;
  double tau = (z - zlo(g)) / (zhi(g) - zlo(g));
  return 1.0 + (g.taper - 1.0) * tau;
}

// Implicit function of the elliptic wall Gamma_1 (Sec. 4.1); F < 0 inside.
__device__ double wall_F(const GeomParams& g, double x, double y, double z) {
  double sg = taper_sigma(g, z);
  double u = (x - g.cx) / (g.a * sg);
  double v = (y - g.cy) / (g.b * sg);
  return (u * u + v * v) - 1.0;
}

// Omega_h of Sec. 2: lattice nodes of Omega plus the Robin planes; Dirichlet end
// planes carry known zeros.
__device__ bool node_inside(const GeomParams& g, int i, int j, int k) {
  if (i < 0 || j < 0 || k < 0 || i >= g.nx || j >= g.ny || k >= g.nz) return false;
  if (g.zbc == SAAMG_Z_DIRICHLET && (k == 0 || k == g.nz - 1)) return false;
  double x = node_coord(g.o[0], i, g.h[0]);
  double y = node_coord(g.o[1], j, g.h[1]);
  double z = node_coord(g.o[2], k, g.h[2]);
  return wall_F(g, x, y, z) < 0.0;
}

// 0 < s <= 1; the lower clamp 2^-20 only guards against rounding.
__device__ double clamp_frac(double s) {
  const double smin = 9.5367431640625e-07;
  if (s < smin) s = smin;
  if (s > 1.0) s = 1.0;
  return s;
}

// Fraction s of Sec. 2 (Fig. 2): the wall point x* = x -/+ s h e_dir nearest to the node.
// dir 0..5 = -x, +x, -y, +y, -z, +z.
__device__ double boundary_fraction(const GeomParams& g, int i, int j, int k, int dir) {
  double x = node_coord(g.o[0], i, g.h[0]);
  double y = node_coord(g.o[1], j, g.h[1]);
  double z = node_coord(g.o[2], k, g.h[2]);
  double sg = taper_sigma(g, z);
  if (dir < 2) {
    double v = (y - g.cy) / (g.b * sg);
    double w = (g.a * sg) * sqrt(1.0 - v * v);
    double s = (dir == 0) ? (x - (g.cx - w)) / g.h[0] : ((g.cx + w) - x) / g.h[0];
    return clamp_frac(s);
  }
  if (dir < 4) {
    double u = (x - g.cx) / (g.a * sg);
    double w = (g.b * sg) * sqrt(1.0 - u * u);
    double s = (dir == 2) ? (y - (g.cy - w)) / g.h[1] : ((g.cy + w) - y) / g.h[1];
    return clamp_frac(s);
  }
  // z: only a taper's cone crosses a z-line, where sigma(z*) = q
  if (g.taper == 1.0 || g.nz < 2) return 1.0;
  double u0 = (x - g.cx) / g.a;
  double v0 = (y - g.cy) / g.b;
  double q = sqrt(u0 * u0 + v0 * v0);
  double tstar = (q - 1.0) / (g.taper - 1.0);
  double zstar = zlo(g) + tstar * (zhi(g) - zlo(g));
  if (dir == 4) return (zstar < z) ? clamp_frac((z - zstar) / g.h[2]) : 1.0;
  return (zstar > z) ? clamp_frac((zstar - z) / g.h[2]) : 1.0;
}

// One direction of a row after substituting the extrapolated outside value into the
// difference star Eq. (6) (g = 0): constant Eq. (7), linear Eq. (8), quadratic Eqs. (9)
// and (10).  dd: diagonal contribution; om/opl: couplings to the minus/plus neighbour.
__device__ void direction_row(int mode, double c, bool in_m, bool in_p, double s, double t,
                              double& dd, double& om, double& opl) {
  om = 0.0;
  opl = 0.0;
  if (in_m && in_p) {
    dd = 2.0 * c;
    om = -c;
    opl = -c;
    return;
  }
  if (!in_m && !in_p) {
    if (mode == SAAMG_BC_CONSTANT) dd = 2.0 * c;
    else if (mode == SAAMG_BC_LINEAR) dd = (1.0 / s + 1.0 / t) * c;
    else dd = (2.0 / (s * t)) * c;
    return;
  }
  double f = in_m ? t : s;
  double off;
  if (mode == SAAMG_BC_CONSTANT) {
    dd = 2.0 * c;
    off = -c;
  } else if (mode == SAAMG_BC_LINEAR) {
    dd = (1.0 + 1.0 / f) * c;
    off = -c;
  } else {
    dd = (2.0 / f) * c;
    off = -(2.0 / (f + 1.0)) * c;
  }
  if (in_m) om = off;
  else opl = off;
}

// Neighbour lookup through the line records: row of (i, line Ln), or -1.
__device__ __forceinline__ int row_in_line(const LineInfo* lines, int Ln, int i) {
  LineInfo l = lines[Ln];
  return (i >= l.lo && i <= l.hi) ? l.start + (i - l.lo) : -1;
}

// Rows of the 6 neighbours (-x,+x,-y,+y,-z,+z) of unknown (i, L), -1 if not an unknown.
__device__ void neighbour_rows(const GeomParams& g, const LineInfo* lines, int L, int i, int row,
                               const LineInfo& me, int nb[6]) {
  int j = L % g.ny, k = L / g.ny;
  nb[0] = (i - 1 >= me.lo) ? row - 1 : -1;
  nb[1] = (i + 1 <= me.hi) ? row + 1 : -1;
  nb[2] = (j > 0) ? row_in_line(lines, L - 1, i) : -1;
  nb[3] = (j < g.ny - 1) ? row_in_line(lines, L + 1, i) : -1;
  nb[4] = (k > 0) ? row_in_line(lines, L - g.ny, i) : -1;
  nb[5] = (k < g.nz - 1) ? row_in_line(lines, L + g.ny, i) : -1;
}

// --- kernels ---------------------------------------------------------------

// Warp per x-line: first/last inside node and count; flags a non-contiguous line.
// Exact inside test of the nodes [a, b] of line (j, k), 32 at a time: first and last inside
// node and their number (warp-uniform results).
__device__ void scan_line(const GeomParams& g, int j, int k, int a, int b, int lane, int& first,
                          int& last, int& cnt) {
  first = INT_MAX;
  last = -1;
  cnt = 0;
  for (int base = a; base <= b; base += 32) {
    const int i = base + lane;
    const bool in = i <= b && node_inside(g, i, j, k);
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (m) {
      if (first == INT_MAX) first = base + __ffs(m) - 1;
      last = base + 31 - __clz(m);
      cnt += __popc(m);
    }
  }
}

// Warp per x-line: first/last inside node and count; flags a non-contiguous line.  The line
// meets the cross-section in |x - cx| < w with w = a sigma sqrt(1 - v^2); nodes two or more
// spacings from either end of that interval are classified the same by the exact test (|F| is
// there far above its rounding error), so only the nodes within two spacings of the ends are
// tested exactly; a line whose ends do not look as expected (an end at the box face, a short
// interval, or any surprise) is scanned node by node.
__global__ void classify_lines_k(GeomParams g, int nlines, LineInfo* lines, int* count,
                                 int* err) {
  const int L = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (L >= nlines) return;
  const int j = L % g.ny, k = L / g.ny;
  int first = INT_MAX, last = -1, cnt = 0;
  bool done = false;
  if (g.zbc == SAAMG_Z_DIRICHLET && (k == 0 || k == g.nz - 1)) {
    done = true;  // known zeros
  } else {
    const double y = node_coord(g.o[1], j, g.h[1]);
    const double z = node_coord(g.o[2], k, g.h[2]);
    const double sg = taper_sigma(g, z);
    const double v = (y - g.cy) / (g.b * sg);
    const double vv = v * v;
    if (vv >= 1.0) {
      done = true;  // u*u + v*v >= 1 for every node: F >= 0
    } else if (vv < 1.0) {
      const double w = (g.a * sg) * sqrt(1.0 - vv);
      const double xl = (g.cx - w - g.o[0]) / g.h[0], xh = (g.cx + w - g.o[0]) / g.h[0];
      const double A = fmax(0.0, ceil(xl) - 2.0), B = fmin((double)(g.nx - 1), floor(xh) + 2.0);
      if (A > B) {
        done = true;  // the interval holds no node, nor any within two spacings
      } else if (B - A >= 64.0) {
        const int a = (int)A, b = (int)B;
        // the five nodes at each end: outside ... inside at the low end, inside ... outside at
        // the high end, with one change each
        const int i = lane < 5 ? a + lane : b - 4 + (lane - 5);
        const bool in = lane < 10 && node_inside(g, i, j, k);
        const unsigned m = __ballot_sync(0xffffffffu, in);
        const unsigned mlo = m & 0x1fu, mhi = (m >> 5) & 0x1fu;
        // low end: bit 0 clear and the set bits contiguous up to bit 4; high end: bit 4 clear
        // and the set bits contiguous from bit 0
        const bool lo_ok = mlo != 0 && (mlo & 1u) == 0 && ((mlo | (mlo - 1u)) & 0x1fu) == 0x1fu &&
                           __popc(mlo) == 5 - (__ffs(mlo) - 1);
        const bool hi_ok = mhi != 0 && (mhi & 0x10u) == 0 && (mhi & (mhi + 1u)) == 0;
        if (lo_ok && hi_ok) {
          first = a + __ffs(mlo) - 1;
          last = b - 4 + (31 - __clz(mhi));
          cnt = last - first + 1;
          done = true;
        }
      } else {
        scan_line(g, j, k, (int)A, (int)B, lane, first, last, cnt);
        done = true;
      }
    }
  }
  if (!done) scan_line(g, j, k, 0, g.nx - 1, lane, first, last, cnt);
  if (lane == 0) {
    LineInfo l;
    l.lo = cnt ? first : 0;
    l.hi = cnt ? last : -1;
    l.start = 0;
    l.rlo = l.hi + 1;
    l.rhi = l.hi;
    l.tstart = 0;
    l.pad0 = l.pad1 = 0;
    lines[L] = l;
    count[L] = cnt;
    if (cnt && cnt != last - first + 1) atomicOr(err, 1);
  }
}

__global__ void chunk_counts_k(const int* count, int nlines, int* nch) {
  int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L < nlines) nch[L] = (count[L] + 31) >> 5;
}

__global__ void set_start_and_chunks_k(LineInfo* lines, const int* start, const int* chunk_start,
                                       const int* count, int nlines, int2* chunks) {
  int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= nlines) return;
  lines[L].start = start[L];
  int c0 = chunk_start[L], cnt = count[L];
  for (int off = 0, c = c0; off < cnt; off += 32, ++c) chunks[c] = make_int2(L, off);
}

// Warp per chunk: the line of each of its rows.
__global__ void row_lines_k(const LineInfo* __restrict__ lines, const int2* __restrict__ chunks,
                            int nchunks, int* __restrict__ rline) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= nchunks) return;
  const int2 ch = chunks[c];
  const LineInfo me = lines[ch.x];
  if (me.lo + ch.y + lane <= me.hi) rline[me.start + ch.y + lane] = ch.x;
}

// Thread per line: row offsets to the four neighbouring lines (0 where a line is missing).
__global__ void line_deltas_k(const LineInfo* __restrict__ lines, int nlines, int ny,
                              int4* __restrict__ nbr) {
  int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= nlines) return;
  const int nz = nlines / ny, j = L % ny, k = L / ny;
  const LineInfo me = lines[L];
  const int base = me.start - me.lo;
  auto delta = [&](int Ln) {
    const LineInfo l = lines[Ln];
    return l.hi >= l.lo ? (l.start - l.lo) - base : 0;
  };
  int4 r;
  r.x = j > 0 ? delta(L - 1) : 0;
  r.y = j < ny - 1 ? delta(L + 1) : 0;
  r.z = k > 0 ? delta(L - ny) : 0;
  r.w = k < nz - 1 ? delta(L + ny) : 0;
  nbr[L] = r;
}

// Regular interior row: all six couplings -c_dir, diagonal 2(cx+cy+cz), scaled; out[5], out[6]
// hold the unscaled diagonal and its diag^-1/2 (the same operations as a general row's).
__global__ void regular_consts_k(GeomParams g, double* out) {
  double dd[3], om, opl;
  for (int ax = 0; ax < 3; ++ax) direction_row(g.mode, g.cdir[ax], true, true, 1.0, 1.0, dd[ax], om, opl);
  double diag = (dd[0] + dd[1]) + dd[2];
  double s = 1.0 / sqrt(diag);
  double ss = s * s;
  out[0] = diag * ss;
  out[1] = (-g.cdir[0]) * ss;
  out[2] = (-g.cdir[1]) * ss;
  out[3] = (-g.cdir[2]) * ss;
  out[4] = 1.0 / out[0];
  out[5] = diag;  // unscaled interior diagonal
  out[6] = s;     // its diag^-1/2
}

// Unscaled row of unknown (i, L) at compact row `row`: diag + 6 couplings into cr[0..6],
// cr[7] = 0; returns s_i = diag^-1/2 and the row length.
__device__ double unscaled_row(const GeomParams& g, const LineInfo* __restrict__ lines, int L,
                               int i, int row, const LineInfo& me, double* __restrict__ cr,
                               int& len) {
  const int j = L % g.ny, k = L / g.ny;
  int nb[6];
  neighbour_rows(g, lines, L, i, row, me, nb);
  double off[6] = {0, 0, 0, 0, 0, 0};
  double dd[3];
  const bool gamma2 = (g.zbc == SAAMG_Z_ROBIN) && (k == 0 || k == g.nz - 1);
  for (int ax = 0; ax < 3; ++ax) {
    const double cdir = g.cdir[ax];
    const int dm = 2 * ax, dp = 2 * ax + 1;
    const bool in_m = nb[dm] >= 0, in_p = nb[dp] >= 0;
    if (ax == 2 && gamma2) {
      // Robin plane, Eq. (11): virtual point u(x') = u(x'') - (2h/d) u(x)
      const bool inner_is_p = (k == 0);
      const bool in_inner = inner_is_p ? in_p : in_m;
      if (in_inner) {
        dd[2] = (2.0 + g.robin) * cdir;
        off[inner_is_p ? dp : dm] = -2.0 * cdir;
      } else {
        // inner neighbour outside the wall: replaced by its one-sided extrapolation
        const double t = boundary_fraction(g, i, j, k, inner_is_p ? dp : dm);
        if (g.mode == SAAMG_BC_CONSTANT) dd[2] = (2.0 + g.robin) * cdir;
        else dd[2] = (g.robin + 2.0 / t) * cdir;
      }
      continue;
    }
    double s = 1.0, t = 1.0;
    if (!in_m) s = boundary_fraction(g, i, j, k, dm);
    if (!in_p) t = boundary_fraction(g, i, j, k, dp);
    direction_row(g.mode, cdir, in_m, in_p, s, t, dd[ax], off[dm], off[dp]);
  }
  double diag = (dd[0] + dd[1]) + dd[2];
  if (gamma2 && g.sym) {
    diag *= 0.5;
    for (int q = 0; q < 6; ++q) off[q] *= 0.5;
  }
  cr[0] = diag;
  len = 1;
  for (int q = 0; q < 6; ++q) {
    cr[1 + q] = off[q];
    len += nb[q] >= 0;
  }
  cr[7] = 0.0;
  return 1.0 / sqrt(diag);
}

// A row is simple when all six neighbours are unknowns and it is not on a Robin plane: its
// unscaled row is the interior one (diagonal rc[5], couplings -c_dir) and s_i = rc[6].
__device__ __forceinline__ bool simple_row(const GeomParams& g, const int nb[6], int L) {
  const int k = L / g.ny;
  const bool gamma2 = (g.zbc == SAAMG_Z_ROBIN) && (k == 0 || k == g.nz - 1);
  return !gamma2 && nb[0] >= 0 && nb[1] >= 0 && nb[2] >= 0 && nb[3] >= 0 && nb[4] >= 0 &&
         nb[5] >= 0;
}

// Warp per chunk, lane per unknown: simple rows get s_i and their row length here; the
// others (near the wall or on a Robin plane, a few per cent) are listed for
// assemble_boundary_k, where every lane of a warp holds one of them (the boundary fractions,
// divisions and square roots run on the FP64 pipe, which would otherwise idle the lanes of
// the simple rows of the same warp).
__global__ void assemble_unscaled_k(GeomParams g, const LineInfo* __restrict__ lines,
                                    const int2* __restrict__ chunks, int nchunks,
                                    double* __restrict__ scale, int* __restrict__ rowlen,
                                    unsigned* __restrict__ ids, const double* __restrict__ rc,
                                    int2* __restrict__ list, int* __restrict__ nlist) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= nchunks) return;  // warp-uniform
  const int2 ch = chunks[c];
  const int L = ch.x;
  const LineInfo me = lines[L];
  const int i = me.lo + ch.y + lane;
  const bool active = i <= me.hi;
  const int row = me.start + ch.y + lane;
  bool simple = false;
  if (active) {
    int nb[6];
    neighbour_rows(g, lines, L, i, row, me, nb);
    simple = simple_row(g, nb, L);
    if (simple) {
      scale[row] = rc[6];
      rowlen[row] = 7;
    }
    ids[row] = (unsigned)i + (unsigned)g.nx * (unsigned)L;
  }
  const unsigned need = __ballot_sync(0xffffffffu, active && !simple);
  if (!need) return;
  int base = 0;
  if (lane == 0) base = atomicAdd(nlist, __popc(need));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (active && !simple) list[base + __popc(need & ((1u << lane) - 1u))] = make_int2(c, lane);
}

// Thread per listed row: the full unscaled row (boundary fractions, Eqs. (7)-(11)), s_i and
// the row length.
__global__ void assemble_boundary_k(GeomParams g, const LineInfo* __restrict__ lines,
                                    const int2* __restrict__ chunks,
                                    const int2* __restrict__ list, const int* __restrict__ nlist,
                                    double* __restrict__ coef, double* __restrict__ scale,
                                    int* __restrict__ rowlen) {
  const int cnt = *nlist;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
    const int2 it = list[e];
    const int2 ch = chunks[it.x];
    const int L = ch.x;
    const LineInfo me = lines[L];
    const int i = me.lo + ch.y + it.y;
    const int row = me.start + ch.y + it.y;
    int len;
    scale[row] = unscaled_row(g, lines, L, i, row, me, coef + 8 * (size_t)row, len);
    rowlen[row] = len;
  }
}

// Warp per chunk: scaled row ahat_ij = a_ij (s_i s_j), CSR fill in ascending column order
// (-z, -y, -x, self, +x, +y, +z), the regular flag (all six neighbours present and the
// coefficients equal the interior ones) and, for the other rows, the scaled row and 1/diag in
// `coef` for the stencil table.  A simple row whose neighbours all have the interior s_j
// is regular: its scaled coefficients are the interior constants rc[0..3], the same products
// in the same order, so it takes them without FP64 work.
__global__ void assemble_scaled_k(GeomParams g, const LineInfo* __restrict__ lines,
                                  const int2* __restrict__ chunks, int nchunks,
                                  double* __restrict__ coef, const double* __restrict__ scale,
                                  const int* __restrict__ rowptr, int* __restrict__ col,
                                  double* __restrict__ val, unsigned char* __restrict__ regular,
                                  unsigned char* __restrict__ nbmask,
                                  const double* __restrict__ rc) {
  int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (c >= nchunks) return;
  int2 ch = chunks[c];
  int L = ch.x;
  LineInfo me = lines[L];
  int i = me.lo + ch.y + lane;
  if (i > me.hi) return;
  int row = me.start + ch.y + lane;
  int nb[6];
  neighbour_rows(g, lines, L, i, row, me, nb);
  const bool simple = simple_row(g, nb, L);
  const long long sreg = __double_as_longlong(rc[6]);
  bool fast = simple && __double_as_longlong(scale[row]) == sreg;
  if (fast) {
#pragma unroll
    for (int q = 0; q < 6; ++q) fast = fast && __double_as_longlong(scale[nb[q]]) == sreg;
  }
  double sc[7];
  bool reg;
  if (fast) {
    sc[0] = rc[0];
    sc[1] = sc[2] = rc[1];
    sc[3] = sc[4] = rc[2];
    sc[5] = sc[6] = rc[3];
    reg = true;
  } else {
    double* cr = coef + 8 * (size_t)row;
    double ur[7];
    if (simple) {  // the interior unscaled row (not stored by the unscaled pass)
      ur[0] = rc[5];
      ur[1] = ur[2] = -g.cdir[0];
      ur[3] = ur[4] = -g.cdir[1];
      ur[5] = ur[6] = -g.cdir[2];
    } else {
      for (int q = 0; q < 7; ++q) ur[q] = cr[q];
    }
    double si = scale[row];
    sc[0] = ur[0] * (si * si);
    reg = true;
    for (int q = 0; q < 6; ++q) {
      if (nb[q] >= 0) {
        sc[1 + q] = ur[1 + q] * (si * scale[nb[q]]);
      } else {
        sc[1 + q] = 0.0;
        reg = false;
      }
    }
    reg = reg && sc[0] == rc[0] && sc[1] == rc[1] && sc[2] == rc[1] && sc[3] == rc[2] &&
          sc[4] == rc[2] && sc[5] == rc[3] && sc[6] == rc[3];
    for (int q = 0; q < 7; ++q) cr[q] = sc[q];
    // 1 / diag: rc[4] is 1.0 / rc[0], the same division
    cr[7] = __double_as_longlong(sc[0]) == __double_as_longlong(rc[0]) ? rc[4] : 1.0 / sc[0];
  }
  const int order[7] = {4, 2, 0, -1, 1, 3, 5};
  int p = rowptr[row];
  for (int o = 0; o < 7; ++o) {
    int q = order[o];
    if (q < 0) {
      col[p] = row;
      val[p] = sc[0];
      ++p;
    } else if (nb[q] >= 0) {
      col[p] = nb[q];
      val[p] = sc[1 + q];
      ++p;
    }
  }
  regular[row] = reg ? 1 : 0;
  unsigned char mk = 0;
  for (int q = 0; q < 6; ++q) mk |= (unsigned char)((nb[q] >= 0) << q);
  nbmask[row] = mk;
}

// Thread per line: longest run of regular rows -> [rlo, rhi]; table rows = the rest.
__global__ void line_runs_k(LineInfo* lines, int nlines, const unsigned char* regular,
                            int* ntab) {
  int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L >= nlines) return;
  LineInfo l = lines[L];
  int cnt = l.hi - l.lo + 1;
  int best_lo = 0, best_len = 0, cur_lo = 0, cur_len = 0;
  for (int t = 0; t < cnt; ++t) {
    if (regular[l.start + t]) {
      if (cur_len == 0) cur_lo = t;
      ++cur_len;
      if (cur_len > best_len) {
        best_len = cur_len;
        best_lo = cur_lo;
      }
    } else {
      cur_len = 0;
    }
  }
  if (best_len > 0) {
    lines[L].rlo = l.lo + best_lo;
    lines[L].rhi = l.lo + best_lo + best_len - 1;
  } else {
    lines[L].rlo = l.hi + 1;
    lines[L].rhi = l.hi;
  }
  ntab[L] = cnt - best_len;
}

__global__ void set_tstart_k(LineInfo* lines, const int* tstart, int nlines) {
  int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L < nlines) lines[L].tstart = tstart[L];
}

// Thread per line: rows in the regular run.
__global__ void run_counts_k(const LineInfo* __restrict__ lines, int nlines, int* __restrict__ cnt) {
  const int L = blockIdx.x * blockDim.x + threadIdx.x;
  if (L < nlines) cnt[L] = max(0, lines[L].rhi - lines[L].rlo + 1);
}

// Warp per line: (compact row, line) of its regular run, at the line's offset in the list.
__global__ void run_rows_k(const LineInfo* __restrict__ lines, int nlines,
                           const int* __restrict__ rstart, int2* __restrict__ rrow) {
  const int L = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (L >= nlines) return;
  const LineInfo l = lines[L];
  const int first = l.start + (l.rlo - l.lo), cnt = l.rhi - l.rlo + 1;
  for (int k = lane; k < cnt; k += 32) rrow[rstart[L] + k] = make_int2(first + k, L);
}

// Warp per chunk: table rows copy their 7 scaled coefficients and 1/diag.
__global__ void fill_table_k(const LineInfo* __restrict__ lines, const int2* __restrict__ chunks,
                             int nchunks, const double* __restrict__ coef,
                             const unsigned char* __restrict__ regular,
                             const double* __restrict__ rc, double* __restrict__ table,
                             float* __restrict__ table32, int* __restrict__ trow) {
  int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (c >= nchunks) return;
  int2 ch = chunks[c];
  LineInfo me = lines[ch.x];
  int i = me.lo + ch.y + lane;
  if (i > me.hi) return;
  if (i >= me.rlo && i <= me.rhi) return;
  int row = me.start + ch.y + lane;
  int t = me.tstart + (i < me.rlo ? i - me.lo : (me.rlo - me.lo) + (i - me.rhi - 1));
  // a regular row outside the line's longest regular run holds the interior constants
  const bool reg = regular[row] != 0;
  trow[t] = row;
  const double cst[8] = {rc[0], rc[1], rc[1], rc[2], rc[2], rc[3], rc[3], rc[4]};
  for (int q = 0; q < 8; ++q) {
    double v = reg ? cst[q] : coef[8 * (size_t)row + q];
    table[8 * (size_t)t + q] = v;
    table32[8 * (size_t)t + q] = (float)v;
  }
}

// Box -> compact right-hand side and initial guess.
__global__ void gather_k(GeomParams g, const LineInfo* __restrict__ lines,
                         const int2* __restrict__ chunks, int nchunks,
                         const double* __restrict__ scale, const double* __restrict__ rho,
                         const double* __restrict__ phi0, double* __restrict__ bhat,
                         double* __restrict__ xhat) {
  int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (c >= nchunks) return;
  int2 ch = chunks[c];
  int L = ch.x;
  LineInfo me = lines[L];
  int i = me.lo + ch.y + lane;
  if (i > me.hi) return;
  int row = me.start + ch.y + lane;
  int k = L / g.ny;
  size_t box = (size_t)i + (size_t)g.nx * (size_t)L;
  bool gamma2 = (g.zbc == SAAMG_Z_ROBIN) && (k == 0 || k == g.nz - 1);
  double bf = (gamma2 && g.sym) ? 0.5 : 1.0;
  double si = scale[row];
  bhat[row] = si * (bf * rho[box]);
  if (xhat) xhat[row] = phi0 ? phi0[box] / si : 0.0;
}

// Every node of the box: the scaled-back unknown on its line run, 0 elsewhere (one pass that
// writes each element once, so phi may be a box array in device or in pinned host memory).
__global__ void scatter_full_k(const GeomParams g, const LineInfo* __restrict__ lines,
                               const double* __restrict__ scale, const double* __restrict__ xhat,
                               size_t nbox, double* __restrict__ phi) {
  for (size_t b = blockIdx.x * (size_t)blockDim.x + threadIdx.x; b < nbox;
       b += (size_t)gridDim.x * blockDim.x) {
    const int L = (int)(b / (size_t)g.nx);
    const int i = (int)(b - (size_t)L * g.nx);
    const LineInfo me = lines[L];
    double v = 0.0;
    if (i >= me.lo && i <= me.hi) {
      const int row = me.start + (i - me.lo);
      v = scale[row] * xhat[row];
    }
    phi[b] = v;
  }
}

inline int warp_blocks(long long warps) { return (int)((warps * 32 + 255) / 256); }

__global__ void chunk_records_k(const LineInfo* __restrict__ lines, const int4* __restrict__ nbr,
                                const int2* __restrict__ chunks, int nchunks,
                                ChunkRec* __restrict__ crec) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nchunks) return;
  const int2 ch = chunks[c];
  const LineInfo me = lines[ch.x];
  const int4 nb = nbr[ch.x];
  ChunkRec r;
  r.row0 = me.start + ch.y;
  r.tl = me.tstart + ch.y;
  r.a = (short)(me.rlo - me.lo - ch.y);
  r.b = (short)(me.rhi - me.lo - ch.y);
  r.n = min(32, me.hi - me.lo + 1 - ch.y);
  r.ym = nb.x;
  r.yp = nb.y;
  r.zm = nb.z;
  r.zp = nb.w;
  crec[c] = r;
}

}  // namespace

void build_operator_data(const GeomParams& g, cudaStream_t s, OperatorData& op) {
  op.g = g;
  // chunk records hold lane offsets within a line as 16-bit values
  if (g.nx > 30000) fail(SAAMG_EINVAL, "more than 30000 nodes along x");
  long long nl = (long long)g.ny * g.nz;
  if (nl > INT_MAX / 32) fail(SAAMG_EINVAL, "grid too large");
  int nlines = (int)nl;
  op.nlines = nlines;
  op.lines.alloc(nlines, s);
  Buf<int> count, start, nch, chstart, err;
  count.alloc(nlines, s);
  start.alloc(nlines, s);
  nch.alloc(nlines, s);
  chstart.alloc(nlines, s);
  err.alloc(1, s);
  fill_int(err.p, 0, 1, s);
  classify_lines_k<<<warp_blocks(nlines), 256, 0, s>>>(g, nlines, op.lines.p, count.p, err.p);
  SAAMG_LAUNCH();
  int herr = 0;
  d2h_sync(&herr, err.p, sizeof(int), s);
  if (herr) fail(SAAMG_EINVAL, "a lattice line meets the domain in more than one interval");
  long long n = exclusive_scan(count.p, start.p, nlines, s);
  if (n > INT_MAX / 8) fail(SAAMG_EINVAL, "too many unknowns for 32-bit indices");
  op.n = (int)n;
  chunk_counts_k<<<(nlines + 255) / 256, 256, 0, s>>>(count.p, nlines, nch.p);
  SAAMG_LAUNCH();
  long long nchunks = exclusive_scan(nch.p, chstart.p, nlines, s);
  op.nchunks = (int)nchunks;
  op.chunks.alloc(nchunks, s);
  set_start_and_chunks_k<<<(nlines + 255) / 256, 256, 0, s>>>(op.lines.p, start.p, chstart.p,
                                                               count.p, nlines, op.chunks.p);
  SAAMG_LAUNCH();
  op.nbr.alloc(nlines, s);
  line_deltas_k<<<(nlines + 255) / 256, 256, 0, s>>>(op.lines.p, nlines, g.ny, op.nbr.p);
  SAAMG_LAUNCH();
  op.rline.alloc(op.n, s);
  if (op.n > 0) {
    row_lines_k<<<warp_blocks(nchunks), 256, 0, s>>>(op.lines.p, op.chunks.p, op.nchunks,
                                                      op.rline.p);
    SAAMG_LAUNCH();
  }

  Buf<double> rc;
  rc.alloc(8, s);
  regular_consts_k<<<1, 1, 0, s>>>(g, rc.p);
  SAAMG_LAUNCH();
  double hrc[5];
  d2h_sync(hrc, rc.p, sizeof(hrc), s);
  op.c0 = hrc[0];
  op.cx = hrc[1];
  op.cy = hrc[2];
  op.cz = hrc[3];
  op.invd0 = hrc[4];

  op.scale.alloc(op.n, s);
  op.ids.alloc(op.n, s);
  op.regular.alloc(op.n, s);
  op.nbmask.alloc(op.n, s);
  Buf<double> coef;
  coef.alloc((size_t)op.n * 8, s);
  Buf<int> rowlen;
  rowlen.alloc(op.n + 1, s);
  if (op.n > 0) {
    Buf<int2> blist;
    Buf<int> bcount;
    blist.alloc(op.n, s);
    bcount.alloc(1, s);
    fill_int(bcount.p, 0, 1, s);
    assemble_unscaled_k<<<warp_blocks(nchunks), 256, 0, s>>>(g, op.lines.p, op.chunks.p,
                                                              op.nchunks, op.scale.p, rowlen.p,
                                                              op.ids.p, rc.p, blist.p, bcount.p);
    SAAMG_LAUNCH();
    assemble_boundary_k<<<sm_count() * 8, 256, 0, s>>>(g, op.lines.p, op.chunks.p, blist.p, bcount.p,
                                                coef.p, op.scale.p, rowlen.p);
    SAAMG_LAUNCH();
  }
  fill_int(rowlen.p + op.n, 0, 1, s);
  op.A.n = op.A.m = op.n;
  op.A.rowptr.alloc(op.n + 1, s);
  long long nnz = exclusive_scan(rowlen.p, op.A.rowptr.p, op.n + 1, s);
  if (nnz > INT_MAX) fail(SAAMG_EINVAL, "more than 2^31 nonzeros");
  op.nnz = op.A.nnz = nnz;
  op.A.col.alloc(nnz, s);
  op.A.val.alloc(nnz, s);
  if (op.n > 0) {
    assemble_scaled_k<<<warp_blocks(nchunks), 256, 0, s>>>(
        g, op.lines.p, op.chunks.p, op.nchunks, coef.p, op.scale.p, op.A.rowptr.p, op.A.col.p,
        op.A.val.p, op.regular.p, op.nbmask.p, rc.p);
    SAAMG_LAUNCH();
  }
  Buf<int> ntab, tstart;
  ntab.alloc(nlines, s);
  tstart.alloc(nlines, s);
  line_runs_k<<<(nlines + 255) / 256, 256, 0, s>>>(op.lines.p, nlines, op.regular.p, ntab.p);
  SAAMG_LAUNCH();
  long long nt = exclusive_scan(ntab.p, tstart.p, nlines, s);
  op.ntable = (int)nt;
  set_tstart_k<<<(nlines + 255) / 256, 256, 0, s>>>(op.lines.p, tstart.p, nlines);
  SAAMG_LAUNCH();
  op.crec.alloc(op.nchunks, s);
  if (op.nchunks > 0) {
    chunk_records_k<<<(op.nchunks + 255) / 256, 256, 0, s>>>(op.lines.p, op.nbr.p, op.chunks.p,
                                                            op.nchunks, op.crec.p);
    SAAMG_LAUNCH();
  }
  {
    Buf<int> rcnt, rstart;
    rcnt.alloc(nlines, s);
    rstart.alloc(nlines, s);
    run_counts_k<<<(nlines + 255) / 256, 256, 0, s>>>(op.lines.p, nlines, rcnt.p);
    SAAMG_LAUNCH();
    op.nrun = (int)exclusive_scan(rcnt.p, rstart.p, nlines, s);
    // every unknown lies in its line's regular run or is a table row: the FP64 passes apply
    // the two lists and nothing else
    if ((long long)op.nrun + op.ntable != op.n)
      fail(SAAMG_ECUDA, "regular-run and table rows do not cover the unknowns");
    op.rrow.alloc((size_t)op.nrun, s);
    if (op.nrun > 0) {
      run_rows_k<<<warp_blocks(nlines), 256, 0, s>>>(op.lines.p, nlines, rstart.p, op.rrow.p);
      SAAMG_LAUNCH();
    }
  }
  op.table.alloc((size_t)nt * 8, s);
  op.table32.alloc((size_t)nt * 8, s);
  op.trow.alloc((size_t)nt, s);
  if (op.n > 0) {
    fill_table_k<<<warp_blocks(nchunks), 256, 0, s>>>(op.lines.p, op.chunks.p, op.nchunks, coef.p,
                                                       op.regular.p, rc.p, op.table.p,
                                                       op.table32.p, op.trow.p);
    SAAMG_LAUNCH();
  }

  SAAMG_CUDA(cudaStreamSynchronize(s));
}

template <>
StencilDev<double> OperatorData::view<double>() const {
  StencilDev<double> v;
  v.cfg = cfg[0];
  v.lines = lines.p;
  v.nbr = nbr.p;
  v.chunks = chunks.p;
  v.crec = crec.p;
  v.nchunks = nchunks;
  v.rline = rline.p;
  v.n = n;
  v.nx = g.nx;
  v.ny = g.ny;
  v.nz = g.nz;
  v.table = table.p;
  v.trow = trow.p;
  v.ntable = ntable;
  v.rrow = rrow.p;
  v.nrun = nrun;
  v.c0 = c0;
  v.cx = cx;
  v.cy = cy;
  v.cz = cz;
  v.invd0 = invd0;
  return v;
}

template <>
StencilDev<float> OperatorData::view<float>() const {
  StencilDev<float> v;
  v.cfg = cfg[1];
  v.lines = lines.p;
  v.nbr = nbr.p;
  v.chunks = chunks.p;
  v.crec = crec.p;
  v.nchunks = nchunks;
  v.rline = rline.p;
  v.n = n;
  v.nx = g.nx;
  v.ny = g.ny;
  v.nz = g.nz;
  v.table = table32.p;
  v.trow = trow.p;
  v.ntable = ntable;
  v.rrow = rrow.p;
  v.nrun = nrun;
  v.c0 = (float)c0;
  v.cx = (float)cx;
  v.cy = (float)cy;
  v.cz = (float)cz;
  v.invd0 = (float)invd0;
  return v;
}

namespace {

// Derivative of the quadratic through the node value p0 and its neighbours along one axis,
// at distances h (unknown neighbour) or s h (wall point, value 0); written with the same
// operations, in the same order, as the CPU reference (this unit is compiled without FMA
// contraction, so the results agree bit for bit).
__device__ double axis_derivative(double h, bool in_m, bool in_p, double pm, double p0,
                                  double pp, double t, double s) {
  if (in_m && in_p) return (pp - pm) / (2.0 * h);
  if (in_m) return (-(s * s) * pm + (s * s - 1.0) * p0) / (h * s * (1.0 + s));
  if (in_p) return ((t * t) * pp - (t * t - 1.0) * p0) / (h * t * (1.0 + t));
  return p0 * (s - t) / (h * s * t);
}

__device__ __forceinline__ bool line_has(const LineInfo& l, int i) { return i >= l.lo && i <= l.hi; }

// E = -grad phi at unknown (i, line L) of chunk offset row `q` in the box.  Neighbours inside
// Omega_h use their phi; an outside neighbour is replaced by the wall point at the boundary
// fraction with phi = 0; on a Robin end plane the z-derivative is the Robin condition's.
__device__ __forceinline__ void gradient_node(const GeomParams& g,
                                              const LineInfo* __restrict__ lines, int L,
                                              const LineInfo& me, int i,
                                              const double* __restrict__ phi,
                                              double* __restrict__ ex, double* __restrict__ ey,
                                              double* __restrict__ ez) {
  const int j = L % g.ny, k = L / g.ny;
  const size_t sy = (size_t)g.nx, sz = (size_t)g.nx * g.ny;
  const size_t q = (size_t)i + sy * (size_t)j + sz * (size_t)k;
  const double p0 = phi[q];
  const double dist = 0.5 * ((double)(g.nz - 1) * g.h[2]);
  const size_t stride[3] = {1, sy, sz};
  double* E[3] = {ex, ey, ez};
  for (int ax = 0; ax < 3; ++ax) {
    double d;
    if (ax == 2 && g.zbc == SAAMG_Z_ROBIN && (k == 0 || k == g.nz - 1)) {
      d = (k == 0 ? 1.0 : -1.0) * p0 / dist;
    } else {
      // membership from the line records (the classification node_inside produced)
      bool in_m, in_p;
      if (ax == 0) {
        in_m = i - 1 >= me.lo;
        in_p = i + 1 <= me.hi;
      } else {
        const int lstride = ax == 1 ? 1 : g.ny;
        const bool has_m = ax == 1 ? j > 0 : k > 0;
        const bool has_p = ax == 1 ? j < g.ny - 1 : k < g.nz - 1;
        in_m = has_m && line_has(lines[L - lstride], i);
        in_p = has_p && line_has(lines[L + lstride], i);
      }
      const double pm = in_m ? phi[q - stride[ax]] : 0.0;
      const double pp = in_p ? phi[q + stride[ax]] : 0.0;
      const double t = in_m ? 1.0 : boundary_fraction(g, i, j, k, 2 * ax);
      const double s = in_p ? 1.0 : boundary_fraction(g, i, j, k, 2 * ax + 1);
      d = axis_derivative(g.h[ax], in_m, in_p, pm, p0, pp, t, s);
    }
    E[ax][q] = -d;
  }
}

// Warp per chunk, lane per unknown: the nodes whose six neighbours are all unknowns (and not
// on a Robin plane) take central differences here; the others -- a few per cent, where the
// boundary fractions, their divisions and square roots would hold a whole warp on the FP64
// pipe for one lane -- are listed for gradient_boundary_k, one per lane of a full warp.
__global__ void field_gradient_k(GeomParams g, const LineInfo* __restrict__ lines,
                                 const int2* __restrict__ chunks, int nchunks,
                                 const double* __restrict__ phi, double* __restrict__ ex,
                                 double* __restrict__ ey, double* __restrict__ ez,
                                 int2* __restrict__ list, int* __restrict__ nlist) {
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= nchunks) return;  // warp-uniform
  const int2 ch = chunks[c];
  const int L = ch.x;
  const LineInfo me = lines[L];
  const int i = me.lo + ch.y + lane;
  const bool active = i <= me.hi;
  bool inner = false;
  if (active) {
    const int j = L % g.ny, k = L / g.ny;
    const bool robin = g.zbc == SAAMG_Z_ROBIN && (k == 0 || k == g.nz - 1);
    inner = !robin && i - 1 >= me.lo && i + 1 <= me.hi && j > 0 && j < g.ny - 1 && k > 0 &&
            k < g.nz - 1 && line_has(lines[L - 1], i) && line_has(lines[L + 1], i) &&
            line_has(lines[L - g.ny], i) && line_has(lines[L + g.ny], i);
    if (inner) {
      const size_t sy = (size_t)g.nx, sz = (size_t)g.nx * g.ny;
      const size_t q = (size_t)i + sy * (size_t)j + sz * (size_t)k;
      // the central differences of axis_derivative, same operations
      ex[q] = -((phi[q + 1] - phi[q - 1]) / (2.0 * g.h[0]));
      ey[q] = -((phi[q + sy] - phi[q - sy]) / (2.0 * g.h[1]));
      ez[q] = -((phi[q + sz] - phi[q - sz]) / (2.0 * g.h[2]));
    }
  }
  const unsigned need = __ballot_sync(0xffffffffu, active && !inner);
  if (!need) return;
  int base = 0;
  if (lane == 0) base = atomicAdd(nlist, __popc(need));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (active && !inner) list[base + __popc(need & ((1u << lane) - 1u))] = make_int2(c, lane);
}

__global__ void gradient_boundary_k(GeomParams g, const LineInfo* __restrict__ lines,
                                    const int2* __restrict__ chunks,
                                    const int2* __restrict__ list, const int* __restrict__ nlist,
                                    const double* __restrict__ phi, double* __restrict__ ex,
                                    double* __restrict__ ey, double* __restrict__ ez) {
  const int cnt = *nlist;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x) {
    const int2 it = list[e];
    const int2 ch = chunks[it.x];
    const LineInfo me = lines[ch.x];
    gradient_node(g, lines, ch.x, me, me.lo + ch.y + it.y, phi, ex, ey, ez);
  }
}

}  // namespace

void field_gradient(const OperatorData& op, const double* phi, double* ex, double* ey,
                    double* ez, cudaStream_t s) {
  const size_t nbox = (size_t)op.g.nx * op.g.ny * op.g.nz;
  SAAMG_CUDA(cudaMemsetAsync(ex, 0, nbox * sizeof(double), s));
  SAAMG_CUDA(cudaMemsetAsync(ey, 0, nbox * sizeof(double), s));
  SAAMG_CUDA(cudaMemsetAsync(ez, 0, nbox * sizeof(double), s));
  if (op.n == 0) return;
  Buf<int2> list;
  Buf<int> count;
  list.alloc(op.n, s);
  count.alloc(1, s);
  fill_int(count.p, 0, 1, s);
  field_gradient_k<<<warp_blocks(op.nchunks), 256, 0, s>>>(op.g, op.lines.p, op.chunks.p,
                                                            op.nchunks, phi, ex, ey, ez, list.p,
                                                            count.p);
  SAAMG_LAUNCH();
  gradient_boundary_k<<<sm_count() * 8, 256, 0, s>>>(op.g, op.lines.p, op.chunks.p, list.p, count.p,
                                              phi, ex, ey, ez);
  SAAMG_LAUNCH();
}

namespace {

// 1 / a_ii of the scaled operator from the stencil data: the regular-run rows' diagonal is the
// interior constant (1 / diag formed once), the table rows carry their own 1 / diag -- the same
// IEEE divisions of the same diagonals as in the CSR, without a pass over it.
__global__ void invd_fill_k(int n, double invd0, double* __restrict__ invd,
                            float* __restrict__ invd32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    invd[i] = invd0;
    if (invd32) invd32[i] = (float)invd0;
  }
}

__global__ void invd_table_k(int ntable, const int* __restrict__ trow,
                             const double* __restrict__ table, double* __restrict__ invd,
                             float* __restrict__ invd32) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntable) return;
  const double v = table[8 * (size_t)t + 7];
  invd[trow[t]] = v;
  if (invd32) invd32[trow[t]] = (float)v;
}

}  // namespace

void stencil_diag_inverse(const OperatorData& op, double* invd, float* invd32, cudaStream_t s) {
  if (op.n == 0) return;
  const size_t need = ((size_t)op.n + 255) / 256;
  const int blocks = (int)(need < (size_t)sm_count() * 16 ? need : (size_t)sm_count() * 16);
  invd_fill_k<<<blocks, 256, 0, s>>>(op.n, op.invd0, invd, invd32);
  SAAMG_LAUNCH();
  if (op.ntable > 0) {
    invd_table_k<<<(op.ntable + 255) / 256, 256, 0, s>>>(op.ntable, op.trow.p, op.table.p, invd,
                                                          invd32);
    SAAMG_LAUNCH();
  }
}

void gather_rhs(const OperatorData& op, const double* rho, const double* phi0, double* bhat,
                double* xhat, cudaStream_t s) {
  if (op.n == 0) return;
  gather_k<<<warp_blocks(op.nchunks), 256, 0, s>>>(op.g, op.lines.p, op.chunks.p, op.nchunks,
                                                    op.scale.p, rho, phi0, bhat, xhat);
  SAAMG_LAUNCH();
}

void scatter_solution(const OperatorData& op, const double* xhat, double* phi, cudaStream_t s) {
  size_t nbox = (size_t)op.g.nx * op.g.ny * op.g.nz;
  if (nbox == 0) return;
  const size_t need = (nbox + 255) / 256;
  const int blocks = (int)(need < (size_t)sm_count() * 16 ? need : (size_t)sm_count() * 16);
  scatter_full_k<<<blocks, 256, 0, s>>>(op.g, op.lines.p, op.scale.p, xhat, nbox, phi);
  SAAMG_LAUNCH();
}

}  // namespace saamg
