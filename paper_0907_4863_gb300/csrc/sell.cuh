// Sliced ELLPACK (SELL-32-sigma) copies of the coarse-level operators A_l (l >= 1), used by
// the V-cycle smoother (internal).  The AMG setup and the transfers keep working on CSR.
//
// Rows are sorted by decreasing length inside windows of kSellWindow rows (stable: equal
// lengths keep their order) and cut into slices of 32 consecutive sorted rows; slice s
// stores its entries column-major, entry k of the slice's lane l at soff[s] + 32 k + l, with
// width (soff[s+1] - soff[s]) / 32 = the longest row of the slice.  A shorter row is padded
// with zero values at its own last column, so the padding adds exact zeros and never
// reads a value the row does not already read.  When every column lies within 32767 of its
// row (aggregates are numbered by their root's lattice index, so a coarse row's neighbours
// are close to it), the columns are stored as 16-bit offsets from the row: 2 bytes per entry
// instead of 4.  One thread owns one row and sums its
// entries in column order; every load of the entry arrays is one contiguous 128-byte
// (float/int) or 256-byte (double) warp access.
#pragma once

#include "csr.cuh"

namespace saamg {

constexpr int kSellWindow = 512;
// smallest level stored as SELL: below it one thread per row leaves most of the GPU idle and
// the CSR kernel with wide row groups is faster
constexpr int kSellMinRows = 100000;

struct DevSell {
  int n = 0, m = 0, nslices = 0;
  long long nnz = 0;            // entries of the matrix
  long long nent = 0;           // stored entries, padding included
  Buf<int> perm;                // sorted position -> row
  Buf<int> soff;                // nslices + 1 slice offsets
  Buf<int> col;                 // column of each stored entry, or (index_bytes == 2) ...
  Buf<short> dcol;              // ... its offset from the row, when every offset fits 16 bits
  int index_bytes = 4;
  Buf<double> val;              // FP64 values (FP64 V-cycle)
  Buf<float> val32;             // FP32 values (mixed precision)
  Buf<__nv_bfloat16> val16;     // BF16 values (mixed precision, BF16 storage)
  size_t bytes() const {
    return perm.bytes() + soff.bytes() + col.bytes() + dcol.bytes() + val.bytes() +
           val32.bytes() + val16.bytes();
  }
};

// S = A in SELL form with the value arrays requested (FP64 / FP32 / BF16 copies of A.val).
void sell_from_csr(const DevCsr& A, DevSell& S, bool f64, bool f32, bool bf16, cudaStream_t s);
// The same for an A whose pattern is that of the matrix `like` holds (a reused hierarchy's
// level): like's layout is copied and only the value arrays are filled.
void sell_like(const DevCsr& A, const DevSell& like, DevSell& S, bool f64, bool f32, bool bf16,
               cudaStream_t s);

// The CSR modes of csr_apply (CSR_CHEB with c1 == 0 does not read d; CSR_SPMV_DINV_DOT
// writes kRedBlocks partial sums of y.y and takes the scale of x from *xscale, 1 if NULL).
template <class TV, class TM>
void sell_apply(int mode, const DevSell& S, const TM* val, const TV* x, TV* y, const TV* b,
                TV* d, const TV* invd, TV c1, TV c2, cudaStream_t s, int kclass,
                double* partials = nullptr, const double* xscale = nullptr);

}  // namespace saamg
