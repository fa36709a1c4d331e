// Particle-grid transfers around the solve of a PIC step (internal).
#pragma once

#include "common.cuh"

namespace saamg {

// rho (box, overwritten) = cloud-in-cell density of the particles (x, y, z, q of length np):
// each particle adds (q / V) times the product of its three hat weights to the 8 nodes
// around it; nodes outside the box are dropped.  NaN everywhere when a charge is not finite.
void deposit_cic(const saamg_grid& grid, int np, const double* x, const double* y,
                 const double* z, const double* q, double* rho, cudaStream_t s);

// E at the particles from the nodal field (ex, ey, ez box arrays), same weights.
void gather_cic(const saamg_grid& grid, const double* ex, const double* ey, const double* ez,
                int np, const double* x, const double* y, const double* z, double* epx,
                double* epy, double* epz, cudaStream_t s);

}  // namespace saamg
