// Equilibrium check of stress spectra (equilibrium.cu): how far a stress field is from the
// balance of momentum div sigma = 0 (Sec. 2, Eq. eq_of_motion), measured spectrally.
#pragma once
#include "internal.h"

namespace hom {

// CTAs per load of the partial-sum kernel on this grid (at most 2 x 152).
int equilibrium_blocks(const Geo& g);

// For each of the nrhs 6-component Kelvin stress spectra at S (unnormalised forward DFT, half
// spectrum in the layout of the z pass), the weighted sum over the half spectrum of
// |xi . sigma_hat(xi)|^2 and of |sigma_hat(xi)|^2 (weight 2 for the columns 0 < kx < N1/2,
// whose conjugates are not stored), one pair of partials per CTA, written to
// part[((rhs0 + l) * 2 + q) * nblk + b] (q = 0, 1); and the zero-frequency coefficients
// sigma_hat(0) to s0[(rhs0 + l) * 6 + i].
template <typename T>
cudaError_t launch_equilibrium_partials(const cx<T>* S, const Geo& g, int nrhs, int rhs0, double* part, double* s0,
                                        int nblk, cudaStream_t s);

// out[l] = sqrt(sum of part[l][0][*]) / |s0[l]|, or that square root / M where the mean vanishes
// up to rounding (|s0[l]| <= 1e-12 sqrt(sum of part[l][1][*])), for l < nrhs; the partials are
// summed in a fixed order.
cudaError_t launch_equilibrium_finish(const double* part, const double* s0, int nrhs, int nblk, long long M,
                                      double* out, cudaStream_t s);

}  // namespace hom
