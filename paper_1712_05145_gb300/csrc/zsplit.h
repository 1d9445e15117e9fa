// Split z pass for deep grids (zpass.cu).  When the fused z pass can only take tiles narrower
// than a 32-byte sector (6 components x N3 complex values per column fill a CTA, e.g. N3 = 512),
// the Lippmann-Schwinger step runs its z stage as three passes instead: the z FFT one component
// at a time (16-column tiles, 128-byte runs), the Green contraction as a coalesced pointwise pass
// over every frequency, and the inverse z FFT one component at a time.
#pragma once
#include "internal.h"

namespace hom {

// eta_hat = -Gamma0_hat(xi) : tau_hat (times a.scale), eta_hat(0) = 0, in place on the 6-component
// spectra of nrhs loads starting at a.S; loads whose a.st entry is inactive are skipped.
template <typename T>
cudaError_t launch_zgreen(const ZArgs<T>& a, int nrhs, cudaStream_t s);

}  // namespace hom
