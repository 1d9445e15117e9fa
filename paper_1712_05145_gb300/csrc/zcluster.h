// Cluster z pass of the Lippmann-Schwinger step (zcluster.cu): the z FFT, the Green contraction
// eta_hat = -Gamma0_hat(xi) : tau_hat (Sec. 2) and the inverse z FFT of a tile of spectrum
// columns, run by a cluster of six CTAs, one per Kelvin component, that meet in distributed
// shared memory for the contraction.
#pragma once
#include "internal.h"

namespace hom {

// Tiling of the cluster z pass for `a.g` and transform type T: fills tc_log2, ntiles, nthr and
// fd_in (division by the tile width).  force_lg >= 0 asks for tiles of 2^force_lg columns if
// they fit.  Returns false when no tile fits (then the single-CTA z pass runs).
template <typename T>
bool zcluster_tiling(ZArgs<T>& a, int force_lg = -1);

// Whether tiles of 2^lg columns fit the cluster z pass on this grid for element size elem.
bool zcluster_tile_fits(const Geo& g, size_t elem, int lg);

// Z_GAMMA on the 6-component spectra of nrhs loads starting at a.S (tiling from zcluster_tiling);
// loads whose a.st entry is inactive are skipped.
template <typename T>
cudaError_t launch_zcluster(const ZArgs<T>& a, int nrhs, cudaStream_t s);

// The TMA variant (FP32): the same tile work, with each CTA's tile loaded by TMA tensor loads that
// complete on an mbarrier and written back by TMA tensor stores.  ztma_fits: whether tiles of 2^lg
// columns can run it on this grid (tiling from zcluster_tiling with that width).  Its bounded wait
// sets bits in a.err when it gives up.
bool ztma_fits(const Geo& g, int lg);
cudaError_t launch_zcluster_tma(const ZArgs<float>& a, int nrhs, cudaStream_t s);

}  // namespace hom
