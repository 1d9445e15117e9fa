// Kernels of the FP32 refinement schedule (bicgstab.cu, aux_kernels.cu).
#pragma once
#include "internal.h"

namespace hom {

// r -= eta on the [6][M] Kelvin fields of nrhs loads, then the load's state gets the FP64 norms
// of the new r: rho = <r, r>_C0 (weights c0h on component 0, c0d on 1..5), res_true = res =
// ||r|| / ||b|| (voxel means), restart = 1.  Loads whose state is inactive are skipped.  part /
// cnt hold per-load partial sums and tickets (pstride slots per load, nblk <= pstride).
cudaError_t launch_restart_residual(float* r, const float* eta, double c0h, double c0d, long long M, RhsState* st,
                                    double* part, int pstride, unsigned* cnt, int nrhs, int nblk, cudaStream_t s);

// a -= b elementwise (n values)
cudaError_t launch_sub_inplace(float* a, const float* b, long long n, cudaStream_t s);

}  // namespace hom
