// Pointwise / layout / reduction kernels used by the host driver (aux_kernels.cu).
#pragma once
#include "internal.h"

namespace hom {

template <typename Tf>
cudaError_t launch_mandel_to_kelvin(const double* in, Tf* out, long long M, int nf, cudaStream_t s);
template <typename Tf>
cudaError_t launch_kelvin_to_mandel(const Tf* in, double* out, long long M, int nf, cudaStream_t s);
// Mandel -> Kelvin of FP64 fields [nf][6][M] in place
cudaError_t launch_mandel_to_kelvin_inplace(double* f, long long M, int nf, cudaStream_t s);
// Kelvin -> Mandel of FP64 fields [nf][6][M] in place
cudaError_t launch_kelvin_to_mandel_inplace(double* f, long long M, int nf, cudaStream_t s);
// x += alpha p per load where the load's CG state has an update pending (RhsState::xpend)
template <typename Tf>
cudaError_t launch_cg_flush(Tf* x, const Tf* p, const RhsState* st, long long per, int n, cudaStream_t s);
// x[i] += d[i] for i < n
cudaError_t launch_add_correction(const float* d, double* x, long long n, cudaStream_t s);
// x += a - b
cudaError_t launch_add_difference(const float* a, const float* b, double* x, long long n, cudaStream_t s);
template <typename Ti, typename To>
cudaError_t launch_convert(const Ti* in, To* out, long long n, cudaStream_t s);
template <typename T>
cudaError_t launch_spec_from_std(const double* in, cx<T>* S, const Geo& g, int nf, int ncomp, int basis,
                                 cudaStream_t s);
template <typename T>
cudaError_t launch_spec_to_std(const cx<T>* S, double* out, const Geo& g, int nf, int ncomp, int basis,
                               cudaStream_t s);
// out[rhs * ncomp + c] = mean over voxels of w(phase, c) * (f[rhs][c] + shift[rhs][c]); with
// rve_loads > 0, load rhs reads the phase array and table of RVE rhs / rve_loads
template <typename Tf>
cudaError_t launch_weighted_mean(const Tf* f, int ncomp, int nrhs, const double* shift, const uint8_t* phase,
                                 const double* mat, int wsel, long long M, double* part, int nblk, double* out,
                                 cudaStream_t s, int rve_loads = 0);

}  // namespace hom
