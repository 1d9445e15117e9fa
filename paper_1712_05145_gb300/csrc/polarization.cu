// Pointwise steps of the polarization scheme (see polarization.h).  One grid-stride kernel over
// the voxels of each load; the six Kelvin components of a voxel share its phase, whose W
// eigenvalues sit in shared memory.  Sums are formed per thread in the field precision and
// reduced in FP64 with a last-CTA ticket, as in the BiCGSTAB updates.
#include "ls_common.cuh"
#include "polarization.h"

namespace hom {

template <typename Tf, int STEP>
__global__ void __launch_bounds__(256) polar_kernel(const PolarArgs<Tf> a) {
  __shared__ double sh[32 + 2];
  __shared__ Tf w[2 * 256];
  __shared__ int flag;
  const int rhs = a.rhs0 + blockIdx.y;
  RhsState& st = a.st[rhs];
  if (STEP == PO_UPDATE && st.active == 0) return;
  for (int i = threadIdx.x; i < a.n_phase; i += blockDim.x) {
    w[i] = a.wt[i * 4 + 2];               // hydrostatic Kelvin eigenvalue of W
    w[a.n_phase + i] = a.wt[i * 4 + 3];   // deviatoric
  }
  __syncthreads();
  const long long M = a.M, off = (long long)rhs * 6 * M;
  const Tf g = (Tf)a.relax, g1 = (Tf)1 - g;
  Tf q = 0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < M; v += (long long)gridDim.x * blockDim.x) {
    const int ph = a.phase[v];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      const long long i = off + c * M + v;
      const Tf wc = w[(c == 0 ? 0 : a.n_phase) + ph];
      if (STEP == PO_UPDATE) {
        const Tf x0 = a.x[i];
        const Tf xn = g1 * x0 + g * (a.r[i] + wc * x0 + (Tf)2 * a.eta[i]);
        a.x[i] = xn;
        const Tf dd = ((Tf)1 - wc) * (xn - x0);
        q += dd * dd;
      } else {
        a.d[i] += ((Tf)1 - wc) * a.x[i];
      }
    }
  }
  if (STEP == PO_FINISH) return;
  double v[1] = {(double)q};
  block_sum_f64<1>(v, sh);
  if (publish_and_collect<1>(v, a.part + (long long)rhs * 2 * a.pstride, a.cnt + rhs, gridDim.x, blockIdx.x, sh,
                             &flag)) {
    if (threadIdx.x == 0) {
      const double d2 = v[0] / (double)M;
      st.res = (st.b2 > 0.0) ? sqrt(d2 / st.b2) : 0.0;
      st.iter += 1;
      if (!isfinite(st.res)) { st.status = 2; st.active = 0; }
      else if (st.res < st.tol) st.active = 0;
      else if (st.iter >= st.max_iter) { st.active = 0; st.status = 1; }
    }
  }
}

template <typename Tf>
cudaError_t launch_polar(int step, const PolarArgs<Tf>& a, int nrhs, int nblk, cudaStream_t s) {
  if (nblk < 1 || nblk > a.pstride || nrhs < 1 || a.n_phase < 1 || a.n_phase > 256) return cudaErrorInvalidValue;
  dim3 grid(nblk, nrhs);
  count_launch();
  switch (step) {
    case PO_UPDATE: polar_kernel<Tf, PO_UPDATE><<<grid, 256, 0, s>>>(a); break;
    case PO_FINISH: polar_kernel<Tf, PO_FINISH><<<grid, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_polar<float>(int, const PolarArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_polar<double>(int, const PolarArgs<double>&, int, int, cudaStream_t);

}  // namespace hom
