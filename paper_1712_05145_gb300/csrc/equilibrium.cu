// Equilibrium check: e = sqrt(<|div sigma|^2>) / |<sigma>| with (div sigma)_hat = i xi . sigma_hat
// on the discrete wave vectors (Nyquist components 0).  By Parseval on the unnormalised DFT,
// <|div sigma|^2> = sum_xi |xi . sigma_hat|^2 / M^2 and <sigma> = sigma_hat(0) / M, so
// e = sqrt(sum_xi |xi . sigma_hat|^2) / |sigma_hat(0)|.  The sum runs over the stored half
// spectrum; a column 0 < kx < N1/2 stands for itself and its conjugate (weight 2), the columns
// kx = 0 and kx = N1/2 hold both members of every conjugate pair (weight 1).  Where the mean
// vanishes up to rounding, |sigma_hat(0)| <= 1e-12 sqrt(sum_xi |sigma_hat|^2) (a zero load),
// e = sqrt(<|div sigma|^2>) = sqrt(sum_xi |xi . sigma_hat|^2) / M instead.
#include "equilibrium.h"
#include "spectral.cuh"

namespace hom {

namespace {
constexpr int kEqThreads = 256;
constexpr double kZeroMean = 1e-12;

template <typename T>
__device__ __forceinline__ cx<double> to_dcx(cx<T> v) {
  return mk<double>((double)v.re, (double)v.im);
}
__device__ __forceinline__ double abs2(cx<double> v) { return v.re * v.re + v.im * v.im; }
}  // namespace

template <typename T>
__global__ void __launch_bounds__(kEqThreads) equilibrium_partial_kernel(const cx<T>* S, const Geo g, int rhs0,
                                                                         double* part, double* s0) {
  __shared__ double sh[64];
  const int lrhs = blockIdx.y, nblk = gridDim.x;
  const long long per = (long long)g.n3 * g.plane_c;   // frequencies of one component
  const long long nmain = (long long)g.n2 * g.h;
  const cx<T>* base = S + (long long)lrhs * 6 * per;
  double acc = 0.0, acc2 = 0.0;
  for (long long q = blockIdx.x * (long long)kEqThreads + threadIdx.x; q < per; q += (long long)nblk * kEqThreads) {
    const int n = (int)(q / g.plane_c);
    const long long f = q - (long long)n * g.plane_c;
    int kx, ky;
    if (f < nmain) { ky = (int)g.fd_h.div((unsigned)f); kx = (int)f - ky * g.h; }
    else { ky = (int)(f - nmain); kx = g.h; }
    cx<double> k[6], t[6], w1, w2, w3;
#pragma unroll
    for (int i = 0; i < 6; ++i) k[i] = to_dcx<T>(base[i * per + q]);
    if (q == 0) {
#pragma unroll
      for (int i = 0; i < 6; ++i) s0[(rhs0 + lrhs) * 6 + i] = k[i].re;
    }
    const double x1 = (double)(kx == g.h ? 0 : kx) * g.xs1;
    const double x2 = (double)wave(ky, g.n2) * g.xs2;
    const double x3 = (double)wave(n, g.n3) * g.xs3;
    kelvin_to_tensor<double>(k, t);
    tensor_dot_xi<double>(t, x1, x2, x3, w1, w2, w3);
    const double wgt = (kx == 0 || kx == g.h) ? 1.0 : 2.0;
    acc += wgt * (abs2(w1) + abs2(w2) + abs2(w3));
    acc2 += wgt * (abs2(k[0]) + abs2(k[1]) + abs2(k[2]) + abs2(k[3]) + abs2(k[4]) + abs2(k[5]));
  }
  double v[2] = {acc, acc2};
  block_sum_f64<2>(v, sh);
  if (threadIdx.x == 0) {
    part[(long long)(rhs0 + lrhs) * 2 * nblk + blockIdx.x] = v[0];
    part[((long long)(rhs0 + lrhs) * 2 + 1) * nblk + blockIdx.x] = v[1];
  }
}

__global__ void __launch_bounds__(kEqThreads) equilibrium_finish_kernel(const double* part, const double* s0, int nblk,
                                                                        double invM, double* out) {
  __shared__ double sh[64];
  const int l = blockIdx.x;
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < nblk; i += kEqThreads) {
    v[0] += part[(long long)l * 2 * nblk + i];
    v[1] += part[((long long)l * 2 + 1) * nblk + i];
  }
  block_sum_f64<2>(v, sh);
  if (threadIdx.x == 0) {
    double d2 = 0.0;
    for (int i = 0; i < 6; ++i) d2 += s0[l * 6 + i] * s0[l * 6 + i];
    const double num = sqrt(v[0]), den = sqrt(d2);
    out[l] = den > kZeroMean * sqrt(v[1]) ? num / den : num * invM;
  }
}

int equilibrium_blocks(const Geo& g) {
  const long long per = (long long)g.n3 * g.plane_c;
  const long long b = (per + kEqThreads - 1) / kEqThreads;
  return (int)(b < 1 ? 1 : (b > 2 * 152 ? 2 * 152 : b));
}

template <typename T>
cudaError_t launch_equilibrium_partials(const cx<T>* S, const Geo& g, int nrhs, int rhs0, double* part, double* s0,
                                        int nblk, cudaStream_t s) {
  if (nrhs < 1 || nrhs > 65535 || nblk < 1) return cudaErrorInvalidValue;
  count_launch();
  equilibrium_partial_kernel<T><<<dim3(nblk, nrhs), kEqThreads, 0, s>>>(S, g, rhs0, part, s0);
  return cudaGetLastError();
}
template cudaError_t launch_equilibrium_partials<double>(const cx<double>*, const Geo&, int, int, double*, double*,
                                                         int, cudaStream_t);
template cudaError_t launch_equilibrium_partials<df64>(const cx<df64>*, const Geo&, int, int, double*, double*, int,
                                                       cudaStream_t);

cudaError_t launch_equilibrium_finish(const double* part, const double* s0, int nrhs, int nblk, long long M,
                                      double* out, cudaStream_t s) {
  if (nrhs < 1 || nblk < 1 || M < 1) return cudaErrorInvalidValue;
  count_launch();
  equilibrium_finish_kernel<<<nrhs, kEqThreads, 0, s>>>(part, s0, nblk, 1.0 / (double)M, out);
  return cudaGetLastError();
}

}  // namespace hom
