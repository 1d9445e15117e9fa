// Pointwise spectral helpers shared by the z pass (Green contraction) and the equilibrium
// check: the Kelvin basis of symmetric tensors, the product with a wave vector, and the
// discrete wave numbers of the half spectrum.
#pragma once
#include "common.cuh"

namespace hom {

// Kelvin components -> symmetric tensor (t11, t22, t33, t23, t13, t12)
template <typename T>
__device__ __forceinline__ void kelvin_to_tensor(const cx<T>* k, cx<T>* t) {
  const T r3 = (T)0.57735026918962576451, r2 = (T)0.70710678118654752440, r6 = (T)0.40824829046386301637;
  t[0] = k[0] * r3 + k[1] * r2 + k[2] * r6;
  t[1] = k[0] * r3 - k[1] * r2 + k[2] * r6;
  t[2] = k[0] * r3 - k[2] * ((T)2 * r6);
  t[3] = k[3] * r2;
  t[4] = k[4] * r2;
  t[5] = k[5] * r2;
}

// w = t xi for a symmetric tensor t
template <typename T>
__device__ __forceinline__ void tensor_dot_xi(const cx<T>* t, T x1, T x2, T x3, cx<T>& w1, cx<T>& w2, cx<T>& w3) {
  w1 = t[0] * x1 + t[5] * x2 + t[4] * x3;
  w2 = t[5] * x1 + t[1] * x2 + t[3] * x3;
  w3 = t[4] * x1 + t[3] * x2 + t[2] * x3;
}

// integer wave number of DFT index j on an axis of length n, Nyquist -> 0 (discrete derivative)
__device__ __forceinline__ int wave(int j, int n) {
  int k = (j >= (n + 1) / 2) ? j - n : j;
  if ((n & 1) == 0 && 2 * j == n) k = 0;
  return k;
}

// Constants of green_from_w for the reference medium (lam0, mu0), or for c0[rve] when c0 is given:
// c1 = 1 / (2 mu0), c2h = (lam0 + mu0) / (2 mu0 (lam0 + 2 mu0))
template <typename T>
__device__ __forceinline__ void green_consts(const double* c0, int rve, double lam0, double mu0, T& c1, T& c2h) {
  if (c0 != nullptr) {
    lam0 = c0[4 * rve];
    mu0 = c0[4 * rve + 1];
  }
  c1 = (T)(1.0 / (2.0 * mu0));
  c2h = (T)((lam0 + mu0) / (2.0 * mu0 * (lam0 + 2.0 * mu0)));
}

// The vector at which Gamma0_hat is evaluated for the half-spectrum frequency (kx, ky, n):
//  green == 0: the discrete wave vector xi (Nyquist components 0);
//  green == 1: the rotated finite-difference symbol q_j = sin(xi_j h/2) prod_{l != j} cos(xi_l h/2)
//  from gtab = [sin | cos](pi j / N1), j <= N1/2, then [sin | cos](pi j / N2), [sin | cos](pi j / N3),
//  j < N, by DFT index (cos exactly 0 at N/2).  Indices past N/2 flip sin and cos of an axis
//  together, which flips q as a whole; Gamma0_hat is even, so the operator is unchanged.
template <typename T>
__device__ __forceinline__ void wave_vector(const Geo& g, int green, const double* gtab, int kx, int ky, int n,
                                            T& x1, T& x2, T& x3) {
  if (green == 0) {
    x1 = (T)((kx == g.h ? 0 : kx) * g.xs1);
    x2 = (T)(wave(ky, g.n2) * g.xs2);
    x3 = (T)(wave(n, g.n3) * g.xs3);
  } else {
    const double* t2 = gtab + 2 * (g.h + 1);
    const double* t3 = t2 + 2 * g.n2;
    const double s1 = __ldg(gtab + kx), c1 = __ldg(gtab + g.h + 1 + kx);
    const double s2 = __ldg(t2 + ky), c2 = __ldg(t2 + g.n2 + ky);
    const double s3 = __ldg(t3 + n), c3 = __ldg(t3 + g.n3 + n);
    x1 = (T)(s1 * c2 * c3);
    x2 = (T)(c1 * s2 * c3);
    x3 = (T)(c1 * c2 * s3);
  }
}

// eta_hat = -Gamma0_hat(xi) : tau_hat in Kelvin components, given w = tau_hat xi.
// Gamma0_hat : tau_hat = v (x) xi + xi (x) v with
// v = w / (2 mu0 |xi|^2) - (lam0 + mu0) / (2 mu0 (lam0 + 2 mu0)) (xi . w) xi / |xi|^4,
// the four-index formula of Sec. 2 contracted with a symmetric tau_hat.
template <typename T>
__device__ __forceinline__ void green_from_w(cx<T>* k, cx<T> w1, cx<T> w2, cx<T> w3, T x1, T x2, T x3, T c1,
                                             T c2h, T scale) {
  const T r3 = (T)0.57735026918962576451, r2 = (T)0.70710678118654752440,
          r6 = (T)0.40824829046386301637, s2 = (T)1.41421356237309504880;
  const T q = x1 * x1 + x2 * x2 + x3 * x3;
  if (q == (T)0) {
#pragma unroll
    for (int i = 0; i < 6; ++i) k[i] = mk<T>(0, 0);
    return;
  }
  const cx<T> s = w1 * x1 + w2 * x2 + w3 * x3;
  const T iq = (T)1 / q;
  const T a1 = c1 * iq * scale;
  const T a2 = c2h * iq * iq * scale;
  const cx<T> v1 = w1 * a1 - s * (a2 * x1);
  const cx<T> v2 = w2 * a1 - s * (a2 * x2);
  const cx<T> v3 = w3 * a1 - s * (a2 * x3);
  const cx<T> e11 = v1 * ((T)-2 * x1), e22 = v2 * ((T)-2 * x2), e33 = v3 * ((T)-2 * x3);
  k[0] = (e11 + e22 + e33) * r3;
  k[1] = (e11 - e22) * r2;
  k[2] = (e11 + e22 - e33 * (T)2) * r6;
  k[3] = (v2 * x3 + v3 * x2) * (-s2);
  k[4] = (v1 * x3 + v3 * x1) * (-s2);
  k[5] = (v1 * x2 + v2 * x1) * (-s2);
}

}  // namespace hom
