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
