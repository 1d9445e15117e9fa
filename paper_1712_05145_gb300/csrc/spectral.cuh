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

}  // namespace hom
