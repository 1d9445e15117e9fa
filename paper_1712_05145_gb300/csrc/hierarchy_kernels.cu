// Pointwise right-hand-side builders of the generalized problems of order alpha
// (Sec. 3 of arXiv:1712.05145: polarization p_alpha and body force g_alpha of the
// Definition, with the separation ansatz u_alpha = X_alpha(y) . grad^(alpha-1) E(Y)),
// and stress fields sigma = C : (E + eps) (Sec. 2, Eq. Hookes_law).
#include "hierarchy.h"

namespace hom {

#define R3 0.57735026918962576451
#define R2 0.70710678118654752440
#define R6 0.40824829046386301637
#define S2 1.41421356237309504880

// Kelvin <-> Cartesian symmetric tensor t = (t11, t22, t33, t23, t13, t12)
__device__ __forceinline__ void k2t(const double* k, double* t) {
  t[0] = k[0] * R3 + k[1] * R2 + k[2] * R6;
  t[1] = k[0] * R3 - k[1] * R2 + k[2] * R6;
  t[2] = k[0] * R3 - 2.0 * k[2] * R6;
  t[3] = k[3] * R2;
  t[4] = k[4] * R2;
  t[5] = k[5] * R2;
}
__device__ __forceinline__ void t2k(const double* t, double* k) {
  k[0] = (t[0] + t[1] + t[2]) * R3;
  k[1] = (t[0] - t[1]) * R2;
  k[2] = (t[0] + t[1] - 2.0 * t[2]) * R6;
  k[3] = t[3] * S2;
  k[4] = t[4] * S2;
  k[5] = t[5] * S2;
}
// component (i, j) of a symmetric tensor stored as (11, 22, 33, 23, 13, 12)
__device__ __forceinline__ int tidx(int i, int j) {
  if (i == j) return i;
  const int s = i + j;  // (1,2) -> 3, (0,2) -> 2 -> 4, (0,1) -> 1 -> 5
  return s == 3 ? 3 : (s == 2 ? 4 : 5);
}
// adds w * sym(v (x) e_k) to t
__device__ __forceinline__ void add_sym_vec_dir(double* t, const double* v, int k, double w) {
  for (int i = 0; i < 3; ++i) {
    if (i == k) t[i] += w * v[i];
    else t[tidx(i, k)] += 0.5 * w * v[i];
  }
}

template <typename Tf>
__global__ void rhs_pointwise_kernel(int order, int nload, const UnitMap map, const RecTable rec,
                                     const Tf* __restrict__ disp,
                                     const Tf* __restrict__ eps,
                                     const Tf* __restrict__ pprev, const double* __restrict__ EK,
                                     const uint8_t* __restrict__ phase, const double* __restrict__ mat, long long M,
                                     Tf* __restrict__ out9, Tf* __restrict__ pf) {
  const long long total = (long long)nload * M;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int L = (int)(id / M);
    const long long v = id - (long long)L * M;
    const int ph = phase[v];
    const double ch = mat[ph * 4 + 2], cd = mat[ph * 4 + 3];
    double t[6] = {0, 0, 0, 0, 0, 0}, g[3];
    if (order == 1) {
      const int u = map.unit[L], k = u % 3, A = map.a0[u / 3];
      double chi[3];
      for (int i = 0; i < 3; ++i) chi[i] = (double)disp[((long long)A * 3 + i) * M + v];
      add_sym_vec_dir(t, chi, k, 1.0);
      double sk[6], st[6];
      for (int c = 0; c < 6; ++c) sk[c] = (c == 0 ? ch : cd) * ((double)eps[((long long)A * 6 + c) * M + v] + EK[A * 6 + c]);
      k2t(sk, st);
      for (int i = 0; i < 3; ++i) g[i] = st[tidx(i, k)];
    } else {
      const int A = L / rec.nK, K = L - A * rec.nK;
      g[0] = g[1] = g[2] = 0.0;
      for (int q = 0; q < rec.nterm[K]; ++q) {
        const int d = rec.dir[K][q];
        const long long Ls = (long long)A * rec.nKprev + rec.src[K][q];
        double u[3], sq[6], tq[6];
        for (int i = 0; i < 3; ++i) u[i] = (double)disp[(Ls * 3 + i) * M + v];
        add_sym_vec_dir(t, u, d, 1.0);
        for (int c = 0; c < 6; ++c)
          sq[c] = (c == 0 ? ch : cd) * (double)eps[(Ls * 6 + c) * M + v] + (double)pprev[(Ls * 6 + c) * M + v];
        k2t(sq, tq);
        for (int i = 0; i < 3; ++i) g[i] += tq[tidx(i, d)];
      }
    }
    double kk[6];
    t2k(t, kk);
    for (int c = 0; c < 6; ++c) {
      const Tf pc = (Tf)((c == 0 ? ch : cd) * kk[c]);
      out9[((long long)L * 9 + c) * M + v] = pc;
      pf[((long long)L * 6 + c) * M + v] = pc;
    }
    for (int i = 0; i < 3; ++i) out9[((long long)L * 9 + 6 + i) * M + v] = (Tf)g[i];
  }
}

template <typename Tf>
__global__ void stress_kernel(const Tf* __restrict__ eps, const double* __restrict__ EK, const Tf* __restrict__ pf,
                              const uint8_t* __restrict__ phase, const double* __restrict__ mat, long long M,
                              double* __restrict__ out) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < M; v += (long long)gridDim.x * blockDim.x) {
    const int ph = phase[v];
    const double ch = mat[ph * 4 + 2], cd = mat[ph * 4 + 3];
    double k[6], m[6];
    for (int c = 0; c < 6; ++c) {
      double e = (double)eps[(long long)c * M + v];
      if (EK) e += EK[c];
      k[c] = (c == 0 ? ch : cd) * e;
      if (pf) k[c] += (double)pf[(long long)c * M + v];
    }
    k2t(k, m);  // Cartesian t, then Mandel = (t11, t22, t33, sqrt2 t23, sqrt2 t13, sqrt2 t12)
    out[v] = m[0];
    out[M + v] = m[1];
    out[2 * M + v] = m[2];
    out[3 * M + v] = m[3] * S2;
    out[4 * M + v] = m[4] * S2;
    out[5 * M + v] = m[5] * S2;
  }
}

static int blocks_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152LL * 32) b = 152LL * 32;
  return (int)(b < 1 ? 1 : b);
}

template <typename Tf>
cudaError_t launch_rhs_pointwise(int order, int nload, const UnitMap& map, const RecTable& rec, const Tf* disp,
                                 const Tf* eps, const Tf* pprev, const double* EK, const uint8_t* phase,
                                 const double* mat, long long M, Tf* out9, Tf* pf, cudaStream_t s) {
  if (order >= 2 && (rec.nK < 1 || rec.nK > kMaxMultisets || (long long)nload != 6LL * rec.nK))
    return cudaErrorInvalidValue;
  count_launch();
  rhs_pointwise_kernel<Tf><<<blocks_for((long long)nload * M), 256, 0, s>>>(order, nload, map, rec, disp, eps,
                                                                             pprev, EK, phase, mat, M, out9, pf);
  return cudaGetLastError();
}

__global__ void combine_loads_kernel(const double* __restrict__ in, int nin, const double* __restrict__ W, int nout,
                                     long long per, double* __restrict__ out) {
  const long long total = (long long)nout * per;
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(id / per);
    const long long i = id - (long long)l * per;
    double acc = 0.0;
    for (int u = 0; u < nin; ++u) acc += W[l * nin + u] * in[(long long)u * per + i];
    out[id] = acc;
  }
}

cudaError_t launch_combine_loads(const double* in, int nin, const double* W, int nout, long long per, double* out,
                                 cudaStream_t s) {
  count_launch();
  combine_loads_kernel<<<blocks_for((long long)nout * per), 256, 0, s>>>(in, nin, W, nout, per, out);
  return cudaGetLastError();
}

template <typename Tf>
cudaError_t launch_stress_field(const Tf* eps, const double* EK, const Tf* pf, const uint8_t* phase,
                                const double* mat, long long M, double* out, cudaStream_t s) {
  count_launch();
  stress_kernel<Tf><<<blocks_for(M), 256, 0, s>>>(eps, EK, pf, phase, mat, M, out);
  return cudaGetLastError();
}

template cudaError_t launch_rhs_pointwise<float>(int, int, const UnitMap&, const RecTable&, const float*,
                                                 const float*, const float*, const double*, const uint8_t*,
                                                 const double*, long long, float*, float*, cudaStream_t);
template cudaError_t launch_rhs_pointwise<double>(int, int, const UnitMap&, const RecTable&, const double*,
                                                  const double*, const double*, const double*, const uint8_t*,
                                                  const double*, long long, double*, double*, cudaStream_t);
template cudaError_t launch_stress_field<float>(const float*, const double*, const float*, const uint8_t*,
                                                const double*, long long, double*, cudaStream_t);
template cudaError_t launch_stress_field<double>(const double*, const double*, const double*, const uint8_t*,
                                                 const double*, long long, double*, cudaStream_t);

}  // namespace hom
