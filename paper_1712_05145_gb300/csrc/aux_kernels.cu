// Pointwise and reduction kernels around the Lippmann-Schwinger step: basis changes
// between the public Mandel vectors and the internal Kelvin components, layout changes
// of spectra, and FP64 voxel means of stresses (the averages behind C_eff, Sec. 2).
#include "aux.h"

namespace hom {

#define R3 0.57735026918962576451
#define R2 0.70710678118654752440
#define R6 0.40824829046386301637

// ---- Mandel <-> Kelvin on real fields [nf][6][M] ------------------------------------
template <typename Tf>
__global__ void mandel_to_kelvin_kernel(const double* __restrict__ in, Tf* __restrict__ out,
                                        long long M, int nf) {
  const long long total = (long long)nf * M;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / M, v = i - f * M;
    const double* a = in + f * 6 * M + v;
    Tf* b = out + f * 6 * M + v;
    const double m0 = a[0], m1 = a[M], m2 = a[2 * M];
    b[0] = (Tf)((m0 + m1 + m2) * R3);
    b[M] = (Tf)((m0 - m1) * R2);
    b[2 * M] = (Tf)((m0 + m1 - 2.0 * m2) * R6);
    b[3 * M] = (Tf)a[3 * M];
    b[4 * M] = (Tf)a[4 * M];
    b[5 * M] = (Tf)a[5 * M];
  }
}

template <typename Tf>
__global__ void kelvin_to_mandel_kernel(const Tf* __restrict__ in, double* __restrict__ out,
                                        long long M, int nf) {
  const long long total = (long long)nf * M;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / M, v = i - f * M;
    const Tf* a = in + f * 6 * M + v;
    double* b = out + f * 6 * M + v;
    const double k0 = (double)a[0], k1 = (double)a[M], k2 = (double)a[2 * M];
    b[0] = k0 * R3 + k1 * R2 + k2 * R6;
    b[M] = k0 * R3 - k1 * R2 + k2 * R6;
    b[2 * M] = k0 * R3 - 2.0 * k2 * R6;
    b[3 * M] = (double)a[3 * M];
    b[4 * M] = (double)a[4 * M];
    b[5 * M] = (double)a[5 * M];
  }
}

// Kelvin -> Mandel of FP64 fields in place: each thread reads a voxel's 6 components before
// writing them back (no restrict: input and output alias)
__global__ void kelvin_to_mandel_inplace_kernel(double* f, long long M, int nf) {
  const long long total = (long long)nf * M;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = i / M, v = i - q * M;
    double* a = f + q * 6 * M + v;
    const double k0 = a[0], k1 = a[M], k2 = a[2 * M];
    a[0] = k0 * R3 + k1 * R2 + k2 * R6;
    a[M] = k0 * R3 - k1 * R2 + k2 * R6;
    a[2 * M] = k0 * R3 - 2.0 * k2 * R6;
  }
}

// Mandel -> Kelvin of FP64 fields in place (input and output alias, as above)
__global__ void mandel_to_kelvin_inplace_kernel(double* f, long long M, int nf) {
  const long long total = (long long)nf * M;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long q = i / M, v = i - q * M;
    double* a = f + q * 6 * M + v;
    const double m0 = a[0], m1 = a[M], m2 = a[2 * M];
    a[0] = (m0 + m1 + m2) * R3;
    a[M] = (m0 - m1) * R2;
    a[2 * M] = (m0 + m1 - 2.0 * m2) * R6;
  }
}

// x += alpha p for each load whose CG state has an update of x pending (the update the next
// forward pass would otherwise apply), fields [n][per]
template <typename Tf>
__global__ void cg_flush_kernel(Tf* __restrict__ x, const Tf* __restrict__ p, const RhsState* __restrict__ st,
                                long long per) {
  const int l = blockIdx.y;
  if (st[l].xpend == 0) return;
  const Tf alpha = (Tf)st[l].alpha;
  Tf* xl = x + (long long)l * per;
  const Tf* pl = p + (long long)l * per;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < per; i += (long long)gridDim.x * blockDim.x)
    xl[i] = xl[i] + alpha * pl[i];
}

template <typename Ti, typename To>
__global__ void convert_kernel(const Ti* __restrict__ in, To* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (To)in[i];
}

static int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 32) b = 152LL * 32;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename Tf>
cudaError_t launch_mandel_to_kelvin(const double* in, Tf* out, long long M, int nf, cudaStream_t s) {
  count_launch();
  mandel_to_kelvin_kernel<Tf><<<grid_for(M * nf, 256), 256, 0, s>>>(in, out, M, nf);
  return cudaGetLastError();
}
template <typename Tf>
cudaError_t launch_kelvin_to_mandel(const Tf* in, double* out, long long M, int nf, cudaStream_t s) {
  count_launch();
  kelvin_to_mandel_kernel<Tf><<<grid_for(M * nf, 256), 256, 0, s>>>(in, out, M, nf);
  return cudaGetLastError();
}
cudaError_t launch_kelvin_to_mandel_inplace(double* f, long long M, int nf, cudaStream_t s) {
  count_launch();
  kelvin_to_mandel_inplace_kernel<<<grid_for(M * nf, 256), 256, 0, s>>>(f, M, nf);
  return cudaGetLastError();
}
cudaError_t launch_mandel_to_kelvin_inplace(double* f, long long M, int nf, cudaStream_t s) {
  count_launch();
  mandel_to_kelvin_inplace_kernel<<<grid_for(M * nf, 256), 256, 0, s>>>(f, M, nf);
  return cudaGetLastError();
}
template <typename Tf>
cudaError_t launch_cg_flush(Tf* x, const Tf* p, const RhsState* st, long long per, int n, cudaStream_t s) {
  long long b = (per + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  count_launch();
  cg_flush_kernel<Tf><<<dim3((unsigned)b, (unsigned)n), 256, 0, s>>>(x, p, st, per);
  return cudaGetLastError();
}
template cudaError_t launch_cg_flush<float>(float*, const float*, const RhsState*, long long, int, cudaStream_t);
template cudaError_t launch_cg_flush<double>(double*, const double*, const RhsState*, long long, int, cudaStream_t);

template <typename Ti, typename To>
cudaError_t launch_convert(const Ti* in, To* out, long long n, cudaStream_t s) {
  count_launch();
  convert_kernel<Ti, To><<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

// x += d (FP64 solution updated by an FP32 correction)
__global__ void add_correction_kernel(const float* __restrict__ d, double* __restrict__ x, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += (double)d[i];
}
cudaError_t launch_add_correction(const float* d, double* x, long long n, cudaStream_t s) {
  count_launch();
  add_correction_kernel<<<grid_for(n, 256), 256, 0, s>>>(d, x, n);
  return cudaGetLastError();
}

// x += a - b (FP64 solution moved by the difference of two FP32 fields: x <- x - (x32 - P x32))
__global__ void add_difference_kernel(const float* __restrict__ a, const float* __restrict__ b, double* __restrict__ x,
                                      long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[i] += (double)a[i] - (double)b[i];
}
cudaError_t launch_add_difference(const float* a, const float* b, double* x, long long n, cudaStream_t s) {
  count_launch();
  add_difference_kernel<<<grid_for(n, 256), 256, 0, s>>>(a, b, x, n);
  return cudaGetLastError();
}

// ---- spectrum layouts ------------------------------------------------------------
// internal: per plane, n2 rows of h values (kx < n1/2) then the n2 Nyquist values;
// standard: [n3][n2][n1/2 + 1] complex.  basis: 0 keep, 1 Mandel->Kelvin, 2 Kelvin->Mandel
// (6-component fields only).
template <typename T>
__device__ __forceinline__ void basis6(cx<double>* v, int basis) {
  if (basis == 1) {
    const cx<double> m0 = v[0], m1 = v[1], m2 = v[2];
    v[0] = (m0 + m1 + m2) * R3;
    v[1] = (m0 - m1) * R2;
    v[2] = (m0 + m1 - m2 * 2.0) * R6;
  } else if (basis == 2) {
    const cx<double> k0 = v[0], k1 = v[1], k2 = v[2];
    v[0] = k0 * R3 + k1 * R2 + k2 * R6;
    v[1] = k0 * R3 - k1 * R2 + k2 * R6;
    v[2] = k0 * R3 - k2 * (2.0 * R6);
  }
}

template <typename T>
__global__ void spec_from_std_kernel(const double* __restrict__ in, cx<T>* __restrict__ S, Geo g,
                                     int nf, int ncomp, int basis) {
  const long long nh = g.h + 1;
  const long long per = (long long)g.n3 * g.n2 * nh;  // frequencies per component
  const long long total = (long long)nf * per;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / per, r = i - f * per;
    const int kx = (int)(r % nh);
    const long long zy = r / nh;
    const int ky = (int)(zy % g.n2), z = (int)(zy / g.n2);
    const long long f_in_plane = (kx < g.h) ? (long long)ky * g.h + kx : (long long)g.n2 * g.h + ky;
    if (ncomp == 6 && basis != 0) {
      cx<double> v[6];
      for (int c = 0; c < 6; ++c) {
        const double* p = in + 2 * ((f * 6 + c) * per + r);
        v[c] = mk<double>(p[0], p[1]);
      }
      basis6<T>(v, basis);
      for (int c = 0; c < 6; ++c)
        S[((f * 6 + c) * g.n3 + z) * g.plane_c + f_in_plane] = mk<T>((T)v[c].re, (T)v[c].im);
    } else {
      for (int c = 0; c < ncomp; ++c) {
        const double* p = in + 2 * ((f * ncomp + c) * per + r);
        S[((f * ncomp + c) * g.n3 + z) * g.plane_c + f_in_plane] = mk<T>((T)p[0], (T)p[1]);
      }
    }
  }
}

template <typename T>
__global__ void spec_to_std_kernel(const cx<T>* __restrict__ S, double* __restrict__ out, Geo g,
                                   int nf, int ncomp, int basis) {
  const long long nh = g.h + 1;
  const long long per = (long long)g.n3 * g.n2 * nh;
  const long long total = (long long)nf * per;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long f = i / per, r = i - f * per;
    const int kx = (int)(r % nh);
    const long long zy = r / nh;
    const int ky = (int)(zy % g.n2), z = (int)(zy / g.n2);
    const long long f_in_plane = (kx < g.h) ? (long long)ky * g.h + kx : (long long)g.n2 * g.h + ky;
    if (ncomp == 6 && basis != 0) {
      cx<double> v[6];
      for (int c = 0; c < 6; ++c) {
        const cx<T> s = S[((f * 6 + c) * g.n3 + z) * g.plane_c + f_in_plane];
        v[c] = mk<double>((double)s.re, (double)s.im);
      }
      basis6<T>(v, basis);
      for (int c = 0; c < 6; ++c) {
        double* p = out + 2 * ((f * 6 + c) * per + r);
        p[0] = v[c].re;
        p[1] = v[c].im;
      }
    } else {
      for (int c = 0; c < ncomp; ++c) {
        const cx<T> s = S[((f * ncomp + c) * g.n3 + z) * g.plane_c + f_in_plane];
        double* p = out + 2 * ((f * ncomp + c) * per + r);
        p[0] = (double)s.re;
        p[1] = (double)s.im;
      }
    }
  }
}

template <typename T>
cudaError_t launch_spec_from_std(const double* in, cx<T>* S, const Geo& g, int nf, int ncomp, int basis,
                                 cudaStream_t s) {
  const long long n = (long long)nf * g.n3 * g.n2 * (g.h + 1);
  count_launch();
  spec_from_std_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(in, S, g, nf, ncomp, basis);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_spec_to_std(const cx<T>* S, double* out, const Geo& g, int nf, int ncomp, int basis,
                               cudaStream_t s) {
  const long long n = (long long)nf * g.n3 * g.n2 * (g.h + 1);
  count_launch();
  spec_to_std_kernel<T><<<grid_for(n, 256), 256, 0, s>>>(S, out, g, nf, ncomp, basis);
  return cudaGetLastError();
}

// ---- FP64 voxel means ------------------------------------------------------------
// Stage 1: block b of (rhs, comp) sums weight(phase) * (field + shift) over a voxel range,
// accumulating each thread's share in FP64.  mat: [n_phase][4] Kelvin eigenvalues
// (C - C0 on k0, on k1..5; C on k0, on k1..5); wsel selects the column pair
// (0: C - C0, 2: C, -1: weight 1).  Stage 2 adds the per-block partials in order.
template <typename Tf>
__global__ void mean_partial_kernel(const Tf* __restrict__ f, int ncomp, const double* __restrict__ shift,
                                    const uint8_t* __restrict__ phase, const double* __restrict__ mat,
                                    int wsel, long long M, int rve_loads, double* __restrict__ part) {
  __shared__ double sh[64];
  const int c = blockIdx.y, rhs = blockIdx.z, nb = gridDim.x;
  const Tf* src = f + ((long long)rhs * ncomp + c) * M;
  if (rve_loads > 0) {   // several RVEs in one handle: this load's phase array and table
    const int rve = rhs / rve_loads;
    phase += (long long)rve * M;
    mat += (long long)rve * 4 * 256;
  }
  const double sft = shift ? shift[rhs * 6 + c] : 0.0;
  const int col = (wsel < 0) ? -1 : wsel + (c == 0 ? 0 : 1);
  double acc = 0.0;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < M; v += (long long)nb * blockDim.x) {
    const double w = (col < 0) ? 1.0 : mat[phase[v] * 4 + col];
    acc += w * ((double)src[v] + sft);
  }
  double vv[1] = {acc};
  block_sum_f64<1>(vv, sh);
  if (threadIdx.x == 0) part[((long long)rhs * ncomp + c) * nb + blockIdx.x] = vv[0];
}

__global__ void mean_final_kernel(const double* __restrict__ part, int nb, long long M, double* out) {
  __shared__ double sh[64];
  const int idx = blockIdx.x;  // rhs * ncomp + c
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[(long long)idx * nb + i];
  double vv[1] = {acc};
  block_sum_f64<1>(vv, sh);
  if (threadIdx.x == 0) out[idx] = vv[0] / (double)M;
}

template <typename Tf>
cudaError_t launch_weighted_mean(const Tf* f, int ncomp, int nrhs, const double* shift, const uint8_t* phase,
                                 const double* mat, int wsel, long long M, double* part, int nblk, double* out,
                                 cudaStream_t s, int rve_loads) {
  dim3 g1(nblk, ncomp, nrhs);
  count_launch();
  mean_partial_kernel<Tf><<<g1, 256, 0, s>>>(f, ncomp, shift, phase, mat, wsel, M, rve_loads, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  count_launch();
  mean_final_kernel<<<nrhs * ncomp, 256, 0, s>>>(part, nblk, M, out);
  return cudaGetLastError();
}

// ---- explicit instantiations -----------------------------------------------------
template cudaError_t launch_mandel_to_kelvin<float>(const double*, float*, long long, int, cudaStream_t);
template cudaError_t launch_mandel_to_kelvin<double>(const double*, double*, long long, int, cudaStream_t);
template cudaError_t launch_kelvin_to_mandel<float>(const float*, double*, long long, int, cudaStream_t);
template cudaError_t launch_kelvin_to_mandel<double>(const double*, double*, long long, int, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double*, float*, long long, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, long long, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double*, double*, long long, cudaStream_t);
template cudaError_t launch_spec_from_std<float>(const double*, cx<float>*, const Geo&, int, int, int, cudaStream_t);
template cudaError_t launch_spec_from_std<double>(const double*, cx<double>*, const Geo&, int, int, int, cudaStream_t);
template cudaError_t launch_spec_to_std<float>(const cx<float>*, double*, const Geo&, int, int, int, cudaStream_t);
template cudaError_t launch_spec_to_std<double>(const cx<double>*, double*, const Geo&, int, int, int, cudaStream_t);
template cudaError_t launch_weighted_mean<float>(const float*, int, int, const double*, const uint8_t*, const double*,
                                                 int, long long, double*, int, double*, cudaStream_t, int);
template cudaError_t launch_weighted_mean<double>(const double*, int, int, const double*, const uint8_t*,
                                                  const double*, int, long long, double*, int, double*, cudaStream_t,
                                                  int);

}  // namespace hom
