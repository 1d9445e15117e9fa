// z-pencil pass of the Lippmann-Schwinger step: z FFTs and the Green contraction.
#include <map>
#include <utility>

#include "ls_common.cuh"
#include "spectral.cuh"
#include "zsplit.h"

namespace hom {

// Pointwise Green contraction of the split z pass: one thread per frequency and load, the six
// Kelvin components read and written with unit stride along the spectrum's flat index.
template <typename T>
__global__ void __launch_bounds__(256) zgreen_kernel(const ZArgs<T> a, int nrhs) {
  const Geo& g = a.g;
  T c1, c2h;
  green_consts<T>(nullptr, 0, a.lam0, a.mu0, c1, c2h);
  const T scale = (T)a.scale;
  const long long per = (long long)g.n3 * g.plane_c;   // frequencies of one component
  const long long nmain = (long long)g.n2 * g.h;
  const long long total = (long long)nrhs * per;
  if (a.prof != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
    atomicAdd(a.prof, (unsigned long long)(total * 12LL * (long long)sizeof(cx<T>)));
    atomicAdd(a.prof + 1, (unsigned long long)total);
  }
  for (long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x; id < total;
       id += (long long)gridDim.x * blockDim.x) {
    const long long lrhs = id / per, q = id - lrhs * per;
    if (a.st != nullptr && a.st[a.rhs0 + lrhs].active == 0) continue;
    if (a.c0 != nullptr) green_consts<T>(a.c0, rve_of(a.rhs0 + (int)lrhs, a.rve_loads), a.lam0, a.mu0, c1, c2h);
    const int n = (int)(q / g.plane_c);
    const long long f = q - (long long)n * g.plane_c;
    int kx, ky;
    if (f < nmain) { ky = (int)g.fd_h.div((unsigned)f); kx = (int)f - ky * g.h; }
    else { ky = (int)(f - nmain); kx = g.h; }
    T x1, x2, x3;
    wave_vector<T>(g, a.green, a.gtab, kx, ky, n, x1, x2, x3);
    cx<T>* base = a.S + lrhs * 6 * per + q;
    cx<T> k[6], tt[6], w1, w2, w3;
#pragma unroll
    for (int i = 0; i < 6; ++i) k[i] = base[i * per];
    kelvin_to_tensor<T>(k, tt);
    tensor_dot_xi<T>(tt, x1, x2, x3, w1, w2, w3);
    green_from_w<T>(k, w1, w2, w3, x1, x2, x3, c1, c2h, scale);
#pragma unroll
    for (int i = 0; i < 6; ++i) base[i * per] = k[i];
  }
}

template <typename T>
cudaError_t launch_zgreen(const ZArgs<T>& a, int nrhs, cudaStream_t s) {
  if (nrhs < 1) return cudaErrorInvalidValue;
  const long long total = (long long)nrhs * a.g.n3 * a.g.plane_c;
  long long blocks = (total + 255) / 256;
  if (blocks > 152LL * 16) blocks = 152LL * 16;
  count_launch();
  zgreen_kernel<T><<<(int)blocks, 256, 0, s>>>(a, nrhs);
  return cudaGetLastError();
}
template cudaError_t launch_zgreen<float>(const ZArgs<float>&, int, cudaStream_t);
template cudaError_t launch_zgreen<double>(const ZArgs<double>&, int, cudaStream_t);
template cudaError_t launch_zgreen<df64>(const ZArgs<df64>&, int, cudaStream_t);

// zpass: one CTA per (tile of 2^tc_log2 spectrum columns, rhs)
template <typename T, int EPT>
__global__ void __launch_bounds__(512) zpass_kernel(const ZArgs<T> a) {
  const int tc_log2 = a.tc_log2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Geo& g = a.g;
  const int tile = blockIdx.x, lrhs = blockIdx.y, rhs = a.rhs0 + lrhs;
  if (a.st != nullptr && a.st[rhs].active == 0) return;
  const int TC = 1 << tc_log2, n3 = g.n3;
  const long long f0 = (long long)tile * TC;
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  const int cstride = a.cstride;
  cx<T>* twz = buf + a.ncomp_in * cstride;   // exp(-2 pi i t / n3)
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int i = tid; i < n3; i += nthr) twz[i] = ldg_cx(a.tw_n3 + i);
  cx<T>* Sr = a.S + (long long)lrhs * a.ncomp_in * n3 * g.plane_c;
  if (a.prof != nullptr && tid == 0) {
    const long long cols = (g.plane_c - f0 < TC) ? g.plane_c - f0 : TC;
    atomicAdd(a.prof, (unsigned long long)((a.ncomp_in + a.ncomp_out) * n3 * cols * (long long)sizeof(cx<T>)));
    atomicAdd(a.prof + 1, (unsigned long long)(n3 * cols));
  }

  const int per_c = n3 * TC;
  {
    // the whole tile is in flight at once: cp.async per element, zeros past the last column
    const int total = a.ncomp_in * per_c;
    for (int e = tid; e < total; e += nthr) {
      const int c = (int)a.fd_comp.div((unsigned)e), ec = e - c * per_c;
      const int tc = ec & (TC - 1), n = ec >> tc_log2;
      const long long f = f0 + tc;
      if (f < g.plane_c) cp_async_elem<sizeof(cx<T>)>(buf + c * cstride + ec, Sr + (long long)(c * n3 + n) * g.plane_c + f);
      else buf[c * cstride + ec] = mk<T>(0, 0);
    }
    cp_async_wait_all();
  }
  __syncthreads();
  const ZAddr za{tc_log2, cstride, TC};
  if (a.mode != Z_INV && a.mode != Z_GREEN) fft_pencils<T, -1, EPT>(buf, za, n3, a.ncomp_in * TC, a.fd_in, twz);

  if (a.mode == Z_GAMMA || a.mode == Z_GREEN || a.mode == Z_DISP || a.mode == Z_RHS) {
    T c1, c2h;
    green_consts<T>(a.c0, rve_of(rhs, a.rve_loads), a.lam0, a.mu0, c1, c2h);
    const T scale = (T)a.scale;
    const long long nmain = (long long)g.n2 * g.h;
    for (int t = tid; t < n3 * TC; t += nthr) {
      const int tc = t & (TC - 1), n = t >> tc_log2;
      const long long f = f0 + tc;
      if (f >= g.plane_c) continue;
      int kx, ky;
      if (f < nmain) { ky = (int)g.fd_h.div((unsigned)f); kx = (int)f - ky * g.h; }
      else { ky = (int)(f - nmain); kx = g.h; }
      // discrete wave vector (Nyquist components taken as 0), or the rotated difference symbol
      T x1, x2, x3;
      wave_vector<T>(g, a.green, a.gtab, kx, ky, n, x1, x2, x3);
      const int e0 = n * TC + tc;
      cx<T> k[6], tt[6], w1, w2, w3;
#pragma unroll
      for (int i = 0; i < 6; ++i) k[i] = buf[i * cstride + e0];
      kelvin_to_tensor<T>(k, tt);
      tensor_dot_xi<T>(tt, x1, x2, x3, w1, w2, w3);
      if (a.mode == Z_DISP) {
        // u_hat = -i (2 w - xi (xi . w) / |xi|^2) / |xi|^2 for eps_hat = i sym(xi (x) u_hat)
        const T q = x1 * x1 + x2 * x2 + x3 * x3;
        cx<T> u[3] = {mk<T>(0, 0), mk<T>(0, 0), mk<T>(0, 0)};
        if (q != (T)0) {
          const cx<T> s = w1 * x1 + w2 * x2 + w3 * x3;
          const T iq = (T)1 / q;
          const T b = iq * scale;
          u[0] = mul_i<T, -1>(w1 * ((T)2 * b) - s * (x1 * iq * b));
          u[1] = mul_i<T, -1>(w2 * ((T)2 * b) - s * (x2 * iq * b));
          u[2] = mul_i<T, -1>(w3 * ((T)2 * b) - s * (x3 * iq * b));
        }
#pragma unroll
        for (int i = 0; i < 3; ++i) buf[i * cstride + e0] = u[i];
      } else {
        if (a.mode == Z_RHS) {
          // (p_hat + theta_hat) xi = p_hat xi - i g_hat, since i theta_hat xi = g_hat (Sec. 3)
          w1 = w1 - mul_i<T, 1>(buf[6 * cstride + e0]);
          w2 = w2 - mul_i<T, 1>(buf[7 * cstride + e0]);
          w3 = w3 - mul_i<T, 1>(buf[8 * cstride + e0]);
        }
        green_from_w<T>(k, w1, w2, w3, x1, x2, x3, c1, c2h, scale);
#pragma unroll
        for (int i = 0; i < 6; ++i) buf[i * cstride + e0] = k[i];
      }
    }
    __syncthreads();
  }

  if (a.mode != Z_FWD && a.mode != Z_GREEN) fft_pencils<T, +1, EPT>(buf, za, n3, a.ncomp_out * TC, a.fd_out, twz);

  for (int e = tid; e < a.ncomp_out * per_c; e += nthr) {
    const int c = (int)a.fd_comp.div((unsigned)e), ec = e - c * per_c;
    const int tc = ec & (TC - 1), n = ec >> tc_log2;
    const long long f = f0 + tc;
    if (f < g.plane_c) Sr[(long long)(c * n3 + n) * g.plane_c + f] = buf[c * cstride + ec];
  }
}

template <typename T>
cudaError_t launch_zpass(const ZArgs<T>& a, int nrhs, cudaStream_t s) {
  // every pencil element must have a thread slot (kEPT per thread, <= 512 threads)
  if ((long long)a.ncomp_in * a.g.n3 * (1LL << a.tc_log2) > (long long)kEPT * a.nthr || a.nthr > 512 ||
      a.ncomp_out > a.ncomp_in)
    return cudaErrorInvalidValue;
  const size_t smem = zpass_smem_bytes(a.g, sizeof(cx<T>), a.ncomp_in, a.tc_log2);
  auto k = zpass_kernel<T, kEPT>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.ntiles, nrhs);
  count_launch();
  k<<<grid, a.nthr, smem, s>>>(a);
  return cudaGetLastError();
}

// resident CTAs per SM of the z pass at `threads` threads and `smem` bytes (0 if it cannot run);
// cached per host thread, since the answer depends only on the arguments
template <typename T>
int zpass_ctas_per_sm(int threads, size_t smem) {
  thread_local std::map<std::pair<int, size_t>, int> cache;
  const auto key = std::make_pair(threads, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  auto k = zpass_kernel<T, kEPT>;
  int nb = 0;
  if (set_smem(k, smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    nb = 0;
  }
  cache[key] = nb;
  return nb;
}
template int zpass_ctas_per_sm<float>(int, size_t);
template int zpass_ctas_per_sm<double>(int, size_t);
template int zpass_ctas_per_sm<df64>(int, size_t);

template cudaError_t launch_zpass<float>(const ZArgs<float>&, int, cudaStream_t);
template cudaError_t launch_zpass<double>(const ZArgs<double>&, int, cudaStream_t);
template cudaError_t launch_zpass<df64>(const ZArgs<df64>&, int, cudaStream_t);

}  // namespace hom
