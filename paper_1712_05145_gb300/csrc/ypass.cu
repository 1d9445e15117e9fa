// Split y pass of the Lippmann-Schwinger step: the y-axis FFT of a tile of 2^ty_log2
// consecutive spectrum columns (kx) of one z-plane.  Between the x and y passes, column 0 of
// every row holds X[0] + i X[n1/2] (two real sequences packed in one complex one).  The forward
// pass separates them after the transform, A = (P + conj P(-k))/2 into column 0 and
// B = (P - conj P(-k))/(2i) into the plane's Nyquist column kx = n1/2; the inverse pass packs
// A + i B before its transform.
#include "ls_common.cuh"

namespace hom {

template <typename T, int DIR, int EPT>
__global__ void __launch_bounds__(512) ypass_kernel(const cx<T>* __restrict__ tw_n2, cx<T>* S, const Geo g,
                                                    int ncomp, int s_ncomp, unsigned long long* prof,
                                                    const RhsState* st, int rhs0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tile = blockIdx.x, z = blockIdx.y;
  const int c = blockIdx.z % ncomp, lrhs = blockIdx.z / ncomp, rhs = rhs0 + lrhs;
  if (st != nullptr && st[rhs].active == 0) return;
  const int n2 = g.n2, h = g.h, lg = g.ty_log2, TY = 1 << lg;
  const int kx0 = tile * TY;
  const int pitch = TY;
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* twy = buf + n2 * pitch;
  const int tid = threadIdx.x, nthr = blockDim.x;
  cx<T>* Sp = S + ((long long)(lrhs * s_ncomp + c) * g.n3 + z) * g.plane_c;
  cx<T>* nyq = Sp + (long long)n2 * h;
  // the column tile goes to shared memory by cp.async while the twiddle table loads
  for (int e = tid; e < n2 * TY; e += nthr) {
    const int y = e >> lg, t = e & (TY - 1);
    cp_async_elem<sizeof(cx<T>)>(buf + y * pitch + t, Sp + (long long)y * h + kx0 + t);
  }
  for (int i = tid; i < n2; i += nthr) twy[i] = ldg_cx(tw_n2 + i);
  if (prof != nullptr && tid == 0) {
    atomicAdd(prof, (unsigned long long)(2LL * n2 * TY * (long long)sizeof(cx<T>) +
                                         (kx0 == 0 ? (long long)n2 * (long long)sizeof(cx<T>) : 0)));
    atomicAdd(prof + 1, (unsigned long long)(n2 * TY));
  }
  cp_async_wait_all();
  __syncthreads();
  if (DIR > 0 && kx0 == 0) {  // pack A + i B
    for (int y = tid; y < n2; y += nthr) {
      const cx<T> v = buf[y * pitch], b = nyq[y];
      buf[y * pitch] = mk<T>(v.re - b.im, v.im + b.re);
    }
    __syncthreads();
  }
  fft_pencils<T, DIR, EPT>(buf, ColAddr{pitch}, n2, TY, g.fd_ty, twy);
  if (DIR < 0 && kx0 == 0) {  // separate A (column 0) and B (Nyquist column)
    for (int ky = tid; 2 * ky <= n2; ky += nthr) {
      const int km = (n2 - ky) % n2;
      const cx<T> pk = buf[ky * pitch], pm = buf[km * pitch];
      const cx<T> ak = (pk + conj(pm)) * (T)0.5;
      const cx<T> bk = mul_i<T, -1>(pk - conj(pm)) * (T)0.5;
      const cx<T> am = (pm + conj(pk)) * (T)0.5;
      const cx<T> bm = mul_i<T, -1>(pm - conj(pk)) * (T)0.5;
      buf[ky * pitch] = ak;
      nyq[ky] = bk;
      if (km != ky) {
        buf[km * pitch] = am;
        nyq[km] = bm;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < n2 * TY; e += nthr) {
    const int y = e >> lg, t = e & (TY - 1);
    Sp[(long long)y * h + kx0 + t] = buf[y * pitch + t];
  }
}

template <typename T>
cudaError_t launch_ypass(const cx<T>* tw_n2, cx<T>* S, const Geo& g, int ncomp, int s_ncomp, int nrhs, int dir,
                         unsigned long long* prof, const RhsState* st, int rhs0, cudaStream_t s) {
  const int TY = 1 << g.ty_log2;
  if ((long long)g.n2 * TY > (long long)kEPT * g.thr_y || g.thr_y > 512 || g.h % TY != 0)
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)(g.n2 * TY + g.n2) * sizeof(cx<T>);
  dim3 grid(g.h / TY, g.n3, ncomp * nrhs);
  if (dir < 0) {
    auto k = ypass_kernel<T, -1, kEPT>;
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    count_launch();
    k<<<grid, g.thr_y, smem, s>>>(tw_n2, S, g, ncomp, s_ncomp, prof, st, rhs0);
  } else {
    auto k = ypass_kernel<T, +1, kEPT>;
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    count_launch();
    k<<<grid, g.thr_y, smem, s>>>(tw_n2, S, g, ncomp, s_ncomp, prof, st, rhs0);
  }
  return cudaGetLastError();
}

template cudaError_t launch_ypass<float>(const cx<float>*, cx<float>*, const Geo&, int, int, int, int,
                                         unsigned long long*, const RhsState*, int, cudaStream_t);
template cudaError_t launch_ypass<double>(const cx<double>*, cx<double>*, const Geo&, int, int, int, int,
                                          unsigned long long*, const RhsState*, int, cudaStream_t);
template cudaError_t launch_ypass<df64>(const cx<df64>*, cx<df64>*, const Geo&, int, int, int, int,
                                        unsigned long long*, const RhsState*, int, cudaStream_t);

}  // namespace hom
