// Split y pass of the Lippmann-Schwinger step: the y-axis FFT of a tile of 2^ty_log2
// consecutive spectrum columns (kx) of one z-plane.  Between the x and y passes, column 0 of
// every row holds X[0] + i X[n1/2] (two real sequences packed in one complex one).  The forward
// pass separates them after the transform, A = (P + conj P(-k))/2 into column 0 and
// B = (P - conj P(-k))/(2i) into the plane's Nyquist column kx = n1/2; the inverse pass packs
// A + i B before its transform.
#include "ls_common.cuh"
#include "tma.cuh"

namespace hom {

// column 0 of the tile <- A + i B (B from the Nyquist column), before the inverse transform
template <typename T>
__device__ __forceinline__ void y_pack(cx<T>* buf, int pitch, const cx<T>* nyq, int n2) {
  for (int y = threadIdx.x; y < n2; y += blockDim.x) {
    const cx<T> v = buf[y * pitch], b = nyq[y];
    buf[y * pitch] = mk<T>(v.re - b.im, v.im + b.re);
  }
}
// column 0 of the transformed tile -> A (column 0) and B (Nyquist column)
template <typename T>
__device__ __forceinline__ void y_separate(cx<T>* buf, int pitch, cx<T>* nyq, int n2) {
  for (int ky = threadIdx.x; 2 * ky <= n2; ky += blockDim.x) {
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
}

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
    y_pack<T>(buf, pitch, nyq, n2);
    __syncthreads();
  }
  fft_pencils<T, DIR, EPT>(buf, ColAddr{pitch}, n2, TY, g.fd_ty, twy);
  if (DIR < 0 && kx0 == 0) {  // separate A (column 0) and B (Nyquist column)
    y_separate<T>(buf, pitch, nyq, n2);
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

// ---- TMA variant (FP32) ------------------------------------------------------------------------
// The same tile work with the tile moved by the tensor-memory accelerator: thread 0 issues the
// tensor loads of the [n2][TY] column tile (one box per 256 rows), which complete on an mbarrier,
// and after the transform the tensor stores.  The Nyquist column (outside the tensor's x extent)
// is read and written with plain accesses by the kx = 0 tile, as above.
constexpr unsigned long long kYtWaitNs = 2000000000ull;  // a tile load that takes 2 s is an error

template <int DIR, int EPT>
__global__ void __launch_bounds__(512) ypass_tma_kernel(const __grid_constant__ CUtensorMap tm,
                                                        const cx<float>* __restrict__ tw_n2, cx<float>* S,
                                                        const Geo g, int ncomp, int s_ncomp,
                                                        unsigned long long* prof, const RhsState* st, int rhs0,
                                                        unsigned* err) {
  extern __shared__ __align__(16) unsigned char yt_smem[];
  const int tile = blockIdx.x, z = blockIdx.y;
  const int c = blockIdx.z % ncomp, lrhs = blockIdx.z / ncomp, rhs = rhs0 + lrhs;
  if (st != nullptr && st[rhs].active == 0) return;
  const int tid = threadIdx.x;
  if ((smem_u32(yt_smem) & 127u) != 0) {   // tensor copies need 128-byte aligned shared addresses
    if (tid == 0 && err != nullptr) atomicOr(err, 2u);
    return;
  }
  const int n2 = g.n2, h = g.h, lg = g.ty_log2, TY = 1 << lg, kx0 = tile * TY;
  const int nbox = (n2 + 255) / 256, rows = n2 / nbox;
  const int plane = (lrhs * s_ncomp + c) * g.n3 + z;   // z-plane index in the tensor
  cx<float>* buf = reinterpret_cast<cx<float>*>(yt_smem);   // [n2][TY]
  cx<float>* twy = buf + n2 * TY;
  const uint32_t bar = smem_u32(twy + n2), sbuf = smem_u32(buf);
  const uint32_t box_bytes = (uint32_t)rows * TY * (uint32_t)sizeof(cx<float>);
  cx<float>* nyq = S + (long long)plane * g.plane_c + (long long)n2 * h;
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(bar, (uint32_t)nbox * box_bytes);
    for (int b = 0; b < nbox; ++b) tma_load_3d(sbuf + b * box_bytes, &tm, kx0, b * rows, plane, bar);
  }
  for (int i = tid; i < n2; i += blockDim.x) twy[i] = ldg_cx(tw_n2 + i);
  if (prof != nullptr && tid == 0) {
    atomicAdd(prof, (unsigned long long)(2LL * n2 * TY * (long long)sizeof(cx<float>) +
                                         (kx0 == 0 ? (long long)n2 * (long long)sizeof(cx<float>) : 0)));
    atomicAdd(prof + 1, (unsigned long long)(n2 * TY));
  }
  __syncthreads();   // the mbarrier is initialised before anyone waits on it
  const bool ok = mbar_wait_bounded(bar, 0, kYtWaitNs);
  if (DIR > 0 && kx0 == 0) {
    y_pack<float>(buf, TY, nyq, n2);
    __syncthreads();
  }
  fft_pencils<float, DIR, EPT>(buf, ColAddr{TY}, n2, TY, g.fd_ty, twy);
  if (DIR < 0 && kx0 == 0) {
    y_separate<float>(buf, TY, nyq, n2);
    __syncthreads();
  }
  fence_proxy_async_smem();   // the transform's shared-memory writes, before the tensor store reads them
  __syncthreads();
  if (tid == 0) {
    for (int b = 0; b < nbox; ++b) tma_store_3d(&tm, kx0, b * rows, plane, sbuf + b * box_bytes);
    bulk_commit();
    bulk_wait_all();   // the stores have finished before the CTA's shared memory is released
  }
  if (!ok && err != nullptr) atomicOr(err, 1u);
}

bool ytma_fits(const Geo& g) {
  // 16-byte tensor strides (even h and an even number of spectrum columns per plane) and whole
  // 16-byte box rows (tiles of 2 columns at least)
  return g.split && g.ty_log2 >= 1 && (g.h % 2) == 0 && (g.plane_c % 2) == 0 && g.h % (1 << g.ty_log2) == 0;
}

cudaError_t launch_ypass_tma(const cx<float>* tw_n2, cx<float>* S, const Geo& g, int ncomp, int s_ncomp, int nrhs,
                             int dir, unsigned long long* prof, const RhsState* st, int rhs0, unsigned* err,
                             cudaStream_t s) {
  const int TY = 1 << g.ty_log2;
  if (!ytma_fits(g) || (long long)g.n2 * TY > (long long)kEPT * g.thr_y || g.thr_y > 512 || nrhs < 1 ||
      ncomp < 1 || ncomp > s_ncomp || (reinterpret_cast<uintptr_t>(S) & 15) != 0)
    return cudaErrorInvalidValue;
  const int nbox = (g.n2 + 255) / 256, rows = g.n2 / nbox;
  const unsigned long long elem = sizeof(cx<float>);
  // the main part of every z-plane of the launch's loads: [s_ncomp nrhs n3 planes][n2][h] (row pitch
  // h, plane pitch plane_c), 8-byte elements
  CUtensorMap tm;
  const unsigned long long dims[3] = {(unsigned long long)g.h, (unsigned long long)g.n2,
                                      (unsigned long long)s_ncomp * nrhs * g.n3};
  const unsigned long long strides[2] = {(unsigned long long)g.h * elem, (unsigned long long)g.plane_c * elem};
  const unsigned box[2] = {(unsigned)TY, (unsigned)rows};
  if (!encode_tensor_3d(&tm, S, dims, strides, box)) return cudaErrorNotSupported;
  const size_t smem = (size_t)(g.n2 * TY + g.n2) * sizeof(cx<float>) + 16;
  dim3 grid(g.h / TY, g.n3, ncomp * nrhs);
  if (dir < 0) {
    auto k = ypass_tma_kernel<-1, kEPT>;
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    count_launch();
    k<<<grid, g.thr_y, smem, s>>>(tm, tw_n2, S, g, ncomp, s_ncomp, prof, st, rhs0, err);
  } else {
    auto k = ypass_tma_kernel<+1, kEPT>;
    cudaError_t e = set_smem(k, smem);
    if (e != cudaSuccess) return e;
    count_launch();
    k<<<grid, g.thr_y, smem, s>>>(tm, tw_n2, S, g, ncomp, s_ncomp, prof, st, rhs0, err);
  }
  return cudaGetLastError();
}

}  // namespace hom
