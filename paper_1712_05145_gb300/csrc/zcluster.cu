// Cluster z pass of the Lippmann-Schwinger step (Sec. 2 of arXiv:1712.05145, Algorithm 1: the
// transform along z, eta_hat = -Gamma0_hat(xi) : tau_hat with eta_hat(0) = 0, the inverse
// transform along z).
//
// A tile is 2^lg consecutive spectrum columns (flat index f of the x-y half-spectrum plane) over
// all N3 z-planes.  Six CTAs form a thread-block cluster; CTA c (its rank) holds component c of
// the tile in its shared memory and runs that component's z FFTs.  The contraction needs all six
// components at a frequency, so after a cluster barrier each CTA contracts one sixth of the
// tile's frequencies, reading and writing the six components in the other CTAs' shared memory
// (distributed shared memory).  A second cluster barrier precedes the inverse z FFTs.
//
// Compared with one CTA holding all six components of a narrower tile, each CTA reads and writes
// runs of 2^lg complex values per z-plane (128 bytes at 16 FP32 columns) instead of 16-32 bytes,
// and at N3 = 512 the z stage stays one pass over the spectrum instead of three.
#include <cooperative_groups.h>

#include "ls_common.cuh"
#include "spectral.cuh"
#include "tma.cuh"
#include "zcluster.h"

namespace cg = cooperative_groups;

namespace hom {

constexpr int kZcComps = 6;            // CTAs per cluster: one per Kelvin component
constexpr int kZcMaxElems = kEPT * 512;
constexpr size_t kZcMaxSmem = 80 * 1024;
// two 512-thread CTAs per SM in FP32 (64 registers); the 16-byte types keep more registers
template <typename T> struct ZcCfg { static constexpr int kMinBlocks = 1; };
template <> struct ZcCfg<float> { static constexpr int kMinBlocks = 2; };

// -Gamma0_hat(xi) : tau_hat at tile element q (column f0 + q mod 2^lg, z-plane q / 2^lg), in place on
// its six Kelvin components k; columns past the plane are left as they are
template <typename T>
__device__ __forceinline__ void contract_point(const Geo& g, const ZArgs<T>& a, long long f0, int lg, int n3, int q,
                                               cx<T>* k, T c1, T c2h, T scale, long long nmain) {
  const int tc = q & ((1 << lg) - 1), n = q >> lg;
  const long long f = f0 + tc;
  if (f >= g.plane_c) return;
  int kx, ky;
  if (f < nmain) { ky = (int)g.fd_h.div((unsigned)f); kx = (int)f - ky * g.h; }
  else { ky = (int)(f - nmain); kx = g.h; }
  // discrete wave vector (Nyquist components taken as 0), or the rotated difference symbol
  T x1, x2, x3;
  wave_vector<T>(g, a.green, a.gtab, kx, ky, n, x1, x2, x3);
  cx<T> tt[6], w1, w2, w3;
  kelvin_to_tensor<T>(k, tt);
  tensor_dot_xi<T>(tt, x1, x2, x3, w1, w2, w3);
  green_from_w<T>(k, w1, w2, w3, x1, x2, x3, c1, c2h, scale);
}

template <typename T, int EPT>
__global__ void __cluster_dims__(kZcComps, 1, 1) __launch_bounds__(512, ZcCfg<T>::kMinBlocks) zcluster_kernel(const ZArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const Geo& g = a.g;
  const int comp = (int)cl.block_rank();
  const int tile = blockIdx.x / kZcComps, lrhs = blockIdx.y, rhs = a.rhs0 + lrhs;
  // the six CTAs of a cluster share the load, so they leave together (before any barrier)
  if (a.st != nullptr && a.st[rhs].active == 0) return;
  const int lg = a.tc_log2, TC = 1 << lg, n3 = g.n3;
  const int per = n3 * TC;   // elements of this CTA's tile
  const long long f0 = (long long)tile * TC;
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);   // [n3][TC]
  cx<T>* twz = buf + per;                             // exp(-2 pi i t / n3)
  const int tid = threadIdx.x, nthr = blockDim.x;

  cx<T>* Sc = a.S + (long long)(lrhs * kZcComps + comp) * n3 * g.plane_c;
  for (int e = tid; e < per; e += nthr) {
    const int tc = e & (TC - 1), n = e >> lg;
    const long long f = f0 + tc;
    if (f < g.plane_c) cp_async_elem<sizeof(cx<T>)>(buf + e, Sc + (long long)n * g.plane_c + f);
    else buf[e] = mk<T>(0, 0);
  }
  for (int i = tid; i < n3; i += nthr) twz[i] = ldg_cx(a.tw_n3 + i);
  const long long cols = (g.plane_c - f0 < TC) ? g.plane_c - f0 : TC;
  if (a.prof != nullptr && tid == 0) {
    atomicAdd(a.prof, (unsigned long long)(2LL * n3 * cols * (long long)sizeof(cx<T>)));
    if (comp == 0) atomicAdd(a.prof + 1, (unsigned long long)(n3 * cols));
  }
  cp_async_wait_all();
  __syncthreads();
  fft_pencils<T, -1, EPT>(buf, ColAddr{TC}, n3, TC, a.fd_in, twz);
  cl.sync();   // every component of the tile is transformed along z

  {
    cx<T>* part[kZcComps];
#pragma unroll
    for (int r = 0; r < kZcComps; ++r) part[r] = cl.map_shared_rank(buf, r);
    T c1, c2h;
    green_consts<T>(a.c0, rve_of(rhs, a.rve_loads), a.lam0, a.mu0, c1, c2h);
    const T scale = (T)a.scale;
    const long long nmain = (long long)g.n2 * g.h;
    const int share = (per + kZcComps - 1) / kZcComps;
    const int q0 = comp * share, q1 = (q0 + share < per) ? q0 + share : per;
    for (int q = q0 + tid; q < q1; q += nthr) {
      cx<T> k[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) k[i] = part[i][q];
      contract_point<T>(g, a, f0, lg, n3, q, k, c1, c2h, scale, nmain);
#pragma unroll
      for (int i = 0; i < 6; ++i) part[i][q] = k[i];
    }
  }
  cl.sync();   // every frequency of the tile is contracted; no CTA touches another's memory after this

  fft_pencils<T, +1, EPT>(buf, ColAddr{TC}, n3, TC, a.fd_in, twz);
  for (int e = tid; e < per; e += nthr) {
    const int tc = e & (TC - 1), n = e >> lg;
    const long long f = f0 + tc;
    if (f < g.plane_c) Sc[(long long)n * g.plane_c + f] = buf[e];
  }
}

// ---- TMA variant (FP32) ------------------------------------------------------------------------
// The same tile work with the tile moved by the tensor-memory accelerator: thread 0 issues the
// tensor loads of the CTA's component (one box per 256 z-planes), which complete on an mbarrier,
// and after the inverse FFTs the tensor stores.  Columns past the plane read as zero and are not
// written.  Several CTAs per SM overlap one tile's copies with other tiles' FFTs.  (A persistent
// form that loops over tiles, loading the next tile during the current one, spills: inside the
// loop the compiler keeps the FFT stages' thread-invariant indexes of every length live, about
// 8 KB of stack per thread.)
constexpr unsigned long long kZtWaitNs = 2000000000ull;  // a tile load that takes 2 s is an error

template <int EPT>
__global__ void __cluster_dims__(kZcComps, 1, 1) __launch_bounds__(512, 2)
    zcluster_tma_kernel(const __grid_constant__ CUtensorMap tm, const ZArgs<float> a) {
  extern __shared__ __align__(16) unsigned char zt_smem[];
  cg::cluster_group cl = cg::this_cluster();
  const Geo& g = a.g;
  const int comp = (int)cl.block_rank();
  const int tile = blockIdx.x / kZcComps, lrhs = blockIdx.y, rhs = a.rhs0 + lrhs;
  if (a.st != nullptr && a.st[rhs].active == 0) return;   // the whole cluster leaves together
  const int tid = threadIdx.x;
  // tensor copies need 128-byte aligned shared addresses; every CTA has the same layout, so on a
  // misaligned base all CTAs leave here, before any cluster barrier
  if ((smem_u32(zt_smem) & 127u) != 0) {
    if (tid == 0 && a.err != nullptr) atomicOr(a.err, 2u);
    return;
  }
  const int lg = a.tc_log2, TC = 1 << lg, n3 = g.n3, per = n3 * TC;
  const int nbox = (n3 + 255) / 256, rows = n3 / nbox;   // a box spans at most 256 z-planes
  const int zc = lrhs * kZcComps + comp;                  // this CTA's component plane in the tensor
  cx<float>* buf = reinterpret_cast<cx<float>*>(zt_smem);   // [n3][TC]
  cx<float>* twz = buf + per;
  const uint32_t bar = smem_u32(twz + n3), sbuf = smem_u32(buf);
  const uint32_t box_bytes = (uint32_t)rows * TC * (uint32_t)sizeof(cx<float>);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
    mbar_arrive_expect_tx(bar, (uint32_t)nbox * box_bytes);
    for (int b = 0; b < nbox; ++b) tma_load_3d(sbuf + b * box_bytes, &tm, tile * TC, b * rows, zc, bar);
  }
  for (int i = tid; i < n3; i += blockDim.x) twz[i] = ldg_cx(a.tw_n3 + i);
  __syncthreads();   // the mbarrier is initialised before anyone waits on it
  const bool ok = mbar_wait_bounded(bar, 0, kZtWaitNs);
  fft_pencils<float, -1, EPT>(buf, ColAddr{TC}, n3, TC, a.fd_in, twz);
  cl.sync();   // every component of the tile is transformed along z
  {
    cx<float>* part[kZcComps];
#pragma unroll
    for (int r = 0; r < kZcComps; ++r) part[r] = cl.map_shared_rank(buf, r);
    float c1, c2h;
    green_consts<float>(a.c0, rve_of(rhs, a.rve_loads), a.lam0, a.mu0, c1, c2h);
    const float scale = (float)a.scale;
    const long long nmain = (long long)g.n2 * g.h, f0 = (long long)tile * TC;
    const int share = (per + kZcComps - 1) / kZcComps;
    const int q0 = comp * share, q1 = (q0 + share < per) ? q0 + share : per;
    for (int q = q0 + tid; q < q1; q += blockDim.x) {
      cx<float> k[6];
#pragma unroll
      for (int i = 0; i < 6; ++i) k[i] = part[i][q];
      contract_point<float>(g, a, f0, lg, n3, q, k, c1, c2h, scale, nmain);
#pragma unroll
      for (int i = 0; i < 6; ++i) part[i][q] = k[i];
    }
  }
  cl.sync();   // no CTA touches another's buffer after this
  fft_pencils<float, +1, EPT>(buf, ColAddr{TC}, n3, TC, a.fd_in, twz);
  fence_proxy_async_smem();   // the inverse FFT's shared-memory writes, before the tensor store reads them
  __syncthreads();
  if (tid == 0) {
    for (int b = 0; b < nbox; ++b) tma_store_3d(&tm, tile * TC, b * rows, zc, sbuf + b * box_bytes);
    bulk_commit();
    if (a.prof != nullptr) {
      const long long f0 = (long long)tile * TC;
      const long long cols = (g.plane_c - f0 < TC) ? g.plane_c - f0 : TC;
      atomicAdd(a.prof, (unsigned long long)(2LL * n3 * cols * (long long)sizeof(cx<float>)));
      if (comp == 0) atomicAdd(a.prof + 1, (unsigned long long)(n3 * cols));
    }
    bulk_wait_all();   // the stores have finished before the CTA's shared memory is released
  }
  if (!ok && a.err != nullptr) atomicOr(a.err, 1u);
}

static size_t zcluster_smem(const Geo& g, size_t elem, int lg) {
  return ((size_t)g.n3 * ((size_t)1 << lg) + g.n3) * elem;
}

bool zcluster_tile_fits(const Geo& g, size_t elem, int lg) {
  return lg >= 0 && lg <= 6 && (long long)g.n3 * (1LL << lg) <= kZcMaxElems &&
         zcluster_smem(g, elem, lg) <= kZcMaxSmem;
}

// Default width: grow the tile while it stays within about 256 threads, or while its runs along
// the flat index are shorter than 128 bytes (one full memory transaction per z-plane).
template <typename T>
bool zcluster_tiling(ZArgs<T>& a, int force_lg) {
  const size_t elem = sizeof(cx<T>);
  if (a.g.n3 < 16) return false;   // shallow grids: the single-CTA z pass has more work per CTA
  int best = -1;
  if (force_lg >= 0 && zcluster_tile_fits(a.g, elem, force_lg)) {
    best = force_lg;
  } else {
    for (int lg = 0; lg <= 6; ++lg) {
      if (!zcluster_tile_fits(a.g, elem, lg)) break;
      if (best < 0 || (long long)a.g.n3 * (1LL << lg) <= 4096 || ((size_t)1 << best) * elem < 128) best = lg;
    }
  }
  if (best < 0) return false;
  a.tc_log2 = best;
  const long long tc = 1LL << best;
  a.ntiles = (int)((a.g.plane_c + tc - 1) / tc);
  const long long e = (long long)a.g.n3 * tc;
  int thr = (int)((e + kEPT - 1) / kEPT);
  thr = ((thr + 31) / 32) * 32;
  a.nthr = thr < 64 ? 64 : thr;
  a.fd_in = make_fastdiv((unsigned)tc);
  return true;
}
template bool zcluster_tiling<float>(ZArgs<float>&, int);
template bool zcluster_tiling<double>(ZArgs<double>&, int);
template bool zcluster_tiling<df64>(ZArgs<df64>&, int);

template <typename T>
cudaError_t launch_zcluster(const ZArgs<T>& a, int nrhs, cudaStream_t s) {
  const long long e = (long long)a.g.n3 * (1LL << a.tc_log2);
  if (a.mode != Z_GAMMA || a.ncomp_in != 6 || a.ncomp_out != 6 || !zcluster_tile_fits(a.g, sizeof(cx<T>), a.tc_log2) ||
      e > (long long)kEPT * a.nthr || a.nthr > 512 || nrhs < 1 || (long long)a.ntiles * kZcComps > 0x7fffffffLL)
    return cudaErrorInvalidValue;
  const size_t smem = zcluster_smem(a.g, sizeof(cx<T>), a.tc_log2);
  auto k = zcluster_kernel<T, kEPT>;
  cudaError_t err = set_smem(k, smem);
  if (err != cudaSuccess) return err;
  dim3 grid((unsigned)(a.ntiles * kZcComps), (unsigned)nrhs);
  count_launch();
  k<<<grid, a.nthr, smem, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_zcluster<float>(const ZArgs<float>&, int, cudaStream_t);
template cudaError_t launch_zcluster<double>(const ZArgs<double>&, int, cudaStream_t);
template cudaError_t launch_zcluster<df64>(const ZArgs<df64>&, int, cudaStream_t);

// ---- TMA variant: host side ----------------------------------------------------------------
bool ztma_fits(const Geo& g, int lg) {
  // the plain cluster tile limits, whole 16-byte box rows (2 columns at least) and 16-byte tensor
  // strides (an even number of spectrum columns per plane)
  return lg >= 1 && g.n3 >= 16 && zcluster_tile_fits(g, sizeof(cx<float>), lg) && (g.plane_c % 2) == 0;
}

cudaError_t launch_zcluster_tma(const ZArgs<float>& a, int nrhs, cudaStream_t s) {
  const Geo& g = a.g;
  const long long per = (long long)g.n3 << a.tc_log2;
  if (a.mode != Z_GAMMA || a.ncomp_in != 6 || a.ncomp_out != 6 || !ztma_fits(g, a.tc_log2) || nrhs < 1 ||
      per > (long long)kEPT * a.nthr || a.nthr > 512 || a.ntiles < 1 ||
      (reinterpret_cast<uintptr_t>(a.S) & 15) != 0)
    return cudaErrorInvalidValue;
  const int nbox = (g.n3 + 255) / 256, rows = g.n3 / nbox;
  const size_t elem = sizeof(cx<float>);
  // the spectra of the launch's loads: [6 nrhs component planes][n3][plane_c] 8-byte elements
  CUtensorMap tm;
  const unsigned long long dims[3] = {(unsigned long long)g.plane_c, (unsigned long long)g.n3,
                                      (unsigned long long)kZcComps * nrhs};
  const unsigned long long strides[2] = {(unsigned long long)g.plane_c * elem,
                                         (unsigned long long)g.n3 * g.plane_c * elem};
  const unsigned box[2] = {1u << a.tc_log2, (unsigned)rows};
  if (!encode_tensor_3d(&tm, a.S, dims, strides, box)) return cudaErrorNotSupported;
  const size_t smem = (size_t)(per + g.n3) * elem + 16;
  auto k = zcluster_tma_kernel<kEPT>;
  cudaError_t err = set_smem(k, smem);
  if (err != cudaSuccess) return err;
  dim3 grid((unsigned)(a.ntiles * kZcComps), (unsigned)nrhs);
  count_launch();
  k<<<grid, a.nthr, smem, s>>>(tm, a);
  return cudaGetLastError();
}

}  // namespace hom
