// Forward plane pass of the Lippmann-Schwinger step (see ls_common.cuh).
#include "ls_common.cuh"

namespace hom {

// ---------------------------------------------------------------------------------
// plane_fwd: one CTA per (z-plane, component, rhs)
template <typename Tf, typename T, int EPT>
__global__ void __launch_bounds__(PlaneCfg<T>::kMaxThreads, PlaneCfg<T>::kMinBlocks)
plane_fwd_kernel(const FwdArgs<Tf, T> a) {
  constexpr int kBatch = PlaneCfg<T>::kBatch;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Geo& g = a.g;
  const int z = blockIdx.x, c = blockIdx.y, lrhs = blockIdx.z, rhs = a.rhs0 + lrhs;
  if (a.st != nullptr && a.st[rhs].active == 0) return;

  const int n1 = g.n1, n2 = g.n2, h = g.h, P = g.P;
  cx<T>* pl = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* nyq = pl + n2 * P;
  cx<T>* twh = nyq + n2;       // rows: exp(-2 pi i t / h)
  cx<T>* twy = twh + h;        // columns: exp(-2 pi i t / n2)
  cx<T>* tw1 = twy + n2;       // R2C split: exp(-2 pi i k / n1), k <= h
  T* tab = reinterpret_cast<T*>(tw1 + h + 1);
  size_t off = align16((size_t)(n2 * P + n2 + 2 * h + n2 + 1) * sizeof(cx<T>) + 2 * a.n_phase * sizeof(T));
  double* sh = reinterpret_cast<double*>(smem_raw + off);
  int* flag = reinterpret_cast<int*>(sh + 64);

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;

  {
    // start the plane's field reads now; they land in L2 while the tables load
    const long long psz = (long long)n2 * n1;
    const long long fo = ((long long)(rhs * a.in_ncomp + c) * g.n3 + z) * psz;
    const unsigned pb = (unsigned)(psz * (long long)sizeof(Tf));
    if (tid == 0 && (pb & 15u) == 0) {
      if (a.mode == FWD_CG) {
        prefetch_l2(a.r + fo, pb);
        if (a.st[rhs].restart == 0) {
          prefetch_l2(a.p + fo, pb);
          prefetch_l2(a.x + fo, pb);
        }
      } else if (a.in != nullptr) {
        prefetch_l2(a.in + fo, pb);
      }
    }
  }
  for (int i = tid; i < h; i += nthr) twh[i] = ldg_cx(a.tw_h + i);
  for (int i = tid; i < n2; i += nthr) twy[i] = ldg_cx(a.tw_n2 + i);
  for (int i = tid; i <= h; i += nthr) tw1[i] = ldg_cx(a.tw_n1 + i);
  const int rve = rve_of(rhs, a.rve_loads);
  if (a.mode != FWD_COPY && a.mode != FWD_C0) {
    const T* mat = a.mat + (long long)rve * kRveTable;
    for (int i = tid; i < a.n_phase; i += nthr) {
      tab[i] = mat[i * 4 + (c == 0 ? 0 : 1)];                 // C - C0 eigenvalue
      tab[a.n_phase + i] = mat[i * 4 + (c == 0 ? 2 : 3)];     // C eigenvalue
    }
  }
  __syncthreads();

  const long long plane_sz = (long long)n2 * n1;
  const long long foff = ((long long)(rhs * a.in_ncomp + c) * g.n3 + z) * plane_sz;
  if (a.prof != nullptr && tid == 0) {
    // algorithmic bytes: field planes read/written once, phase bytes, spectrum plane written
    long long fields = (a.mode == FWD_CG) ? (a.st[rhs].restart ? 2 : 5)
                                          : ((a.mode == FWD_COPY || a.mode == FWD_C0 || a.in != nullptr) ? 1 : 0);
    long long b = fields * plane_sz * (long long)sizeof(Tf) + g.plane_c * (long long)sizeof(cx<T>);
    if (a.mode != FWD_COPY && a.mode != FWD_C0) b += plane_sz;
    atomicAdd(a.prof, (unsigned long long)b);
    atomicAdd(a.prof + 1, (unsigned long long)plane_sz);
  }
  const uint8_t* php = a.phase + (long long)rve * g.M + (long long)z * plane_sz;
  T acc = (T)0;

  if (a.mode == FWD_TAU || a.mode == FWD_STRESS) {
    const T ec = (a.E != nullptr) ? (T)a.E[rhs * 6 + c] : (T)0;
    const T* w = (a.mode == FWD_TAU) ? tab : tab + a.n_phase;
    #pragma unroll 4
    for (int row = warp; row < n2; row += nwarp) {
      for (int c2 = lane; c2 < h; c2 += 32) {
        const long long o = (long long)row * n1 + 2 * c2;
        Tf v0 = 0, v1 = 0;
        if (a.in != nullptr) ld2<Tf>(a.in + foff + o, v0, v1);
        const uchar2 ph = *reinterpret_cast<const uchar2*>(php + o);
        pl[row * P + c2] = mk<T>(w[ph.x] * ((T)v0 + ec), w[ph.y] * ((T)v1 + ec));
      }
    }
  } else if (a.mode == FWD_CG) {
    // Flat element index e = row * h + col; the loads of kBatch elements per thread are issued
    // before the first store of p (which the compiler must assume may alias r).
    const RhsState& s = a.st[rhs];
    const bool restart = (s.restart != 0);
    const T beta = restart ? (T)0 : (T)s.beta;
    const T alpha = restart ? (T)0 : (T)s.alpha;
    const Tf* rp = a.r + foff;
    Tf* pp = a.p + foff;
    Tf* xp = a.x + foff;
    const int total = n2 * h;
    for (int e0 = tid; e0 < total; e0 += kBatch * nthr) {
      Tf r0[kBatch], r1[kBatch], p0[kBatch], p1[kBatch], x0[kBatch], x1[kBatch];
      uchar2 ph[kBatch];
      int rw[kBatch];
      #pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int e = e0 + j * nthr;
        rw[j] = (int)g.fd_h.div((unsigned)e);
        p0[j] = 0;
        p1[j] = 0;
        if (e < total) {
          const int o = rw[j] * n1 + 2 * (e - rw[j] * h);
          ld2<Tf>(rp + o, r0[j], r1[j]);
          if (!restart) {   // a restart neither reads the old p nor has an update of x pending
            ld2<Tf>(pp + o, p0[j], p1[j]);
            ld2<Tf>(xp + o, x0[j], x1[j]);
          }
          ph[j] = *reinterpret_cast<const uchar2*>(php + o);
        }
      }
      #pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int e = e0 + j * nthr;
        if (e < total) {
          const int col = e - rw[j] * h, o = rw[j] * n1 + 2 * col;
          if (!restart) st2<Tf>(xp + o, (Tf)((T)x0[j] + alpha * (T)p0[j]), (Tf)((T)x1[j] + alpha * (T)p1[j]));
          const T q0 = (T)r0[j] + beta * (T)p0[j];
          const T q1 = (T)r1[j] + beta * (T)p1[j];
          st2<Tf>(pp + o, (Tf)q0, (Tf)q1);
          const T c0 = tab[a.n_phase + ph[j].x], c1 = tab[a.n_phase + ph[j].y];
          acc += c0 * q0 * q0 + c1 * q1 * q1;
          pl[rw[j] * P + col] = mk<T>(c0 * q0, c1 * q1);
        }
      }
    }
  } else {  // FWD_COPY, FWD_C0
    T ch, cd;
    c0_weights<T>(a.c0, rve, a.c0h, a.c0d, ch, cd);
    const T w = (a.mode == FWD_C0) ? (c == 0 ? ch : cd) : (T)1;
    #pragma unroll 4
    for (int row = warp; row < n2; row += nwarp) {
      for (int c2 = lane; c2 < h; c2 += 32) {
        const long long o = (long long)row * n1 + 2 * c2;
        Tf v0, v1;
        ld2<Tf>(a.in + foff + o, v0, v1);
        pl[row * P + c2] = mk<T>(w * (T)v0, w * (T)v1);
      }
    }
  }
  __syncthreads();

  // x axis: length-h complex FFT of the packed rows z[n] = x[2n] + i x[2n+1]
  fft_pencils<T, -1, EPT>(pl, RowAddr{P}, h, n2, g.fd_n2, twh);

  // R2C split: X[k] = (Z[k] + conj Z[h-k])/2 - i W^k (Z[k] - conj Z[h-k])/2, W = e^{-2 pi i/n1}.
  // X[0] and X[n1/2] are real and share slot 0 as X[0] + i X[n1/2].
  {
    const int nk = h / 2 + 1;
    for (int t = tid; t < n2 * nk; t += nthr) {
      const int row = t % n2, k = t / n2;
      cx<T>* R = pl + row * P;
      if (k == 0) {
        const cx<T> z0 = R[0];
        R[0] = mk<T>(z0.re + z0.im, z0.re - z0.im);
      } else if (2 * k == h) {
        R[k] = conj(R[k]);
      } else {
        const cx<T> za = R[k], zb = R[h - k];
        const cx<T> wa = tw1[k], wb = tw1[h - k];
        // X[k]
        cx<T> e = (za + conj(zb)) * (T)0.5;
        cx<T> o = mul_i<T, -1>(za - conj(zb)) * (T)0.5;
        const cx<T> xa = e + cmul(wa, o);
        // X[h-k]
        e = (zb + conj(za)) * (T)0.5;
        o = mul_i<T, -1>(zb - conj(za)) * (T)0.5;
        const cx<T> xb = e + cmul(wb, o);
        R[k] = xa;
        R[h - k] = xb;
      }
    }
  }
  __syncthreads();

  // y axis: columns kx = 0..h-1 (column 0 carries X[0] + i X[n1/2])
  fft_pencils<T, -1, EPT>(pl, ColAddr{P}, n2, h, g.fd_h, twy);

  // separate column 0 into the kx = 0 column (A) and the Nyquist column kx = n1/2 (B):
  // A[k] = (P[k] + conj P[-k])/2,  B[k] = (P[k] - conj P[-k])/(2i)
  for (int ky = tid; 2 * ky <= n2; ky += nthr) {
    const int km = (n2 - ky) % n2;
    const cx<T> pk = pl[ky * P], pm = pl[km * P];
    const cx<T> ak = (pk + conj(pm)) * (T)0.5;
    const cx<T> bk = mul_i<T, -1>(pk - conj(pm)) * (T)0.5;
    const cx<T> am = (pm + conj(pk)) * (T)0.5;
    const cx<T> bm = mul_i<T, -1>(pm - conj(pk)) * (T)0.5;
    pl[ky * P] = ak;
    nyq[ky] = bk;
    if (km != ky) {
      pl[km * P] = am;
      nyq[km] = bm;
    }
  }
  __syncthreads();

  cx<T>* Sp = a.S + ((long long)(lrhs * a.ncomp + c) * g.n3 + z) * g.plane_c;
  // the spectrum plane is contiguous (row pitch h): flat index e = row * h + col
  for (int e = tid; e < n2 * h; e += nthr) {
    const int row = (int)g.fd_h.div((unsigned)e);
    Sp[e] = pl[row * P + (e - row * h)];
  }
  for (int ky = tid; ky < n2; ky += nthr) Sp[(long long)n2 * h + ky] = nyq[ky];

  if (a.mode == FWD_CG) {
    double v[1] = {(double)acc};
    block_sum_f64<1>(v, sh);
    const int ncta = a.ncomp * g.n3;
    if (publish_and_collect<1>(v, a.part + (long long)rhs * 2 * ncta, a.cnt + rhs, ncta, c * g.n3 + z,
                               sh, flag)) {
      if (threadIdx.x == 0) finalize_state(FIN_ENERGY, a.st[rhs], v, 1.0 / (double)g.M);
    }
  }
}

void geo_finish(Geo& g) {
  g.fd_h = make_fastdiv((unsigned)g.h);
  g.fd_n2 = make_fastdiv((unsigned)g.n2);
  // split passes: x pass with rb rows of h values per CTA (<= kEPT * 256 elements),
  // y pass with 2^ty_log2 columns (a power of two dividing h, <= 16) of n2 values per CTA
  const long long nrows = (long long)g.n2 * g.n3;
  long long rb = (kEPT * 256) / g.h;
  if (rb < 1) rb = 1;
  if (rb > nrows) rb = nrows;
  g.rb = (int)rb;
  g.nrb = (int)((nrows + rb - 1) / rb);
  int tx = (int)((rb * g.h + kEPT - 1) / kEPT);
  tx = ((tx + 31) / 32) * 32;
  g.thr_x = tx < 64 ? 64 : tx;
  g.fd_rb = make_fastdiv((unsigned)g.rb);
  int lg = 0;
  while (lg < 4 && (g.h % (2 << lg)) == 0 && (long long)g.n2 * (2 << lg) <= (long long)kEPT * 512) ++lg;
  set_ytile(g, lg);
}

bool ytile_fits(const Geo& g, int lg) {
  return lg >= 0 && lg <= 4 && (g.h % (1 << lg)) == 0 && (long long)g.n2 * (1 << lg) <= (long long)kEPT * 512;
}

void set_ytile(Geo& g, int lg) {
  g.ty_log2 = lg;
  int ty = (int)(((long long)g.n2 * (1 << lg) + kEPT - 1) / kEPT);
  ty = ((ty + 31) / 32) * 32;
  g.thr_y = ty < 64 ? 64 : ty;
  g.fd_ty = make_fastdiv((unsigned)(1 << lg));
}

size_t plane_smem_bytes(const Geo& g, size_t elem) {
  size_t b = (size_t)(g.n2 * g.P + g.n2 + 2 * g.h + g.n2 + 1) * elem + 2 * 256 * elem;
  b = (b + 15) & ~size_t(15);
  return b + 64 * sizeof(double) + 16;
}
size_t zpass_smem_bytes(const Geo& g, size_t elem, int ncomp, int tc_log2) {
  const size_t tc = (size_t)1 << tc_log2;
  const size_t cstride = g.n3 * tc + ((g.n3 % 2 == 0) ? tc : 0);
  return ((size_t)ncomp * cstride + g.n3) * elem;
}

// z-pass tile: 2^lg consecutive spectrum columns (lg <= 4) whose pencils fit kEPT elements per
// thread at <= 512 threads and <= 64 KB of shared memory.  Among the tiles whose row reads cover
// at least one 32-byte sector, the one with the most resident warps per SM wins (ties: the
// wider tile); at 128^3 in FP32 that is 4 columns (192 threads, 5 CTAs per SM) rather than 8
// (384 threads, 2 CTAs per SM at the kernel's register count).
static int zpass_threads(int ncomp, int n3, int lg) {
  const long long e = (long long)ncomp * n3 * (1LL << lg);
  int thr = (int)((e + kEPT - 1) / kEPT);
  thr = ((thr + 31) / 32) * 32;
  return thr < 128 ? 128 : thr;
}

bool zpass_tile_fits(const Geo& g, size_t elem, int ncomp, int lg) {
  return lg >= 0 && lg <= 4 && (size_t)ncomp * g.n3 * ((size_t)1 << lg) <= (size_t)kEPT * 512 &&
         zpass_smem_bytes(g, elem, ncomp, lg) <= 64 * 1024;
}

template <typename T>
void zpass_tiling(ZArgs<T>& a, int force_lg) {
  const size_t elem = sizeof(cx<T>);
  int best_lg = -1;
  long long best_warps = -1;
  const bool forced = force_lg >= 0 && zpass_tile_fits(a.g, elem, a.ncomp_in, force_lg);
  if (forced) best_lg = force_lg;
  for (int lg = 4; lg >= 0 && !forced; --lg) {
    if (!zpass_tile_fits(a.g, elem, a.ncomp_in, lg)) continue;
    if (best_lg >= 0 && ((size_t)1 << lg) * elem < 32) break;   // narrower than a sector
    const int thr = zpass_threads(a.ncomp_in, a.g.n3, lg);
    const long long warps =
        (long long)zpass_ctas_per_sm<T>(thr, zpass_smem_bytes(a.g, elem, a.ncomp_in, lg)) * (thr / 32);
    if (best_lg < 0 || warps > best_warps) {
      best_lg = lg;
      best_warps = warps;
    }
  }
  const int lg = best_lg < 0 ? 0 : best_lg;
  a.tc_log2 = lg;
  const long long tc = 1LL << lg;
  a.ntiles = (int)((a.g.plane_c + tc - 1) / tc);
  // component stride = n3 * tc, padded to an odd multiple of tc so that the 2 to 4 components
  // a warp touches fall in different shared-memory banks
  a.cstride = (int)(a.g.n3 * tc + ((a.g.n3 % 2 == 0) ? tc : 0));
  a.fd_in = make_fastdiv((unsigned)(a.ncomp_in * tc));
  a.fd_out = make_fastdiv((unsigned)(a.ncomp_out * tc));
  a.fd_comp = make_fastdiv((unsigned)(a.g.n3 * tc));
  a.nthr = zpass_threads(a.ncomp_in, a.g.n3, lg);
}
template void zpass_tiling<float>(ZArgs<float>&, int);
template void zpass_tiling<double>(ZArgs<double>&, int);
template void zpass_tiling<df64>(ZArgs<df64>&, int);

template <typename Tf, typename T>
cudaError_t launch_plane_fwd(const FwdArgs<Tf, T>& a, int nrhs, cudaStream_t s) {
  const int thr = plane_threads<T>(a.g);
  if ((long long)a.g.n2 * a.g.h > (long long)PlaneCfg<T>::kEPT * thr || thr > PlaneCfg<T>::kMaxThreads ||
      a.n_phase > 256)
    return cudaErrorInvalidValue;
  const size_t smem = plane_smem_bytes(a.g, sizeof(cx<T>));
  auto k = plane_fwd_kernel<Tf, T, PlaneCfg<T>::kEPT>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.g.n3, a.ncomp, nrhs);
  count_launch();
  k<<<grid, thr, smem, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_plane_fwd<float, float>(const FwdArgs<float, float>&, int, cudaStream_t);
template cudaError_t launch_plane_fwd<double, double>(const FwdArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_plane_fwd<double, df64>(const FwdArgs<double, df64>&, int, cudaStream_t);

}  // namespace hom
