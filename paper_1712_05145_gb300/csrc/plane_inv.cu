// Inverse plane pass of the Lippmann-Schwinger step with the solver epilogues.
#include "ls_common.cuh"

namespace hom {

// ---------------------------------------------------------------------------------
// plane_inv: one CTA per (z-plane, component, rhs)
template <typename Tf, typename T, int EPT>
__global__ void __launch_bounds__(PlaneCfg<T>::kMaxThreads, PlaneCfg<T>::kMinBlocks)
plane_inv_kernel(const InvArgs<Tf, T> a) {
  constexpr int kBatch = PlaneCfg<T>::kBatch;
  const int s_ncomp = a.s_ncomp;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Geo& g = a.g;
  const int z = blockIdx.x, c = blockIdx.y, lrhs = blockIdx.z, rhs = a.rhs0 + lrhs;
  if (a.st != nullptr && a.st[rhs].active == 0) return;
  T c0h, c0d;
  c0_weights<T>(a.c0, rve_of(rhs, a.rve_loads), a.c0h, a.c0d, c0h, c0d);
  const int n1 = g.n1, n2 = g.n2, h = g.h, P = g.P;
  cx<T>* pl = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* twh = pl + n2 * P + n2;   // rows: exp(-2 pi i t / h)
  cx<T>* twy = twh + h;            // columns: exp(-2 pi i t / n2)
  cx<T>* tw1 = twy + n2;           // C2R merge: exp(-2 pi i k / n1), k <= h
  size_t off = align16((size_t)(n2 * P + n2 + 2 * h + n2 + 1) * sizeof(cx<T>));
  double* sh = reinterpret_cast<double*>(smem_raw + off);
  int* flag = reinterpret_cast<int*>(sh + 64);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  {
    // the epilogue's field planes are fetched into L2 while the transforms run
    const long long psz = (long long)n2 * n1;
    const unsigned pb = (unsigned)(psz * (long long)sizeof(Tf));
    if (tid == 0 && (pb & 15u) == 0) {
      if (a.mode == INV_CG) {
        const long long fo = ((long long)(rhs * 6 + c) * g.n3 + z) * psz;
        prefetch_l2(a.r + fo, pb);
      } else {
        const long long fo = ((long long)(rhs * a.out_ncomp + c) * g.n3 + z) * psz;
        if (a.b != nullptr) prefetch_l2(a.b + fo, (unsigned)(psz * (long long)sizeof(double)));
        if (a.xsub != nullptr) prefetch_l2(a.xsub + fo, (unsigned)(psz * (long long)sizeof(double)));
        if (a.fin == FIN_BASIC && a.prev != nullptr) prefetch_l2(a.prev + fo, pb);
      }
    }
  }
  // the spectrum plane (contiguous, row pitch h: flat index e = row * h + col) goes to shared
  // memory (row pitch P) by cp.async while the twiddle tables load; the Nyquist column kx = n1/2
  // lands in the n2 slots after the plane
  const cx<T>* Sp = a.S + ((long long)(lrhs * s_ncomp + c) * g.n3 + z) * g.plane_c;
  const int nmain = n2 * h;
  cx<T>* nyq = pl + n2 * P;
  for (int e = tid; e < nmain; e += nthr) {
    const int row = (int)g.fd_h.div((unsigned)e), col = e - row * h;
    cp_async_elem<sizeof(cx<T>)>(pl + row * P + col, Sp + e);
  }
  for (int ky = tid; ky < n2; ky += nthr) cp_async_elem<sizeof(cx<T>)>(nyq + ky, Sp + nmain + ky);
  for (int i = tid; i < h; i += nthr) twh[i] = ldg_cx(a.tw_h + i);
  for (int i = tid; i < n2; i += nthr) twy[i] = ldg_cx(a.tw_n2 + i);
  for (int i = tid; i <= h; i += nthr) tw1[i] = ldg_cx(a.tw_n1 + i);

  if (a.prof != nullptr && tid == 0) {
    const long long psz = (long long)n2 * n1;
    long long fields = (a.mode == INV_CG) ? 2 : 1 + (a.fin == FIN_BASIC);
    long long b = fields * psz * (long long)sizeof(Tf) + g.plane_c * (long long)sizeof(cx<T>);
    if (a.b != nullptr) b += psz * (long long)sizeof(double);
    if (a.xsub != nullptr) b += psz * (long long)sizeof(double);
    atomicAdd(a.prof, (unsigned long long)b);
    atomicAdd(a.prof + 1, (unsigned long long)psz);
  }
  cp_async_wait_all();
  __syncthreads();
  for (int row = tid; row < n2; row += nthr) {   // pack kx = 0 (A) and kx = n1/2 (B) as A + i B
    const cx<T> v = pl[row * P], b = nyq[row];
    pl[row * P] = mk<T>(v.re - b.im, v.im + b.re);
  }
  __syncthreads();

  fft_pencils<T, +1, EPT>(pl, ColAddr{P}, n2, h, g.fd_h, twy);

  // C2R merge: Z[k] = X[k] + conj X[h-k] + i W^{-k} (X[k] - conj X[h-k]),  W = e^{-2 pi i/n1};
  // slot 0 holds X[0] + i X[n1/2]
  {
    const int nk = h / 2 + 1;
    for (int t = tid; t < n2 * nk; t += nthr) {
      const int row = t % n2, k = t / n2;
      cx<T>* R = pl + row * P;
      if (k == 0) {
        const T x0 = R[0].re, xn = R[0].im;
        R[0] = mk<T>(x0 + xn, x0 - xn);
      } else if (2 * k == h) {
        R[k] = conj(R[k]) * (T)2;
      } else {
        const cx<T> xa = R[k], xb = R[h - k];
        const cx<T> wa = conj(tw1[k]), wb = conj(tw1[h - k]);
        const cx<T> za = (xa + conj(xb)) + mul_i<T, 1>(cmul(wa, xa - conj(xb)));
        const cx<T> zb = (xb + conj(xa)) + mul_i<T, 1>(cmul(wb, xb - conj(xa)));
        R[k] = za;
        R[h - k] = zb;
      }
    }
  }
  __syncthreads();

  fft_pencils<T, +1, EPT>(pl, RowAddr{P}, h, n2, g.fd_n2, twh);

  // epilogue on the real plane: x[2n] = Re z[n], x[2n+1] = Im z[n]
  const long long plane_sz = (long long)n2 * n1;
  T q0 = 0, q1 = 0;
  if (a.mode == INV_STORE) {
    const long long foff = ((long long)(rhs * a.out_ncomp + c) * g.n3 + z) * plane_sz;
    const T cw = (c == 0) ? c0h : c0d;
    #pragma unroll 4
    for (int row = warp; row < n2; row += nwarp) {
      for (int c2 = lane; c2 < h; c2 += 32) {
        const long long o = foff + (long long)row * n1 + 2 * c2;
        const cx<T> e = pl[row * P + c2];
        T v0 = a.out_scale * e.re, v1 = a.out_scale * e.im;
        if (a.b != nullptr) { double b0, b1; ld2<double>(a.b + o, b0, b1); v0 += (T)b0; v1 += (T)b1; }
        if (a.xsub != nullptr) { double s0, s1; ld2<double>(a.xsub + o, s0, s1); v0 -= (T)s0; v1 -= (T)s1; }
        if (a.fin == FIN_BASIC) {
          Tf p0, p1;
          ld2<Tf>(a.prev + o, p0, p1);
          const T d0 = v0 - (T)p0, d1 = v1 - (T)p1;
          q0 += d0 * d0 + d1 * d1;
        } else {
          q0 += cw * (v0 * v0 + v1 * v1);
        }
        q1 += v0 * v0 + v1 * v1;
        st2<Tf>(a.out + o, (Tf)v0, (Tf)v1);
      }
    }
  } else {  // INV_CG: q = A p = Gamma0 * (C : p) = -eta, r -= alpha q (x += alpha p: next forward pass)
    // Flat element index e = row * h + col; each thread issues the loads of kBatch elements
    // before the first store, so that they are in flight together (a store to r may alias the
    // next load for the compiler, which would otherwise serialise load -> store chains).
    const long long foff = ((long long)(rhs * 6 + c) * g.n3 + z) * plane_sz;
    const T alpha = (T)a.st[rhs].alpha;
    const T cw = (c == 0) ? c0h : c0d;
    Tf* rp = a.r + foff;
    const int total = n2 * h;
    for (int e0 = tid; e0 < total; e0 += kBatch * nthr) {
      Tf r0[kBatch], r1[kBatch];
      int rw[kBatch];
      #pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int e = e0 + j * nthr;
        rw[j] = (int)g.fd_h.div((unsigned)e);
        if (e < total) {
          const int o = rw[j] * n1 + 2 * (e - rw[j] * h);
          ld2<Tf>(rp + o, r0[j], r1[j]);
        }
      }
      #pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int e = e0 + j * nthr;
        if (e < total) {
          const int col = e - rw[j] * h, o = rw[j] * n1 + 2 * col;
          const cx<T> v = pl[rw[j] * P + col];
          const T ra = (T)r0[j] + alpha * v.re, rb = (T)r1[j] + alpha * v.im;
          st2<Tf>(rp + o, (Tf)ra, (Tf)rb);
          q0 += cw * (ra * ra + rb * rb);
          q1 += ra * ra + rb * rb;
        }
      }
    }
  }

  if (a.fin != FIN_NONE) {
    double v[2] = {(double)q0, (double)q1};
    block_sum_f64<2>(v, sh);
    const int ncta = a.ncomp * g.n3;
    if (publish_and_collect<2>(v, a.part + (long long)rhs * 2 * ncta, a.cnt + rhs, ncta, c * g.n3 + z,
                               sh, flag)) {
      if (threadIdx.x == 0) finalize_state(a.fin, a.st[rhs], v, 1.0 / (double)g.M);
    }
  }
}

template <typename Tf, typename T>
cudaError_t launch_plane_inv(const InvArgs<Tf, T>& a, int nrhs, cudaStream_t s) {
  const int thr = plane_threads<T>(a.g);
  if ((long long)a.g.n2 * a.g.h > (long long)PlaneCfg<T>::kEPT * thr || thr > PlaneCfg<T>::kMaxThreads)
    return cudaErrorInvalidValue;
  const size_t smem = plane_smem_bytes(a.g, sizeof(cx<T>));
  auto k = plane_inv_kernel<Tf, T, PlaneCfg<T>::kEPT>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.g.n3, a.ncomp, nrhs);
  count_launch();
  k<<<grid, thr, smem, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_plane_inv<float, float>(const InvArgs<float, float>&, int, cudaStream_t);
template cudaError_t launch_plane_inv<double, double>(const InvArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_plane_inv<float, double>(const InvArgs<float, double>&, int, cudaStream_t);
template cudaError_t launch_plane_inv<float, df64>(const InvArgs<float, df64>&, int, cudaStream_t);
template cudaError_t launch_plane_inv<double, df64>(const InvArgs<double, df64>&, int, cudaStream_t);

}  // namespace hom
