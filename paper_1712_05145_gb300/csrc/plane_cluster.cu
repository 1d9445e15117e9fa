// Cluster plane passes of the Lippmann-Schwinger step for x-y planes larger than one CTA's shared
// memory (e.g. 512 x 512: 256 x 512 complex values, 1 MB in FP32).
//
// Q CTAs (a thread-block cluster, Q = 2, 4, 8 or 16) transform one (load, component, z-plane)
// together.  CTA q owns rows [qR, (q+1)R) of the plane (R = N2 / Q) for the x-axis work and
// columns [qCb, (q+1)Cb) of the half spectrum (Cb = (N1/2) / Q) for the y-axis work; between the
// two the plane is transposed through distributed shared memory: each CTA reads its column block
// out of the other CTAs' row blocks.  The forward pass applies the same prologues as plane_fwd
// (polarization, Eq. auxiliary_problem; stress; CG direction; copy; C0) to its rows, runs the
// packed real-to-complex row FFT, the transpose, the column FFT and writes its columns of the
// spectrum; the inverse pass reads its columns, runs the inverse column FFT, the transpose, the
// complex-to-real merge and row FFT, and the same epilogues as plane_inv (store, fixed-point step,
// CG vector updates) with their FP64 reductions.
//
// Compared with the split x and y passes, the intermediate half spectrum between the x and y
// transforms never leaves the chip: two fewer spectrum sweeps through HBM per direction.
#include <cooperative_groups.h>

#include <vector>

#include "ls_common.cuh"
#include "plane_cluster.h"

namespace cg = cooperative_groups;

namespace hom {

constexpr int kPcMaxThreads = 1024;
constexpr size_t kPcMaxSmem = 200 * 1024;

// Shared-memory layout of a cluster plane CTA (complex elements of T unless noted):
//   buf  [R][P] rows (x phase), reused as [N2][Cb] columns (y phase)   R * P >= N2 * Cb
//   nyq  [N2]   Nyquist column kx = N1/2 (CTA 0)
//   twh  [h]    exp(-2 pi i t / h);   twy [N2] exp(-2 pi i t / N2);   tw1 [h + 1] exp(-2 pi i k / N1)
//   tab  [2 * 256] T: per-phase eigenvalues (C - C0, C) of this component
//   sh   64 doubles + flag (FP64 block reduction)
static size_t pc_smem_bytes(const Geo& g, size_t elem, size_t real) {
  size_t b = (size_t)(g.pc_R * g.P + g.n2 + g.h + g.n2 + g.h + 1) * elem + 2 * 256 * real;
  b = (b + 15) & ~size_t(15);
  return b + 64 * sizeof(double) + 16;
}

template <typename Tf, typename T, int EPT>
__global__ void __launch_bounds__(kPcMaxThreads, 1) plane_fwd_cluster_kernel(const FwdArgs<Tf, T> a) {
  constexpr int kBatch = PlaneCfg<T>::kBatch;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const Geo& g = a.g;
  const int Q = g.pc_Q, R = g.pc_R, Cb = g.pc_Cb;
  const int q = (int)cl.block_rank();
  const int z = blockIdx.x / Q, c = blockIdx.y, lrhs = blockIdx.z, rhs = a.rhs0 + lrhs;
  // the Q CTAs of a cluster share the load, so they leave together (before any barrier)
  if (a.st != nullptr && a.st[rhs].active == 0) return;
  const int n1 = g.n1, n2 = g.n2, h = g.h, P = g.P;
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* nyq = buf + R * P;
  cx<T>* twh = nyq + n2;
  cx<T>* twy = twh + h;
  cx<T>* tw1 = twy + n2;
  T* tab = reinterpret_cast<T*>(tw1 + h + 1);
  size_t off = align16((size_t)(R * P + n2 + h + n2 + h + 1) * sizeof(cx<T>) + 2 * 256 * sizeof(T));
  double* sh = reinterpret_cast<double*>(smem_raw + off);
  int* flag = reinterpret_cast<int*>(sh + 64);
  const int tid = threadIdx.x, nthr = blockDim.x;

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

  const int y0 = q * R;                                   // first plane row of this CTA
  const long long plane_sz = (long long)n2 * n1;
  const long long foff = ((long long)(rhs * a.in_ncomp + c) * g.n3 + z) * plane_sz + (long long)y0 * n1;
  const long long blk_sz = (long long)R * n1;             // voxels of this CTA's rows
  if (a.prof != nullptr && tid == 0) {
    long long fields = (a.mode == FWD_CG) ? (a.st[rhs].restart ? 2 : 5)
                                          : ((a.mode == FWD_COPY || a.mode == FWD_C0 || a.in != nullptr) ? 1 : 0);
    long long b = fields * blk_sz * (long long)sizeof(Tf) + (long long)n2 * Cb * (long long)sizeof(cx<T>);
    if (q == 0) b += (long long)n2 * (long long)sizeof(cx<T>);
    if (a.mode != FWD_COPY && a.mode != FWD_C0) b += blk_sz;
    atomicAdd(a.prof, (unsigned long long)b);
    atomicAdd(a.prof + 1, (unsigned long long)blk_sz);
  }
  const uint8_t* php = a.phase + (long long)rve * g.M + (long long)z * plane_sz + (long long)y0 * n1;
  T acc = (T)0;
  const int total = R * h;   // complex elements of this CTA's rows (flat index e = row * h + col)

  if (a.mode == FWD_TAU || a.mode == FWD_STRESS) {
    const T ec = (a.E != nullptr) ? (T)a.E[rhs * 6 + c] : (T)0;
    const T* w = (a.mode == FWD_TAU) ? tab : tab + a.n_phase;
    for (int e = tid; e < total; e += nthr) {
      const int row = (int)g.fd_h.div((unsigned)e), col = e - row * h;
      const long long o = (long long)row * n1 + 2 * col;
      Tf v0 = 0, v1 = 0;
      if (a.in != nullptr) ld2<Tf>(a.in + foff + o, v0, v1);
      const uchar2 ph = *reinterpret_cast<const uchar2*>(php + o);
      buf[row * P + col] = mk<T>(w[ph.x] * ((T)v0 + ec), w[ph.y] * ((T)v1 + ec));
    }
  } else if (a.mode == FWD_CG) {
    // the loads of kBatch elements per thread are issued before the first store of p
    const RhsState& s = a.st[rhs];
    const bool restart = (s.restart != 0);
    const T beta = restart ? (T)0 : (T)s.beta;
    const T alpha = restart ? (T)0 : (T)s.alpha;
    const Tf* rp = a.r + foff;
    Tf* pp = a.p + foff;
    Tf* xp = a.x + foff;
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
          buf[rw[j] * P + col] = mk<T>(c0 * q0, c1 * q1);
        }
      }
    }
  } else {  // FWD_COPY, FWD_C0
    T ch, cd;
    c0_weights<T>(a.c0, rve, a.c0h, a.c0d, ch, cd);
    const T w = (a.mode == FWD_C0) ? (c == 0 ? ch : cd) : (T)1;
    for (int e = tid; e < total; e += nthr) {
      const int row = (int)g.fd_h.div((unsigned)e), col = e - row * h;
      const long long o = (long long)row * n1 + 2 * col;
      Tf v0, v1;
      ld2<Tf>(a.in + foff + o, v0, v1);
      buf[row * P + col] = mk<T>(w * (T)v0, w * (T)v1);
    }
  }
  __syncthreads();

  // x axis on this CTA's rows: length-h complex FFT of z[n] = x[2n] + i x[2n+1], then the R2C split
  fft_pencils<T, -1, EPT>(buf, RowAddr{P}, h, R, g.pc_fdR, twh);
  {
    const int nk = h / 2 + 1;
    for (int t = tid; t < R * nk; t += nthr) {
      const int k = (int)g.pc_fdR.div((unsigned)t), row = t - k * R;
      cx<T>* Rw = buf + row * P;
      if (k == 0) {
        const cx<T> z0 = Rw[0];
        Rw[0] = mk<T>(z0.re + z0.im, z0.re - z0.im);
      } else if (2 * k == h) {
        Rw[k] = conj(Rw[k]);
      } else {
        const cx<T> za = Rw[k], zb = Rw[h - k];
        const cx<T> wa = tw1[k], wb = tw1[h - k];
        cx<T> e = (za + conj(zb)) * (T)0.5;
        cx<T> o = mul_i<T, -1>(za - conj(zb)) * (T)0.5;
        const cx<T> xa = e + cmul(wa, o);
        e = (zb + conj(za)) * (T)0.5;
        o = mul_i<T, -1>(zb - conj(za)) * (T)0.5;
        const cx<T> xb = e + cmul(wb, o);
        Rw[k] = xa;
        Rw[h - k] = xb;
      }
    }
  }
  cl.sync();   // every row of the plane is transformed along x

  // transpose: this CTA's column block [q Cb, (q+1) Cb) of all n2 rows, element e = y * Cb + j
  {
    cx<T> v[EPT];
    const int ncol = n2 * Cb;
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * nthr;
      if (e < ncol) {
        const int y = (int)g.pc_fdCb.div((unsigned)e), j = e - y * Cb;
        const int src = (int)g.pc_fdR.div((unsigned)y), r = y - src * R;
        const cx<T>* rb = cl.map_shared_rank(buf, src);
        v[i] = rb[r * P + q * Cb + j];
      }
    }
    cl.sync();   // every CTA has read its columns; the row blocks may be overwritten
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * nthr;
      if (e < ncol) buf[e] = v[i];   // column layout [y][j], pitch Cb
    }
  }
  __syncthreads();

  // y axis: Cb columns of length n2 (CTA 0's column 0 carries X[0] + i X[n1/2])
  fft_pencils<T, -1, EPT>(buf, ColAddr{Cb}, n2, Cb, g.pc_fdCb, twy);
  if (q == 0) {
    // separate column 0 into kx = 0 (A) and the Nyquist column kx = n1/2 (B)
    for (int ky = tid; 2 * ky <= n2; ky += nthr) {
      const int km = (n2 - ky) % n2;
      const cx<T> pk = buf[ky * Cb], pm = buf[km * Cb];
      const cx<T> ak = (pk + conj(pm)) * (T)0.5;
      const cx<T> bk = mul_i<T, -1>(pk - conj(pm)) * (T)0.5;
      const cx<T> am = (pm + conj(pk)) * (T)0.5;
      const cx<T> bm = mul_i<T, -1>(pm - conj(pk)) * (T)0.5;
      buf[ky * Cb] = ak;
      nyq[ky] = bk;
      if (km != ky) {
        buf[km * Cb] = am;
        nyq[km] = bm;
      }
    }
    __syncthreads();
  }

  cx<T>* Sp = a.S + ((long long)(lrhs * a.ncomp + c) * g.n3 + z) * g.plane_c;
  for (int e = tid; e < n2 * Cb; e += nthr) {
    const int y = (int)g.pc_fdCb.div((unsigned)e), j = e - y * Cb;
    Sp[(long long)y * h + q * Cb + j] = buf[e];
  }
  if (q == 0)
    for (int ky = tid; ky < n2; ky += nthr) Sp[(long long)n2 * h + ky] = nyq[ky];

  if (a.mode == FWD_CG) {
    double v[1] = {(double)acc};
    block_sum_f64<1>(v, sh);
    const int ncta = a.ncomp * g.n3 * Q;
    if (publish_and_collect<1>(v, a.part + (long long)rhs * 2 * ncta, a.cnt + rhs, ncta, (c * g.n3 + z) * Q + q,
                               sh, flag)) {
      if (threadIdx.x == 0) finalize_state(FIN_ENERGY, a.st[rhs], v, 1.0 / (double)g.M);
    }
  }
}

template <typename Tf, typename T, int EPT>
__global__ void __launch_bounds__(kPcMaxThreads, 1) plane_inv_cluster_kernel(const InvArgs<Tf, T> a) {
  constexpr int kBatch = PlaneCfg<T>::kBatch;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const Geo& g = a.g;
  const int Q = g.pc_Q, R = g.pc_R, Cb = g.pc_Cb;
  const int q = (int)cl.block_rank();
  const int z = blockIdx.x / Q, c = blockIdx.y, lrhs = blockIdx.z, rhs = a.rhs0 + lrhs;
  if (a.st != nullptr && a.st[rhs].active == 0) return;
  const int n1 = g.n1, n2 = g.n2, h = g.h, P = g.P;
  T c0h, c0d;
  c0_weights<T>(a.c0, rve_of(rhs, a.rve_loads), a.c0h, a.c0d, c0h, c0d);
  cx<T>* buf = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* nyq = buf + R * P;
  cx<T>* twh = nyq + n2;
  cx<T>* twy = twh + h;
  cx<T>* tw1 = twy + n2;
  size_t off = align16((size_t)(R * P + n2 + h + n2 + h + 1) * sizeof(cx<T>) + 2 * 256 * sizeof(T));
  double* sh = reinterpret_cast<double*>(smem_raw + off);
  int* flag = reinterpret_cast<int*>(sh + 64);
  const int tid = threadIdx.x, nthr = blockDim.x;

  // this CTA's column block of the spectrum plane goes to shared memory by cp.async (column layout
  // [y][j], pitch Cb) while the twiddle tables load; CTA 0 also fetches the Nyquist column
  const cx<T>* Sp = a.S + ((long long)(lrhs * a.s_ncomp + c) * g.n3 + z) * g.plane_c;
  for (int e = tid; e < n2 * Cb; e += nthr) {
    const int y = (int)g.pc_fdCb.div((unsigned)e), j = e - y * Cb;
    cp_async_elem<sizeof(cx<T>)>(buf + e, Sp + (long long)y * h + q * Cb + j);
  }
  if (q == 0)
    for (int ky = tid; ky < n2; ky += nthr) cp_async_elem<sizeof(cx<T>)>(nyq + ky, Sp + (long long)n2 * h + ky);
  for (int i = tid; i < h; i += nthr) twh[i] = ldg_cx(a.tw_h + i);
  for (int i = tid; i < n2; i += nthr) twy[i] = ldg_cx(a.tw_n2 + i);
  for (int i = tid; i <= h; i += nthr) tw1[i] = ldg_cx(a.tw_n1 + i);
  const int y0 = q * R;
  const long long plane_sz = (long long)n2 * n1;
  const long long blk_sz = (long long)R * n1;
  if (a.prof != nullptr && tid == 0) {
    long long fields = (a.mode == INV_CG) ? 2 : 1 + (a.fin == FIN_BASIC);
    long long b = fields * blk_sz * (long long)sizeof(Tf) + (long long)n2 * Cb * (long long)sizeof(cx<T>);
    if (q == 0) b += (long long)n2 * (long long)sizeof(cx<T>);
    if (a.b != nullptr) b += blk_sz * (long long)sizeof(double);
    if (a.xsub != nullptr) b += blk_sz * (long long)sizeof(double);
    atomicAdd(a.prof, (unsigned long long)b);
    atomicAdd(a.prof + 1, (unsigned long long)blk_sz);
  }
  cp_async_wait_all();
  __syncthreads();
  if (q == 0) {   // pack kx = 0 (A) and kx = n1/2 (B) as A + i B
    for (int y = tid; y < n2; y += nthr) {
      const cx<T> v = buf[y * Cb], b = nyq[y];
      buf[y * Cb] = mk<T>(v.re - b.im, v.im + b.re);
    }
    __syncthreads();
  }
  fft_pencils<T, +1, EPT>(buf, ColAddr{Cb}, n2, Cb, g.pc_fdCb, twy);
  cl.sync();   // every column of the plane is transformed along y

  // transpose: this CTA's rows [y0, y0 + R) of all h columns, element e = r * h + kx
  {
    cx<T> v[EPT];
    const int nrow = R * h;
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * nthr;
      if (e < nrow) {
        const int r = (int)g.fd_h.div((unsigned)e), kx = e - r * h;
        const int src = (int)g.pc_fdCb.div((unsigned)kx), j = kx - src * Cb;
        const cx<T>* cb = cl.map_shared_rank(buf, src);
        v[i] = cb[(y0 + r) * Cb + j];
      }
    }
    cl.sync();   // every CTA has read its rows; the column blocks may be overwritten
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const int e = tid + i * nthr;
      if (e < nrow) {
        const int r = (int)g.fd_h.div((unsigned)e), kx = e - r * h;
        buf[r * P + kx] = v[i];
      }
    }
  }
  __syncthreads();

  // C2R merge: Z[k] = X[k] + conj X[h-k] + i W^{-k} (X[k] - conj X[h-k]); slot 0 holds X[0] + i X[n1/2]
  {
    const int nk = h / 2 + 1;
    for (int t = tid; t < R * nk; t += nthr) {
      const int k = (int)g.pc_fdR.div((unsigned)t), row = t - k * R;
      cx<T>* Rw = buf + row * P;
      if (k == 0) {
        const T x0 = Rw[0].re, xn = Rw[0].im;
        Rw[0] = mk<T>(x0 + xn, x0 - xn);
      } else if (2 * k == h) {
        Rw[k] = conj(Rw[k]) * (T)2;
      } else {
        const cx<T> xa = Rw[k], xb = Rw[h - k];
        const cx<T> wa = conj(tw1[k]), wb = conj(tw1[h - k]);
        const cx<T> za = (xa + conj(xb)) + mul_i<T, 1>(cmul(wa, xa - conj(xb)));
        const cx<T> zb = (xb + conj(xa)) + mul_i<T, 1>(cmul(wb, xb - conj(xa)));
        Rw[k] = za;
        Rw[h - k] = zb;
      }
    }
  }
  __syncthreads();
  fft_pencils<T, +1, EPT>(buf, RowAddr{P}, h, R, g.pc_fdR, twh);

  // epilogue on this CTA's rows of the real plane: x[2n] = Re z[n], x[2n+1] = Im z[n]
  T q0 = 0, q1 = 0;
  const int total = R * h;
  if (a.mode == INV_STORE) {
    const long long foff = ((long long)(rhs * a.out_ncomp + c) * g.n3 + z) * plane_sz + (long long)y0 * n1;
    const T cw = (c == 0) ? c0h : c0d;
    for (int e = tid; e < total; e += nthr) {
      const int row = (int)g.fd_h.div((unsigned)e), c2 = e - row * h;
      const long long o = foff + (long long)row * n1 + 2 * c2;
      const cx<T> v = buf[row * P + c2];
      T v0 = a.out_scale * v.re, v1 = a.out_scale * v.im;
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
  } else {  // INV_CG: q = A p = Gamma0 * (C : p) = -eta, r -= alpha q (x += alpha p: next forward pass)
    const long long foff = ((long long)(rhs * 6 + c) * g.n3 + z) * plane_sz + (long long)y0 * n1;
    const T alpha = (T)a.st[rhs].alpha;
    const T cw = (c == 0) ? c0h : c0d;
    Tf* rp = a.r + foff;
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
          const cx<T> v = buf[rw[j] * P + col];
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
    const int ncta = a.ncomp * g.n3 * Q;
    if (publish_and_collect<2>(v, a.part + (long long)rhs * 2 * ncta, a.cnt + rhs, ncta, (c * g.n3 + z) * Q + q,
                               sh, flag)) {
      if (threadIdx.x == 0) finalize_state(a.fin, a.st[rhs], v, 1.0 / (double)g.M);
    }
  }
}

// Clusters of this kernel that fit the GPU at once for a cluster of Q CTAs (0 if none, or if the
// size is not supported).  Sizes above 8 need the non-portable opt-in, set here per kernel.
template <typename K>
static int max_active_clusters(K kernel, int Q, int thr, size_t smem) {
  if (set_smem(kernel, smem) != cudaSuccess ||
      (Q > 8 && cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(Q * 64), 1, 1);
  cfg.blockDim = dim3((unsigned)thr, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

static void pc_shape(Geo& g, int Q) {
  g.pc_Q = Q;
  g.pc_R = g.n2 / Q;
  g.pc_Cb = g.h / Q;
  int thr = (int)(((long long)g.n2 * g.h / Q + kEPT - 1) / kEPT);
  thr = ((thr + 31) / 32) * 32;
  g.pc_thr = thr < 128 ? 128 : thr;
  g.pc_fdR = make_fastdiv((unsigned)g.pc_R);
  g.pc_fdCb = make_fastdiv((unsigned)g.pc_Cb);
}

// Picks the cluster size for the plane of g (FP32 transforms) among Q in {2, 4, 8, 16} that divide
// N2 and N1/2 and leave at most 16 elements per thread of a 1024-thread CTA within the shared-memory
// bound.  The smallest Q with at most 8192 elements per CTA (512 threads, so that two CTAs share an
// SM and one's memory phase overlaps the other's transforms) comes first, then the smallest Q with
// more; a shape is taken only if the GPU can hold at least one such cluster of both kernels.
bool plane_cluster_setup(Geo& g) {
  g.pc_Q = 0;
  const long long e = (long long)g.n2 * g.h;
  std::vector<int> order;
  for (int pass = 0; pass < 2; ++pass)
    for (int Q : {2, 4, 8, 16}) {
      const long long per = e / Q;
      if (g.n2 % Q != 0 || g.h % Q != 0 || per > (long long)kEPT * kPcMaxThreads) continue;
      if ((pass == 0) != (per <= (long long)kEPT * 512)) continue;
      order.push_back(Q);
    }
  for (int Q : order) {
    Geo t = g;
    pc_shape(t, Q);
    const size_t smem = pc_smem_bytes(t, sizeof(cx<float>), sizeof(float));
    if (smem > kPcMaxSmem) continue;
    if (max_active_clusters(plane_fwd_cluster_kernel<float, float, kEPT>, Q, t.pc_thr, smem) < 1 ||
        max_active_clusters(plane_inv_cluster_kernel<float, float, kEPT>, Q, t.pc_thr, smem) < 1)
      continue;
    g = t;
    return true;
  }
  return false;
}

template <typename K, typename A>
static cudaError_t launch_cluster(K kernel, const A& a, int nrhs, int ncomp, cudaStream_t s) {
  const Geo& g = a.g;
  if (g.pc_Q < 2 || g.pc_Q > 16 || g.pc_thr > kPcMaxThreads || (long long)g.pc_R * g.h > (long long)kEPT * g.pc_thr ||
      (long long)g.n2 * g.pc_Cb > (long long)kEPT * g.pc_thr || g.pc_R * g.pc_Q != g.n2 || g.pc_Cb * g.pc_Q != g.h ||
      nrhs < 1 || ncomp < 1 || ncomp > 65535 || nrhs > 65535)
    return cudaErrorInvalidValue;
  const size_t smem = pc_smem_bytes(g, sizeof(cx<float>), sizeof(float));
  cudaError_t e = set_smem(kernel, smem);
  if (e == cudaSuccess && g.pc_Q > 8) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(g.pc_Q * g.n3), (unsigned)ncomp, (unsigned)nrhs);
  cfg.blockDim = dim3((unsigned)g.pc_thr, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)g.pc_Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, kernel, a);
}

cudaError_t launch_plane_fwd_cluster(const FwdArgs<float, float>& a, int nrhs, cudaStream_t s) {
  if (a.n_phase > 256) return cudaErrorInvalidValue;
  return launch_cluster(plane_fwd_cluster_kernel<float, float, kEPT>, a, nrhs, a.ncomp, s);
}
cudaError_t launch_plane_inv_cluster(const InvArgs<float, float>& a, int nrhs, cudaStream_t s) {
  return launch_cluster(plane_inv_cluster_kernel<float, float, kEPT>, a, nrhs, a.ncomp, s);
}

}  // namespace hom
