// Split x passes of the Lippmann-Schwinger step, for x-y planes larger than one CTA holds
// (and as an alternative schedule for smaller ones).  The forward x pass applies the same
// prologues as plane_fwd (polarization, stress, CG direction, copy, C0) to a block of rows and
// transforms each row with the packed real-to-complex FFT; the inverse x pass applies the
// complex-to-real merge, the row FFT and the same epilogues as plane_inv.  The y transforms
// run in ypass.cu between them; the spectrum layout is the one of the fused plane kernels,
// except that column 0 still holds X[0] + i X[n1/2] of every row between the x and y passes.
#include "ls_common.cuh"

namespace hom {

// FP32 forward x pass: at most 64 registers, so four 256-thread CTAs fit an SM (74 registers and
// three CTAs without the bound); the extra resident warps hide its field loads (512^3: 3.65 ->
// 3.39 ms per launch), without spills.  The FP64 and double-float forms: at most 128 registers,
// two CTAs per SM (with a bound of one CTA the double-float form takes 156 registers and runs 30 %
// slower).
template <typename T> struct XfCfg { static constexpr int kMinBlocks = 2; };
template <> struct XfCfg<float> { static constexpr int kMinBlocks = 4; };

template <typename Tf, typename T, int EPT>
__global__ void __launch_bounds__(256, XfCfg<T>::kMinBlocks) xpass_fwd_kernel(const FwdArgs<Tf, T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Geo& g = a.g;
  const int blk = blockIdx.x, c = blockIdx.y, lrhs = blockIdx.z, rhs = a.rhs0 + lrhs;
  if (a.st != nullptr && a.st[rhs].active == 0) return;
  const int n1 = g.n1, h = g.h, P = g.P, rb = g.rb;
  const long long nrows = (long long)g.n2 * g.n3;
  const long long r0 = (long long)blk * rb;
  const int nr = (int)((nrows - r0 < rb) ? nrows - r0 : rb);

  cx<T>* pl = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* twh = pl + rb * P;
  cx<T>* tw1 = twh + h;
  T* tab = reinterpret_cast<T*>(tw1 + h + 1);
  size_t off = align16((size_t)(rb * P + 2 * h + 1) * sizeof(cx<T>) + 2 * a.n_phase * sizeof(T));
  double* sh = reinterpret_cast<double*>(smem_raw + off);
  int* flag = reinterpret_cast<int*>(sh + 64);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;

  if (tid == 0) {
    // this block's rows are contiguous in every field: their reads start into L2 now, while the
    // tables load (one bulk prefetch per field)
    const long long cb = (long long)(rhs * a.in_ncomp + c) * g.M + r0 * n1;
    const unsigned fb = (unsigned)((long long)nr * n1 * (long long)sizeof(Tf));
    if (a.mode == FWD_CG) {
      prefetch_l2_if_aligned(a.r + cb, fb);
      if (a.st[rhs].restart == 0) {
        prefetch_l2_if_aligned(a.p + cb, fb);
        prefetch_l2_if_aligned(a.x + cb, fb);
      }
    } else if (a.in != nullptr) {
      prefetch_l2_if_aligned(a.in + cb, fb);
    }
    if (a.mode != FWD_COPY && a.mode != FWD_C0)
      prefetch_l2_if_aligned(a.phase + (long long)rve_of(rhs, a.rve_loads) * g.M + r0 * n1, (unsigned)(nr * n1));
  }
  for (int i = tid; i < h; i += nthr) twh[i] = ldg_cx(a.tw_h + i);
  for (int i = tid; i <= h; i += nthr) tw1[i] = ldg_cx(a.tw_n1 + i);
  const int rve = rve_of(rhs, a.rve_loads);
  if (a.mode != FWD_COPY && a.mode != FWD_C0) {
    const T* mat = a.mat + (long long)rve * kRveTable;
    for (int i = tid; i < a.n_phase; i += nthr) {
      tab[i] = mat[i * 4 + (c == 0 ? 0 : 1)];
      tab[a.n_phase + i] = mat[i * 4 + (c == 0 ? 2 : 3)];
    }
  }
  const uint8_t* phase = a.phase + (long long)rve * g.M;
  __syncthreads();

  const long long cbase = (long long)(rhs * a.in_ncomp + c) * g.M;  // this component's field
  if (a.prof != nullptr && tid == 0) {
    const long long vox = (long long)nr * n1;
    long long fields = (a.mode == FWD_CG) ? (a.st[rhs].restart ? 2 : 5)
                                          : ((a.mode == FWD_COPY || a.mode == FWD_C0 || a.in != nullptr) ? 1 : 0);
    long long b = fields * vox * (long long)sizeof(Tf) + (long long)nr * h * (long long)sizeof(cx<T>);
    if (a.mode != FWD_COPY && a.mode != FWD_C0) b += vox;
    atomicAdd(a.prof, (unsigned long long)b);
    atomicAdd(a.prof + 1, (unsigned long long)vox);
  }
  T acc = (T)0;
  const RhsState* sp = (a.mode == FWD_CG) ? a.st + rhs : nullptr;
  const bool restart = sp ? (sp->restart != 0) : true;
  const T beta = restart ? (T)0 : (T)sp->beta;
  const T alpha = restart ? (T)0 : (T)sp->alpha;
  const T ec = (a.E != nullptr && (a.mode == FWD_TAU || a.mode == FWD_STRESS)) ? (T)a.E[rhs * 6 + c] : (T)0;
  const T* w = (a.mode == FWD_TAU) ? tab : tab + a.n_phase;
  T ch, cd;
  c0_weights<T>(a.c0, rve, a.c0h, a.c0d, ch, cd);
  const T wc = (a.mode == FWD_C0) ? (c == 0 ? ch : cd) : (T)1;

  if (a.mode == FWD_CG) {
    // Flat index e = row * h + col over this block's rows (contiguous in the field); the loads of
    // kBatch elements per thread are issued before the first store of p, which the compiler must
    // assume may alias r, so that they are in flight together.
    constexpr int kBatch = PlaneCfg<T>::kBatch;
    const Tf* rp = a.r + cbase + r0 * n1;
    Tf* pp = a.p + cbase + r0 * n1;
    Tf* xp = a.x + cbase + r0 * n1;
    const uint8_t* php = phase + r0 * n1;
    const int total = nr * h;
    for (int e0 = tid; e0 < rb * h; e0 += kBatch * nthr) {
      Tf q0r[kBatch], q1r[kBatch], p0[kBatch], p1[kBatch], x0[kBatch], x1[kBatch];
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
          ld2<Tf>(rp + o, q0r[j], q1r[j]);
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
        if (e >= rb * h) continue;
        const int col = e - rw[j] * h;
        cx<T> val = mk<T>(0, 0);
        if (e < total) {
          const int o = rw[j] * n1 + 2 * col;
          if (!restart) st2<Tf>(xp + o, (Tf)((T)x0[j] + alpha * (T)p0[j]), (Tf)((T)x1[j] + alpha * (T)p1[j]));
          const T q0 = (T)q0r[j] + beta * (T)p0[j], q1 = (T)q1r[j] + beta * (T)p1[j];
          st2<Tf>(pp + o, (Tf)q0, (Tf)q1);
          const T c0 = tab[a.n_phase + ph[j].x], c1 = tab[a.n_phase + ph[j].y];
          acc += c0 * q0 * q0 + c1 * q1 * q1;
          val = mk<T>(c0 * q0, c1 * q1);
        }
        pl[rw[j] * P + col] = val;
      }
    }
  } else {
#pragma unroll 4
    for (int lr = warp; lr < rb; lr += nwarp) {
      for (int c2 = lane; c2 < h; c2 += 32) {
        cx<T> val = mk<T>(0, 0);
        if (lr < nr) {
          const long long o = (r0 + lr) * n1 + 2 * c2;
          if (a.mode == FWD_TAU || a.mode == FWD_STRESS) {
            Tf v0 = 0, v1 = 0;
            if (a.in != nullptr) ld2<Tf>(a.in + cbase + o, v0, v1);
            const uchar2 ph = *reinterpret_cast<const uchar2*>(phase + o);
            val = mk<T>(w[ph.x] * ((T)v0 + ec), w[ph.y] * ((T)v1 + ec));
          } else {
            Tf v0, v1;
            ld2<Tf>(a.in + cbase + o, v0, v1);
            val = mk<T>(wc * (T)v0, wc * (T)v1);
          }
        }
        pl[lr * P + c2] = val;
      }
    }
  }
  __syncthreads();

  fft_pencils<T, -1, EPT>(pl, RowAddr{P}, h, rb, g.fd_rb, twh);

  // R2C split (as in plane_fwd); slot 0 keeps X[0] + i X[n1/2] for the y pass
  {
    const int nk = h / 2 + 1;
    for (int t = tid; t < rb * nk; t += nthr) {
      const int row = t % rb, k = t / rb;
      cx<T>* R = pl + row * P;
      if (k == 0) {
        const cx<T> z0 = R[0];
        R[0] = mk<T>(z0.re + z0.im, z0.re - z0.im);
      } else if (2 * k == h) {
        R[k] = conj(R[k]);
      } else {
        const cx<T> za = R[k], zb = R[h - k];
        const cx<T> wa = tw1[k], wb = tw1[h - k];
        cx<T> e = (za + conj(zb)) * (T)0.5;
        cx<T> o = mul_i<T, -1>(za - conj(zb)) * (T)0.5;
        const cx<T> xa = e + cmul(wa, o);
        e = (zb + conj(za)) * (T)0.5;
        o = mul_i<T, -1>(zb - conj(za)) * (T)0.5;
        const cx<T> xb = e + cmul(wb, o);
        R[k] = xa;
        R[h - k] = xb;
      }
    }
  }
  __syncthreads();

  cx<T>* Sc = a.S + (long long)(lrhs * a.ncomp + c) * g.n3 * g.plane_c;
#pragma unroll 4
  for (int lr = warp; lr < nr; lr += nwarp) {
    const unsigned gr = (unsigned)(r0 + lr);
    const unsigned zz = g.fd_n2.div(gr), yy = gr - zz * (unsigned)g.n2;
    cx<T>* dst = Sc + (long long)zz * g.plane_c + (long long)yy * h;
    for (int col = lane; col < h; col += 32) dst[col] = pl[lr * P + col];
  }

  if (a.mode == FWD_CG) {
    double v[1] = {(double)acc};
    block_sum_f64<1>(v, sh);
    const int ncta = a.ncomp * g.nrb;
    if (publish_and_collect<1>(v, a.part + (long long)rhs * 2 * ncta, a.cnt + rhs, ncta, c * g.nrb + blk, sh,
                               flag)) {
      if (threadIdx.x == 0) finalize_state(FIN_ENERGY, a.st[rhs], v, 1.0 / (double)g.M);
    }
  }
}

template <typename Tf, typename T, int EPT>
__global__ void __launch_bounds__(256) xpass_inv_kernel(const InvArgs<Tf, T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Geo& g = a.g;
  const int blk = blockIdx.x, c = blockIdx.y, lrhs = blockIdx.z, rhs = a.rhs0 + lrhs;
  if (a.st != nullptr && a.st[rhs].active == 0) return;
  const int n1 = g.n1, h = g.h, P = g.P, rb = g.rb;
  const long long nrows = (long long)g.n2 * g.n3;
  const long long r0 = (long long)blk * rb;
  const int nr = (int)((nrows - r0 < rb) ? nrows - r0 : rb);
  cx<T>* pl = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* twh = pl + rb * P;
  cx<T>* tw1 = twh + h;
  size_t off = align16((size_t)(rb * P + 2 * h + 1) * sizeof(cx<T>));
  double* sh = reinterpret_cast<double*>(smem_raw + off);
  int* flag = reinterpret_cast<int*>(sh + 64);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  if (tid == 0) {
    // the epilogue's field rows (contiguous) start into L2 while the transforms run
    const unsigned fb = (unsigned)((long long)nr * n1 * (long long)sizeof(Tf));
    if (a.mode == INV_CG) {
      prefetch_l2_if_aligned(a.r + (long long)(rhs * 6 + c) * g.M + r0 * n1, fb);
    } else {
      const long long cb = (long long)(rhs * a.out_ncomp + c) * g.M + r0 * n1;
      const unsigned db = (unsigned)((long long)nr * n1 * (long long)sizeof(double));
      if (a.b != nullptr) prefetch_l2_if_aligned(a.b + cb, db);
      if (a.xsub != nullptr) prefetch_l2_if_aligned(a.xsub + cb, db);
      if (a.fin == FIN_BASIC && a.prev != nullptr) prefetch_l2_if_aligned(a.prev + cb, fb);
    }
  }
  // the block's spectrum rows go to shared memory by cp.async while the twiddle tables load
  const cx<T>* Sc = a.S + (long long)(lrhs * a.s_ncomp + c) * g.n3 * g.plane_c;
#pragma unroll 4
  for (int lr = warp; lr < rb; lr += nwarp) {
    if (lr < nr) {
      const unsigned gr = (unsigned)(r0 + lr);
      const unsigned zz = g.fd_n2.div(gr), yy = gr - zz * (unsigned)g.n2;
      const cx<T>* src = Sc + (long long)zz * g.plane_c + (long long)yy * h;
      for (int col = lane; col < h; col += 32) cp_async_elem<sizeof(cx<T>)>(pl + lr * P + col, src + col);
    } else {
      for (int col = lane; col < h; col += 32) pl[lr * P + col] = mk<T>(0, 0);
    }
  }
  for (int i = tid; i < h; i += nthr) twh[i] = ldg_cx(a.tw_h + i);
  for (int i = tid; i <= h; i += nthr) tw1[i] = ldg_cx(a.tw_n1 + i);
  if (a.prof != nullptr && tid == 0) {
    const long long vox = (long long)nr * n1;
    long long fields = (a.mode == INV_CG) ? 2 : 1 + (a.fin == FIN_BASIC);
    long long b = fields * vox * (long long)sizeof(Tf) + (long long)nr * h * (long long)sizeof(cx<T>);
    if (a.b != nullptr) b += vox * (long long)sizeof(double);
    if (a.xsub != nullptr) b += vox * (long long)sizeof(double);
    atomicAdd(a.prof, (unsigned long long)b);
    atomicAdd(a.prof + 1, (unsigned long long)vox);
  }
  cp_async_wait_all();
  __syncthreads();

  // C2R merge (as in plane_inv); slot 0 holds X[0] + i X[n1/2]
  {
    const int nk = h / 2 + 1;
    for (int t = tid; t < rb * nk; t += nthr) {
      const int row = t % rb, k = t / rb;
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

  fft_pencils<T, +1, EPT>(pl, RowAddr{P}, h, rb, g.fd_rb, twh);

  T q0 = 0, q1 = 0;
  T ch, cd;
  c0_weights<T>(a.c0, rve_of(rhs, a.rve_loads), a.c0h, a.c0d, ch, cd);
  const T cw = (c == 0) ? ch : cd;
  if (a.mode == INV_STORE) {
    const long long cbase = (long long)(rhs * a.out_ncomp + c) * g.M;
#pragma unroll 4
    for (int lr = warp; lr < nr; lr += nwarp) {
      for (int c2 = lane; c2 < h; c2 += 32) {
        const long long o = cbase + (r0 + lr) * n1 + 2 * c2;
        const cx<T> e = pl[lr * P + c2];
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
  } else {  // INV_CG: r -= alpha A p with A p = -eta (x += alpha p: next forward pass)
    // flat index e = row * h + col; kBatch elements' loads in flight before the first store
    constexpr int kBatch = PlaneCfg<T>::kBatch;
    const long long cbase = (long long)(rhs * 6 + c) * g.M + r0 * n1;
    const T alpha = (T)a.st[rhs].alpha;
    Tf* rp = a.r + cbase;
    const int total = nr * h;
    for (int e0 = tid; e0 < total; e0 += kBatch * nthr) {
      Tf s0[kBatch], s1[kBatch];
      int rw[kBatch];
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int e = e0 + j * nthr;
        rw[j] = (int)g.fd_h.div((unsigned)e);
        if (e < total) {
          const int o = rw[j] * n1 + 2 * (e - rw[j] * h);
          ld2<Tf>(rp + o, s0[j], s1[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kBatch; ++j) {
        const int e = e0 + j * nthr;
        if (e < total) {
          const int col = e - rw[j] * h, o = rw[j] * n1 + 2 * col;
          const cx<T> v = pl[rw[j] * P + col];
          const T ra = (T)s0[j] + alpha * v.re, rb_ = (T)s1[j] + alpha * v.im;
          st2<Tf>(rp + o, (Tf)ra, (Tf)rb_);
          q0 += cw * (ra * ra + rb_ * rb_);
          q1 += ra * ra + rb_ * rb_;
        }
      }
    }
  }
  if (a.fin != FIN_NONE) {
    double v[2] = {(double)q0, (double)q1};
    block_sum_f64<2>(v, sh);
    const int ncta = a.ncomp * g.nrb;
    if (publish_and_collect<2>(v, a.part + (long long)rhs * 2 * ncta, a.cnt + rhs, ncta, c * g.nrb + blk, sh,
                               flag)) {
      if (threadIdx.x == 0) finalize_state(a.fin, a.st[rhs], v, 1.0 / (double)g.M);
    }
  }
}

static size_t xpass_smem_bytes(const Geo& g, size_t elem) {
  size_t b = (size_t)(g.rb * g.P + 2 * g.h + 1) * elem + 2 * 256 * elem;
  b = (b + 15) & ~size_t(15);
  return b + 64 * sizeof(double) + 16;
}

template <typename Tf, typename T>
cudaError_t launch_xpass_fwd(const FwdArgs<Tf, T>& a, int nrhs, cudaStream_t s) {
  if ((long long)a.g.rb * a.g.h > (long long)kEPT * a.g.thr_x || a.g.thr_x > 256 || a.n_phase > 256)
    return cudaErrorInvalidValue;
  const size_t smem = xpass_smem_bytes(a.g, sizeof(cx<T>));
  auto k = xpass_fwd_kernel<Tf, T, kEPT>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.g.nrb, a.ncomp, nrhs);
  count_launch();
  k<<<grid, a.g.thr_x, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename Tf, typename T>
cudaError_t launch_xpass_inv(const InvArgs<Tf, T>& a, int nrhs, cudaStream_t s) {
  if ((long long)a.g.rb * a.g.h > (long long)kEPT * a.g.thr_x || a.g.thr_x > 256) return cudaErrorInvalidValue;
  const size_t smem = xpass_smem_bytes(a.g, sizeof(cx<T>));
  auto k = xpass_inv_kernel<Tf, T, kEPT>;
  cudaError_t e = set_smem(k, smem);
  if (e != cudaSuccess) return e;
  dim3 grid(a.g.nrb, a.ncomp, nrhs);
  count_launch();
  k<<<grid, a.g.thr_x, smem, s>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_xpass_fwd<float, float>(const FwdArgs<float, float>&, int, cudaStream_t);
template cudaError_t launch_xpass_fwd<double, double>(const FwdArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_xpass_inv<float, float>(const InvArgs<float, float>&, int, cudaStream_t);
template cudaError_t launch_xpass_inv<double, double>(const InvArgs<double, double>&, int, cudaStream_t);
template cudaError_t launch_xpass_inv<float, double>(const InvArgs<float, double>&, int, cudaStream_t);
template cudaError_t launch_xpass_fwd<double, df64>(const FwdArgs<double, df64>&, int, cudaStream_t);
template cudaError_t launch_xpass_inv<float, df64>(const InvArgs<float, df64>&, int, cudaStream_t);
template cudaError_t launch_xpass_inv<double, df64>(const InvArgs<double, df64>&, int, cudaStream_t);

}  // namespace hom
