// Device building blocks shared by the Lippmann-Schwinger kernels: a complex
// type, exact small-radix DFTs held in registers, and a Stockham autosort stage
// that a whole CTA runs over pencils held in shared memory.
//
// FFT convention (Sec. 2, periodic Lippmann-Schwinger equation as a Fourier series):
// forward  X[k] = sum_n x[n] exp(-2 pi i n k / N)   (DIR = -1, unnormalised)
// inverse  x[n] = sum_k X[k] exp(+2 pi i n k / N)   (DIR = +1, unnormalised)
// The 1/M of the Fourier coefficients is applied once, inside the Green contraction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hom {

// Double-float number: the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi) / 2), about
// 48 significant bits.  The FP32 mode's FP64 passes (residuals, literal checks, projections) run
// in it: on this GPU the FP64 pipe executes a small fraction of the FP32 rate, and these passes
// need about 1e-12 relative accuracy, not 53 bits.  Sums use Knuth's TwoSum and Dekker's
// FastTwoSum, products an FMA-exact product (the standard error-free transformations); the
// division goes through double and is used once per frequency only.
struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ constexpr df64(float f) : hi(f), lo(0.0f) {}
  __host__ __device__ constexpr df64(int i) : df64((double)i) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};
__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return df64(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return df64(s, b - (s - a));
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df64 operator/(df64 a, df64 b) { return df64((double)a / (double)b); }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }
__device__ __forceinline__ bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df64 a, df64 b) { return !(a == b); }

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

template <typename T> __device__ __forceinline__ cx<T> mk(T a, T b) { cx<T> r; r.re = a; r.im = b; return r; }
template <typename T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk<T>(a.re + b.re, a.im + b.im); }
template <typename T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk<T>(a.re - b.re, a.im - b.im); }
template <typename T> __device__ __forceinline__ cx<T> operator*(cx<T> a, T s) { return mk<T>(a.re * s, a.im * s); }
template <typename T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T> __device__ __forceinline__ cx<T> conj(cx<T> a) { return mk<T>(a.re, -a.im); }
// read-only cached load of a complex value
__device__ __forceinline__ cx<float> ldg_cx(const cx<float>* p) {
  float2 f = __ldg(reinterpret_cast<const float2*>(p));
  return mk<float>(f.x, f.y);
}
__device__ __forceinline__ cx<double> ldg_cx(const cx<double>* p) {
  double2 f = __ldg(reinterpret_cast<const double2*>(p));
  return mk<double>(f.x, f.y);
}
__device__ __forceinline__ cx<df64> ldg_cx(const cx<df64>* p) {
  float4 f = __ldg(reinterpret_cast<const float4*>(p));
  return mk<df64>(df64(f.x, f.y), df64(f.z, f.w));
}
// multiply by +i (s = +1) or -i (s = -1)
template <typename T, int S> __device__ __forceinline__ cx<T> mul_i(cx<T> a) {
  return S > 0 ? mk<T>(-a.im, a.re) : mk<T>(a.im, -a.re);
}

// cos(2 pi j / 48) for j = 0..12 (first quadrant); the twiddles of every radix used
// here (2, 3, 4, 6, 8, 12, 16) are multiples of 2 pi / 48.
__host__ __device__ constexpr double cos48(int j) {
  return j == 0 ? 1.0
       : j == 1 ? 0.99144486137381041114
       : j == 2 ? 0.96592582628906828675
       : j == 3 ? 0.92387953251128675613
       : j == 4 ? 0.86602540378443864676
       : j == 5 ? 0.79335334029123516458
       : j == 6 ? 0.70710678118654752440
       : j == 7 ? 0.60876142900872063942
       : j == 8 ? 0.5
       : j == 9 ? 0.38268343236508977173
       : j == 10 ? 0.25881904510252076235
       : j == 11 ? 0.13052619222005159155
       : 0.0;
}
// cos and sin of 2 pi m / 48 for any integer m, reduced by quadrant.
__host__ __device__ constexpr double cosm48(int m) {
  return ((m % 48) + 48) % 48 <= 12 ? cos48(((m % 48) + 48) % 48)
       : ((m % 48) + 48) % 48 <= 24 ? -cos48(24 - ((m % 48) + 48) % 48)
       : ((m % 48) + 48) % 48 <= 36 ? -cos48(((m % 48) + 48) % 48 - 24)
       : cos48(48 - ((m % 48) + 48) % 48);
}
__host__ __device__ constexpr double sinm48(int m) { return cosm48(12 - m); }

// v *= exp(DIR * 2 pi i * m / R), exact for multiples of a quarter turn.
template <typename T, int R, int M, int DIR>
__device__ __forceinline__ cx<T> twiddle_c(cx<T> v) {
  constexpr int m = ((M % R) + R) % R;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (4 * m == R) {            // quarter turn: multiply by DIR*i
    return mul_i<T, DIR>(v);
  } else if constexpr (2 * m == R) {
    return mk<T>(-v.re, -v.im);
  } else if constexpr (4 * m == 3 * R) {
    return mul_i<T, -DIR>(v);
  } else {
    constexpr int q = 48 / R * m;
    const T c = (T)cosm48(q);
    const T s = (T)(DIR * sinm48(q));
    return mk<T>(v.re * c - v.im * s, v.re * s + v.im * c);
  }
}

// ---- small DFTs in registers ----------------------------------------------
template <typename T, int DIR>
__device__ __forceinline__ void dft2(cx<T>& a, cx<T>& b) {
  cx<T> t = a;
  a = t + b;
  b = t - b;
}

template <typename T, int DIR>
__device__ __forceinline__ void dft3(cx<T>& a, cx<T>& b, cx<T>& c) {
  // W3 = exp(DIR 2 pi i / 3) = -1/2 + DIR i sqrt(3)/2
  const T h = (T)0.86602540378443864676;
  cx<T> s = b + c, d = b - c;
  cx<T> a0 = a;
  a = a0 + s;
  cx<T> m = mk<T>(a0.re - (T)0.5 * s.re, a0.im - (T)0.5 * s.im);
  cx<T> r = mul_i<T, DIR>(d) * h;
  b = m + r;
  c = m - r;
}

// Generic R = R1 * R2 decomposition (Cooley-Tukey in registers): input index
// n = R2*n1 + n2, output index k = k1 + R1*k2.
template <typename T, int R, int DIR> struct SmallDFT;

template <typename T, int DIR> struct SmallDFT<T, 1, DIR> {
  __device__ __forceinline__ static void run(cx<T>*) {}
};
template <typename T, int DIR> struct SmallDFT<T, 2, DIR> {
  __device__ __forceinline__ static void run(cx<T>* v) { dft2<T, DIR>(v[0], v[1]); }
};
template <typename T, int DIR> struct SmallDFT<T, 3, DIR> {
  __device__ __forceinline__ static void run(cx<T>* v) { dft3<T, DIR>(v[0], v[1], v[2]); }
};
template <typename T, int DIR> struct SmallDFT<T, 4, DIR> {
  __device__ __forceinline__ static void run(cx<T>* v) {
    cx<T> a = v[0] + v[2], b = v[0] - v[2];
    cx<T> c = v[1] + v[3], d = mul_i<T, DIR>(v[1] - v[3]);
    v[0] = a + c;
    v[2] = a - c;
    v[1] = b + d;
    v[3] = b - d;
  }
};

template <int R> struct Split { static constexpr int R1 = (R % 4 == 0 && R > 4) ? 4 : (R % 3 == 0 ? 3 : 2); };

template <typename T, int R, int DIR> struct SmallDFT {
  static constexpr int R1 = Split<R>::R1;
  static constexpr int R2 = R / R1;
  template <int N2>
  __device__ __forceinline__ static void inner(cx<T>* v, cx<T> (&y)[R1][R2]) {
    if constexpr (N2 < R2) {
      cx<T> t[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) t[n1] = v[R2 * n1 + N2];
      SmallDFT<T, R1, DIR>::run(t);
      tw_row<N2, 0>(t);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) y[k1][N2] = t[k1];
      inner<N2 + 1>(v, y);
    }
  }
  template <int N2, int K1>
  __device__ __forceinline__ static void tw_row(cx<T>* t) {
    if constexpr (K1 < R1) {
      t[K1] = twiddle_c<T, R, N2 * K1, DIR>(t[K1]);
      tw_row<N2, K1 + 1>(t);
    }
  }
  __device__ __forceinline__ static void run(cx<T>* v) {
    cx<T> y[R1][R2];
    inner<0>(v, y);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      SmallDFT<T, R2, DIR>::run(y[k1]);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = y[k1][k2];
    }
  }
};

// ---- Stockham autosort stage over pencils in shared memory ------------------
// Pencil p, element n lives at buf[addr(p, n)].  N (axis length) and NS (product of the
// radices of the earlier stages) are compile-time constants.  tw[t] = exp(-2 pi i t / N)
// (host-computed, usually staged in shared memory), conjugated for DIR = +1.  Each thread runs
// up to MAXT radix-R tasks; task t covers pencil t mod npen and butterfly t div npen, so
// consecutive threads touch consecutive pencils.  All loads of a stage complete (barrier)
// before any store, so the stage works in place.

// q = n / d for 0 <= n < 2^31 with a precomputed multiplier (Granlund-Montgomery round-up)
struct FastDiv {
  unsigned d, m, s;
  __device__ __forceinline__ unsigned div(unsigned n) const { return (__umulhi(n, m) + n) >> s; }
};
inline FastDiv make_fastdiv(unsigned d) {
  unsigned s = 0;
  while ((1u << s) < d) ++s;
  const unsigned long long m = ((1ull << 32) * ((1ull << s) - d)) / d + 1;
  FastDiv f;
  f.d = d;
  f.m = (unsigned)m;
  f.s = s;
  return f;
}

struct RowAddr {   // pencils are rows: addr = p * pitch + n (odd pitch: conflict-free across rows)
  int pitch;
  __device__ __forceinline__ int operator()(int p, int n) const { return p * pitch + n; }
};
struct ColAddr {   // pencils are columns: addr = p + n * pitch
  int pitch;
  __device__ __forceinline__ int operator()(int p, int n) const { return p + n * pitch; }
};
struct ZAddr {     // pencil p = c * 2^tc_log2 + tc: addr = c*cstride + n*tcp + tc
  int tc_log2, cstride, tcp;
  __device__ __forceinline__ int operator()(int p, int n) const {
    return (p >> tc_log2) * cstride + n * tcp + (p & ((1 << tc_log2) - 1));
  }
};

template <typename T, int N, int NS, int R, int DIR, int MAXT, typename Addr>
__device__ __forceinline__ void stockham_stage(cx<T>* buf, const Addr& addr, int npen, const FastDiv& npd,
                                               const cx<T>* tw) {
  constexpr int per = N / R;
  constexpr int tstep = N / (NS * R);
  const int ntask = npen * per;
  cx<T> v[MAXT][R];
  int pen[MAXT], base[MAXT];
#pragma unroll
  for (int i = 0; i < MAXT; ++i) {
    const int t = threadIdx.x + i * blockDim.x;
    pen[i] = -1;
    if (t < ntask) {
      const int j = (int)npd.div((unsigned)t);
      const int p = t - j * npen;
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = buf[addr(p, j + r * per)];
      const int k = j % NS;
      if (NS > 1) {
        const int st = k * tstep;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cx<T> w = tw[st * r];
          if (DIR > 0) w.im = -w.im;
          v[i][r] = cmul(v[i][r], w);
        }
      }
      SmallDFT<T, R, DIR>::run(v[i]);
      pen[i] = p;
      base[i] = (j - k) * R + k;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < MAXT; ++i) {
    if (pen[i] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[addr(pen[i], base[i] + r * NS)] = v[i][r];
    }
  }
  __syncthreads();
}

// Fixed radix sequences, one per supported axis length.  Each length is a straight-line run
// of stages (no runtime loop over stage kinds): register allocation then takes the maximum
// over the stages rather than their union, and every stride is a compile-time constant.
template <typename T, int DIR, int EPT, int N, int NS, int... Rs>
struct StageSeq;
template <typename T, int DIR, int EPT, int N, int NS>
struct StageSeq<T, DIR, EPT, N, NS> {
  template <typename Addr>
  __device__ __forceinline__ static void run(cx<T>*, const Addr&, int, const FastDiv&, const cx<T>*) {}
};
template <typename T, int DIR, int EPT, int N, int NS, int R, int... Rs>
struct StageSeq<T, DIR, EPT, N, NS, R, Rs...> {
  template <typename Addr>
  __device__ __forceinline__ static void run(cx<T>* b, const Addr& a, int npen, const FastDiv& npd,
                                             const cx<T>* tw) {
    stockham_stage<T, N, NS, R, DIR, (EPT + R - 1) / R>(b, a, npen, npd, tw);
    StageSeq<T, DIR, EPT, N, NS * R, Rs...>::run(b, a, npen, npd, tw);
  }
};

// Axis lengths the kernels accept (host side checks with fft_length_supported).  The z axis may
// also have length 1 (a two-dimensional cell, see z_length_supported).
__host__ __device__ constexpr bool fft_length_supported(int n) {
  return n == 2 || n == 3 || n == 4 || n == 6 || n == 8 || n == 12 || n == 16 || n == 24 ||
         n == 32 || n == 48 || n == 64 || n == 96 || n == 128 || n == 192 || n == 256 ||
         n == 384 || n == 512;
}
__host__ __device__ constexpr bool z_length_supported(int n) { return n == 1 || fft_length_supported(n); }

// Runs the FFT of length n on `npen` pencils (npd divides by npen).  EPT bounds elements per
// thread: the caller guarantees npen * n <= EPT * blockDim.x.
template <typename T, int DIR, int EPT, typename Addr>
__device__ __forceinline__ void fft_pencils(cx<T>* buf, const Addr& addr, int n, int npen, const FastDiv& npd,
                                            const cx<T>* tw) {
#define HOM_SEQ(NN, ...) \
  case NN: StageSeq<T, DIR, EPT, NN, 1, __VA_ARGS__>::run(buf, addr, npen, npd, tw); break;
  switch (n) {
    case 1: break;  // a single plane along z (two-dimensional cells): the identity
    HOM_SEQ(2, 2)
    HOM_SEQ(3, 3)
    HOM_SEQ(4, 4)
    HOM_SEQ(6, 6)
    HOM_SEQ(8, 8)
    HOM_SEQ(12, 12)
    HOM_SEQ(16, 16)
    HOM_SEQ(24, 8, 3)
    HOM_SEQ(32, 8, 4)
    HOM_SEQ(48, 16, 3)
    HOM_SEQ(64, 16, 4)
    HOM_SEQ(96, 16, 6)
    HOM_SEQ(128, 16, 8)
    HOM_SEQ(192, 16, 12)
    HOM_SEQ(256, 16, 16)
    HOM_SEQ(384, 16, 8, 3)
    HOM_SEQ(512, 8, 8, 8)
    default: break;
  }
#undef HOM_SEQ
}

// ---- FP64 block reduction ---------------------------------------------------
// Sums NQ per-thread values (already accumulated in T) into FP64; thread 0 gets the
// block totals.  Warp shuffles, then shared memory across warps.
template <int NQ>
__device__ __forceinline__ void block_sum_f64(double (&v)[NQ], double* sh /* >= 32*NQ */) {
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[warp * NQ + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += sh[w * NQ + q];
      v[q] = s;
    }
  }
  __syncthreads();
}

}  // namespace hom
