// The Lippmann-Schwinger step on the GPU (Sec. 2 of arXiv:1712.05145, Algorithm 1):
//
//   plane_fwd : polarization tau = (C - C0) : (eps + E)         (Eq. auxiliary_problem)
//               fused with the x-axis R2C and y-axis FFT of one z-plane
//   zpass     : z-axis FFT, eta_hat = -Gamma0_hat(xi) : tau_hat  (Green operator, Sec. 2)
//               with eta_hat(0) = 0, inverse z-axis FFT
//   plane_inv : inverse y FFT and x-axis C2R of one z-plane fused with the update
//               (fixed-point step, CG vector updates, residuals) and FP64 reductions
//
// Strain-like fields are stored in the Kelvin basis of symmetric tensors
//   k0 = tr(e)/sqrt3, k1 = (e11-e22)/sqrt2, k2 = (e11+e22-2e33)/sqrt6,
//   k3 = sqrt2 e23, k4 = sqrt2 e13, k5 = sqrt2 e12,
// an orthonormal basis in which every isotropic stiffness is diagonal (3K on k0, 2mu on
// k1..k5).  The polarization of component c therefore needs only component c, and
// one CTA transforms one (rhs, component, z-plane) without touching the others.
#pragma once
#include "internal.h"

namespace hom {

constexpr int kEPT = 16;
// Launch shape of the plane kernels per compute precision: 16 elements per thread, CTAs of up
// to 512 threads.  (8 elements per thread with 1024-thread CTAs and 32 registers, which doubles
// the resident warps, measured slower at 128^3: the extra radix stage and register spills cost
// more than the occupancy gained.)  kBatch: elements per thread whose global loads the prologue
// and epilogue loops issue together.
template <typename T> struct PlaneCfg;
template <> struct PlaneCfg<float> {   // 64 registers: 2 CTAs per SM
  static constexpr int kEPT = 16, kMaxThreads = 512, kMinBlocks = 2, kBatch = 4;
};
template <> struct PlaneCfg<double> {
  static constexpr int kEPT = 16, kMaxThreads = 512, kMinBlocks = 1, kBatch = 4;
};
template <> struct PlaneCfg<df64> {
  static constexpr int kEPT = 16, kMaxThreads = 512, kMinBlocks = 1, kBatch = 4;
};
// threads of a plane CTA: every element of the n2 x h plane has a slot, whole warps, >= 128
template <typename T>
inline int plane_threads(const Geo& g) {
  const long long e = (long long)g.n2 * g.h;
  int thr = (int)((e + PlaneCfg<T>::kEPT - 1) / PlaneCfg<T>::kEPT);
  thr = ((thr + 31) / 32) * 32;
  return thr < 128 ? 128 : thr;
}
// An FP32 Krylov sweep (state flag `stall`) whose residual has not halved for kStallIters
// iterations ends (the FP64 residual sweep then restarts it, or reports non-convergence).
// Below kNearFloor (relative residual) an FP32 sweep is close to its rounding floor and a
// shorter window applies.  FP64 sweeps run to the tolerance or the iteration cap.
constexpr int kStallIters = 100;
constexpr int kStallItersNearFloor = 25;
constexpr double kNearFloor = 1e-5;

// ---------------------------------------------------------------------------------
// several RVEs of one grid in one handle: load r belongs to RVE r / rve_loads (rve_loads > 0)
__device__ __forceinline__ int rve_of(int rhs, int rve_loads) { return rve_loads > 0 ? rhs / rve_loads : 0; }
constexpr int kRveTable = 4 * 256;   // per-phase table entries of one RVE

// Kelvin eigenvalues of C0 (3 lam0 + 2 mu0, 2 mu0) of an RVE: from c0[rve] = (lam0, mu0, 3 lam0 + 2 mu0,
// 2 mu0) when given (computed on the host, like h and d), else (h, d)
template <typename T>
__device__ __forceinline__ void c0_weights(const double* c0, int rve, T h, T d, T& ch, T& cd) {
  if (c0 != nullptr) {
    ch = (T)c0[4 * rve + 2];
    cd = (T)c0[4 * rve + 3];
  } else {
    ch = h;
    cd = d;
  }
}

// ---------------------------------------------------------------------------------
// small helpers
template <typename Tf> struct Pair;
template <> struct Pair<float> { using V = float2; };
template <> struct Pair<double> { using V = double2; };

template <typename Tf>
__device__ __forceinline__ void ld2(const Tf* p, Tf& a, Tf& b) {
  typename Pair<Tf>::V v = *reinterpret_cast<const typename Pair<Tf>::V*>(p);
  a = v.x;
  b = v.y;
}
template <typename Tf>
__device__ __forceinline__ void st2(Tf* p, Tf a, Tf b) {
  typename Pair<Tf>::V v;
  v.x = a;
  v.y = b;
  *reinterpret_cast<typename Pair<Tf>::V*>(p) = v;
}

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

// Asynchronous global -> shared copy of one complex value (cp.async, 8 or 16 bytes, both
// addresses aligned to it): a CTA's copies of a whole tile are in flight together without
// staging registers.  cp_async_wait_all commits them and waits for all of this thread's copies.
template <int BYTES>
__device__ __forceinline__ void cp_async_elem(void* smem, const void* gmem) {
  static_assert(BYTES == 8 || BYTES == 16, "cp.async copies 8 or 16 bytes here");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Bulk prefetch of a contiguous global range into L2 (TMA, sm_90+).  bytes must be a multiple
// of 16 and ptr 16-byte aligned; the range must lie inside one allocation.  Issued by one thread.
__device__ __forceinline__ void prefetch_l2(const void* ptr, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(ptr), "r"(bytes) : "memory");
}

// The same where the range allows it (16-byte aligned start and size); otherwise nothing.
__device__ __forceinline__ void prefetch_l2_if_aligned(const void* ptr, unsigned bytes) {
  if (bytes != 0 && (bytes & 15u) == 0 && (reinterpret_cast<unsigned long long>(ptr) & 15ull) == 0)
    prefetch_l2(ptr, bytes);
}

// Publishes this block's NQ totals (valid in thread 0 after block_sum_f64) and lets the
// block that draws the last ticket sum all ncta partials in a fixed order.  Returns
// true in that block, with the grand totals in thread 0's v.
template <int NQ>
__device__ __forceinline__ bool publish_and_collect(double (&v)[NQ], double* part, unsigned* cnt, int ncta, int cta,
                                    double* sh, int* flag) {
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) part[q * ncta + cta] = v[q];
    __threadfence();
    const unsigned t = atomicAdd(cnt, 1u);
    *flag = (t == (unsigned)(ncta - 1)) ? 1 : 0;
  }
  __syncthreads();
  const bool last = (*flag != 0);
  if (last) {
    __threadfence();
    double s[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) s[q] = 0.0;
    for (int i = threadIdx.x; i < ncta; i += blockDim.x) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) s[q] += __ldcg(part + q * ncta + i);
    }
    block_sum_f64<NQ>(s, sh);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] = s[q];
      *cnt = 0u;
    }
  }
  return last;
}

__device__ __forceinline__ void finalize_state(int kind, RhsState& s, const double* v, double invM) {
  switch (kind) {
    case FIN_ENERGY: {
      const double pAp = v[0] * invM;
      s.pAp = pAp;
      s.xpend = 0;   // this forward pass applied the previous iteration's update of x
      s.alpha = (pAp != 0.0) ? s.rho / pAp : 0.0;
      if (!isfinite(s.alpha)) { s.status = 2; s.active = 0; }
      break;
    }
    case FIN_CG: {
      const double rho = v[0] * invM, rr = v[1] * invM;
      s.beta = (s.rho != 0.0) ? rho / s.rho : 0.0;
      s.rho = rho;
      s.res = (s.b2 > 0.0) ? sqrt(rr / s.b2) : 0.0;
      s.iter += 1;
      s.restart = 0;
      s.xpend = 1;
      if (!isfinite(s.res) || !isfinite(s.beta)) { s.status = 2; s.active = 0; }
      else if (s.res < s.tol) s.active = 0;
      else if (s.iter >= s.max_iter) { s.active = 0; s.status = 1; }
      else if (s.res < 0.5 * s.best) { s.best = s.res; s.best_iter = s.iter; }
      else if (s.stall && s.iter - s.best_iter >= (s.res < kNearFloor ? kStallItersNearFloor : kStallIters))
        s.active = 0;  // sweep stalled: hand over to the FP64 residual sweep
      break;
    }
    case FIN_BASIC: {
      const double d2 = v[0] * invM;
      s.res = (s.b2 > 0.0) ? sqrt(d2 / s.b2) : 0.0;
      s.iter += 1;
      if (!isfinite(s.res)) { s.status = 2; s.active = 0; }
      else if (s.res < s.tol) s.active = 0;
      else if (s.iter >= s.max_iter) { s.active = 0; s.status = 1; }
      break;
    }
    case FIN_RHS: {
      s.rho = v[0] * invM;
      s.b2 = v[1] * invM;
      s.res = 1.0;
      s.res_true = 1.0;
      s.restart = 1;
      if (!isfinite(s.b2)) { s.status = 2; s.active = 0; }
      break;
    }
    case FIN_RESID: {
      s.rho = v[0] * invM;
      s.res_true = (s.b2 > 0.0) ? sqrt(v[1] * invM / s.b2) : 0.0;
      s.res = s.res_true;
      s.restart = 1;
      if (!isfinite(s.res_true)) { s.status = 2; s.active = 0; }
      break;
    }
    default: break;
  }
}

// Dynamic shared memory above 48 KB needs an opt-in; the carveout asks for the largest shared
// memory partition so that the occupancy is not limited by a small default carveout.  The
// opt-in is a per-function, per-context limit shared by every host thread, so it is always set
// to the device maximum rather than to this launch's size: with per-launch values, a thread
// launching a small grid could lower the limit between another thread's set and its launch.
// The limit only bounds a launch; occupancy follows the bytes each launch asks for.
inline int smem_optin_max() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return v;
}

template <typename K>
inline cudaError_t set_smem(K kernel, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                       (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  if (bytes <= 48 * 1024) return cudaSuccess;
  const int optin = smem_optin_max();
  if ((long long)bytes > optin) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

}  // namespace hom
