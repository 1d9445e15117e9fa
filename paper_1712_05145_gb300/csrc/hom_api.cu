// Host driver and C ABI of libhom (see include/hom.h).
//
// A handle owns the RVE on the device (phase array, per-phase Kelvin eigenvalues of
// C - C0 and C, twiddle tables), the spectrum scratch, the per-load solver state and the
// correctors of every solved order.  Solvers run entirely on the device: the host only
// launches kernels and reads back a few status words every `check_every` iterations.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <string>
#include <type_traits>
#include <vector>

#include "aux.h"
#include "equilibrium.h"
#include "hierarchy.h"
#include "plane_cluster.h"
#include "polarization.h"
#include "zcluster.h"
#include "zsplit.h"
#include "hom.h"
#include "internal.h"

using namespace hom;

namespace hom {
std::atomic<long long>& launch_counter() {
  static std::atomic<long long> n{0};
  return n;
}
void count_launch() { launch_counter().fetch_add(1, std::memory_order_relaxed); }
}  // namespace hom

namespace {

const double kSqrt2 = 1.41421356237309504880;
const double kR3 = 0.57735026918962576451, kR2 = 0.70710678118654752440, kR6 = 0.40824829046386301637;

void mandel_to_kelvin6(const double* m, double* k) {
  k[0] = (m[0] + m[1] + m[2]) * kR3;
  k[1] = (m[0] - m[1]) * kR2;
  k[2] = (m[0] + m[1] - 2.0 * m[2]) * kR6;
  k[3] = m[3];
  k[4] = m[4];
  k[5] = m[5];
}
void kelvin_to_mandel6(const double* k, double* m) {
  m[0] = k[0] * kR3 + k[1] * kR2 + k[2] * kR6;
  m[1] = k[0] * kR3 - k[1] * kR2 + k[2] * kR6;
  m[2] = k[0] * kR3 - 2.0 * k[2] * kR6;
  m[3] = k[3];
  m[4] = k[4];
  m[5] = k[5];
}

}  // namespace

struct OrderData {
  bool solved = false;
  bool disp_ok = false;   // displacement correctors computed for the current strains
  int nloads = 0;
  int cap = 0;            // loads the buffers below hold (>= nloads)
  void* eps = nullptr;    // Tf [nloads][6][M] Kelvin strain fluctuation
  void* disp = nullptr;   // Tf [nloads][3][M] displacement corrector
  void* pf = nullptr;     // Tf [nloads][6][M] Kelvin polarization p_alpha (orders >= 1)
  std::vector<double> loadsK;  // order 0: [nloads][6] Kelvin macroscopic strains
  std::vector<double> eff;     // [6][nloads] Mandel mean stresses
  bool unit = true;            // orders >= 1: the loads are the unit loads (not combinations)
};

struct hom_ctx {
  Geo g{};
  int nphase = 0;
  double lam0 = 0, mu0 = 0;
  hom_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  bool fp32 = true;
  uint8_t* d_phase = nullptr;
  double* d_mat64 = nullptr;
  float* d_mat32 = nullptr;
  cx<double>* d_tw64 = nullptr;
  df64* d_mat_df = nullptr;     // the FP64 tables as double-float (FP32 mode's FP64 passes)
  cx<df64>* d_tw_df = nullptr;
  cx<float>* d_tw32 = nullptr;
  long long tw_off[4] = {0, 0, 0, 0};
  void* d_S = nullptr;  // compute-precision spectrum, `chunk` loads (>= 9 component planes)
  size_t S_rhs_bytes = 0;
  int chunk = 1;
  int S_comps = 6;      // component planes d_S holds (per z-plane set)
  cx<double>* d_S64 = nullptr;  // FP64 spectrum for residual sweeps and RHS builds (FP32 mode)
  int chunk64 = 1;
  int S64_comps = 6;
  int cap = 0;  // loads the state / partial arrays hold
  RhsState* d_st = nullptr;
  double* d_part = nullptr;  // [2][cap][2][6*n3]
  unsigned* d_cnt = nullptr; // [2][cap]
  double* d_E = nullptr;     // [cap][6]
  double* d_mpart = nullptr; // mean reduction partials
  double* d_mout = nullptr;
  int mblk = 64;
  void* d_work[4] = {nullptr, nullptr, nullptr, nullptr};
  int ztile_lg[2] = {-1, -1};  // z-pass tile width forced by the autotuner (FP32, FP64); -1: rule
  int zc_lg[2] = {-1, -1};     // cluster z-pass tile width forced by the autotuner; -1: rule
  bool zc_off[2] = {false, false};  // the autotuner found the single-CTA z pass faster
  bool zc_tma = false;         // FP32 cluster z pass: the TMA form (z_mode 0 and 2, or the autotuner's pick)
  bool y_tma = false;          // FP32 split y pass: the TMA form (y_mode 0 and 1, or the autotuner's pick)
  unsigned* d_kerr = nullptr;  // bits set by kernels whose bounded waits gave up
  bool pc_off = false;         // the autotuner found the split x and y passes faster than the cluster ones
  bool tuned = false;
  void* d_bicg = nullptr;    // BiCGSTAB fields r_hat, v, s, t (the polarization scheme: eta)
  std::vector<double> kelvin;  // [n_phase][4] host copy of the material table: C - C0, C
  double* d_polar64 = nullptr; // [n_phase][4] polarization-scheme table (c0 w, w), built on first use
  float* d_polar32 = nullptr;
  double* d_gtab = nullptr;    // rotated finite-difference Green operator: sin, cos of pi j / N per axis
  int n_rve = 1;               // RVE slots of one grid (hom_options.n_rve)
  int rve_loads = 0;           // n_rve > 1: loads per slot (6, the unit loads); 0 with one RVE
  double* d_c0 = nullptr;      // n_rve > 1: [slot][4] (lambda0, mu0, 3 lambda0 + 2 mu0, 2 mu0)
  std::vector<double> c0_host; // n_rve > 1: host copy of d_c0
  size_t bicg_bytes = 0;
  size_t work_bytes[4] = {0, 0, 0, 0};
  OrderData ord[kMaxOrder + 1];
  size_t bytes = 0;
  std::vector<void*> allocs;
  std::string err;
  // per-kernel accounting (hom_profile)
  bool prof_on = false;
  unsigned long long* d_prof = nullptr;  // [HOM_KERNEL_COUNT][bytes, units]
  struct Pending { int kind; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[HOM_KERNEL_COUNT] = {};
  long long prof_launches[HOM_KERNEL_COUNT] = {};
};

namespace {

hom_status fail(hom_ctx* c, hom_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CK(...)                                                                                \
  do {                                                                                         \
    cudaError_t e_ = (__VA_ARGS__);                                                            \
    if (e_ != cudaSuccess)                                                                     \
      return fail(c, HOM_ERR_CUDA, "%s failed: %s (%s:%d)", #__VA_ARGS__,                      \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                                 \
  } while (0)

#define CKS(...)                         \
  do {                                   \
    hom_status s_ = (__VA_ARGS__);       \
    if (s_ != HOM_OK) return s_;         \
  } while (0)

hom_status dalloc(hom_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(c, HOM_ERR_NOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  c->bytes += bytes;
  c->allocs.push_back(*p);
  return HOM_OK;
}

void dfree(hom_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  c->bytes -= bytes;
  c->allocs.erase(std::remove(c->allocs.begin(), c->allocs.end(), p), c->allocs.end());
}

size_t field_bytes(const hom_ctx* c, int nf, int ncomp) {
  return (size_t)nf * ncomp * (size_t)c->g.M * (c->fp32 ? sizeof(float) : sizeof(double));
}

// grows work buffer i to at least `bytes`
hom_status work(hom_ctx* c, int i, size_t bytes, void** out) {
  if (c->work_bytes[i] < bytes) {
    dfree(c, c->d_work[i], c->work_bytes[i]);
    c->d_work[i] = nullptr;
    c->work_bytes[i] = 0;
    CKS(dalloc(c, &c->d_work[i], bytes));
    c->work_bytes[i] = bytes;
  }
  *out = c->d_work[i];
  return HOM_OK;
}

// partial sums one load's reducing kernel publishes at most (one per CTA)
size_t ncta_max(const hom_ctx* c) {
  return 6 * (size_t)std::max(c->g.n3 * std::max(1, c->g.pc_Q), c->g.split ? c->g.nrb : 0) + 64;
}

// grows the per-load state, partial and load arrays to `n` loads
hom_status ensure_cap(hom_ctx* c, int n) {
  if (n <= c->cap) return HOM_OK;
  const size_t ncta = ncta_max(c);
  if (c->d_st) {
    dfree(c, c->d_st, sizeof(RhsState) * c->cap);
    dfree(c, c->d_part, sizeof(double) * 2 * c->cap * 2 * ncta);
    dfree(c, c->d_cnt, sizeof(unsigned) * 2 * c->cap);
    dfree(c, c->d_E, sizeof(double) * 6 * c->cap);
    dfree(c, c->d_mpart, sizeof(double) * (size_t)c->cap * 9 * c->mblk);
    dfree(c, c->d_mout, sizeof(double) * (size_t)c->cap * 9);
  }
  c->cap = n;
  CKS(dalloc(c, (void**)&c->d_st, sizeof(RhsState) * n));
  CKS(dalloc(c, (void**)&c->d_part, sizeof(double) * 2 * n * 2 * ncta));
  CKS(dalloc(c, (void**)&c->d_cnt, sizeof(unsigned) * 2 * n));
  CKS(dalloc(c, (void**)&c->d_E, sizeof(double) * 6 * n));
  CKS(dalloc(c, (void**)&c->d_mpart, sizeof(double) * (size_t)n * 9 * c->mblk));
  CKS(dalloc(c, (void**)&c->d_mout, sizeof(double) * (size_t)n * 9));
  CK(cudaMemsetAsync(c->d_cnt, 0, sizeof(unsigned) * 2 * n, c->stream));
  CK(cudaMemsetAsync(c->d_st, 0, sizeof(RhsState) * n, c->stream));
  return HOM_OK;
}

double* part_fwd(hom_ctx* c) { return c->d_part; }
double* part_inv(hom_ctx* c) { return c->d_part + (size_t)c->cap * 2 * ncta_max(c); }
unsigned* cnt_fwd(hom_ctx* c) { return c->d_cnt; }
unsigned* cnt_inv(hom_ctx* c) { return c->d_cnt + c->cap; }

template <typename T> const T* mat_ptr(hom_ctx* c);
template <> const float* mat_ptr<float>(hom_ctx* c) { return c->d_mat32; }
template <> const double* mat_ptr<double>(hom_ctx* c) { return c->d_mat64; }
template <> const df64* mat_ptr<df64>(hom_ctx* c) { return c->d_mat_df; }
template <typename T> const cx<T>* tw(hom_ctx* c, int i);
template <> const cx<float>* tw<float>(hom_ctx* c, int i) { return c->d_tw32 + c->tw_off[i]; }
template <> const cx<double>* tw<double>(hom_ctx* c, int i) { return c->d_tw64 + c->tw_off[i]; }
template <> const cx<df64>* tw<df64>(hom_ctx* c, int i) { return c->d_tw_df + c->tw_off[i]; }

template <typename Tf, typename T>
FwdArgs<Tf, T> fwd_args(hom_ctx* c, int mode, int ncomp, int in_ncomp) {
  FwdArgs<Tf, T> a{};
  a.g = c->g;
  a.mode = mode;
  a.ncomp = ncomp;
  a.in_ncomp = in_ncomp;
  a.phase = c->d_phase;
  a.mat = mat_ptr<T>(c);
  a.n_phase = c->nphase;
  a.c0h = (T)(3.0 * c->lam0 + 2.0 * c->mu0);
  a.c0d = (T)(2.0 * c->mu0);
  a.rve_loads = c->rve_loads;
  a.c0 = c->rve_loads > 0 ? c->d_c0 : nullptr;
  a.part = part_fwd(c);
  a.cnt = cnt_fwd(c);
  a.prof = c->prof_on ? c->d_prof + 2 * (HOM_KERNEL_PLANE_FWD + (sizeof(T) == 8 ? 3 : 0)) : nullptr;
  a.tw_h = tw<T>(c, 0);
  a.tw_n1 = tw<T>(c, 1);
  a.tw_n2 = tw<T>(c, 2);
  return a;
}
template <typename T>
ZArgs<T> z_args(hom_ctx* c, int mode, int nin, int nout) {
  ZArgs<T> a{};
  a.g = c->g;
  a.mode = mode;
  a.ncomp_in = nin;
  a.ncomp_out = nout;
  a.lam0 = c->lam0;
  a.mu0 = c->mu0;
  a.rve_loads = c->rve_loads;
  a.c0 = c->rve_loads > 0 ? c->d_c0 : nullptr;
  a.scale = 1.0 / (double)c->g.M;
  a.prof = c->prof_on ? c->d_prof + 2 * (HOM_KERNEL_ZPASS + (sizeof(T) == 8 ? 3 : 0)) : nullptr;
  a.tw_n3 = tw<T>(c, 3);
  a.green = c->opt.green_operator;
  a.gtab = c->d_gtab;
  a.err = c->d_kerr;
  zpass_tiling<T>(a, c->ztile_lg[sizeof(T) == 8 ? 1 : 0]);
  return a;
}
template <typename Tf, typename T>
InvArgs<Tf, T> inv_args(hom_ctx* c, int mode, int fin, int ncomp, int out_ncomp, int s_ncomp) {
  InvArgs<Tf, T> a{};
  a.g = c->g;
  a.mode = mode;
  a.fin = fin;
  a.ncomp = ncomp;
  a.out_ncomp = out_ncomp;
  a.s_ncomp = s_ncomp;
  a.c0h = (T)(3.0 * c->lam0 + 2.0 * c->mu0);
  a.c0d = (T)(2.0 * c->mu0);
  a.rve_loads = c->rve_loads;
  a.c0 = c->rve_loads > 0 ? c->d_c0 : nullptr;
  a.out_scale = (T)1;
  a.part = part_inv(c);
  a.cnt = cnt_inv(c);
  a.prof = c->prof_on ? c->d_prof + 2 * (HOM_KERNEL_PLANE_INV + (sizeof(T) == 8 ? 3 : 0)) : nullptr;
  a.tw_h = tw<T>(c, 0);
  a.tw_n1 = tw<T>(c, 1);
  a.tw_n2 = tw<T>(c, 2);
  return a;
}

template <typename T> cx<T>* spec(hom_ctx* c, int* chunk);
template <> cx<float>* spec<float>(hom_ctx* c, int* chunk) {
  *chunk = c->chunk;
  return reinterpret_cast<cx<float>*>(c->d_S);
}
template <> cx<double>* spec<double>(hom_ctx* c, int* chunk) {
  if (c->fp32) {
    *chunk = c->chunk64;
    return c->d_S64;
  }
  *chunk = c->chunk;
  return reinterpret_cast<cx<double>*>(c->d_S);
}
template <> cx<df64>* spec<df64>(hom_ctx* c, int* chunk) {   // same bytes per value as double
  return reinterpret_cast<cx<df64>*>(spec<double>(c, chunk));
}

cudaEvent_t pool_event(hom_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Sums the device time of every completed accounted launch (synchronizes the stream).
hom_status prof_drain(hom_ctx* c) {
  if (c->pending.empty()) return HOM_OK;
  CK(cudaStreamSynchronize(c->stream));
  for (auto& p : c->pending) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, p.a, p.b));
    c->prof_ms[p.kind] += ms;
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pending.clear();
  return HOM_OK;
}

// profile kind of an LS-step kernel transforming in precision T
template <typename T>
int kind_of(int k) { return k + (sizeof(T) == 8 ? 3 : 0); }

// Launches one LS-step kernel; while accounting is on, brackets it with CUDA events.
template <typename F>
hom_status timed_launch(hom_ctx* c, int kind, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (c->prof_on) {
    a = pool_event(c);
    b = pool_event(c);
    CK(cudaEventRecord(a, c->stream));
  }
  CK(launch());
  if (c->prof_on) {
    CK(cudaEventRecord(b, c->stream));
    c->pending.push_back({kind, a, b});
    c->prof_launches[kind] += 1;
    if (c->pending.size() > 4096) CKS(prof_drain(c));
  }
  return HOM_OK;
}

// The split y pass of one chunk: its TMA variant for FP32 transforms where chosen and possible.
template <typename T>
cudaError_t ypass(hom_ctx* c, const cx<T>* tw_n2, cx<T>* S, int ncomp, int s_ncomp, int n, int dir,
                  unsigned long long* yp, const RhsState* st, int rhs0) {
  if constexpr (std::is_same<T, float>::value) {
    if (c->y_tma && ytma_fits(c->g))
      return launch_ypass_tma(tw_n2, S, c->g, ncomp, s_ncomp, n, dir, yp, st, rhs0, c->d_kerr, c->stream);
  }
  return launch_ypass<T>(tw_n2, S, c->g, ncomp, s_ncomp, n, dir, yp, st, rhs0, c->stream);
}

// Forward x-y transform of one chunk: the fused plane kernel, or the split x and y passes.
template <typename Tf, typename T>
hom_status fwd_xy(hom_ctx* c, const FwdArgs<Tf, T>& fa, int n) {
  if (!c->g.split)
    return timed_launch(c, kind_of<T>(HOM_KERNEL_PLANE_FWD), [&] { return launch_plane_fwd<Tf, T>(fa, n, c->stream); });
  if constexpr (std::is_same<T, float>::value && std::is_same<Tf, float>::value) {
    if (c->g.pc_Q > 0 && !c->pc_off)   // one cluster per plane, transposed in distributed shared memory
      return timed_launch(c, kind_of<T>(HOM_KERNEL_PLANE_FWD), [&] { return launch_plane_fwd_cluster(fa, n, c->stream); });
  }
  CKS(timed_launch(c, kind_of<T>(HOM_KERNEL_PLANE_FWD), [&] { return launch_xpass_fwd<Tf, T>(fa, n, c->stream); }));
  const int yk = sizeof(T) == 8 ? HOM_KERNEL_YPASS_F64 : HOM_KERNEL_YPASS;
  unsigned long long* yp = c->prof_on ? c->d_prof + 2 * yk : nullptr;
  return timed_launch(c, yk, [&] {
    return ypass<T>(c, fa.tw_n2, fa.S, fa.ncomp, fa.ncomp, n, -1, yp, fa.st, fa.rhs0);
  });
}

// Inverse x-y transform of one chunk with the epilogue of `ia`.
template <typename Tf, typename T>
hom_status inv_xy(hom_ctx* c, const InvArgs<Tf, T>& ia, int n) {
  if (!c->g.split)
    return timed_launch(c, kind_of<T>(HOM_KERNEL_PLANE_INV), [&] { return launch_plane_inv<Tf, T>(ia, n, c->stream); });
  if constexpr (std::is_same<T, float>::value && std::is_same<Tf, float>::value) {
    if (c->g.pc_Q > 0 && !c->pc_off)
      return timed_launch(c, kind_of<T>(HOM_KERNEL_PLANE_INV), [&] { return launch_plane_inv_cluster(ia, n, c->stream); });
  }
  const int yk = sizeof(T) == 8 ? HOM_KERNEL_YPASS_F64 : HOM_KERNEL_YPASS;
  unsigned long long* yp = c->prof_on ? c->d_prof + 2 * yk : nullptr;
  CKS(timed_launch(c, yk, [&] {
    return ypass<T>(c, ia.tw_n2, const_cast<cx<T>*>(ia.S), ia.ncomp, ia.s_ncomp, n, +1, yp, ia.st, ia.rhs0);
  }));
  return timed_launch(c, kind_of<T>(HOM_KERNEL_PLANE_INV), [&] { return launch_xpass_inv<Tf, T>(ia, n, c->stream); });
}

// One full LS pass (plane_fwd, zpass, plane_inv) over loads [0, nrhs), chunk by chunk.  The
// forward kernel reads fields of type Tf1, the inverse kernel writes fields of type Tf3, and the
// transforms run in T.
template <typename Tf1, typename Tf3, typename T>
hom_status ls_pass(hom_ctx* c, int nrhs, FwdArgs<Tf1, T> fa, ZArgs<T> za, InvArgs<Tf3, T> ia,
                   const std::vector<int>* active = nullptr) {
  int chunk;
  cx<T>* S = spec<T>(c, &chunk);
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    const int n = std::min(chunk, nrhs - r0);
    if (active) {
      bool any = false;
      for (int i = r0; i < r0 + n; ++i) any = any || (*active)[i];
      if (!any) continue;
    }
    fa.rhs0 = za.rhs0 = ia.rhs0 = r0;
    fa.S = S;
    za.S = S;
    ia.S = S;
    CKS(fwd_xy<Tf1, T>(c, fa, n));
    ZArgs<T> zc = za;
    const int zi = sizeof(T) == 8 ? 1 : 0;
    if (za.mode == Z_GAMMA && za.ncomp_in == 6 && za.ncomp_out == 6 && c->opt.z_mode != 1 && !c->zc_off[zi] &&
        zcluster_tiling<T>(zc, c->zc_lg[zi])) {
      // one pass: six CTAs per tile, the contraction in distributed shared memory
      bool tma = false;
      if constexpr (std::is_same<T, float>::value) tma = c->zc_tma && ztma_fits(c->g, zc.tc_log2);
      if (tma) {
        if constexpr (std::is_same<T, float>::value)
          CKS(timed_launch(c, kind_of<T>(HOM_KERNEL_ZPASS), [&] { return launch_zcluster_tma(zc, n, c->stream); }));
      } else {
        CKS(timed_launch(c, kind_of<T>(HOM_KERNEL_ZPASS), [&] { return launch_zcluster<T>(zc, n, c->stream); }));
      }
    } else if (za.mode == Z_GAMMA && za.ncomp_in == 6 && ((size_t)1 << za.tc_log2) * sizeof(cx<T>) < 32) {
      // deep grid: the fused z tiles would be narrower than a sector; split the z stage into
      // per-component z FFTs (one "load" per component, all loads of the chunk processed) and
      // a pointwise contraction
      ZArgs<T> zf = z_args<T>(c, Z_FWD, 1, 1);
      zpass_tiling<T>(zf, -1);
      zf.S = S;
      ZArgs<T> zi = zf;
      zi.mode = Z_INV;
      CKS(timed_launch(c, kind_of<T>(HOM_KERNEL_ZPASS), [&] { return launch_zpass<T>(zf, 6 * n, c->stream); }));
      CKS(timed_launch(c, kind_of<T>(HOM_KERNEL_ZPASS), [&] { return launch_zgreen<T>(za, n, c->stream); }));
      CKS(timed_launch(c, kind_of<T>(HOM_KERNEL_ZPASS), [&] { return launch_zpass<T>(zi, 6 * n, c->stream); }));
    } else {
      CKS(timed_launch(c, kind_of<T>(HOM_KERNEL_ZPASS), [&] { return launch_zpass<T>(za, n, c->stream); }));
    }
    CKS(inv_xy<Tf3, T>(c, ia, n));
  }
  return HOM_OK;
}

// Reads the kernels' error word (bits of bounded waits that gave up) and clears it.
hom_status check_kernel_flags(hom_ctx* c) {
  if (!c->d_kerr) return HOM_OK;
  unsigned f = 0;
  CK(cudaMemcpyAsync(&f, c->d_kerr, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (f == 0) return HOM_OK;
  CK(cudaMemsetAsync(c->d_kerr, 0, sizeof(unsigned), c->stream));
  return fail(c, HOM_ERR_CUDA, "a kernel gave up a bounded wait (flags 0x%x): its results are invalid", f);
}

hom_status read_states(hom_ctx* c, int n, std::vector<RhsState>& h) {
  h.resize(n);
  CK(cudaMemcpyAsync(h.data(), c->d_st, sizeof(RhsState) * n, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return check_kernel_flags(c);
}
hom_status write_states(hom_ctx* c, const std::vector<RhsState>& h) {
  CK(cudaMemcpyAsync(c->d_st, h.data(), sizeof(RhsState) * h.size(), cudaMemcpyHostToDevice, c->stream));
  return HOM_OK;
}

template <typename Tf>
size_t tbytes(const hom_ctx* c, int nf, int ncomp) {
  return (size_t)nf * ncomp * (size_t)c->g.M * sizeof(Tf);
}

// x <- Gamma0 * (C0 : x), the C0-orthogonal projection onto compatible fields, in FP64.  The
// FP32 corrections carry rounding noise that is not compatible; left in x, the compatible-
// subspace residual below would turn it into a compatible error scaled by the stiffness
// contrast.  Projected, x differs from the solution only by compatible errors the residual sees.
template <typename TC>
hom_status project_compatible_t(hom_ctx* c, int n, double* x64, const std::vector<int>* act) {
  auto fa = fwd_args<double, TC>(c, FWD_C0, 6, 6);
  fa.in = x64;
  fa.st = c->d_st;
  auto za = z_args<TC>(c, Z_GAMMA, 6, 6);
  za.st = c->d_st;
  auto ia = inv_args<double, TC>(c, INV_STORE, FIN_NONE, 6, 6, 6);
  ia.out = x64;
  ia.out_scale = (TC)(-1.0);
  ia.st = c->d_st;
  return ls_pass<double, double, TC>(c, n, fa, za, ia, act);
}
// FP64 mode computes in double; the FP32 mode's FP64 passes compute in double-float, which
// keeps about 48 bits (far more than these checks need) at a fraction of the FP64 pipe's cost.
hom_status project_compatible(hom_ctx* c, int n, double* x64, const std::vector<int>* act) {
  return c->fp32 ? project_compatible_t<df64>(c, n, x64, act) : project_compatible_t<double>(c, n, x64, act);
}

// Equilibrium error of sigma = C : (epsK + E) for n loads (Kelvin FP64 fields, E in c->d_E): the
// stress spectrum (plane pass in FWD_STRESS mode, then the z FFT one component at a time), its
// weighted sum of |xi . sigma_hat|^2 per CTA, and one finishing kernel for all loads.  T is the
// transform type (double, or double-float in the FP32 mode).  out: device double [n].
template <typename T>
hom_status equilibrium_t(hom_ctx* c, int n, const double* epsK, double* d_part, double* d_s0, double* d_out) {
  const int nblk = equilibrium_blocks(c->g);
  int chunk;
  cx<T>* S = spec<T>(c, &chunk);
  for (int r0 = 0; r0 < n; r0 += chunk) {
    const int m = std::min(chunk, n - r0);
    auto fa = fwd_args<double, T>(c, FWD_STRESS, 6, 6);
    fa.in = epsK;
    fa.E = c->d_E;
    fa.rhs0 = r0;
    fa.S = S;
    CKS((fwd_xy<double, T>(c, fa, m)));
    ZArgs<T> zf = z_args<T>(c, Z_FWD, 1, 1);
    zpass_tiling<T>(zf, -1);
    zf.S = S;
    CKS(timed_launch(c, kind_of<T>(HOM_KERNEL_ZPASS), [&] { return launch_zpass<T>(zf, 6 * m, c->stream); }));
    CK(launch_equilibrium_partials<T>(S, c->g, m, r0, d_part, d_s0, nblk, c->stream));
  }
  CK(launch_equilibrium_finish(d_part, d_s0, n, nblk, c->g.M, d_out, c->stream));
  return HOM_OK;
}

// The same projection computed in FP32: x32 = fp32(x), p32 = Gamma0 * (C0 : x32) in FP32, and
// x += p32 - x32, which removes the incompatible part of x up to FP32 rounding of the projection
// (about 1e-7 of ||x||).  x32 and p32 are FP32 scratch of n loads.
hom_status project_compatible_fp32(hom_ctx* c, int n, double* x64, float* x32, float* p32,
                                   const std::vector<int>* act) {
  // only the loads of `act` are touched: the conversion and the correction run load by load
  const long long per = 6 * c->g.M;
  for (int i = 0; i < n; ++i)
    if (!act || (*act)[i]) CK((launch_convert<double, float>(x64 + i * per, x32 + i * per, per, c->stream)));
  auto fa = fwd_args<float, float>(c, FWD_C0, 6, 6);
  fa.in = x32;
  fa.st = c->d_st;
  auto za = z_args<float>(c, Z_GAMMA, 6, 6);
  za.st = c->d_st;
  auto ia = inv_args<float, float>(c, INV_STORE, FIN_NONE, 6, 6, 6);
  ia.out = p32;
  ia.out_scale = -1.0f;
  ia.st = c->d_st;
  CKS((ls_pass<float, float, float>(c, n, fa, za, ia, act)));
  for (int i = 0; i < n; ++i)
    if (!act || (*act)[i]) CK(launch_add_difference(p32 + i * per, x32 + i * per, x64 + i * per, per, c->stream));
  return HOM_OK;
}

// FP64 residual sweep r = b - A x, evaluated as b - Gamma0 * (C : (x + E)) (Eq. cg_form with
// A = Gamma0 * C on compatible fields): equal to the literal residual on compatible x, and
// itself exactly compatible, so CG restarts inside the subspace where A is self-adjoint in the
// C0 product.  x and b are FP64; r is written in the iteration precision Tf.
template <typename Tf, typename TC>
hom_status residual_sweep_t(hom_ctx* c, int n, const double* dE, const double* b64, const double* x64, Tf* r,
                          int fin, const std::vector<int>* act) {
  auto fa = fwd_args<double, TC>(c, FWD_STRESS, 6, 6);
  fa.in = x64;
  fa.E = dE;
  fa.st = c->d_st;
  auto za = z_args<TC>(c, Z_GAMMA, 6, 6);
  za.st = c->d_st;
  auto ia = inv_args<Tf, TC>(c, INV_STORE, fin, 6, 6, 6);
  ia.out = r;
  ia.b = b64;
  ia.st = c->d_st;
  return ls_pass<double, Tf, TC>(c, n, fa, za, ia, act);
}
template <typename Tf>
hom_status residual_sweep(hom_ctx* c, int n, const double* dE, const double* b64, const double* x64, Tf* r,
                          int fin, const std::vector<int>* act) {
  return c->fp32 ? residual_sweep_t<Tf, df64>(c, n, dE, b64, x64, r, fin, act)
                 : residual_sweep_t<Tf, double>(c, n, dE, b64, x64, r, fin, act);
}

// out = A in = Gamma0 * (C : in) for compatible in (Eq. cg_form), one LS pass with the sign of
// eta reversed; loads whose device state is inactive are skipped.
template <typename Tf>
hom_status apply_A(hom_ctx* c, int n, const Tf* in, Tf* out, const std::vector<int>* act) {
  auto fa = fwd_args<Tf, Tf>(c, FWD_STRESS, 6, 6);
  fa.in = in;
  fa.st = c->d_st;
  auto za = z_args<Tf>(c, Z_GAMMA, 6, 6);
  za.st = c->d_st;
  auto ia = inv_args<Tf, Tf>(c, INV_STORE, FIN_NONE, 6, 6, 6);
  ia.out = out;
  ia.out_scale = (Tf)-1;
  ia.st = c->d_st;
  return ls_pass<Tf, Tf, Tf>(c, n, fa, za, ia, act);
}

// Autotuner (hom_options.autotune): times one operator application per candidate launch shape
// on this handle's grid and keeps the fastest per load.  The candidates are the loads per launch
// (1, 2, 3, 4, 6, 8, 12, ... up to the spectrum scratch's capacity, at most 12), the z stages
// that fit (the single-CTA z pass with tiles of 2^0 .. 2^4 columns, the cluster z pass with tiles
// of at least 32 bytes per z-plane) and, on planes above one CTA, the cluster plane passes against
// the split x and y passes; then the split y pass's tile width.  It tunes the passes of the
// iteration precision T.
// Tuning cache (HOM_TUNE_CACHE): one line per tuned handle kind,
//   key: n1 n2 n3 precision transform-bytes z_mode pass_mode n_rve green chunk-capacity y_mode
//   value: chunk zc_off zc_lg ztile_lg pc_off ty_log2 zc_tma y_tma
// The last line with a matching key wins.  A shape read back is one the tuner itself produced for
// the same grid and options, so it is valid for this handle.
std::string tune_key(const hom_ctx* c, size_t tbytes) {
  char b[192];
  std::snprintf(b, sizeof(b), "%d %d %d %d %zu %d %d %d %d %d %d", c->g.n1, c->g.n2, c->g.n3, c->opt.precision, tbytes,
                c->opt.z_mode, c->opt.pass_mode, c->n_rve, c->opt.green_operator, c->chunk, c->opt.y_mode);
  return b;
}

bool tune_cache_load(hom_ctx* c, const char* path, const std::string& key, int idx) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool hit = false;
  int v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  while (std::fgets(line, sizeof(line), f)) {
    const char* bar = std::strchr(line, '|');
    if (!bar || std::string(line, (size_t)(bar - line)) != key + " ") continue;
    int w[8];
    if (std::sscanf(bar + 1, "%d %d %d %d %d %d %d %d", &w[0], &w[1], &w[2], &w[3], &w[4], &w[5], &w[6], &w[7]) == 8) {
      std::memcpy(v, w, sizeof(v));
      hit = true;
    }
  }
  std::fclose(f);
  if (!hit || v[0] < 1 || v[0] > c->chunk || v[5] < 0 || v[5] > 4 || (c->g.split && !ytile_fits(c->g, v[5]))) return false;
  c->chunk = v[0];
  c->zc_off[idx] = v[1] != 0;
  c->zc_lg[idx] = v[2];
  c->ztile_lg[idx] = v[3];
  c->pc_off = v[4] != 0;
  if (c->g.split) set_ytile(c->g, v[5]);
  if (idx == 0) {
    c->zc_tma = v[6] != 0;
    c->y_tma = v[7] != 0;
  }
  return true;
}

void tune_cache_store(const hom_ctx* c, const char* path, const std::string& key, int idx) {
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s | %d %d %d %d %d %d %d %d\n", key.c_str(), c->chunk, c->zc_off[idx] ? 1 : 0, c->zc_lg[idx],
               c->ztile_lg[idx], c->pc_off ? 1 : 0, c->g.ty_log2, c->zc_tma ? 1 : 0, c->y_tma ? 1 : 0);
  std::fclose(f);
}

template <typename T>
hom_status autotune(hom_ctx* c) {
  const char* cache = std::getenv("HOM_TUNE_CACHE");
  const std::string key = tune_key(c, sizeof(T));
  if (cache && *cache && tune_cache_load(c, cache, key, sizeof(T) == 8 ? 1 : 0)) {
    c->tuned = true;
    return HOM_OK;
  }
  const int nt = std::min(c->chunk, 12);
  std::vector<int> chunks;
  for (int k : {1, 2, 3, 4, 6, 8, 12})
    if (k <= nt) chunks.push_back(k);
  // z-stage candidates: (0, lg) the single-CTA z pass with 2^lg columns, (1, lg) the cluster z
  // pass with per-element copies, (2, lg) its TMA form (FP32 transforms).  z_mode 1 keeps the
  // single-CTA pass, 2 the TMA form and 3 the per-element form where they fit.
  std::vector<std::pair<int, int>> zcand, zplain, ztma;
  for (int lg = 0; lg <= 4; ++lg)
    if (zpass_tile_fits(c->g, sizeof(cx<T>), 6, lg)) zcand.push_back({0, lg});
  if (c->opt.z_mode != 1) {
    for (int lg = 0; lg <= 6; ++lg) {
      ZArgs<T> probe{};
      probe.g = c->g;
      if (((size_t)1 << lg) * sizeof(cx<T>) >= 32 && zcluster_tiling<T>(probe, lg) && probe.tc_log2 == lg) {
        zplain.push_back({1, lg});
        if (std::is_same<T, float>::value && ztma_fits(c->g, lg)) ztma.push_back({2, lg});
      }
    }
  }
  if (c->opt.z_mode == 2 && !ztma.empty()) {
    zcand = ztma;
  } else if ((c->opt.z_mode == 3 || (c->opt.z_mode == 2 && !std::is_same<T, float>::value)) && !zplain.empty()) {
    zcand = zplain;
  } else {
    zcand.insert(zcand.end(), zplain.begin(), zplain.end());
    zcand.insert(zcand.end(), ztma.begin(), ztma.end());
  }
  if (zcand.empty()) return HOM_OK;
  const size_t fb = tbytes<T>(c, nt, 6);
  void *vin, *vout;
  CKS(work(c, 0, fb, &vin));
  CKS(work(c, 1, fb, &vout));
  CK(cudaMemsetAsync(vin, 0, fb, c->stream));
  CKS(ensure_cap(c, nt));
  std::vector<RhsState> st(nt);
  for (auto& s : st) {
    s = RhsState{};
    s.active = 1;
  }
  CKS(write_states(c, st));
  const int chunk0 = c->chunk, idx = sizeof(T) == 8 ? 1 : 0;
  cudaEvent_t e0 = pool_event(c), e1 = pool_event(c);
  // x-y candidates: the cluster plane passes where the grid has them (FP32 transforms), and the split passes
  std::vector<bool> pcand = {false};
  if (std::is_same<T, float>::value && c->g.pc_Q > 0) pcand.push_back(true);
  double best = 1e300;
  int best_chunk = chunk0, best_lg = -1, best_kind = 0;
  bool best_pc_off = false;
  for (bool pc_off : pcand)
  for (int ck : chunks) {
    for (const auto& zk : zcand) {
      const int lg = zk.second;
      c->pc_off = pc_off;
      c->chunk = ck;
      c->zc_off[idx] = (zk.first == 0);
      if (std::is_same<T, float>::value) c->zc_tma = (zk.first == 2);
      if (zk.first == 0) c->ztile_lg[idx] = lg;
      else c->zc_lg[idx] = lg;
      CKS(apply_A<T>(c, nt, reinterpret_cast<const T*>(vin), reinterpret_cast<T*>(vout), nullptr));  // warm-up
      CK(cudaEventRecord(e0, c->stream));
      for (int rep = 0; rep < 2; ++rep)
        CKS(apply_A<T>(c, nt, reinterpret_cast<const T*>(vin), reinterpret_cast<T*>(vout), nullptr));
      CK(cudaEventRecord(e1, c->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_chunk = ck;
        best_lg = lg;
        best_kind = zk.first;
        best_pc_off = pc_off;
      }
    }
  }
  c->pc_off = best_pc_off;
  c->chunk = best_chunk;
  c->zc_off[idx] = (best_kind == 0);
  if (std::is_same<T, float>::value) c->zc_tma = (best_kind == 2);
  if (best_kind == 0) {
    c->ztile_lg[idx] = best_lg;
    c->zc_lg[idx] = -1;
  } else {
    c->zc_lg[idx] = best_lg;
    c->ztile_lg[idx] = -1;
  }
  // then, where the split y pass runs, its tile width (2^2 .. 2^4 columns) and, for FP32
  // transforms, its tile copies (per-element asynchronous copies or TMA; y_mode 1 keeps TMA) with
  // the rest fixed
  if (c->g.split && (c->g.pc_Q == 0 || c->pc_off || !std::is_same<T, float>::value)) {
    constexpr bool f32 = std::is_same<T, float>::value;
    const int lg0 = c->g.ty_log2;
    const bool tma0 = f32 && c->y_tma;
    int best_y = lg0;
    bool best_tma = tma0;
    for (int lg = 2; lg <= 4; ++lg)
    for (int t = 0; t < 2; ++t) {
      const bool tma = (t == 1);
      if (!ytile_fits(c->g, lg) || (lg == lg0 && tma == tma0)) continue;
      if (tma && !f32) continue;
      if (f32 && ((c->opt.y_mode == 1 && !tma) || (c->opt.y_mode == 2 && tma))) continue;
      set_ytile(c->g, lg);
      if (tma && !ytma_fits(c->g)) continue;
      if (f32) c->y_tma = tma;
      CKS(apply_A<T>(c, nt, reinterpret_cast<const T*>(vin), reinterpret_cast<T*>(vout), nullptr));
      CK(cudaEventRecord(e0, c->stream));
      for (int rep = 0; rep < 2; ++rep)
        CKS(apply_A<T>(c, nt, reinterpret_cast<const T*>(vin), reinterpret_cast<T*>(vout), nullptr));
      CK(cudaEventRecord(e1, c->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        best_y = lg;
        best_tma = tma;
      }
    }
    set_ytile(c->g, best_y);
    if (f32) c->y_tma = best_tma;
  }
  c->ev_pool.push_back(e0);
  c->ev_pool.push_back(e1);
  c->tuned = true;
  if (cache && *cache) tune_cache_store(c, cache, key, idx);
  return HOM_OK;
}

// One BiCGSTAB sweep on A x = r from the current x (FP64 mode: the solution; FP32 mode: the
// correction d), until every load's device state is inactive.
template <typename Tf>
hom_status bicgstab_sweep(hom_ctx* c, int n, Tf* x, Tf* r, Tf* p, std::vector<RhsState>& st, std::vector<int>& act) {
  const size_t fb = tbytes<Tf>(c, n, 6);
  if (c->bicg_bytes < 4 * fb) {
    if (c->d_bicg) dfree(c, c->d_bicg, c->bicg_bytes);
    c->d_bicg = nullptr;
    c->bicg_bytes = 0;
    CKS(dalloc(c, &c->d_bicg, 4 * fb));
    c->bicg_bytes = 4 * fb;
  }
  char* w = reinterpret_cast<char*>(c->d_bicg);
  BicgArgs<Tf> a;
  a.x = x;
  a.r = r;
  a.p = p;
  a.rh = reinterpret_cast<Tf*>(w);
  a.v = reinterpret_cast<Tf*>(w + fb);
  a.s = reinterpret_cast<Tf*>(w + 2 * fb);
  a.t = reinterpret_cast<Tf*>(w + 3 * fb);
  a.M = c->g.M;
  a.st = c->d_st;
  a.part = part_fwd(c);
  a.pstride = (int)ncta_max(c);
  a.cnt = cnt_fwd(c);
  // enough CTAs per load to cover the SMs several times over, within the partial-sum slots
  const int nblk = std::max(1, std::min(a.pstride, std::max(64, (152 * 8) / n)));
  CK(launch_bicg<Tf>(BI_RESTART, a, n, nblk, c->stream));
  bool any = true;
  while (any) {
    for (int k = 0; k < c->opt.check_every; ++k) {
      CKS(apply_A<Tf>(c, n, a.p, a.v, &act));
      CK(launch_bicg<Tf>(BI_ALPHA, a, n, nblk, c->stream));
      CK(launch_bicg<Tf>(BI_S, a, n, nblk, c->stream));
      CKS(apply_A<Tf>(c, n, a.s, a.t, &act));
      CK(launch_bicg<Tf>(BI_OMEGA, a, n, nblk, c->stream));
      CK(launch_bicg<Tf>(BI_X, a, n, nblk, c->stream));
      CK(launch_bicg<Tf>(BI_P, a, n, nblk, c->stream));
    }
    CKS(read_states(c, n, st));
    any = false;
    for (int i = 0; i < n; ++i) {
      act[i] = st[i].active;
      any = any || act[i];
    }
  }
  return HOM_OK;
}

// Per-phase table of the polarization scheme, [n_phase][4] in Kelvin eigenvalues: c0 w and w for
// the hydrostatic and the deviatoric modes, w = (c - c0) / (c + c0) = eigenvalue of
// W = (C - C0) (C + C0)^-1.  The first two entries take the place of C - C0 in a FWD_TAU pass,
// which then transforms C0 : W x.
template <typename Tf> Tf*& polar_table_slot(hom_ctx* c);
template <> float*& polar_table_slot<float>(hom_ctx* c) { return c->d_polar32; }
template <> double*& polar_table_slot<double>(hom_ctx* c) { return c->d_polar64; }
template <typename Tf>
hom_status polar_table(hom_ctx* c, const Tf** out) {
  Tf*& slot = polar_table_slot<Tf>(c);
  if (!slot) {
    const double c0[2] = {3.0 * c->lam0 + 2.0 * c->mu0, 2.0 * c->mu0};
    std::vector<Tf> t(4 * 256, (Tf)0);
    for (int i = 0; i < c->nphase; ++i) {
      for (int m = 0; m < 2; ++m) {
        const double cp = c->kelvin[4 * i + 2 + m];
        const double w = (cp - c0[m]) / (cp + c0[m]);
        t[4 * i + m] = (Tf)(c0[m] * w);
        t[4 * i + 2 + m] = (Tf)w;
      }
    }
    void* p;
    CKS(dalloc(c, &p, sizeof(Tf) * 4 * 256));
    slot = reinterpret_cast<Tf*>(p);
    CK(cudaMemcpyAsync(slot, t.data(), sizeof(Tf) * 4 * 256, cudaMemcpyHostToDevice, c->stream));
  }
  *out = slot;
  return HOM_OK;
}

// One polarization-scheme sweep on A d' = r (Eq. cg_form) for the active loads, from x = r:
//   x <- (1 - g) x + g (r + W x + 2 eta),  eta = -Gamma0 * (C0 : W x)  (an LS pass),
// until each load's Cauchy quantity ||(I - W)(x_{k+1} - x_k)|| / ||b|| meets its tolerance; then
// d += (I - W) x for the loads that ran.  x lives in the p buffer, eta in the BiCGSTAB scratch.
template <typename Tf>
hom_status polar_sweep(hom_ctx* c, int n, Tf* d, const Tf* r, Tf* x, std::vector<RhsState>& st,
                       std::vector<int>& act) {
  const size_t fb = tbytes<Tf>(c, n, 6);
  if (c->bicg_bytes < fb) {
    if (c->d_bicg) dfree(c, c->d_bicg, c->bicg_bytes);
    c->d_bicg = nullptr;
    c->bicg_bytes = 0;
    CKS(dalloc(c, &c->d_bicg, fb));
    c->bicg_bytes = fb;
  }
  const Tf* wt;
  CKS(polar_table<Tf>(c, &wt));
  CK(cudaMemcpyAsync(x, r, fb, cudaMemcpyDeviceToDevice, c->stream));
  PolarArgs<Tf> a;
  a.x = x;
  a.r = r;
  a.eta = reinterpret_cast<const Tf*>(c->d_bicg);
  a.d = d;
  a.phase = c->d_phase;
  a.wt = wt;
  a.n_phase = c->nphase;
  a.relax = (c->opt.polarization_variant == 1) ? 0.5 : 1.0;
  a.M = c->g.M;
  a.rhs0 = 0;
  a.st = c->d_st;
  a.part = part_fwd(c);
  a.pstride = (int)ncta_max(c);
  a.cnt = cnt_fwd(c);
  const int nblk = std::max(1, std::min(a.pstride, std::max(64, (152 * 8) / n)));
  const std::vector<int> ran = act;
  bool any = true;
  while (any) {
    for (int k = 0; k < c->opt.check_every; ++k) {
      auto fa = fwd_args<Tf, Tf>(c, FWD_TAU, 6, 6);
      fa.mat = wt;
      fa.in = x;
      fa.st = c->d_st;
      auto za = z_args<Tf>(c, Z_GAMMA, 6, 6);
      za.st = c->d_st;
      auto ia = inv_args<Tf, Tf>(c, INV_STORE, FIN_NONE, 6, 6, 6);
      ia.out = reinterpret_cast<Tf*>(c->d_bicg);
      ia.st = c->d_st;
      CKS((ls_pass<Tf, Tf, Tf>(c, n, fa, za, ia, &act)));
      CK(launch_polar<Tf>(PO_UPDATE, a, n, nblk, c->stream));
    }
    CKS(read_states(c, n, st));
    any = false;
    for (int i = 0; i < n; ++i) {
      act[i] = st[i].active;
      any = any || act[i];
    }
  }
  for (int i0 = 0; i0 < n;) {   // d += (I - W) x over each run of loads that took part
    if (!ran[i0]) { ++i0; continue; }
    int i1 = i0;
    while (i1 < n && ran[i1]) ++i1;
    a.rhs0 = i0;
    CK(launch_polar<Tf>(PO_FINISH, a, i1 - i0, nblk, c->stream));
    i0 = i1;
  }
  return HOM_OK;
}

// FP64 residual of the operator of Eq. cg_form itself, r = b - A x with A = Id + Gamma0 * (C - C0):
// one LS pass, tau = (C - C0) : (x + E), r = -Gamma0 * tau + b - x (for order 0, b is the E term
// inside tau).  Unlike residual_sweep it sees an incompatible part of x, so a value below tol
// certifies the solution without a projection.
template <typename Tf, typename TC>
hom_status literal_residual_t(hom_ctx* c, int n, const double* dE, const double* b64, const double* x64, Tf* r,
                            const std::vector<int>* act) {
  auto fa = fwd_args<double, TC>(c, FWD_TAU, 6, 6);
  fa.in = x64;
  fa.E = dE;
  fa.st = c->d_st;
  auto za = z_args<TC>(c, Z_GAMMA, 6, 6);
  za.st = c->d_st;
  auto ia = inv_args<Tf, TC>(c, INV_STORE, FIN_RESID, 6, 6, 6);
  ia.out = r;
  ia.b = b64;
  ia.xsub = x64;
  ia.st = c->d_st;
  return ls_pass<double, Tf, TC>(c, n, fa, za, ia, act);
}
template <typename Tf>
hom_status literal_residual(hom_ctx* c, int n, const double* dE, const double* b64, const double* x64, Tf* r,
                            const std::vector<int>* act) {
  return c->fp32 ? literal_residual_t<Tf, df64>(c, n, dE, b64, x64, r, act)
                 : literal_residual_t<Tf, double>(c, n, dE, b64, x64, r, act);
}

// Solves A x = b (Eq. cg_form) for n loads; b = -Gamma0 * (C : E) for Kelvin loads dE (order 0,
// device [n][6]) or b = b64 (higher orders).  The solution x64 is FP64 in both precisions.
//  FP64 mode (Tf = double): Basic Scheme or CG in FP64 directly on x64.
//  FP32 mode (Tf = float): iterative refinement -- each sweep runs FP32 CG on A d = r from d = 0
//  (FP64 reductions), then x64 += d and an FP64 residual sweep restarts the next one.
template <typename Tf>
hom_status solve_system(hom_ctx* c, int n, const double* dE, const double* b64, double* x64, double tol,
                        hom_solve_info* info) {
  const bool mixed = sizeof(Tf) == sizeof(float);
  CKS(ensure_cap(c, n));
  const size_t fb = tbytes<Tf>(c, n, 6);
  void *vr, *vp, *vd = nullptr;
  CKS(work(c, 0, fb, &vr));
  CKS(work(c, 1, fb, &vp));
  if (mixed) CKS(work(c, 3, fb, &vd));
  Tf* r = reinterpret_cast<Tf*>(vr);
  Tf* p = reinterpret_cast<Tf*>(vp);
  Tf* d = mixed ? reinterpret_cast<Tf*>(vd) : reinterpret_cast<Tf*>(x64);
  const bool basic = (c->opt.scheme == HOM_BASIC);
  const bool bicg = (c->opt.scheme == HOM_BICGSTAB);
  const bool polar = (c->opt.scheme == HOM_POLARIZATION);
  // an FP32 sweep is asked for a reduction FP32 can deliver relative to its starting residual
  // The first sweep starts from b and aims at the tolerance itself where FP32 can reach it
  // (relative residuals down to kFirstSweepFloor); later sweeps ask for kSweepGain relative to
  // the FP64 residual they restart from.
  const double kSweepGain = 1e-5, kFirstSweepTarget = 1e-4;
  const double tol_inner = (mixed && !basic) ? std::max(0.5 * tol, kFirstSweepTarget) : (mixed ? 0.5 * tol : tol);
  // The FP32 corrections leave an incompatible part in x: CG's step lengths reach C0 / C_min
  // along the soft phases' directions and multiply the FP32 rounding of each direction p by as
  // much (4.4e-5 of ||b|| at 128^3 and contrast 100).  The residual form b - Gamma0 * (C : x)
  // does not see it, but the operator of Eq. cg_form does.  So in FP32 mode:
  //  * a sweep that aimed at the tolerance is verified with the literal residual b - A x (one
  //    FP64 pass, which sees the incompatible part); below tol the load is done;
  //  * otherwise x is projected onto compatible fields and CG restarts from the residual of the
  //    projected x (two FP64 passes).  The first sweep aims only at kFirstSweepTarget: the
  //    projection after it perturbs the residual by about the incompatible part anyway, and the
  //    later sweeps, whose corrections are small, leave a negligible incompatible part.
  // The polarization scheme's iterates are compatible only at the fixed point, so it takes the
  // same verification in both precisions.
  const bool project = mixed || polar;

  std::vector<RhsState> st(n);
  for (int i = 0; i < n; ++i) {
    RhsState s{};
    s.tol = tol_inner;
    s.max_iter = c->opt.max_iter;
    s.active = 1;
    s.restart = 1;
    s.best = 1e300;
    s.best_iter = 0;
    s.stall = mixed ? 1 : 0;   // FP64 CG runs to the tolerance: a restart there only loses information
    st[i] = s;
  }
  CKS(write_states(c, st));
  std::vector<int> refine(n, 0), done(n, 0), act(n, 1);

  if (basic) {
    // eps_0 = b (Algorithm 1 INIT); eps_{k+1} = b + T(eps_k), here T(eps_k + E) (+ b field)
    Tf* buf[2] = {d, p};
    {
      auto fa = fwd_args<Tf, Tf>(c, FWD_TAU, 6, 6);
      fa.E = dE;
      fa.st = c->d_st;
      auto za = z_args<Tf>(c, Z_GAMMA, 6, 6);
      za.st = c->d_st;
      auto ia = inv_args<Tf, Tf>(c, INV_STORE, FIN_RHS, 6, 6, 6);
      ia.out = buf[0];
      ia.b = b64;
      ia.st = c->d_st;
      CKS((ls_pass<Tf, Tf, Tf>(c, n, fa, za, ia)));
    }
    int it = 0;
    while (true) {
      for (int k = 0; k < c->opt.check_every; ++k, ++it) {
        auto fa = fwd_args<Tf, Tf>(c, FWD_TAU, 6, 6);
        fa.in = buf[it & 1];
        fa.E = dE;
        fa.st = c->d_st;
        auto za = z_args<Tf>(c, Z_GAMMA, 6, 6);
        za.st = c->d_st;
        auto ia = inv_args<Tf, Tf>(c, INV_STORE, FIN_BASIC, 6, 6, 6);
        ia.out = buf[(it + 1) & 1];
        ia.prev = buf[it & 1];
        ia.b = b64;
        ia.st = c->d_st;
        CKS((ls_pass<Tf, Tf, Tf>(c, n, fa, za, ia, &act)));
      }
      CKS(read_states(c, n, st));
      bool any = false;
      for (int i = 0; i < n; ++i) {
        act[i] = st[i].active;
        any = any || st[i].active;
      }
      if (!any) break;
    }
    // the iterate of load i sits in buf[iter_i & 1]
    const size_t one = tbytes<Tf>(c, 1, 6);
    for (int i = 0; i < n; ++i) {
      const Tf* src = reinterpret_cast<const Tf*>(reinterpret_cast<const char*>(buf[st[i].iter & 1]) + one * i);
      if (mixed) {
        CK((launch_convert<Tf, double>(src, x64 + (size_t)i * 6 * c->g.M, 6 * c->g.M, c->stream)));
      } else if (st[i].iter & 1) {
        CK(cudaMemcpyAsync(reinterpret_cast<char*>(x64) + one * i, src, one, cudaMemcpyDeviceToDevice, c->stream));
      }
    }
    // report the FP64 residual of the fixed point (the Cauchy quantity stays in `res`)
    std::vector<RhsState> before = st;
    for (int i = 0; i < n; ++i) st[i].active = 1;
    CKS(write_states(c, st));
    std::vector<int> all(n, 1);
    if (mixed) CKS(literal_residual<Tf>(c, n, dE, b64, x64, r, &all));   // sees an incompatible part
    else CKS(residual_sweep<Tf>(c, n, dE, b64, x64, r, FIN_RESID, &all));
    CKS(read_states(c, n, st));
    for (int i = 0; i < n; ++i) {
      st[i].res = before[i].res;
      st[i].status = before[i].status;
      done[i] = (before[i].status == 0);
    }
  } else {
    CK(cudaMemsetAsync(x64, 0, tbytes<double>(c, n, 6), c->stream));
    if (mixed) CK(cudaMemsetAsync(d, 0, fb, c->stream));
    // initial residual r = b (x = 0)
    if (dE != nullptr) {
      auto fa = fwd_args<Tf, Tf>(c, FWD_TAU, 6, 6);
      fa.E = dE;
      fa.st = c->d_st;
      auto za = z_args<Tf>(c, Z_GAMMA, 6, 6);
      za.st = c->d_st;
      auto ia = inv_args<Tf, Tf>(c, INV_STORE, FIN_RHS, 6, 6, 6);
      ia.out = r;
      ia.st = c->d_st;
      CKS((ls_pass<Tf, Tf, Tf>(c, n, fa, za, ia)));
    } else {
      CKS(residual_sweep<Tf>(c, n, nullptr, b64, x64, r, FIN_RHS, nullptr));
    }
    CKS(read_states(c, n, st));
    for (int i = 0; i < n; ++i) {
      if (st[i].b2 == 0.0) {  // b = 0: x = 0 is exact
        done[i] = 1;
        act[i] = 0;
        st[i].active = 0;
        st[i].res_true = 0.0;
        st[i].res = 0.0;
      }
    }
    CKS(write_states(c, st));
    while (true) {
      bool any = false;
      for (int i = 0; i < n; ++i) any = any || act[i];
      if (bicg && any) {
        CKS(bicgstab_sweep<Tf>(c, n, d, r, p, st, act));
        any = false;
      }
      if (polar && any) {
        CKS(polar_sweep<Tf>(c, n, d, r, p, st, act));
        any = false;
      }
      while (any) {
        for (int k = 0; k < c->opt.check_every; ++k) {
          auto fa = fwd_args<Tf, Tf>(c, FWD_CG, 6, 6);
          fa.r = r;
          fa.p = p;
          fa.x = d;
          fa.st = c->d_st;
          auto za = z_args<Tf>(c, Z_GAMMA, 6, 6);
          za.st = c->d_st;
          auto ia = inv_args<Tf, Tf>(c, INV_CG, FIN_CG, 6, 6, 6);
          ia.r = r;
          ia.st = c->d_st;
          CKS((ls_pass<Tf, Tf, Tf>(c, n, fa, za, ia, &act)));
        }
        CKS(read_states(c, n, st));
        any = false;
        bool pend = false;
        for (int i = 0; i < n; ++i) {
          act[i] = st[i].active;
          any = any || act[i];
          pend = pend || (!act[i] && st[i].xpend);
        }
        if (!any && pend) {
          // the last iteration's x += alpha p, which a following forward pass would have applied
          CK(launch_cg_flush<Tf>(d, p, c->d_st, 6 * c->g.M, n, c->stream));
          for (int i = 0; i < n; ++i) st[i].xpend = 0;
          CKS(write_states(c, st));
        }
      }
      if (mixed) {  // x += d, d = 0
        CK(launch_add_correction(reinterpret_cast<const float*>(d), x64, (long long)n * 6 * c->g.M, c->stream));
        CK(cudaMemsetAsync(d, 0, fb, c->stream));
      }
      bool need = false;
      for (int i = 0; i < n; ++i) {
        const bool run = !done[i] && st[i].status == 0;
        st[i].active = run ? 1 : 0;
        act[i] = run;
        need = need || run;
      }
      if (!need) break;
      CKS(write_states(c, st));
      if (project) {
        // loads whose sweep aimed at the tolerance: the literal residual decides
        std::vector<int> check(n, 0);
        bool any_check = false;
        for (int i = 0; i < n; ++i) {
          check[i] = act[i] && st[i].tol <= tol;
          any_check = any_check || check[i];
        }
        if (any_check) {
          for (int i = 0; i < n; ++i) st[i].active = check[i];
          CKS(write_states(c, st));
          CKS(literal_residual<Tf>(c, n, dE, b64, x64, r, &check));
          CKS(read_states(c, n, st));
          bool rest = false;
          for (int i = 0; i < n; ++i) {
            if (check[i] && st[i].res_true < tol) {
              done[i] = 1;
              act[i] = 0;
            }
            st[i].active = act[i];
            rest = rest || act[i];
          }
          CKS(write_states(c, st));
          if (!rest) break;
        }
        // after a load's loose first sweep an FP32 projection suffices: its rounding (~1e-7 of ||x||)
        // is far below the tolerance and the literal check at the end sees whatever is left; later
        // projections run at FP64 accuracy.  The choice is made per load, so a load's arithmetic does
        // not depend on the other loads solved with it.
        std::vector<int> loose(n, 0), tight(n, 0);
        bool any_loose = false, any_tight = false;
        for (int i = 0; i < n; ++i) {
          if (!act[i]) continue;
          if (refine[i] > 0 || st[i].tol <= tol) tight[i] = 1, any_tight = true;
          else loose[i] = 1, any_loose = true;
        }
        if (any_loose) {
          for (int i = 0; i < n; ++i) st[i].active = loose[i];
          CKS(write_states(c, st));
          CKS(project_compatible_fp32(c, n, x64, reinterpret_cast<float*>(d), reinterpret_cast<float*>(r), &loose));
          CK(cudaMemsetAsync(d, 0, fb, c->stream));   // d was scratch; the next sweep starts from 0
        }
        if (any_tight) {
          for (int i = 0; i < n; ++i) st[i].active = tight[i];
          CKS(write_states(c, st));
          CKS(project_compatible(c, n, x64, &tight));
        }
        for (int i = 0; i < n; ++i) st[i].active = act[i];
        CKS(write_states(c, st));
      }
      CKS(residual_sweep<Tf>(c, n, dE, b64, x64, r, FIN_RESID, &act));
      CKS(read_states(c, n, st));
      bool again = false;
      for (int i = 0; i < n; ++i) {
        if (!act[i]) continue;
        if (st[i].res_true < tol) {
          done[i] = 1;
          st[i].active = 0;
        } else if (refine[i] < c->opt.max_refine && st[i].iter < st[i].max_iter) {
          refine[i] += 1;
          st[i].active = 1;  // restart CG from the FP64 residual
          st[i].tol = mixed ? std::max(0.5 * tol, kSweepGain * st[i].res_true) : 0.5 * tol;
          st[i].best = 1e300;
          st[i].best_iter = st[i].iter;
          again = true;
        } else {
          st[i].active = 0;
          st[i].status = 1;
        }
        act[i] = st[i].active;
      }
      CKS(write_states(c, st));
      if (!again) break;
    }
  }

  hom_status worst = HOM_OK;
  for (int i = 0; i < n; ++i) {
    hom_status si = HOM_OK;
    if (st[i].status == 2) si = HOM_ERR_NUMERIC;
    else if (st[i].status == 1 || !done[i] || (basic && st[i].res_true >= tol && st[i].res >= tol))
      si = HOM_ERR_NOT_CONVERGED;
    if (info) {
      info[i].iterations = st[i].iter;
      info[i].refinements = refine[i];
      info[i].status = si;
      info[i].reserved = 0;
      info[i].rel_residual = st[i].res;
      info[i].rel_residual_fp64 = st[i].res_true;
    }
    if (si == HOM_ERR_NUMERIC) worst = si;
    else if (si != HOM_OK && worst == HOM_OK) worst = si;
  }
  if (worst == HOM_ERR_NOT_CONVERGED) fail(c, worst, "at least one load did not reach the tolerance");
  if (worst == HOM_ERR_NUMERIC) fail(c, worst, "NaN or Inf in a reduction");
  return worst;
}

// The fields of an order for nloads loads.  The buffers only grow, so a handle that solves batches
// of varying size (a resident serving handle) allocates once for its largest one.
hom_status alloc_order(hom_ctx* c, int order, int nloads, bool with_p) {
  OrderData& o = c->ord[order];
  if (o.eps && o.cap >= nloads && (!with_p || o.pf)) {
    o.nloads = nloads;
    return HOM_OK;
  }
  const int cap = std::max(nloads, o.cap);
  if (o.eps) dfree(c, o.eps, tbytes<double>(c, o.cap, 6));
  if (o.disp) dfree(c, o.disp, tbytes<double>(c, o.cap, 3));
  if (o.pf) dfree(c, o.pf, tbytes<double>(c, o.cap, 6));
  o.eps = o.disp = o.pf = nullptr;
  o.nloads = nloads;
  o.cap = cap;
  CKS(dalloc(c, &o.eps, tbytes<double>(c, cap, 6)));
  CKS(dalloc(c, &o.disp, tbytes<double>(c, cap, 3)));
  if (with_p) CKS(dalloc(c, &o.pf, tbytes<double>(c, cap, 6)));
  return HOM_OK;
}

// mean stress <C : (eps + E)> (order 0) or <C : eps + p> (higher orders), Mandel [6][n]
hom_status mean_stress(hom_ctx* c, int order, std::vector<double>& eff) {
  OrderData& o = c->ord[order];
  const int n = o.nloads;
  CKS(ensure_cap(c, n));
  std::vector<double> hk(n * 6), hp(n * 6, 0.0);
  if (order == 0)
    CK(cudaMemcpyAsync(c->d_E, o.loadsK.data(), sizeof(double) * 6 * n, cudaMemcpyHostToDevice, c->stream));
  CK(launch_weighted_mean<double>(reinterpret_cast<const double*>(o.eps), 6, n, order == 0 ? c->d_E : nullptr,
                                  c->d_phase, c->d_mat64, 2, c->g.M, c->d_mpart, c->mblk, c->d_mout, c->stream,
                                  c->rve_loads));
  CK(cudaMemcpyAsync(hk.data(), c->d_mout, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, c->stream));
  if (order > 0) {
    CK(launch_weighted_mean<double>(reinterpret_cast<const double*>(o.pf), 6, n, nullptr, c->d_phase, c->d_mat64,
                                    -1, c->g.M, c->d_mpart, c->mblk, c->d_mout, c->stream));
    CK(cudaMemcpyAsync(hp.data(), c->d_mout, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  eff.assign(6 * n, 0.0);
  for (int j = 0; j < n; ++j) {
    double k[6], m[6];
    for (int i = 0; i < 6; ++i) k[i] = hk[j * 6 + i] + hp[j * 6 + i];
    kelvin_to_mandel6(k, m);
    for (int i = 0; i < 6; ++i) eff[i * n + j] = m[i];
  }
  return HOM_OK;
}

// Displacement correctors u (e_y(u) = eps, zero mean) of every load of `order`, in FP64:
// forward FFT of the strain, u_hat = -i (2 eps_hat xi - xi (xi . eps_hat xi)/|xi|^2)/|xi|^2,
// inverse FFT of the 3 components.
hom_status displacements(hom_ctx* c, int order) {
  OrderData& o = c->ord[order];
  if (o.disp_ok) return HOM_OK;
  const int n = o.nloads;
  int chunk;
  cx<double>* S = spec<double>(c, &chunk);
  chunk = std::max(1, (c->fp32 ? c->S64_comps : c->S_comps) / 6);
  for (int r0 = 0; r0 < n; r0 += chunk) {
    const int m = std::min(chunk, n - r0);
    auto fa = fwd_args<double, double>(c, FWD_COPY, 6, 6);
    fa.in = reinterpret_cast<const double*>(o.eps);
    fa.rhs0 = r0;
    fa.S = S;
    CKS((fwd_xy<double, double>(c, fa, m)));
    auto za = z_args<double>(c, Z_DISP, 6, 3);
    za.S = S;
    za.rhs0 = r0;
    CKS(timed_launch(c, HOM_KERNEL_ZPASS_F64, [&] { return launch_zpass<double>(za, m, c->stream); }));
    auto ia = inv_args<double, double>(c, INV_STORE, FIN_NONE, 3, 3, 6);
    ia.S = S;
    ia.rhs0 = r0;
    ia.out = reinterpret_cast<double*>(o.disp);
    CKS((inv_xy<double, double>(c, ia, m)));
  }
  o.disp_ok = true;
  return HOM_OK;
}

// Right-hand sides b = -Gamma0 * (p_alpha + theta_alpha) of order 1 or 2 (Sec. 3, modified
// initialization), in FP64, with p_alpha kept in pf for the effective tensor.
// Multisets K of `o` directions, in the load order of order o: o = 1: k; o = 2: the Mandel
// pairs (11, 22, 33, 23, 13, 12); o >= 3: sorted tuples in lexicographic order.
std::vector<std::vector<int>> order_multisets(int o) {
  std::vector<std::vector<int>> out;
  if (o == 1) return {{0}, {1}, {2}};
  if (o == 2) return {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
  std::vector<int> cur;
  std::function<void(int)> rec = [&](int start) {
    if ((int)cur.size() == o) {
      out.push_back(cur);
      return;
    }
    for (int d = start; d < 3; ++d) {
      cur.push_back(d);
      rec(d);
      cur.pop_back();
    }
  };
  rec(0);
  return out;
}

int loads_of_order(int o) { return o == 0 ? 6 : 6 * (o + 1) * (o + 2) / 2; }

// For every multiset K of order o >= 2: the distinct directions j of K and the position of
// K - e_j among the multisets of order o - 1.
RecTable rec_table(int o) {
  RecTable t{};
  const auto cur = order_multisets(o), prev = order_multisets(o - 1);
  t.nK = (int)cur.size();
  t.nKprev = (int)prev.size();
  for (int k = 0; k < t.nK; ++k) {
    int n = 0;
    for (int j = 0; j < 3; ++j) {
      auto it = std::find(cur[k].begin(), cur[k].end(), j);
      if (it == cur[k].end()) continue;
      std::vector<int> rest = cur[k];
      rest.erase(rest.begin() + (it - cur[k].begin()));
      std::sort(rest.begin(), rest.end());
      int idx = -1;
      for (int q = 0; q < t.nKprev && idx < 0; ++q) {
        std::vector<int> pq = prev[q];
        std::sort(pq.begin(), pq.end());
        if (pq == rest) idx = q;
      }
      t.dir[k][n] = j;
      t.src[k][n] = idx;
      ++n;
    }
    t.nterm[k] = n;
  }
  return t;
}

// Right-hand sides of order `order` (b = -Gamma0 * (p + theta), Sec. 3) and the polarizations p:
// order 1 for the nu unit loads map.unit[0..nu) (order-0 correctors through map.a0), order 2 for
// the 36 unit loads.
hom_status build_rhs(hom_ctx* c, int order, double* b, double* pf, const UnitMap& map, int nu) {
  const int n = (order == 1) ? nu : loads_of_order(order);
  const RecTable rec = (order >= 2) ? rec_table(order) : RecTable{};
  CKS(displacements(c, order - 1));
  const OrderData& lo = c->ord[order - 1];
  void* v9;
  CKS(work(c, 3, tbytes<double>(c, n, 9), &v9));
  double* f9 = reinterpret_cast<double*>(v9);
  CKS(ensure_cap(c, std::max(n, 6)));
  if (order == 1)
    CK(cudaMemcpyAsync(c->d_E, c->ord[0].loadsK.data(), sizeof(double) * c->ord[0].loadsK.size(),
                       cudaMemcpyHostToDevice, c->stream));
  CK(launch_rhs_pointwise<double>(order, n, map, rec, reinterpret_cast<const double*>(lo.disp),
                                  reinterpret_cast<const double*>(lo.eps),
                                  order >= 2 ? reinterpret_cast<const double*>(lo.pf) : nullptr, c->d_E, c->d_phase,
                                  c->d_mat64, c->g.M, f9, pf, c->stream));
  int chunk;
  cx<double>* S = spec<double>(c, &chunk);
  chunk = std::max(1, (c->fp32 ? c->S64_comps : c->S_comps) / 9);
  for (int r0 = 0; r0 < n; r0 += chunk) {
    const int m = std::min(chunk, n - r0);
    auto fa = fwd_args<double, double>(c, FWD_COPY, 9, 9);
    fa.in = f9;
    fa.rhs0 = r0;
    fa.S = S;
    CKS((fwd_xy<double, double>(c, fa, m)));
    auto za = z_args<double>(c, Z_RHS, 9, 6);
    za.S = S;
    za.rhs0 = r0;
    CKS(timed_launch(c, HOM_KERNEL_ZPASS_F64, [&] { return launch_zpass<double>(za, m, c->stream); }));
    auto ia = inv_args<double, double>(c, INV_STORE, FIN_NONE, 6, 6, 9);
    ia.S = S;
    ia.rhs0 = r0;
    ia.out = b;
    CKS((inv_xy<double, double>(c, ia, m)));
  }
  return HOM_OK;
}

hom_status export_field(hom_ctx* c, int order, int load, int kind, double* d) {
  if (kind == HOM_FIELD_DISPLACEMENT) CKS(displacements(c, order));
  const OrderData& o = c->ord[order];
  const long long M = c->g.M;
  const double* eps = reinterpret_cast<const double*>(o.eps) + (long long)load * 6 * M;
  if (kind == HOM_FIELD_STRAIN) {
    CK(launch_kelvin_to_mandel<double>(eps, d, M, 1, c->stream));
  } else if (kind == HOM_FIELD_DISPLACEMENT) {
    CK(cudaMemcpyAsync(d, reinterpret_cast<const double*>(o.disp) + (long long)load * 3 * M, sizeof(double) * 3 * M,
                       cudaMemcpyDeviceToDevice, c->stream));
  } else {
    const double* ek = nullptr;
    if (order == 0) {
      CK(cudaMemcpyAsync(c->d_E, &o.loadsK[load * 6], sizeof(double) * 6, cudaMemcpyHostToDevice, c->stream));
      ek = c->d_E;
    }
    CK(launch_stress_field<double>(eps, ek,
                                   order > 0 ? reinterpret_cast<const double*>(o.pf) + (long long)load * 6 * M : nullptr,
                                   c->d_phase, c->d_mat64, M, d, c->stream));
  }
  return HOM_OK;
}

template <typename Tf>
hom_status solve_order0(hom_ctx* c, int n, const double* loads, double tol, hom_solve_info* info) {
  CKS(alloc_order(c, 0, n, false));
  OrderData& o = c->ord[0];
  o.solved = false;
  o.loadsK.assign(6 * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double m[6] = {0, 0, 0, 0, 0, 0};
    if (loads) for (int j = 0; j < 6; ++j) m[j] = loads[i * 6 + j];
    else m[i % 6] = 1.0;   // the unit loads (of each RVE slot in turn)
    mandel_to_kelvin6(m, &o.loadsK[i * 6]);
  }
  CKS(ensure_cap(c, n));
  CK(cudaMemcpyAsync(c->d_E, o.loadsK.data(), sizeof(double) * 6 * n, cudaMemcpyHostToDevice, c->stream));
  hom_status s = solve_system<Tf>(c, n, c->d_E, nullptr, reinterpret_cast<double*>(o.eps), tol, info);
  if (s != HOM_OK && s != HOM_ERR_NOT_CONVERGED) return s;
  CKS(mean_stress(c, 0, o.eff));
  o.disp_ok = false;
  o.solved = (s == HOM_OK);
  return s;
}

// order-0 load index holding the unit Mandel strain e_A, for each A (-1 if none)
void unit_order0_loads(const hom_ctx* c, int a0[6]) {
  const OrderData& o = c->ord[0];
  for (int A = 0; A < 6; ++A) a0[A] = -1;
  for (int i = 0; i < o.nloads; ++i) {
    double m[6];
    kelvin_to_mandel6(&o.loadsK[i * 6], m);
    for (int A = 0; A < 6; ++A) {
      bool unit = true;
      for (int j = 0; j < 6; ++j) unit = unit && std::fabs(m[j] - (j == A ? 1.0 : 0.0)) < 1e-14;
      if (unit && a0[A] < 0) a0[A] = i;
    }
  }
}

// Order 1 or 2 (the paper's alpha = 2, 3).  Order 1 solves the 18 unit loads (W = NULL) or n
// combinations of them, W [n][18]; order 2 solves its 36 unit loads from the 18 unit loads of
// order 1.
template <typename Tf>
hom_status solve_higher(hom_ctx* c, int order, int n, const double* W, double tol, hom_solve_info* info) {
  if (!c->ord[order - 1].solved) return fail(c, HOM_ERR_ORDER, "order %d needs a converged order %d", order, order - 1);
  UnitMap map{};
  int nu = 0;
  std::vector<double> Wu;  // W restricted to the unit loads used, [n][nu]
  if (order == 1) {
    int a0[6];
    unit_order0_loads(c, a0);
    for (int u = 0; u < 18; ++u) {
      bool used = (W == nullptr);
      for (int l = 0; l < n && !used; ++l) used = (W[l * 18 + u] != 0.0);
      if (!used) continue;
      if (a0[u / 3] < 0)
        return fail(c, HOM_ERR_ORDER, "order-1 load (A=%d, k=%d) needs the unit order-0 load e_%d", u / 3, u % 3,
                    u / 3);
      map.unit[nu++] = u;
    }
    for (int A = 0; A < 6; ++A) map.a0[A] = a0[A] < 0 ? 0 : a0[A];
    if (nu == 0) return fail(c, HOM_ERR_ARG, "every order-1 load is zero");
    if (W != nullptr) {
      Wu.assign((size_t)n * nu, 0.0);
      for (int l = 0; l < n; ++l)
        for (int j = 0; j < nu; ++j) Wu[(size_t)l * nu + j] = W[l * 18 + map.unit[j]];
    }
  } else if (!c->ord[order - 1].unit) {
    return fail(c, HOM_ERR_ORDER, "order %d needs order %d solved for its unit loads", order, order - 1);
  }
  CKS(alloc_order(c, order, n, true));
  OrderData& o = c->ord[order];
  o.solved = false;
  o.unit = (W == nullptr);
  void* vb;
  CKS(work(c, 2, tbytes<double>(c, n, 6), &vb));
  double* b = reinterpret_cast<double*>(vb);
  if (order == 1 && W != nullptr) {
    // the unit right-hand sides and polarizations, then their combinations (both linear in the load)
    void *bu = nullptr, *pu = nullptr, *dW = nullptr;
    const size_t ub = tbytes<double>(c, nu, 6);
    hom_status st = dalloc(c, &bu, ub);
    if (st == HOM_OK) st = dalloc(c, &pu, ub);
    if (st == HOM_OK) st = dalloc(c, &dW, sizeof(double) * Wu.size());
    if (st == HOM_OK) st = build_rhs(c, 1, reinterpret_cast<double*>(bu), reinterpret_cast<double*>(pu), map, nu);
    if (st == HOM_OK &&
        cudaMemcpyAsync(dW, Wu.data(), sizeof(double) * Wu.size(), cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
      st = fail(c, HOM_ERR_CUDA, "copy of the load combinations failed");
    const long long per = 6LL * c->g.M;
    if (st == HOM_OK && launch_combine_loads(reinterpret_cast<const double*>(bu), nu,
                                             reinterpret_cast<const double*>(dW), n, per, b,
                                             c->stream) != cudaSuccess)
      st = fail(c, HOM_ERR_CUDA, "combine_loads launch failed");
    if (st == HOM_OK && launch_combine_loads(reinterpret_cast<const double*>(pu), nu,
                                             reinterpret_cast<const double*>(dW), n, per,
                                             reinterpret_cast<double*>(o.pf), c->stream) != cudaSuccess)
      st = fail(c, HOM_ERR_CUDA, "combine_loads launch failed");
    if (cudaStreamSynchronize(c->stream) != cudaSuccess && st == HOM_OK)
      st = fail(c, HOM_ERR_CUDA, "building the order-1 combinations failed");
    if (bu) dfree(c, bu, ub);
    if (pu) dfree(c, pu, ub);
    if (dW) dfree(c, dW, sizeof(double) * Wu.size());
    if (st != HOM_OK) return st;
  } else {
    CKS(build_rhs(c, order, b, reinterpret_cast<double*>(o.pf), map, order == 1 ? nu : n));
  }
  hom_status s = solve_system<Tf>(c, n, nullptr, b, reinterpret_cast<double*>(o.eps), tol, info);
  if (s != HOM_OK && s != HOM_ERR_NOT_CONVERGED) return s;
  CKS(mean_stress(c, order, o.eff));
  o.disp_ok = false;
  o.solved = (s == HOM_OK);
  return s;
}

void twiddles(int n, std::vector<cx<double>>& out) {
  for (int t = 0; t < n; ++t) {
    const double a = -2.0 * M_PI * (double)t / (double)n;
    cx<double> w;
    w.re = std::cos(a);
    w.im = std::sin(a);
    out.push_back(w);
  }
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

HOM_API void hom_default_options(hom_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = HOM_FP32_REFINE;
  opt->scheme = HOM_CG;
  opt->max_iter = 2000;
  opt->check_every = 8;
  opt->max_refine = 6;
  opt->rhs_chunk = 0;
  opt->spectrum_budget_bytes = 1024LL << 20;
  opt->cuda_stream = nullptr;
}

HOM_API const char* hom_status_string(hom_status s) {
  switch (s) {
    case HOM_OK: return "HOM_OK";
    case HOM_ERR_ARG: return "HOM_ERR_ARG";
    case HOM_ERR_SIZE: return "HOM_ERR_SIZE";
    case HOM_ERR_NOMEM: return "HOM_ERR_NOMEM";
    case HOM_ERR_NOT_CONVERGED: return "HOM_ERR_NOT_CONVERGED";
    case HOM_ERR_ORDER: return "HOM_ERR_ORDER";
    case HOM_ERR_NUMERIC: return "HOM_ERR_NUMERIC";
    case HOM_ERR_TIMEOUT: return "HOM_ERR_TIMEOUT";
    case HOM_ERR_CUDA: return "HOM_ERR_CUDA";
  }
  return "HOM_ERR_UNKNOWN";
}

HOM_API const char* hom_last_error(hom_t h) { return h ? h->err.c_str() : "null handle"; }

HOM_API int64_t hom_device_bytes(hom_t h) { return h ? (int64_t)h->bytes : 0; }

HOM_API hom_status hom_launch_config(hom_t c, int32_t* loads_per_launch, int32_t* ztile_log2) {
  if (!c) return HOM_ERR_ARG;
  if (loads_per_launch) *loads_per_launch = c->chunk;
  if (ztile_log2) *ztile_log2 = c->ztile_lg[c->fp32 ? 0 : 1];
  return HOM_OK;
}

HOM_API hom_status hom_ypass_config(hom_t c, int32_t* tile_log2, int32_t* tma) {
  if (!c) return HOM_ERR_ARG;
  const bool fp32_split = c->fp32 && c->g.split && (c->g.pc_Q == 0 || c->pc_off);
  if (tile_log2) *tile_log2 = c->g.split ? c->g.ty_log2 : -1;
  if (tma) *tma = (fp32_split && c->y_tma && ytma_fits(c->g)) ? 1 : 0;
  return HOM_OK;
}

HOM_API hom_status hom_plane_config(hom_t c, int32_t* cluster_ctas) {
  if (!c) return HOM_ERR_ARG;
  if (cluster_ctas) *cluster_ctas = (c->g.pc_Q > 0 && !c->pc_off) ? c->g.pc_Q : 0;
  return HOM_OK;
}

HOM_API hom_status hom_zpass_config(hom_t c, int32_t* cluster, int32_t* tile_log2) {
  if (!c) return HOM_ERR_ARG;
  const int zi = c->fp32 ? 0 : 1;
  ZArgs<float> p32{};
  ZArgs<double> p64{};
  p32.g = c->g;
  p64.g = c->g;
  bool on = c->opt.z_mode != 1 && !c->zc_off[zi];
  if (on) on = c->fp32 ? zcluster_tiling<float>(p32, c->zc_lg[zi]) : zcluster_tiling<double>(p64, c->zc_lg[zi]);
  const bool tma = on && c->fp32 && c->zc_tma && ztma_fits(c->g, p32.tc_log2);
  if (cluster) *cluster = tma ? 2 : (on ? 1 : 0);
  if (tile_log2) *tile_log2 = on ? (c->fp32 ? p32.tc_log2 : p64.tc_log2) : c->ztile_lg[zi];
  return HOM_OK;
}

HOM_API int64_t hom_launch_count(void) { return hom::launch_counter().load(std::memory_order_relaxed); }

HOM_API int64_t hom_estimate_bytes(const int32_t grid[3], int32_t order, int32_t precision) {
  if (!grid) return -1;
  const long long n1 = grid[0], n2 = grid[1], n3 = grid[2];
  if (n1 < 4 || (n1 & 1) || !fft_length_supported((int)(n1 / 2)) || !fft_length_supported((int)n2) ||
      !z_length_supported((int)n3) || order < 0 || order > kMaxOrder)
    return -1;
  const bool fp32 = (precision == HOM_FP32_REFINE);
  const long long M = n1 * n2 * n3, plane_c = n2 * (n1 / 2 + 1);
  const long long budget = 1024LL << 20;
  auto scratch = [&](long long elem) {
    const long long per = 6 * n3 * plane_c * elem;
    long long chunk = std::max(1LL, budget / per);
    chunk = std::min(chunk, 64LL);
    return per / 6 * std::max(6 * chunk, 9LL);
  };
  long long b = M + (1LL << 20);                 // phase, tables, states
  b += scratch(fp32 ? 8 : 16);
  if (fp32) b += scratch(16);
  const long long nl = loads_of_order(order), tf = fp32 ? 4 : 8;
  b += 2 * nl * 6 * M * tf;                      // r, p
  long long slot3 = fp32 ? nl * 6 * M * 4 : 0;   // FP32 correction d
  if (order >= 1) {
    b += nl * 6 * M * 8;                         // right-hand sides
    slot3 = std::max(slot3, nl * 9 * M * 8);     // p and g of the right-hand-side build
  }
  b += slot3;
  b += 6 * 9 * M * 8;                            // order-0 strain and displacement
  for (int o = 1; o <= order; ++o)               // strain, displacement, polarization of each order
    b += (long long)loads_of_order(o) * 15 * M * 8;
  return (int64_t)((double)b * 1.05) + (16LL << 20);
}

HOM_API hom_status hom_profile(hom_t c, int32_t enable) {
  if (!c) return HOM_ERR_ARG;
  CKS(prof_drain(c));
  if (enable) {
    if (!c->d_prof) CKS(dalloc(c, (void**)&c->d_prof, sizeof(unsigned long long) * 2 * HOM_KERNEL_COUNT));
    CK(cudaMemsetAsync(c->d_prof, 0, sizeof(unsigned long long) * 2 * HOM_KERNEL_COUNT, c->stream));
    for (int k = 0; k < HOM_KERNEL_COUNT; ++k) {
      c->prof_ms[k] = 0.0;
      c->prof_launches[k] = 0;
    }
  }
  c->prof_on = (enable != 0);
  return HOM_OK;
}

HOM_API hom_status hom_profile_read(hom_t c, hom_kernel_stat* out) {
  if (!c || !out) return HOM_ERR_ARG;
  CKS(prof_drain(c));
  unsigned long long hp[2 * HOM_KERNEL_COUNT] = {};
  if (c->d_prof) {
    CK(cudaMemcpyAsync(hp, c->d_prof, sizeof(hp), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  for (int k = 0; k < HOM_KERNEL_COUNT; ++k) {
    out[k].launches = c->prof_launches[k];
    out[k].bytes = (int64_t)hp[2 * k];
    out[k].voxel_comps = (int64_t)hp[2 * k + 1];
    out[k].ms = c->prof_ms[k];
  }
  return HOM_OK;
}

HOM_API void hom_destroy(hom_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& p : h->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  for (void* p : h->allocs) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// Copies one RVE into slot `slot` of the handle: the phase array (host or device source, every
// value < n_phase), the per-phase Kelvin eigenvalues of C - C0 and C in FP64, FP32 and
// double-float, and the reference medium.  Synchronous on the handle's stream.
hom_status set_rve_data(hom_ctx* c, int slot, const uint8_t* phase, int n_phase, const double* lame, double lambda0,
                        double mu0) {
  const Geo& g = c->g;
  std::vector<uint8_t> hph((size_t)g.M);
  if (is_device_ptr(phase)) {
    CK(cudaMemcpy(hph.data(), phase, (size_t)g.M, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(hph.data(), phase, (size_t)g.M);
  }
  for (size_t i = 0; i < hph.size(); ++i)
    if (hph[i] >= n_phase) return fail(c, HOM_ERR_ARG, "phase value %d >= n_phase %d", (int)hph[i], n_phase);
  // per-phase Kelvin eigenvalues: C - C0 (3 dK, 2 dmu), C (3K, 2mu)
  std::vector<double> m64(4 * 256, 0.0);
  std::vector<float> m32(4 * 256, 0.0f);
  for (int i = 0; i < n_phase; ++i) {
    const double l = lame[2 * i], m = lame[2 * i + 1];
    if (!std::isfinite(l) || !std::isfinite(m)) return fail(c, HOM_ERR_ARG, "non-finite Lame parameter");
    m64[4 * i + 0] = 3.0 * (l - lambda0) + 2.0 * (m - mu0);
    m64[4 * i + 1] = 2.0 * (m - mu0);
    m64[4 * i + 2] = 3.0 * l + 2.0 * m;
    m64[4 * i + 3] = 2.0 * m;
    for (int j = 0; j < 4; ++j) m32[4 * i + j] = (float)m64[4 * i + j];
  }
  std::vector<df64> mdf(4 * 256, df64(0.0f, 0.0f));
  for (int i = 0; i < 4 * 256; ++i) mdf[i] = df64(m64[i]);
  const size_t t = (size_t)slot * 4 * 256;
  CK(cudaMemcpyAsync(c->d_phase + (size_t)slot * g.M, hph.data(), (size_t)g.M, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_mat64 + t, m64.data(), sizeof(double) * 4 * 256, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_mat32 + t, m32.data(), sizeof(float) * 4 * 256, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->d_mat_df + t, mdf.data(), sizeof(df64) * 4 * 256, cudaMemcpyHostToDevice, c->stream));
  if (c->n_rve > 1) {
    // the C0 weights are computed here as the one-RVE path computes its scalar c0h, c0d, so that a
    // slot's arithmetic is that of a handle holding its RVE alone
    double* w = &c->c0_host[4 * slot];
    w[0] = lambda0;
    w[1] = mu0;
    w[2] = 3.0 * lambda0 + 2.0 * mu0;
    w[3] = 2.0 * mu0;
    CK(cudaMemcpyAsync(c->d_c0 + 4 * slot, w, sizeof(double) * 4, cudaMemcpyHostToDevice, c->stream));
  } else {
    c->nphase = n_phase;
    c->lam0 = lambda0;
    c->mu0 = mu0;
    c->kelvin.assign(m64.begin(), m64.begin() + 4 * n_phase);
  }
  CK(cudaStreamSynchronize(c->stream));
  return HOM_OK;
}

HOM_API hom_status hom_create(const int32_t grid[3], const uint8_t* phase, int32_t n_phase, const double* lame,
                              double lambda0, double mu0, const hom_options* opt, hom_t* out) {
  hom_ctx* c = nullptr;
  if (!grid || !phase || !lame || !out) return HOM_ERR_ARG;
  if (n_phase < 1 || n_phase > 256) return HOM_ERR_ARG;
  if (!(mu0 != 0.0) || !(lambda0 + 2.0 * mu0 != 0.0) || !std::isfinite(lambda0) || !std::isfinite(mu0))
    return HOM_ERR_ARG;
  const int n1 = grid[0], n2 = grid[1], n3 = grid[2];
  if (n1 < 4 || (n1 & 1) || !fft_length_supported(n1 / 2) || !fft_length_supported(n2) ||
      !z_length_supported(n3))
    return HOM_ERR_SIZE;
  const int pass_mode = opt ? opt->pass_mode : 0;
  if (pass_mode < 0 || pass_mode > 3) return HOM_ERR_ARG;
  if (opt && (opt->z_mode < 0 || opt->z_mode > 3)) return HOM_ERR_ARG;
  if (opt && (opt->y_mode < 0 || opt->y_mode > 2)) return HOM_ERR_ARG;
  if (opt && opt->green_operator != HOM_GREEN_SPECTRAL && opt->green_operator != HOM_GREEN_ROTATED) return HOM_ERR_ARG;
  if (pass_mode == 1 && (long long)(n1 / 2) * n2 > 8192) return HOM_ERR_SIZE;

  c = new hom_ctx();
  hom_default_options(&c->opt);
  if (opt) c->opt = *opt;
  if (c->opt.max_iter < 1) c->opt.max_iter = 1;
  if (c->opt.check_every < 1) c->opt.check_every = 1;
  if (c->opt.max_refine < 0) c->opt.max_refine = 0;
  if (c->opt.spectrum_budget_bytes <= 0) c->opt.spectrum_budget_bytes = 1024LL << 20;
  if (c->opt.precision != HOM_FP64 && c->opt.precision != HOM_FP32_REFINE) { delete c; return HOM_ERR_ARG; }
  if (c->opt.scheme != HOM_BASIC && c->opt.scheme != HOM_CG && c->opt.scheme != HOM_BICGSTAB &&
      c->opt.scheme != HOM_POLARIZATION) {
    delete c;
    return HOM_ERR_ARG;
  }
  if (c->opt.scheme == HOM_POLARIZATION) {
    // |w| = |c - c0| / (c + c0) <= 1 needs positive reference moduli and non-negative phase moduli
    bool ok = (mu0 > 0.0) && (3.0 * lambda0 + 2.0 * mu0 > 0.0) &&
              (c->opt.polarization_variant == 0 || c->opt.polarization_variant == 1);
    for (int i = 0; i < n_phase && ok; ++i)
      ok = (2.0 * lame[2 * i + 1] >= 0.0) && (3.0 * lame[2 * i] + 2.0 * lame[2 * i + 1] >= 0.0);
    if (!ok) {
      delete c;
      return HOM_ERR_ARG;
    }
  }
  c->fp32 = (c->opt.precision == HOM_FP32_REFINE);
  c->nphase = n_phase;
  c->lam0 = lambda0;
  c->mu0 = mu0;
  c->n_rve = c->opt.n_rve < 1 ? 1 : c->opt.n_rve;
  if (c->n_rve > kMaxRve || (c->n_rve > 1 && c->opt.scheme == HOM_POLARIZATION)) {
    delete c;
    return HOM_ERR_ARG;
  }
  c->rve_loads = c->n_rve > 1 ? 6 : 0;
  cudaGetDevice(&c->device);
  if (c->opt.cuda_stream) {
    c->stream = reinterpret_cast<cudaStream_t>(c->opt.cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return HOM_ERR_CUDA;
    }
    c->own_stream = true;
  }

  Geo& g = c->g;
  g.n1 = n1;
  g.n2 = n2;
  g.n3 = n3;
  g.h = n1 / 2;
  g.P = (g.h & 1) ? g.h : g.h + 1;
  g.M = (long long)n1 * n2 * n3;
  g.plane_c = (long long)n2 * (g.h + 1);
  geo_finish(g);
  g.split = (pass_mode >= 2 || (pass_mode == 0 && (long long)g.n2 * g.h > 8192)) ? 1 : 0;
  const int nmax = std::max(n1, std::max(n2, n3));
  g.xs1 = 2.0 * M_PI * nmax / n1;
  g.xs2 = 2.0 * M_PI * nmax / n2;
  g.xs3 = 2.0 * M_PI * nmax / n3;

  auto bail = [&](hom_status s) {
    hom_destroy(c);
    return s;
  };
  // FP32 transforms of split planes run as cluster plane passes (pass_mode 0 or 3)
  if (g.split && pass_mode != 2 && c->fp32 && !plane_cluster_setup(g) && pass_mode == 3) return bail(HOM_ERR_SIZE);

  // phase arrays and per-phase tables of every RVE slot (all filled with the given RVE)
  hom_status s;
  if (c->n_rve > 1) c->nphase = 256;   // slots may differ in their phase counts; tables are padded
  if ((s = dalloc(c, (void**)&c->d_phase, (size_t)g.M * c->n_rve)) != HOM_OK) return bail(s);
  if ((s = dalloc(c, (void**)&c->d_mat64, sizeof(double) * 4 * 256 * c->n_rve)) != HOM_OK) return bail(s);
  if ((s = dalloc(c, (void**)&c->d_mat32, sizeof(float) * 4 * 256 * c->n_rve)) != HOM_OK) return bail(s);
  if ((s = dalloc(c, (void**)&c->d_mat_df, sizeof(df64) * 4 * 256 * c->n_rve)) != HOM_OK) return bail(s);
  if (c->n_rve > 1) {
    if ((s = dalloc(c, (void**)&c->d_c0, sizeof(double) * 4 * c->n_rve)) != HOM_OK) return bail(s);
    c->c0_host.assign(4 * c->n_rve, 0.0);
  }
  for (int slot = 0; slot < c->n_rve; ++slot)
    if ((s = set_rve_data(c, slot, phase, n_phase, lame, lambda0, mu0)) != HOM_OK) return bail(s);

  // twiddle tables exp(-2 pi i t / L) for L = h, n1, n2, n3 (host libm, FP64)
  std::vector<cx<double>> t64;
  const int lens[4] = {g.h, n1, n2, n3};
  for (int i = 0; i < 4; ++i) {
    c->tw_off[i] = (long long)t64.size();
    twiddles(lens[i], t64);
  }
  std::vector<cx<float>> t32(t64.size());
  for (size_t i = 0; i < t64.size(); ++i) {
    t32[i].re = (float)t64[i].re;
    t32[i].im = (float)t64[i].im;
  }
  if ((s = dalloc(c, (void**)&c->d_tw64, sizeof(cx<double>) * t64.size())) != HOM_OK) return bail(s);
  if ((s = dalloc(c, (void**)&c->d_tw32, sizeof(cx<float>) * t32.size())) != HOM_OK) return bail(s);
  cudaMemcpy(c->d_tw64, t64.data(), sizeof(cx<double>) * t64.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(c->d_tw32, t32.data(), sizeof(cx<float>) * t32.size(), cudaMemcpyHostToDevice);
  std::vector<cx<df64>> tdf(t64.size());
  for (size_t i = 0; i < t64.size(); ++i) {
    tdf[i].re = df64(t64[i].re);
    tdf[i].im = df64(t64[i].im);
  }
  if ((s = dalloc(c, (void**)&c->d_tw_df, sizeof(cx<df64>) * tdf.size())) != HOM_OK) return bail(s);
  cudaMemcpy(c->d_tw_df, tdf.data(), sizeof(cx<df64>) * tdf.size(), cudaMemcpyHostToDevice);

  // the rotated finite-difference operator's per-axis table: sin(pi j / N), cos(pi j / N) by DFT index
  // (j <= N1/2 on the half-spectrum axis), cos exactly 0 at j = N/2
  if (c->opt.green_operator == HOM_GREEN_ROTATED) {
    std::vector<double> gt;
    auto axis = [&](int n, int count) {
      for (int j = 0; j < count; ++j) gt.push_back(std::sin(M_PI * j / n));
      for (int j = 0; j < count; ++j) gt.push_back(2 * j == n ? 0.0 : std::cos(M_PI * j / n));
    };
    axis(n1, g.h + 1);
    axis(n2, n2);
    axis(n3, n3);
    if ((s = dalloc(c, (void**)&c->d_gtab, sizeof(double) * gt.size())) != HOM_OK) return bail(s);
    cudaMemcpy(c->d_gtab, gt.data(), sizeof(double) * gt.size(), cudaMemcpyHostToDevice);
  }

  // spectrum scratch
  const size_t elem = c->fp32 ? sizeof(cx<float>) : sizeof(cx<double>);
  c->S_rhs_bytes = (size_t)6 * n3 * (size_t)g.plane_c * elem;
  const size_t budget = (size_t)c->opt.spectrum_budget_bytes;
  c->chunk = c->opt.rhs_chunk > 0 ? c->opt.rhs_chunk : (int)std::max<size_t>(1, budget / c->S_rhs_bytes);
  c->chunk = std::min(c->chunk, 64);
  c->S_comps = std::max(6 * c->chunk, 9);
  if ((s = dalloc(c, &c->d_S, c->S_rhs_bytes / 6 * c->S_comps)) != HOM_OK) return bail(s);
  if (c->fp32) {
    const size_t b64 = (size_t)6 * n3 * (size_t)g.plane_c * sizeof(cx<double>);
    c->chunk64 = (int)std::max<size_t>(1, budget / b64);
    c->chunk64 = std::min(c->chunk64, 64);
    c->S64_comps = std::max(6 * c->chunk64, 9);
    if ((s = dalloc(c, (void**)&c->d_S64, b64 / 6 * c->S64_comps)) != HOM_OK) return bail(s);
  }
  if ((s = ensure_cap(c, 6)) != HOM_OK) return bail(s);
  if ((s = dalloc(c, (void**)&c->d_kerr, sizeof(unsigned))) != HOM_OK) return bail(s);
  if (cudaMemsetAsync(c->d_kerr, 0, sizeof(unsigned), c->stream) != cudaSuccess) return bail(HOM_ERR_CUDA);
  c->zc_tma = (c->opt.z_mode == 0 || c->opt.z_mode == 2);
  c->y_tma = (c->opt.y_mode != 2);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(HOM_ERR_CUDA);
  *out = c;
  return HOM_OK;
}

HOM_API hom_status hom_solve(hom_t c, int32_t order, int32_t n_loads, const double* loads, double tol,
                             hom_solve_info* info) {
  if (!c) return HOM_ERR_ARG;
  if (!(tol > 0.0)) return fail(c, HOM_ERR_ARG, "tol must be > 0");
  if (order < 0 || order > kMaxOrder) return fail(c, HOM_ERR_ARG, "order must be in 0..%d", kMaxOrder);
  for (int k = order + 1; k <= kMaxOrder; ++k) c->ord[k].solved = false;
  if (c->opt.autotune && !c->tuned) {
    hom_status t = c->fp32 ? autotune<float>(c) : autotune<double>(c);
    if (t != HOM_OK) return t;
  }
  if (c->n_rve > 1) {
    // several RVE slots: the 6 unit loads of the first n_loads / 6 slots (all slots for 0)
    if (order != 0 || loads) return fail(c, HOM_ERR_ARG, "a handle with several RVEs solves order 0, unit loads only");
    const int n = n_loads > 0 ? n_loads : 6 * c->n_rve;
    if (n % 6 != 0 || n > 6 * c->n_rve) return fail(c, HOM_ERR_ARG, "n_loads must be 6 x (RVE slots to solve)");
    return c->fp32 ? solve_order0<float>(c, n, nullptr, tol, info) : solve_order0<double>(c, n, nullptr, tol, info);
  }
  if (order == 0) {
    int n = loads ? n_loads : 6;
    if (n < 1 || n > 64) return fail(c, HOM_ERR_ARG, "n_loads must be in 1..64");
    return c->fp32 ? solve_order0<float>(c, n, loads, tol, info) : solve_order0<double>(c, n, loads, tol, info);
  }
  if (c->opt.green_operator != HOM_GREEN_SPECTRAL)
    return fail(c, HOM_ERR_ARG, "the higher-order problems are built with the spectral Green operator only");
  if (order >= 2 && loads) return fail(c, HOM_ERR_ARG, "orders >= 2 take only their unit loads (loads = NULL)");
  int n = loads_of_order(order);
  if (order == 1 && loads) {
    n = n_loads;
    if (n < 1 || n > 64) return fail(c, HOM_ERR_ARG, "n_loads must be in 1..64");
  }
  c->ord[order].solved = false;
  return c->fp32 ? solve_higher<float>(c, order, n, loads, tol, info)
                 : solve_higher<double>(c, order, n, loads, tol, info);
}

HOM_API hom_status hom_set_rve(hom_t c, int32_t slot, const uint8_t* phase, int32_t n_phase, const double* lame,
                               double lambda0, double mu0) {
  if (!c || !phase || !lame) return HOM_ERR_ARG;
  if (slot < 0 || slot >= c->n_rve) return fail(c, HOM_ERR_ARG, "slot out of range");
  if (n_phase < 1 || n_phase > 256) return fail(c, HOM_ERR_ARG, "n_phase must be in 1..256");
  if (!(mu0 != 0.0) || !(lambda0 + 2.0 * mu0 != 0.0) || !std::isfinite(lambda0) || !std::isfinite(mu0))
    return fail(c, HOM_ERR_ARG, "degenerate reference medium");
  if (c->opt.scheme == HOM_POLARIZATION) {
    bool ok = (mu0 > 0.0) && (3.0 * lambda0 + 2.0 * mu0 > 0.0);
    for (int i = 0; i < n_phase && ok; ++i)
      ok = (2.0 * lame[2 * i + 1] >= 0.0) && (3.0 * lame[2 * i] + 2.0 * lame[2 * i + 1] >= 0.0);
    if (!ok) return fail(c, HOM_ERR_ARG, "the polarization scheme needs non-negative moduli");
  }
  CK(cudaStreamSynchronize(c->stream));   // no pass of the previous RVE still reads the tables
  CKS(set_rve_data(c, slot, phase, n_phase, lame, lambda0, mu0));
  // the polarization tables and every solved order belonged to the previous microstructure
  dfree(c, c->d_polar64, sizeof(double) * 4 * 256);
  dfree(c, c->d_polar32, sizeof(float) * 4 * 256);
  c->d_polar64 = nullptr;
  c->d_polar32 = nullptr;
  for (int k = 0; k <= kMaxOrder; ++k) {
    c->ord[k].solved = false;
    c->ord[k].disp_ok = false;
    c->ord[k].eff.clear();
  }
  return HOM_OK;
}

HOM_API hom_status hom_effective(hom_t c, int32_t order, double* out) {
  if (!c || !out) return HOM_ERR_ARG;
  if (order < 0 || order > kMaxOrder) return fail(c, HOM_ERR_ARG, "order must be in 0..%d", kMaxOrder);
  const OrderData& o = c->ord[order];
  if (o.eff.empty()) return fail(c, HOM_ERR_ORDER, "order %d has not been solved", order);
  std::memcpy(out, o.eff.data(), sizeof(double) * o.eff.size());
  return HOM_OK;
}

HOM_API hom_status hom_get_field(hom_t c, int32_t order, int32_t load, int32_t kind, double* dst,
                                 int32_t dst_on_device) {
  if (!c || !dst) return HOM_ERR_ARG;
  if (order < 0 || order > kMaxOrder) return fail(c, HOM_ERR_ARG, "order must be in 0..%d", kMaxOrder);
  const OrderData& o = c->ord[order];
  if (!o.eps || o.eff.empty()) return fail(c, HOM_ERR_ORDER, "order %d has not been solved", order);
  if (load < 0 || load >= o.nloads) return fail(c, HOM_ERR_ARG, "load out of range");
  if (kind != HOM_FIELD_STRAIN && kind != HOM_FIELD_DISPLACEMENT && kind != HOM_FIELD_STRESS)
    return fail(c, HOM_ERR_ARG, "unknown field kind");
  if (kind == HOM_FIELD_DISPLACEMENT && c->opt.green_operator != HOM_GREEN_SPECTRAL)
    return fail(c, HOM_ERR_ARG, "displacements are recovered with the spectral operator only");
  const int nc = (kind == HOM_FIELD_DISPLACEMENT) ? 3 : 6;
  const size_t nbytes = sizeof(double) * nc * (size_t)c->g.M;
  double* d = dst;
  void* tmp = nullptr;
  if (!dst_on_device) {
    CKS(work(c, 2, std::max(nbytes, c->work_bytes[2]), &tmp));
    d = reinterpret_cast<double*>(tmp);
  }
  hom_status s = export_field(c, order, load, kind, d);
  if (s != HOM_OK) return s;
  if (!dst_on_device) CK(cudaMemcpyAsync(dst, d, nbytes, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return HOM_OK;
}

HOM_API hom_status hom_equilibrium_error(hom_t c, int32_t nrhs, const double* eps, const double* E, double* out) {
  if (!c || !out) return HOM_ERR_ARG;
  if (c->n_rve > 1) return fail(c, HOM_ERR_ARG, "the equilibrium diagnostic takes a handle with one RVE");
  if (c->opt.green_operator != HOM_GREEN_SPECTRAL)
    return fail(c, HOM_ERR_ARG, "the equilibrium diagnostic measures the spectral divergence only");
  const OrderData& o = c->ord[0];
  if (!eps) {
    if (!o.eps || o.eff.empty()) return fail(c, HOM_ERR_ORDER, "order 0 has not been solved");
    if (nrhs != o.nloads) return fail(c, HOM_ERR_ARG, "nrhs must equal the %d solved order-0 loads", o.nloads);
  } else if (nrhs < 1 || nrhs > 64) {
    return fail(c, HOM_ERR_ARG, "1 to 64 fields per call");
  }
  CKS(ensure_cap(c, nrhs));
  std::vector<double> ek(6 * nrhs, 0.0);
  if (!eps) ek = o.loadsK;
  else if (E) for (int i = 0; i < nrhs; ++i) mandel_to_kelvin6(E + 6 * i, &ek[6 * i]);
  CK(cudaMemcpyAsync(c->d_E, ek.data(), sizeof(double) * 6 * nrhs, cudaMemcpyHostToDevice, c->stream));
  const double* epsK = reinterpret_cast<const double*>(o.eps);
  if (eps) {
    void* vin;
    CKS(work(c, 0, std::max(tbytes<double>(c, nrhs, 6), c->work_bytes[0]), &vin));
    CK(launch_mandel_to_kelvin<double>(eps, (double*)vin, c->g.M, nrhs, c->stream));
    epsK = (const double*)vin;
  }
  const int nblk = equilibrium_blocks(c->g);
  void* vred;
  CKS(work(c, 1, std::max(sizeof(double) * (size_t)nrhs * (2 * nblk + 7), c->work_bytes[1]), &vred));
  double* d_part = (double*)vred;
  double* d_s0 = d_part + (size_t)nrhs * 2 * nblk;
  double* d_out = d_s0 + (size_t)nrhs * 6;
  CKS(c->fp32 ? equilibrium_t<df64>(c, nrhs, epsK, d_part, d_s0, d_out)
              : equilibrium_t<double>(c, nrhs, epsK, d_part, d_s0, d_out));
  CK(cudaMemcpyAsync(out, d_out, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return HOM_OK;
}

HOM_API hom_status hom_ls_apply(hom_t c, int32_t nrhs, const double* eps_in, const double* E, double* eps_out) {
  if (!c || !eps_out || nrhs < 1 || nrhs > 64) return HOM_ERR_ARG;
  CKS(ensure_cap(c, nrhs));
  std::vector<double> ek(6 * nrhs, 0.0);
  if (E) for (int i = 0; i < nrhs; ++i) mandel_to_kelvin6(E + 6 * i, &ek[6 * i]);
  CK(cudaMemcpyAsync(c->d_E, ek.data(), sizeof(double) * 6 * nrhs, cudaMemcpyHostToDevice, c->stream));
  void *vin = nullptr, *vout;
  const size_t fb = field_bytes(c, nrhs, 6);
  CKS(work(c, 1, fb, &vout));
  if (eps_in) CKS(work(c, 0, fb, &vin));
  if (c->fp32) {
    if (eps_in) CK(launch_mandel_to_kelvin<float>(eps_in, (float*)vin, c->g.M, nrhs, c->stream));
    auto fa = fwd_args<float, float>(c, FWD_TAU, 6, 6);
    fa.in = (const float*)vin;
    fa.E = c->d_E;
    auto za = z_args<float>(c, Z_GAMMA, 6, 6);
    auto ia = inv_args<float, float>(c, INV_STORE, FIN_NONE, 6, 6, 6);
    ia.out = (float*)vout;
    CKS((ls_pass<float, float>(c, nrhs, fa, za, ia)));
    CK(launch_kelvin_to_mandel<float>((const float*)vout, eps_out, c->g.M, nrhs, c->stream));
  } else {
    if (eps_in) CK(launch_mandel_to_kelvin<double>(eps_in, (double*)vin, c->g.M, nrhs, c->stream));
    auto fa = fwd_args<double, double>(c, FWD_TAU, 6, 6);
    fa.in = (const double*)vin;
    fa.E = c->d_E;
    auto za = z_args<double>(c, Z_GAMMA, 6, 6);
    auto ia = inv_args<double, double>(c, INV_STORE, FIN_NONE, 6, 6, 6);
    ia.out = (double*)vout;
    CKS((ls_pass<double, double>(c, nrhs, fa, za, ia)));
    CK(launch_kelvin_to_mandel<double>((const double*)vout, eps_out, c->g.M, nrhs, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return check_kernel_flags(c);
}

}  // extern "C"

namespace {
template <typename T>
hom_status fft_fwd_impl(hom_ctx* c, int nf, const double* f, double* fhat) {
  void *vin, *vs;
  CKS(work(c, 0, sizeof(T) * (size_t)nf * c->g.M, &vin));
  const size_t sb = sizeof(cx<T>) * (size_t)nf * c->g.n3 * c->g.plane_c;
  CKS(work(c, 2, sb, &vs));
  CK((launch_convert<double, T>(f, (T*)vin, (long long)nf * c->g.M, c->stream)));
  // the nf fields are the components of one load for the x-y transforms (fused plane kernel or
  // split x and y passes), and nf one-component loads for the z transforms
  auto fa = fwd_args<T, T>(c, FWD_COPY, nf, nf);
  fa.in = (const T*)vin;
  fa.S = (cx<T>*)vs;
  CKS((fwd_xy<T, T>(c, fa, 1)));
  auto za = z_args<T>(c, Z_FWD, 1, 1);
  zpass_tiling<T>(za, -1);
  za.S = (cx<T>*)vs;
  CK(launch_zpass<T>(za, nf, c->stream));
  CK(launch_spec_to_std<T>((const cx<T>*)vs, fhat, c->g, 1, nf, 0, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return check_kernel_flags(c);   // the split y pass may run in its TMA form
}
template <typename T>
hom_status fft_inv_impl(hom_ctx* c, int nf, const double* fhat, double* f) {
  void *vout, *vs;
  CKS(work(c, 0, sizeof(T) * (size_t)nf * c->g.M, &vout));
  const size_t sb = sizeof(cx<T>) * (size_t)nf * c->g.n3 * c->g.plane_c;
  CKS(work(c, 2, sb, &vs));
  CK(launch_spec_from_std<T>(fhat, (cx<T>*)vs, c->g, 1, nf, 0, c->stream));
  auto za = z_args<T>(c, Z_INV, 1, 1);
  zpass_tiling<T>(za, -1);
  za.S = (cx<T>*)vs;
  CK(launch_zpass<T>(za, nf, c->stream));
  auto ia = inv_args<T, T>(c, INV_STORE, FIN_NONE, nf, nf, nf);
  ia.S = (const cx<T>*)vs;
  ia.out = (T*)vout;
  CKS((inv_xy<T, T>(c, ia, 1)));
  CK((launch_convert<T, double>((const T*)vout, f, (long long)nf * c->g.M, c->stream)));
  CK(cudaStreamSynchronize(c->stream));
  return check_kernel_flags(c);   // the split y pass may run in its TMA form
}
template <typename T>
hom_status green_impl(hom_ctx* c, int nrhs, const double* th, double* eh) {
  void* vs;
  const size_t sb = sizeof(cx<T>) * (size_t)nrhs * 6 * c->g.n3 * c->g.plane_c;
  CKS(work(c, 2, sb, &vs));
  CK(launch_spec_from_std<T>(th, (cx<T>*)vs, c->g, nrhs, 6, 1, c->stream));
  auto za = z_args<T>(c, Z_GREEN, 6, 6);
  za.S = (cx<T>*)vs;
  za.scale = 1.0;
  CK(launch_zpass<T>(za, nrhs, c->stream));
  CK(launch_spec_to_std<T>((const cx<T>*)vs, eh, c->g, nrhs, 6, 2, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return HOM_OK;
}
}  // namespace

extern "C" {

HOM_API hom_status hom_fft_forward(hom_t c, int32_t nfield, const double* f, double* fhat) {
  if (!c || !f || !fhat || nfield < 1 || nfield > 64) return HOM_ERR_ARG;
  return c->fp32 ? fft_fwd_impl<float>(c, nfield, f, fhat) : fft_fwd_impl<double>(c, nfield, f, fhat);
}
HOM_API hom_status hom_fft_inverse(hom_t c, int32_t nfield, const double* fhat, double* f) {
  if (!c || !f || !fhat || nfield < 1 || nfield > 64) return HOM_ERR_ARG;
  return c->fp32 ? fft_inv_impl<float>(c, nfield, fhat, f) : fft_inv_impl<double>(c, nfield, fhat, f);
}
HOM_API hom_status hom_green_apply(hom_t c, int32_t nrhs, const double* tau_hat, double* eta_hat) {
  if (!c || !tau_hat || !eta_hat || nrhs < 1 || nrhs > 64) return HOM_ERR_ARG;
  return c->fp32 ? green_impl<float>(c, nrhs, tau_hat, eta_hat) : green_impl<double>(c, nrhs, tau_hat, eta_hat);
}

}  // extern "C"
