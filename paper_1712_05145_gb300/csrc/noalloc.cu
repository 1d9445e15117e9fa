// hom_ls_apply_noalloc: one Lippmann-Schwinger step (the same kernels as hom_ls_apply, FP64)
// for callers that cannot allocate device memory -- code running where cudaMalloc is not
// allowed or not wanted, such as inside another library's memory pool, a real-time loop that
// must not allocate, or a process whose allocator is owned by someone else.
//
// Instead of a handle's buffers, this entry point keeps its scratch (spectrum of one load,
// twiddle tables, per-phase eigenvalues, macroscopic strains) in one file-scope device array
// of kNoallocScratchBytes.  Every GPU that loads the library holds that array until the
// process exits.  The caller passes the phase array, the input field and the output field.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "aux.h"
#include "hom.h"
#include "internal.h"

namespace hom {
namespace {

constexpr size_t kNoallocScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
thread_local std::string g_noalloc_err;

hom_status noalloc_fail(hom_status s, const std::string& msg) {
  g_noalloc_err = msg;
  return s;
}

// true for memory the GPU addresses directly (device or managed); clears the error a host
// pointer leaves behind
bool device_pointer(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array for the current device.  The first call on a device
// resolves it with cudaGetSymbolAddress; the array's host-side name is not a device address.
hom_status scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(HOM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(HOM_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return noalloc_fail(HOM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = reinterpret_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return HOM_OK;
}

}  // namespace

// Bytes of the scratch array the allocation-free step needs for a grid and load count.
size_t noalloc_scratch_need(int n1, int n2, int n3, int nrhs) {
  const size_t plane_c = (size_t)n2 * (n1 / 2 + 1);
  size_t b = align256((size_t)6 * n3 * plane_c * sizeof(cx<double>));        // spectrum, one load
  b += align256((size_t)(n1 / 2 + n1 + n2 + n3) * sizeof(cx<double>));       // twiddles
  b += align256((size_t)4 * 256 * sizeof(double));                           // per-phase eigenvalues
  b += align256((size_t)6 * nrhs * sizeof(double));                          // macroscopic strains
  return b;
}

}  // namespace hom

using namespace hom;

extern "C" {

HOM_API hom_status hom_ls_apply_noalloc(const int32_t grid[3], const uint8_t* phase, int32_t n_phase,
                                        const double* lame, double lambda0, double mu0, int32_t nrhs,
                                        const double* eps_in, const double* E, double* eps_out,
                                        void* cuda_stream) {
  if (!grid || !phase || !lame || !eps_out || nrhs < 1 || nrhs > 64 || n_phase < 1 || n_phase > 256)
    return noalloc_fail(HOM_ERR_ARG, "hom_ls_apply_noalloc: null pointer or count out of range");
  if (!(mu0 != 0.0) || !(lambda0 + 2.0 * mu0 != 0.0))
    return noalloc_fail(HOM_ERR_ARG, "hom_ls_apply_noalloc: degenerate reference medium");
  const int n1 = grid[0], n2 = grid[1], n3 = grid[2];
  if (n1 < 4 || (n1 & 1) || !fft_length_supported(n1 / 2) || !fft_length_supported(n2) ||
      !z_length_supported(n3) || (long long)(n1 / 2) * n2 > 8192)
    return noalloc_fail(HOM_ERR_SIZE, "hom_ls_apply_noalloc: grid axis not supported");
  const size_t need = noalloc_scratch_need(n1, n2, n3, nrhs);
  if (need > kNoallocScratchBytes)
    return noalloc_fail(HOM_ERR_SIZE, "hom_ls_apply_noalloc: grid needs " + std::to_string(need) +
                                          " bytes of scratch, more than the fixed " +
                                          std::to_string(kNoallocScratchBytes));
  // every array the kernels touch must be device memory: a host pointer would fault on the GPU
  if (!device_pointer(phase))
    return noalloc_fail(HOM_ERR_ARG, "hom_ls_apply_noalloc: phase must be a device pointer");
  if (!device_pointer(eps_out) || (eps_in != nullptr && !device_pointer(eps_in)))
    return noalloc_fail(HOM_ERR_ARG, "hom_ls_apply_noalloc: eps_in and eps_out must be device pointers");
  const size_t field_bytes = sizeof(double) * 6 * (size_t)n1 * n2 * n3 * nrhs;
  const bool in_place = (eps_in == eps_out);
  if (eps_in != nullptr && !in_place) {
    const char* a = reinterpret_cast<const char*>(eps_in);
    const char* b = reinterpret_cast<const char*>(eps_out);
    if (a < b + field_bytes && b < a + field_bytes)
      return noalloc_fail(HOM_ERR_ARG, "hom_ls_apply_noalloc: eps_in and eps_out overlap without being equal");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  unsigned char* base = nullptr;
  hom_status st = scratch_address(&base);
  if (st != HOM_OK) return st;

  Geo g{};
  g.n1 = n1;
  g.n2 = n2;
  g.n3 = n3;
  g.h = n1 / 2;
  g.P = (g.h & 1) ? g.h : g.h + 1;
  g.M = (long long)n1 * n2 * n3;
  g.plane_c = (long long)n2 * (g.h + 1);
  geo_finish(g);
  const int nmax = n1 > n2 ? (n1 > n3 ? n1 : n3) : (n2 > n3 ? n2 : n3);
  g.xs1 = 2.0 * M_PI * nmax / n1;
  g.xs2 = 2.0 * M_PI * nmax / n2;
  g.xs3 = 2.0 * M_PI * nmax / n3;

  // carve the scratch: spectrum | twiddles (h, n1, n2, n3) | eigenvalues | loads
  size_t off = 0;
  cx<double>* S = reinterpret_cast<cx<double>*>(base + off);
  off += align256((size_t)6 * n3 * g.plane_c * sizeof(cx<double>));
  cx<double>* tw = reinterpret_cast<cx<double>*>(base + off);
  off += align256((size_t)(g.h + n1 + n2 + n3) * sizeof(cx<double>));
  double* mat = reinterpret_cast<double*>(base + off);
  off += align256((size_t)4 * 256 * sizeof(double));
  double* dE = reinterpret_cast<double*>(base + off);

  // host-side tables (host memory only), copied into the scratch on the caller's stream
  std::vector<cx<double>> htw;
  htw.reserve(g.h + n1 + n2 + n3);
  const int lens[4] = {g.h, n1, n2, n3};
  long long tw_off[4];
  for (int i = 0; i < 4; ++i) {
    tw_off[i] = (long long)htw.size();
    for (int t = 0; t < lens[i]; ++t) {
      const double a = -2.0 * M_PI * (double)t / (double)lens[i];
      cx<double> w;
      w.re = std::cos(a);
      w.im = std::sin(a);
      htw.push_back(w);
    }
  }
  std::vector<double> hmat(4 * 256, 0.0);
  for (int i = 0; i < n_phase; ++i) {
    const double l = lame[2 * i], m = lame[2 * i + 1];
    hmat[4 * i + 0] = 3.0 * (l - lambda0) + 2.0 * (m - mu0);
    hmat[4 * i + 1] = 2.0 * (m - mu0);
    hmat[4 * i + 2] = 3.0 * l + 2.0 * m;
    hmat[4 * i + 3] = 2.0 * m;
  }
  const double r3 = 0.57735026918962576451, r2 = 0.70710678118654752440, r6 = 0.40824829046386301637;
  std::vector<double> hE(6 * nrhs, 0.0);
  if (E) {
    for (int i = 0; i < nrhs; ++i) {
      const double* m = E + 6 * i;
      double* k = &hE[6 * i];
      k[0] = (m[0] + m[1] + m[2]) * r3;
      k[1] = (m[0] - m[1]) * r2;
      k[2] = (m[0] + m[1] - 2.0 * m[2]) * r6;
      k[3] = m[3];
      k[4] = m[4];
      k[5] = m[5];
    }
  }
#define NA_CK(call)                                                                           \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return noalloc_fail(HOM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
  } while (0)
  NA_CK(cudaMemcpyAsync(tw, htw.data(), sizeof(cx<double>) * htw.size(), cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(mat, hmat.data(), sizeof(double) * hmat.size(), cudaMemcpyHostToDevice, s));
  NA_CK(cudaMemcpyAsync(dE, hE.data(), sizeof(double) * hE.size(), cudaMemcpyHostToDevice, s));

  // Kelvin components of the input into the output buffer; the step then runs in place there
  if (in_place) {
    NA_CK(launch_mandel_to_kelvin_inplace(eps_out, g.M, nrhs, s));
  } else if (eps_in) {
    NA_CK(launch_mandel_to_kelvin<double>(eps_in, eps_out, g.M, nrhs, s));
  } else {
    NA_CK(cudaMemsetAsync(eps_out, 0, field_bytes, s));
  }

  FwdArgs<double, double> fa{};
  fa.g = g;
  fa.mode = FWD_TAU;
  fa.ncomp = 6;
  fa.in_ncomp = 6;
  fa.phase = phase;
  fa.mat = mat;
  // the kernels stage a table of n_phase rows in shared memory and index it by the raw phase
  // byte, which this entry point does not scan; the table holds all 256 rows (zero past the
  // caller's n_phase), so every byte value stays inside it
  fa.n_phase = 256;
  fa.in = eps_out;
  fa.E = dE;
  fa.S = S;
  fa.tw_h = tw + tw_off[0];
  fa.tw_n1 = tw + tw_off[1];
  fa.tw_n2 = tw + tw_off[2];
  ZArgs<double> za{};
  za.g = g;
  za.mode = Z_GAMMA;
  za.ncomp_in = 6;
  za.ncomp_out = 6;
  za.S = S;
  za.lam0 = lambda0;
  za.mu0 = mu0;
  za.scale = 1.0 / (double)g.M;
  za.tw_n3 = tw + tw_off[3];
  zpass_tiling<double>(za);
  InvArgs<double, double> ia{};
  ia.g = g;
  ia.mode = INV_STORE;
  ia.fin = FIN_NONE;
  ia.ncomp = 6;
  ia.out_ncomp = 6;
  ia.s_ncomp = 6;
  ia.S = S;
  ia.c0h = 3.0 * lambda0 + 2.0 * mu0;
  ia.c0d = 2.0 * mu0;
  ia.out_scale = 1.0;
  ia.out = eps_out;
  ia.tw_h = fa.tw_h;
  ia.tw_n1 = fa.tw_n1;
  ia.tw_n2 = fa.tw_n2;
  // one load at a time through the single-load spectrum; the forward pass has consumed a
  // load's input before the inverse pass overwrites it
  for (int r = 0; r < nrhs; ++r) {
    fa.rhs0 = za.rhs0 = ia.rhs0 = r;
    NA_CK((launch_plane_fwd<double, double>(fa, 1, s)));
    NA_CK(launch_zpass<double>(za, 1, s));
    NA_CK((launch_plane_inv<double, double>(ia, 1, s)));
  }
  NA_CK(launch_kelvin_to_mandel_inplace(eps_out, g.M, nrhs, s));
#undef NA_CK
  g_noalloc_err.clear();
  return HOM_OK;
}

HOM_API const char* hom_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

}  // extern "C"
