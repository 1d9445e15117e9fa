/*
 * hom.h -- C ABI of libhom, an sm_103a (GB300) implementation of FFT-based
 * homogenization with higher-order terms after Dietrich, Merkert and Simeon,
 * "Derivation of higher-order terms in FFT-based numerical homogenization"
 * (arXiv:1712.05145).
 *
 * The library solves, on one GPU, the periodic Lippmann-Schwinger equation of
 * quasi-static linear elasticity on a voxel representative volume element
 * (Sec. 2: Hooke's law, balance of momentum, polarization problem, Lippmann-
 * Schwinger equation with the closed-form isotropic Green operator Gamma0_hat)
 * with the Basic Scheme or its CG form (Algorithm 1, Eq. cg_form), and the
 * generalized problems of order alpha of Sec. 3 (Definition of the generalized
 * homogenization problem, theta_alpha closed form, modified initialization).
 *
 * Conventions shared by every entry point
 *  - Grid (N1, N2, N3), N1 the fastest axis.  Cubic voxels of edge h = 1/max(N);
 *    cubic grids are exactly the unit torus [-1/2, 1/2)^3 of Sec. 2.
 *  - Scalar voxel arrays are [N3][N2][N1]; fields are [field][component][N3][N2][N1].
 *  - Symmetric tensors are Mandel 6-vectors (11, 22, 33, sqrt2*23, sqrt2*13, sqrt2*12);
 *    vectors are 3 components (x1, x2, x3).  6x6 and 6xK matrices are row-major.
 *  - Orders are counted from 0: order 0 is the classical cell problem (the paper's
 *    alpha = 1), order o >= 1 is the paper's alpha = o + 1 (orders up to 6).
 *  - Unit loads: order 0, load A = 0..5 is the Mandel unit strain E^A; order 1,
 *    load 3*A + k is E(Y) = E^A Y_k (18 loads); order 2, load 6*A + P is
 *    E(Y) = E^A Y_k Y_l / (1 + delta_kl) with (k, l) the P-th Mandel pair (36 loads);
 *    order o >= 3, E(Y) = E^A Y^K / K! for the multisets K of o directions in
 *    lexicographic order (6 (o+1)(o+2)/2 loads: 60, 90, 126, 168 for o = 3 to 6).
 *  - Spectral operators use the discrete wave vector xi_i = 2 pi k_i / (N_i h) with the
 *    Nyquist component (k_i = N_i/2 on even axes) taken as 0.
 *  - Errors are returned as hom_status; no C++ exception crosses the ABI.  After an
 *    error, hom_last_error(h) describes it.  A handle is used by one host thread at a
 *    time; all its GPU work runs on the stream given in hom_options (default: a stream
 *    the handle creates).
 *  - Device pointers must be allocated on the device that was current at hom_create.
 */
#ifndef HOM_H
#define HOM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HOM_API __attribute__((visibility("default")))

typedef struct hom_ctx* hom_t;

typedef enum {
  HOM_OK = 0,
  HOM_ERR_ARG = 1,           /* invalid argument (null pointer, bad index, bad option) */
  HOM_ERR_SIZE = 2,          /* grid axis not supported (see hom_create) */
  HOM_ERR_NOMEM = 3,         /* device allocation failed */
  HOM_ERR_NOT_CONVERGED = 4, /* iteration cap reached before the tolerance */
  HOM_ERR_ORDER = 5,         /* lower-order correctors missing */
  HOM_ERR_NUMERIC = 6,       /* NaN or Inf met in a reduction */
  HOM_ERR_TIMEOUT = 7,       /* a bounded device wait expired */
  HOM_ERR_CUDA = 8           /* CUDA runtime error (text in hom_last_error) */
} hom_status;

enum { HOM_FP64 = 0, HOM_FP32_REFINE = 1 };
enum { HOM_BASIC = 0, HOM_CG = 1, HOM_BICGSTAB = 2, HOM_POLARIZATION = 3 };
enum { HOM_FIELD_STRAIN = 0, HOM_FIELD_DISPLACEMENT = 1, HOM_FIELD_STRESS = 2 };
enum { HOM_GREEN_SPECTRAL = 0, HOM_GREEN_ROTATED = 1 };

typedef struct {
  int32_t precision;       /* HOM_FP64: FP64 fields and FFTs.  HOM_FP32_REFINE: FP32 fields and
                              FFTs, FP64 reductions, FP64 residual-correction sweeps. */
  int32_t scheme;          /* HOM_BASIC (fixed point), HOM_CG (CG on A eps = b, C0 product),
                              HOM_BICGSTAB (BiCGSTAB on A eps = b, L2 products; the solver the
                              paper ran for its CG-version, Sec. 4; iterations count full steps,
                              each with two operator applications) or HOM_POLARIZATION (the
                              polarization scheme cited in Sec. 1: the fixed point
                              x = b + (I - 2 Gamma0 * C0) W x, W = (C - C0)(C + C0)^-1,
                              eps = (I - W) x, one LS pass per iteration; it contracts by
                              max |(c - c0)/(c + c0)| over the phases' Kelvin moduli c, so C0
                              near the geometric mean of the phases converges fastest.  Needs
                              mu0 > 0, 3 lambda0 + 2 mu0 > 0 and non-negative phase moduli) */
  int32_t max_iter;        /* iteration cap per load (inner iterations in FP32_REFINE) */
  int32_t check_every;     /* iterations between host convergence checks (>= 1) */
  int32_t max_refine;      /* FP32_REFINE: cap on FP64 residual-correction sweeps */
  int32_t rhs_chunk;       /* loads whose spectra are transformed per launch; 0 = choose so
                              that the spectrum scratch fits spectrum_budget_bytes */
  int64_t spectrum_budget_bytes; /* target size of the spectrum scratch (0 = 1 GiB).  More loads
                              per launch give the latency-bound kernels more CTAs; at 128^3 FP32
                              the default transforms all 6 unit loads per launch */
  void* cuda_stream;       /* cudaStream_t to run on; NULL = the handle's own stream */
  int32_t pass_mode;       /* x-y transforms: 0 = fused plane kernels when a plane fits one CTA,
                              else (FP32 transforms) cluster plane passes, whose CTAs transpose
                              the plane through distributed shared memory, or split x and y
                              passes; 1 = always fused (fails if a plane does not fit); 2 = always
                              split; 3 = always cluster for FP32 transforms (fails if no cluster
                              shape fits), split for the FP64-accurate passes */
  int32_t autotune;        /* 1: before the first solve, time one operator application per
                              candidate launch shape (loads per launch, z stage and tile width,
                              cluster or split plane passes, y tile width and copy form) on this grid and keep
                              the fastest; 0 (default): fixed rules.  When the environment
                              variable HOM_TUNE_CACHE names a file, a shape tuned earlier for the
                              same grid and options is read from it instead of timing again, and a
                              newly tuned one is appended to it. */
  int32_t polarization_variant; /* HOM_POLARIZATION: 0 = x <- T(x) (Eyre-Milton, Monchiet-Bonnet);
                              1 = x <- (x + T(x)) / 2 (the averaged, augmented-Lagrangian form,
                              which also converges where a phase modulus is 0) */
  int32_t z_mode;          /* z stage of the LS step: 0 = cluster z pass (six CTAs, one per Kelvin
                              component, meeting in distributed shared memory for the Green
                              contraction) where its tile fits, else the single-CTA z pass; for FP32
                              transforms its tiles move by TMA tensor loads and stores where that
                              fits (N3 >= 16, an even number of spectrum columns per plane); the
                              autotuner may pick any of these forms;
                              1 = always the single-CTA z pass (three passes on deep grids);
                              2 = the cluster z pass in its TMA form where that fits, else as 0;
                              3 = the cluster z pass with per-element asynchronous copies where its
                              tile fits, else as 0.  The two copy forms give identical results for
                              the same tile width. */
  int32_t green_operator;  /* HOM_GREEN_SPECTRAL (0): Gamma0_hat of Sec. 2 at the discrete wave
                              vector (Nyquist components 0).  HOM_GREEN_ROTATED (1): the Green
                              operator of the rotated finite-difference discretisation (corner
                              displacements, voxel-centre strains, derivatives averaged over the four
                              voxel edges along an axis; one of the discrete operators of the FFT
                              schemes Sec. 1 cites): Gamma0_hat evaluated at q_j = sin(xi_j h/2)
                              prod_{l != j} cos(xi_l h/2), zero where q = 0.  Order 0 only; the
                              equilibrium diagnostic stays spectral and is not offered with it. */
  int32_t n_rve;           /* RVE slots of one grid held by the handle (1..10, 0 = 1).  With more than
                              one, every LS launch carries the loads of all slots: load r belongs to
                              slot r / 6, and each slot has its own phase array, per-phase table and
                              reference medium (hom_set_rve).  Such a handle solves order 0 for the
                              6 unit loads of each slot (hom_solve with loads = NULL, n_loads =
                              6 x slots, 0 = all) with CG, BiCGSTAB or the Basic Scheme; hom_effective
                              returns the 6 x (6 x slots) mean stresses, one 6 x 6 block per slot. */
  int32_t y_mode;          /* tile copies of the split y pass (FP32 transforms): 0 = TMA tensor loads
                              and stores where they fit (an even N1/2 and an even number of spectrum
                              columns per plane), else per-element asynchronous copies; the
                              autotuner may pick either; 1 = TMA where it fits, kept by the
                              autotuner; 2 = per-element copies.  Results are identical. */
  int32_t reserved[1];
} hom_options;

typedef struct {
  int32_t iterations;        /* iterations performed (inner iterations summed over sweeps) */
  int32_t refinements;       /* FP64 residual-correction sweeps performed */
  int32_t status;            /* hom_status of this load */
  int32_t reserved;
  double rel_residual;       /* last relative residual tracked by the iteration */
  double rel_residual_fp64;  /* ||b - A eps||_L2 / ||b||_L2 of Eq. cg_form recomputed at the end at FP64
                                accuracy: native FP64 in HOM_FP64, double-float arithmetic (a pair of
                                floats, about 48 significant bits) in HOM_FP32_REFINE */
} hom_solve_info;

/* Fills *opt with defaults: HOM_FP32_REFINE, HOM_CG, max_iter 2000, check_every 8,
 * max_refine 6, rhs_chunk 0, spectrum_budget_bytes 1 GiB, own stream. */
HOM_API void hom_default_options(hom_options* opt);

/* Creates a handle for one voxel RVE (Sec. 2: C(x) piecewise isotropic, reference C0).
 *  grid[3]     N1, N2, N3.  N1 even with N1/2, N2 and N3 in {2,3,4,6,8,12,16,24,32,48,64,96,
 *              128,192,256,384,512}; N3 may also be 1, a two-dimensional cell (every field is
 *              constant along y3 and xi3 = 0: plane strain, or plane stress with the plane-stress
 *              Lame parameter 2 lambda mu / (lambda + 2 mu) in place of lambda).  Planes with
 *              (N1/2) * N2 <= 8192 can use the fused plane kernels; larger ones use split x and y
 *              passes or cluster plane passes (hom_options.pass_mode).
 *  phase       uint8 [N3][N2][N1], host or device pointer (auto-detected); copied.
 *  n_phase     1..256; every phase index must be < n_phase.
 *  lame        double [n_phase][2] host array of (lambda, mu) per phase; copied.  Phases are
 *              isotropic, like every material of the paper (Sec. 4): the boundary takes no full
 *              6 x 6 stiffness per phase, and the kernels rely on C being diagonal in the Kelvin
 *              basis (3K, 2mu).
 *  lambda0,mu0 Lame parameters of the reference medium C0 (mu0 != 0, lambda0+2mu0 != 0).
 *  opt         options (NULL = defaults); the stream pointer is borrowed, not owned.
 *  out         receives the handle (owned by the caller; release with hom_destroy).
 * Allocates device memory for the RVE and the scratch; errors leave *out unset. */
HOM_API hom_status hom_create(const int32_t grid[3], const uint8_t* phase, int32_t n_phase,
                              const double* lame, double lambda0, double mu0,
                              const hom_options* opt, hom_t* out);

/* Solves problem `order` (0 to 6: the paper's alpha = order + 1) for its loads to relative
 * residual tol:
 * ||b - A eps||_L2 / ||b||_L2 < tol with A = Id + Gamma0 * (C - C0) (Eq. cg_form); for the
 * Basic Scheme this is the paper's Cauchy quantity ||eps_{n+1} - eps_n|| / ||eps_0||.
 *  order 0: n_loads macroscopic strains, loads = double [n_loads][6] Mandel host array, or
 *           loads = NULL for the 6 unit loads (n_loads ignored).  n_loads <= 64.
 *  order 1: loads = NULL for the 18 unit loads grad E = E^A (x) e_k (load 3A+k, A the Mandel
 *           component, k the direction), or loads = double [n_loads][18] host array of
 *           coefficients of those unit loads (n_loads <= 64), each solved as one system.
 *           Every unit load used needs the unit strain e_A among the converged order-0 loads.
 *  order o >= 2: requires order o - 1 solved for its unit loads; loads must be NULL.  The unit
 *           loads are E(Y) = E^A Y^K / K! for the multisets K of o directions: 6 x (o+1)(o+2)/2
 *           loads (36, 60, 90, 126, 168 for o = 2 to 6), load A * nK + (index of K), K ordered as the
 *           Mandel pairs (11, 22, 33, 23, 13, 12) for o = 2 and lexicographically (sorted
 *           tuples, 111 < 112 < ... < 333) for o >= 3.
 *  info     host array of one hom_solve_info per load (nullable); caller-owned.
 * The correctors stay on the device, owned by the handle, until hom_destroy or the next
 * solve of the same order.  Returns HOM_ERR_NOT_CONVERGED if any load missed tol. */
HOM_API hom_status hom_solve(hom_t h, int32_t order, int32_t n_loads, const double* loads,
                             double tol, hom_solve_info* info);

/* Effective tensors as FP64 voxel means of the stress of each load (host array out):
 *  order 0: 6 x n_loads, column A = <C : (E^A + eps^A)> (the 6x6 C_eff for unit loads);
 *  order 1: 6 x n_loads (18 for the unit loads), column = <C : eps_2 + p_2> (mean order-2
 *           stress of the paper's alpha = 2);
 *  order o >= 2: 6 x (its loads), column = <C : eps_{o+1} + p_{o+1}>. */
HOM_API hom_status hom_effective(hom_t h, int32_t order, double* out);

/* Replaces the microstructure of RVE slot `slot` (0 .. n_rve - 1) of a handle without any device
 * allocation: phase (host or device, copied; every value < n_phase), n_phase, lame and the
 * reference medium as hom_create.  The grid and options stay.  Solved orders of the handle are
 * discarded.  Waits for the handle's stream.  This lets a server keep handles of the grids it
 * sees resident and refill them per request (the paper has no counterpart). */
HOM_API hom_status hom_set_rve(hom_t h, int32_t slot, const uint8_t* phase, int32_t n_phase, const double* lame,
                               double lambda0, double mu0);

/* Copies one corrector field of a solved order to dst (double):
 *  HOM_FIELD_STRAIN       6 x [N3][N2][N1] Mandel strain fluctuation eps;
 *  HOM_FIELD_DISPLACEMENT 3 x [N3][N2][N1] zero-mean displacement u with e_y(u) = eps;
 *  HOM_FIELD_STRESS       6 x [N3][N2][N1] Mandel stress (C : (E + eps) for order 0,
 *                         C : eps + p for orders >= 1).
 * dst is a device pointer if dst_on_device != 0, else a host pointer. */
HOM_API hom_status hom_get_field(hom_t h, int32_t order, int32_t load, int32_t kind, double* dst,
                                 int32_t dst_on_device);

/* Equilibrium error of stress fields sigma = C : (E + eps) (Sec. 2, Eq. Hookes_law): how far
 * sigma is from the balance of momentum div sigma = 0 (Eq. eq_of_motion), in the spectral form
 * of Moulinec and Suquet (the paper's reference for the Basic Scheme),
 *   out[l] = sqrt(< |div sigma|^2 >) / |<sigma>|,   (div sigma)_hat(xi) = i xi . sigma_hat(xi),
 * with the discrete wave vectors of the Green operator (Nyquist components 0), <.> the voxel
 * mean and |.| the Frobenius norm.  Where the mean vanishes up to rounding (|<sigma>| <=
 * 1e-12 sqrt(<|sigma|^2>), e.g. a zero load), out[l] = sqrt(< |div sigma|^2 >).  A
 * solution of the discrete Lippmann-Schwinger equation has out = 0 up to its residual.
 *   eps != NULL: device double [nrhs][6][N3][N2][N1] Mandel strain fluctuations (nrhs <= 64),
 *                E host double [nrhs][6] Mandel (NULL = zero);
 *   eps == NULL: the handle's order-0 solutions and their loads (nrhs = their count, E unused;
 *                HOM_ERR_ORDER if order 0 has not been solved).
 * out: host double [nrhs].  Computed at FP64 accuracy (double, or double-float transforms in
 * HOM_FP32_REFINE).  Not part of a solve; costs one forward transform per field. */
HOM_API hom_status hom_equilibrium_error(hom_t h, int32_t nrhs, const double* eps, const double* E,
                                         double* out);

/* One Lippmann-Schwinger step on caller device buffers (Sec. 2, Algorithm 1 loop body):
 *   eps_out = -Gamma0 * [(C - C0) : (eps_in + E)]
 * eps_in, eps_out: device double [nrhs][6][N3][N2][N1] Mandel (eps_in NULL = zero field);
 * E: host double [nrhs][6] Mandel (NULL = zero).  Computed in the handle's precision. */
HOM_API hom_status hom_ls_apply(hom_t h, int32_t nrhs, const double* eps_in, const double* E,
                                double* eps_out);

/* Forward 3-D real-to-complex DFT, X[k] = sum_n x[n] exp(-2 pi i k.n/N) (unnormalised):
 * f: device double [nfield][N3][N2][N1]; fhat: device double complex (interleaved re, im)
 * [nfield][N3][N2][N1/2+1]; 1 <= nfield <= 64.  Computed in the handle's precision. */
HOM_API hom_status hom_fft_forward(hom_t h, int32_t nfield, const double* f, double* fhat);

/* Inverse of hom_fft_forward without the 1/M factor: f[n] = sum_k X[k] exp(+2 pi i k.n/N)
 * over the Hermitian-completed spectrum.  fhat is not modified. */
HOM_API hom_status hom_fft_inverse(hom_t h, int32_t nfield, const double* fhat, double* f);

/* Green contraction at every frequency of the half spectrum (Sec. 2, Gamma0_hat formula):
 *   eta_hat(xi) = -Gamma0_hat(xi) : tau_hat(xi),  eta_hat = 0 where xi = 0,
 * tau_hat, eta_hat: device double complex [nrhs][6][N3][N2][N1/2+1] Mandel. */
HOM_API hom_status hom_green_apply(hom_t h, int32_t nrhs, const double* tau_hat, double* eta_hat);

/* Per-kernel accounting for performance measurement (off by default).
 * Kernel kinds of the Lippmann-Schwinger step, with FFTs in FP32 (0..2) or at FP64 accuracy (3..5:
 * double in HOM_FP64, double-float in the FP64-accurate passes of HOM_FP32_REFINE): */
enum {
  HOM_KERNEL_PLANE_FWD = 0, HOM_KERNEL_ZPASS = 1, HOM_KERNEL_PLANE_INV = 2,
  HOM_KERNEL_PLANE_FWD_F64 = 3, HOM_KERNEL_ZPASS_F64 = 4, HOM_KERNEL_PLANE_INV_F64 = 5,
  HOM_KERNEL_YPASS = 6, HOM_KERNEL_YPASS_F64 = 7,  /* split y pass (x passes count as plane kinds) */
  HOM_KERNEL_COUNT = 8
};

typedef struct {
  int64_t launches;     /* kernel launches */
  int64_t bytes;        /* algorithmic bytes: every input and output element the working CTAs
                           must read or write once (fields, phase bytes, spectrum scratch) */
  int64_t voxel_comps;  /* voxel-component units (plane kernels) or spectrum-column units
                           (z pass) processed by CTAs that did work */
  double ms;            /* device time summed over launches (CUDA events on the handle's stream) */
} hom_kernel_stat;

/* enable != 0 starts accounting (and resets the counters); 0 stops it.  While enabled each
 * LS-step launch is bracketed by CUDA events and counts its bytes on the device. */
HOM_API hom_status hom_profile(hom_t h, int32_t enable);

/* Reads the counters into out[HOM_KERNEL_COUNT] (host array); synchronizes the stream. */
HOM_API hom_status hom_profile_read(hom_t h, hom_kernel_stat* out);

/* One Lippmann-Schwinger step without any device allocation, for callers that cannot allocate
 * device memory: code that runs inside another library's memory pool or under an allocator it
 * does not own, or a loop that must not call cudaMalloc.  The paper has no counterpart; this is
 * the step of hom_ls_apply (FP64) with its scratch in a fixed device array of 16 MiB inside the
 * library, which every GPU that loads the library holds until the process exits.
 *  grid, phase    as hom_create (N3 = 1 is a two-dimensional cell), but phase must be a device
 *                 pointer (not copied).  Its values must be < n_phase.  The call does not scan
 *                 it: a value >= n_phase reads a zero row of the per-phase table, which keeps
 *                 every access in bounds but gives a meaningless result for that voxel.
 *  n_phase, lame  as hom_create (lame is a host array); lambda0, mu0 the reference medium.
 *  eps_in, eps_out device double [nrhs][6][N3][N2][N1] Mandel (eps_in NULL = zero field);
 *                 eps_in == eps_out computes in place; other overlaps return HOM_ERR_ARG, and so
 *                 do host pointers.  E host double [nrhs][6] Mandel (NULL = zero); 1 <= nrhs <= 64.
 *  cuda_stream    cudaStream_t the work is queued on (NULL = legacy default stream).  The small
 *                 tables (twiddles, per-phase eigenvalues, E) are copied from pageable host
 *                 memory with cudaMemcpyAsync, so the call may block the calling thread until
 *                 the stream reaches those copies; the result is ready when the stream is.
 * Limit: the spectrum of one load, 96 * N3 * N2 * (N1/2 + 1) bytes, plus small tables must fit
 * the 16 MiB (64^3 fits, 128 x 64 x 64 does not); larger grids return HOM_ERR_SIZE.
 * The first call on a device resolves the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  Every call shares the array: calls that overlap
 * on the GPU (other streams, other threads) race and must be serialized by the caller.
 * Errors are described by hom_noalloc_last_error() (per host thread). */
HOM_API hom_status hom_ls_apply_noalloc(const int32_t grid[3], const uint8_t* phase, int32_t n_phase,
                                        const double* lame, double lambda0, double mu0, int32_t nrhs,
                                        const double* eps_in, const double* E, double* eps_out,
                                        void* cuda_stream);

/* Text of the calling thread's last hom_ls_apply_noalloc error ("" after a success). */
HOM_API const char* hom_noalloc_last_error(void);

/* Device bytes a handle with default options needs to solve `order` (0 to 6) on this grid in
 * `precision`, as counted from its allocations (used for admission by the server); -1 if the
 * grid is not supported. */
HOM_API int64_t hom_estimate_bytes(const int32_t grid[3], int32_t order, int32_t precision);

/* ---- request server: continuous batching of RVE solves (no counterpart in the paper) ----
 * Requests are copied on submission and queued.  max_active worker threads admit queued requests
 * first-fit against a device-memory budget as soon as a worker is free:
 *  - an admitted order-0 request takes with it up to max_batch - 1 further queued order-0 requests
 *    of the same grid, precision, scheme and tolerance; they are solved in one handle with one RVE
 *    slot each (hom_options.n_rve), so every launch of the solve carries all of their loads;
 *  - handles stay resident per (grid, precision, scheme, order, slots) and are refilled with the
 *    next requests by hom_set_rve, so admission allocates no device memory once a kind has been
 *    seen; idle handles of other kinds are destroyed, least recently used first, when a new kind
 *    does not fit the budget;
 *  - every handle runs on its own stream, so different grids' launches overlap on the device.
 * Each load's arithmetic is that of its RVE solved alone (per-load solver state and refinement
 * decisions, per-slot tables and reference media), so a request's result does not depend on what
 * it was batched or overlapped with. */
typedef struct hom_server_ctx* hom_server_t;

typedef struct {
  int32_t grid[3];
  const uint8_t* phase;    /* host [N3][N2][N1], copied at submission */
  int32_t n_phase;
  const double* lame;      /* host [n_phase][2], copied */
  double lambda0, mu0;
  int32_t order;           /* 0 or 1 (order 1 also solves order 0) */
  int32_t precision;       /* HOM_FP32_REFINE or HOM_FP64 */
  int32_t scheme;          /* HOM_CG, HOM_BASIC or HOM_BICGSTAB */
  int32_t reserved;
  double tol;
} hom_request;

typedef struct {
  int32_t done;            /* 0 while queued or running */
  int32_t status;          /* hom_status of the solve */
  int32_t iterations;      /* CG / fixed-point iterations summed over all loads */
  int32_t order;
  double queue_ms, run_ms, latency_ms;  /* submission -> start -> end (host steady clock) */
  double c_eff[36];        /* 6x6 Mandel, row-major */
  double d1[108];          /* 6x18 Mandel (order 1) */
  char message[160];       /* hom_last_error text of a failed request, "" on success */
} hom_result;

/* budget_bytes <= 0: 85 % of the free device memory at creation.  1 <= max_active <= 64;
 * 1 <= max_batch <= 10 RVEs per batched handle (1: every request alone in its handle).
 * hom_server_create is hom_server_create_batched with max_batch = 8. */
HOM_API hom_status hom_server_create_batched(int64_t budget_bytes, int32_t max_active, int32_t max_batch,
                                             hom_server_t* out);
HOM_API hom_status hom_server_create(int64_t budget_bytes, int32_t max_active, hom_server_t* out);
/* Batches run, requests run in them, and handles created so far (each pointer nullable). */
HOM_API hom_status hom_server_counters(hom_server_t s, int64_t* batches, int64_t* requests_run,
                                       int64_t* handles_created);
/* Queues a request; *id identifies it.  HOM_ERR_NOMEM if it can never fit the budget. */
HOM_API hom_status hom_server_submit(hom_server_t s, const hom_request* req, int64_t* id);
/* Copies the result if the request is done (out->done = 1), else sets out->done = 0. */
HOM_API hom_status hom_server_poll(hom_server_t s, int64_t id, hom_result* out);
/* Blocks until the request is done, then copies its result. */
HOM_API hom_status hom_server_wait(hom_server_t s, int64_t id, hom_result* out);
/* Queue length, running requests and the device bytes the server's handles hold or have reserved
 * (each pointer nullable). */
HOM_API hom_status hom_server_stats(hom_server_t s, int64_t* queued, int64_t* running, int64_t* bytes_in_use);
/* Waits for every queued and running request, then releases the server. */
HOM_API void hom_server_destroy(hom_server_t s);

/* Bytes of device memory the handle holds now. */
HOM_API int64_t hom_device_bytes(hom_t h);

/* Launch shape of the handle's iteration passes: loads transformed per launch and the z-pass
 * tile width as log2 of its columns (-1: chosen per launch by the occupancy rule).  After an
 * autotuned solve these are the tuned values.  Pointers nullable. */
HOM_API hom_status hom_launch_config(hom_t h, int32_t* loads_per_launch, int32_t* ztile_log2);

/* x-y passes of the handle's FP32 transforms: *cluster_ctas = CTAs per plane of the cluster plane
 * passes (hom_options.pass_mode), 0 when the fused plane kernels or the split x and y passes run. */
HOM_API hom_status hom_plane_config(hom_t h, int32_t* cluster_ctas);

/* split y pass of the handle's iteration passes: *tile_log2 its tile width as log2 of its columns
 * (-1 when the grid's x-y transforms are not split), *tma = 1 when its FP32 tiles move by TMA tensor
 * loads and stores (hom_options.y_mode and the autotuner's pick).  Pointers nullable. */
HOM_API hom_status hom_ypass_config(hom_t h, int32_t* tile_log2, int32_t* tma);

/* z stage of the handle's iteration passes: *cluster = 1 for the cluster z pass, 2 for its TMA
 * form, 0 for the single-CTA z pass (hom_options.z_mode); *tile_log2 its tile width as log2 of its
 * columns (-1: the default rule).  Pointers nullable. */
HOM_API hom_status hom_zpass_config(hom_t h, int32_t* cluster, int32_t* tile_log2);

/* Kernels this library has launched in this process so far, over all handles, servers and the
 * allocation-free entry point (a host-side count of launches issued, not of launches finished). */
HOM_API int64_t hom_launch_count(void);

/* Text of the last error on this handle ("" if none); valid until the next call. */
HOM_API const char* hom_last_error(hom_t h);

/* Static name of a status code. */
HOM_API const char* hom_status_string(hom_status s);

/* Releases the handle and all device memory it holds (NULL is a no-op). */
HOM_API void hom_destroy(hom_t h);

#ifdef __cplusplus
}
#endif

#endif /* HOM_H */
