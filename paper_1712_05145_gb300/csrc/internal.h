// Internal (C++) interface between the host driver and the CUDA kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace hom {

constexpr int kMaxRve = 10;   // RVE slots of one handle (6 unit loads each, at most 64 loads per solve)

// Geometry of one voxel grid and its spectrum layout.
//  fields   [rhs][comp][n3][n2][n1]            real, x fastest
//  spectrum [rhs][comp][n3][plane_c]           complex; one x-y plane holds the
//           n2 x h half-spectrum rows (kx < n1/2, row pitch h) followed by the
//           n2 values of the Nyquist column kx = n1/2.
struct Geo {
  int n1, n2, n3, h;     // h = n1 / 2 (n1 even)
  int P;                 // shared-memory row pitch of a plane (complex elements, odd)
  long long M;           // voxels
  long long plane_c;     // n2 * (h + 1)
  FastDiv fd_h, fd_n2;   // division by h and n2 (pencil counts of the column and row FFTs)
  // split passes (grids whose x-y plane does not fit one CTA, or by choice):
  int split;             // 1: x pass + y pass kernels instead of the fused plane kernels
  int rb, nrb, thr_x;    // x pass: rows per CTA, row blocks per component, threads
  FastDiv fd_rb;         // division by rb
  int ty_log2, thr_y;    // y pass: 2^ty_log2 consecutive columns per CTA, threads
  FastDiv fd_ty;         // division by 2^ty_log2
  double xs1, xs2, xs3;  // physical frequency per integer wave number: 2 pi Nmax / N_i
  // cluster plane passes (split grids, FP32 transforms): pc_Q CTAs per plane (0: not used), each
  // with pc_R = n2 / pc_Q rows and pc_Cb = h / pc_Q spectrum columns, pc_thr threads
  int pc_Q, pc_R, pc_Cb, pc_thr;
  FastDiv pc_fdR, pc_fdCb;  // division by pc_R and pc_Cb
};

// Per right-hand-side solver state, kept on the device (FP64).
struct RhsState {
  double rho;        // <r, r>_C0
  double alpha, beta;
  double pAp;        // <p, A p>_C0 = <p, C p>
  double b2;         // ||b||^2 (voxel mean)
  double res;        // latest relative residual (recursive / Cauchy)
  double res_true;   // FP64 residual ||b - A x|| / ||b||
  double tol;        // inner stopping tolerance
  double best;       // smallest residual of the current sweep (stall detection)
  int iter;          // iterations done
  int max_iter;
  int active;        // 1 while the inner iteration runs
  int restart;       // 1: next CG step starts from p = r
  int status;        // 0 ok, 1 not converged, 2 numeric
  int best_iter;     // iteration at which `best` was last halved
  // BiCGSTAB (L2 inner products): rho = <r_hat, r>, alpha, omega, beta; rr = <r, r>
  double omega;
  double rr;
  int sconv;         // 1: the half step s already met the tolerance (omega = 0, x += alpha p)
  int stall;         // 1: end the sweep when the residual stalls (FP32 sweeps of the refinement)
  int xpend;         // CG: x += alpha p of the last iteration is still to be applied (the next
                     // forward pass applies it while it reads p; after a sweep, cg_flush does)
};

// FWD_TAU: tau = (C - C0) : (in + E)     (polarization, Eq. auxiliary_problem)
// FWD_STRESS: tau = C : (in + E)         (stress; -Gamma0 * sigma is the equilibrium residual)
// FWD_CG: x += alpha p, p = r + beta p, tau = C : p   (CG: the previous iteration's update of x and
//         the new direction; A p = Gamma0 * (C : p) on compatible p)
// FWD_COPY: tau = in                     (plain transform)
// FWD_C0: tau = C0 : in                  (-Gamma0 * (C0 : in) is minus the compatible part of in)
enum FwdMode { FWD_TAU = 0, FWD_CG = 1, FWD_COPY = 2, FWD_STRESS = 3, FWD_C0 = 4 };
// Z_GAMMA: forward z FFT, -Gamma0_hat contraction, inverse z FFT (the LS step)
// Z_FWD / Z_INV: forward / inverse z FFT only; Z_GREEN: contraction only (no FFT)
// Z_DISP: forward z FFT of a strain, displacement u_hat (3 components), inverse z FFT
// Z_RHS: forward z FFT of (p, g), -Gamma0_hat : (p_hat + theta_hat), inverse z FFT
enum ZMode { Z_GAMMA = 0, Z_FWD = 1, Z_INV = 2, Z_DISP = 3, Z_RHS = 4, Z_GREEN = 5 };
enum InvMode { INV_STORE = 0, INV_CG = 1 };
enum FinKind { FIN_NONE = 0, FIN_RHS = 1, FIN_BASIC = 2, FIN_CG = 3, FIN_RESID = 4, FIN_ENERGY = 5 };

template <typename Tf, typename T>
struct FwdArgs {
  Geo g;
  int mode, ncomp, in_ncomp;   // components transformed; components per rhs of `in`
  const uint8_t* phase;
  const T* mat;                // [n_phase][4] Kelvin eigenvalues: C-C0 (h, dev), C (h, dev)
  T c0h, c0d;                  // FWD_C0: C0 Kelvin eigenvalues 3 lam0 + 2 mu0, 2 mu0
  int n_phase;
  int rve_loads;               // > 0: the handle holds several RVEs, rve_loads consecutive loads each;
                               // load r reads phase + (r / rve_loads) M and its RVE's 256-row table
  const double* c0;            // rve_loads > 0: [rve][4] (lambda0, mu0, 3 lambda0 + 2 mu0, 2 mu0) per RVE
  const Tf* in;                // FWD_TAU: strain (nullable); FWD_COPY: field
  const double* E;             // FWD_TAU: [rhs][6] Kelvin macroscopic strain (nullable)
  const Tf* r;                 // FWD_CG
  Tf* p;                       // FWD_CG (read old p, write new p)
  Tf* x;                       // FWD_CG (x += alpha p with the old p, except at a restart)
  cx<T>* S;                    // chunk spectrum
  int rhs0;                    // global rhs index of the chunk's first rhs
  RhsState* st;                // nullable
  double* part;                // [rhs][2][ncta] partial sums
  unsigned* cnt;               // [rhs] tickets
  unsigned long long* prof;    // nullable: [bytes, units] of this kernel kind
  const cx<T>* tw_h;
  const cx<T>* tw_n1;
  const cx<T>* tw_n2;
};

template <typename T>
struct ZArgs {
  Geo g;
  int mode, ncomp_in, ncomp_out;
  int tc_log2;           // tile: 2^tc_log2 consecutive spectrum columns
  int ntiles;            // ceil(plane_c / 2^tc_log2)
  int nthr;              // threads per CTA
  int cstride;           // shared-memory stride between components (padded against bank conflicts)
  FastDiv fd_in, fd_out; // division by ncomp_in * 2^tc_log2 and ncomp_out * 2^tc_log2
  FastDiv fd_comp;       // division by n3 * 2^tc_log2 (elements of one component in a tile)
  cx<T>* S;
  int rhs0;
  const RhsState* st;
  double lam0, mu0;
  int rve_loads;         // > 0: loads per RVE of a several-RVE handle, whose reference media are
  const double* c0;      //   c0[rve][4] = (lambda0, mu0, 3 lambda0 + 2 mu0, 2 mu0) in place of lam0, mu0
  double scale;          // factor applied with the spectral operator (1/M after a forward FFT)
  int green;             // 0: spectral wave vector; 1: rotated finite-difference vector q (gtab)
  const double* gtab;    // green == 1: sin, cos of pi j / N per axis (see wave_vector)
  unsigned long long* prof;
  const cx<T>* tw_n3;
  unsigned* err;         // nullable: bits set by kernels whose bounded waits gave up (1) or whose
                         // shared-memory layout was unusable (2)
};

template <typename Tf, typename T>
struct InvArgs {
  Geo g;
  int mode, fin, ncomp, out_ncomp;
  int s_ncomp;           // components per rhs in the spectrum
  const cx<T>* S;
  int rhs0;
  T c0h, c0d;            // C0 Kelvin eigenvalues: 3 lam0 + 2 mu0, 2 mu0
  int rve_loads;         // > 0: loads per RVE of a several-RVE handle, whose reference media are
  const double* c0;      //   c0[rve][4] = (lambda0, mu0, 3 lambda0 + 2 mu0, 2 mu0) in place of c0h, c0d
  T out_scale;           // INV_STORE: out = out_scale * eta (+ b)
  Tf* out;               // INV_STORE
  const double* b;       // INV_STORE: added right-hand-side field, FP64 (nullable)
  const double* xsub;    // INV_STORE: subtracted field, FP64 (nullable): out = scale*eta + b - xsub
  const Tf* prev;        // INV_STORE: previous iterate for the Cauchy difference (nullable)
  Tf* r;                 // INV_CG: r += alpha eta (= r - alpha A p)
  RhsState* st;
  double* part;
  unsigned* cnt;
  unsigned long long* prof;
  const cx<T>* tw_h;
  const cx<T>* tw_n1;
  const cx<T>* tw_n2;
};

// BiCGSTAB vector updates with their FP64 reductions (one kernel per step kind, see bicgstab.cu)
enum BicgStep { BI_RESTART = 0, BI_ALPHA = 1, BI_S = 2, BI_OMEGA = 3, BI_X = 4, BI_P = 5 };
template <typename Tf>
struct BicgArgs {
  Tf *x, *r, *rh, *p, *v, *s, *t;  // [rhs][6][M] each
  long long M;
  RhsState* st;                    // [rhs]
  double* part;                    // [rhs][2][pstride] partial sums
  int pstride;
  unsigned* cnt;                   // [rhs] tickets
};
template <typename Tf>
cudaError_t launch_bicg(int step, const BicgArgs<Tf>& a, int nrhs, int nblk, cudaStream_t s);

template <typename Tf, typename T>
cudaError_t launch_plane_fwd(const FwdArgs<Tf, T>& a, int nrhs, cudaStream_t s);
// split passes: x pass (prologue + row R2C), y pass over column tiles, x inverse pass
template <typename Tf, typename T>
cudaError_t launch_xpass_fwd(const FwdArgs<Tf, T>& a, int nrhs, cudaStream_t s);
template <typename T>
cudaError_t launch_ypass(const cx<T>* tw_n2, cx<T>* S, const Geo& g, int ncomp, int s_ncomp, int nrhs, int dir,
                         unsigned long long* prof, const RhsState* st, int rhs0, cudaStream_t s);
// the y pass with its column tiles moved by TMA tensor loads and stores (FP32 transforms); ytma_fits:
// whether the grid's split y pass can run it (even h and plane, tiles of 2 columns at least); err:
// nullable word whose bits the kernel sets when its bounded wait gives up (1)
bool ytma_fits(const Geo& g);
cudaError_t launch_ypass_tma(const cx<float>* tw_n2, cx<float>* S, const Geo& g, int ncomp, int s_ncomp, int nrhs,
                             int dir, unsigned long long* prof, const RhsState* st, int rhs0, unsigned* err,
                             cudaStream_t s);
template <typename Tf, typename T>
cudaError_t launch_xpass_inv(const InvArgs<Tf, T>& a, int nrhs, cudaStream_t s);
template <typename T>
cudaError_t launch_zpass(const ZArgs<T>& a, int nrhs, cudaStream_t s);
template <typename Tf, typename T>
cudaError_t launch_plane_inv(const InvArgs<Tf, T>& a, int nrhs, cudaStream_t s);

size_t plane_smem_bytes(const Geo& g, size_t elem);
size_t zpass_smem_bytes(const Geo& g, size_t elem, int ncomp, int tc_log2);
// fills fd_h, fd_n2 and the split-pass tiling of a geometry whose n1, n2, n3 are set
void geo_finish(Geo& g);
// y pass tiles of 2^lg columns (ty_log2, thr_y, fd_ty); whether such tiles fit the y pass
void set_ytile(Geo& g, int lg);
bool ytile_fits(const Geo& g, int lg);
// resident CTAs per SM of the z pass for a launch shape (occupancy query, cached)
template <typename T>
int zpass_ctas_per_sm(int threads, size_t smem);
// z-pass tiling for ncomp input components: fills tc_log2, ntiles, nthr.  force_lg >= 0 asks for
// tiles of 2^force_lg columns (used when it fits); otherwise the occupancy rule picks the width.
template <typename T>
void zpass_tiling(ZArgs<T>& a, int force_lg = -1);
// whether tiles of 2^lg columns fit the z pass for ncomp input components (threads, shared memory)
bool zpass_tile_fits(const Geo& g, size_t elem, int ncomp, int lg);

// counts one kernel launch of this library (process-wide; read by hom_launch_count)
void count_launch();

}  // namespace hom
