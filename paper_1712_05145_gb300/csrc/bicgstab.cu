// BiCGSTAB on the Lippmann-Schwinger system A eps = b (Eq. cg_form), the Krylov solver the paper
// ran for its CG-version (Sec. 4).  The two operator applications per iteration, v = A p and
// t = A s, are LS passes (A = Gamma0 * (C : .) on compatible fields); this file holds the vector
// updates between them.  Each step is one grid-stride kernel over the [6][M] field of every
// active load, with FP64 block sums and a last-block ticket that updates the load's state:
//   BI_RESTART  r_hat = r, p = r                      rho = <r, r>
//   BI_ALPHA    (reads v = A p)                       alpha = rho / <r_hat, v>
//   BI_S        s = r - alpha v                       sconv = ||s|| / ||b|| < tol
//   BI_OMEGA    (reads t = A s)                       omega = <t, s> / <t, t>   (0 if sconv)
//   BI_X        x += alpha p + omega s, r = s - omega t
//                                                     rho' = <r_hat, r>, res = ||r|| / ||b||,
//                                                     beta = (rho' / rho) (alpha / omega)
//   BI_P        p = r + beta (p - omega v), or r_hat = r, p = r after a breakdown (rho' = 0 or
//               omega = 0), in which case BI_X has already set rho = <r, r>.
#include "ls_common.cuh"

namespace hom {

__device__ __forceinline__ void bicg_finalize(int step, RhsState& s, const double* v, double invM) {
  switch (step) {
    case BI_RESTART: {
      s.rho = v[0] * invM;
      s.rr = s.rho;
      s.restart = 0;
      s.sconv = 0;
      if (!isfinite(s.rho)) { s.status = 2; s.active = 0; }
      break;
    }
    case BI_ALPHA: {
      const double rv = v[0] * invM;
      s.alpha = (rv != 0.0) ? s.rho / rv : 0.0;
      s.sconv = 0;
      if (!isfinite(s.alpha)) { s.status = 2; s.active = 0; }
      break;
    }
    case BI_S: {
      const double ss = v[0] * invM;
      s.sconv = (s.b2 > 0.0 && sqrt(ss / s.b2) < s.tol) ? 1 : 0;
      break;
    }
    case BI_OMEGA: {
      const double ts = v[0] * invM, tt = v[1] * invM;
      s.omega = (s.sconv || tt <= 0.0) ? 0.0 : ts / tt;
      if (!isfinite(s.omega)) { s.status = 2; s.active = 0; }
      break;
    }
    case BI_X: {
      const double rho = v[0] * invM, rr = v[1] * invM;
      s.rr = rr;
      s.res = (s.b2 > 0.0) ? sqrt(rr / s.b2) : 0.0;
      s.iter += 1;
      if (s.omega != 0.0 && rho != 0.0 && s.rho != 0.0) {
        s.beta = (rho / s.rho) * (s.alpha / s.omega);
        s.rho = rho;
        s.restart = 0;
      } else {  // breakdown: restart from r_hat = r
        s.beta = 0.0;
        s.rho = rr;
        s.restart = 1;
      }
      if (!isfinite(s.res) || !isfinite(s.beta)) { s.status = 2; s.active = 0; }
      else if (s.res < s.tol) s.active = 0;
      else if (s.iter >= s.max_iter) { s.active = 0; s.status = 1; }
      else if (s.res < 0.5 * s.best) { s.best = s.res; s.best_iter = s.iter; }
      else if (s.stall && s.iter - s.best_iter >= (s.res < kNearFloor ? kStallItersNearFloor : kStallIters))
        s.active = 0;  // stalled: hand over to the FP64 residual sweep
      break;
    }
    default: break;
  }
}

template <typename Tf, int STEP>
__global__ void __launch_bounds__(256) bicg_kernel(const BicgArgs<Tf> a) {
  __shared__ double sh[64 + 2];
  __shared__ int flag;
  const int rhs = blockIdx.y;
  RhsState& st = a.st[rhs];
  if (st.active == 0) return;
  const long long per = 6LL * a.M, off = (long long)rhs * per;
  const Tf al = (Tf)st.alpha, om = (Tf)st.omega, be = (Tf)st.beta;
  const bool restart = (STEP == BI_P) && st.restart != 0;
  Tf q0 = 0, q1 = 0;   // per-thread partials in the field precision, block and grid sums in FP64
  for (long long i = off + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < off + per;
       i += (long long)gridDim.x * blockDim.x) {
    if (STEP == BI_RESTART) {
      const Tf r = a.r[i];
      a.rh[i] = r;
      a.p[i] = r;
      q0 += r * r;
    } else if (STEP == BI_ALPHA) {
      q0 += a.rh[i] * a.v[i];
    } else if (STEP == BI_S) {
      const Tf s = a.r[i] - al * a.v[i];
      a.s[i] = s;
      q0 += s * s;
    } else if (STEP == BI_OMEGA) {
      const Tf t = a.t[i], s = a.s[i];
      q0 += t * s;
      q1 += t * t;
    } else if (STEP == BI_X) {
      const Tf s = a.s[i];
      a.x[i] += al * a.p[i] + om * s;
      const Tf r = s - om * a.t[i];
      a.r[i] = r;
      q0 += a.rh[i] * r;
      q1 += r * r;
    } else {  // BI_P
      const Tf r = a.r[i];
      if (restart) {
        a.rh[i] = r;
        a.p[i] = r;
      } else {
        a.p[i] = r + be * (a.p[i] - om * a.v[i]);
      }
    }
  }
  if (STEP == BI_P) return;
  double v[2] = {(double)q0, (double)q1};
  block_sum_f64<2>(v, sh);
  if (publish_and_collect<2>(v, a.part + (long long)rhs * 2 * a.pstride, a.cnt + rhs, gridDim.x, blockIdx.x, sh,
                             &flag)) {
    if (threadIdx.x == 0) bicg_finalize(STEP, st, v, 1.0 / (double)a.M);
  }
}

template <typename Tf>
cudaError_t launch_bicg(int step, const BicgArgs<Tf>& a, int nrhs, int nblk, cudaStream_t s) {
  if (nblk < 1 || nblk > a.pstride || nrhs < 1) return cudaErrorInvalidValue;
  dim3 grid(nblk, nrhs);
  count_launch();
  switch (step) {
    case BI_RESTART: bicg_kernel<Tf, BI_RESTART><<<grid, 256, 0, s>>>(a); break;
    case BI_ALPHA: bicg_kernel<Tf, BI_ALPHA><<<grid, 256, 0, s>>>(a); break;
    case BI_S: bicg_kernel<Tf, BI_S><<<grid, 256, 0, s>>>(a); break;
    case BI_OMEGA: bicg_kernel<Tf, BI_OMEGA><<<grid, 256, 0, s>>>(a); break;
    case BI_X: bicg_kernel<Tf, BI_X><<<grid, 256, 0, s>>>(a); break;
    case BI_P: bicg_kernel<Tf, BI_P><<<grid, 256, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_bicg<float>(int, const BicgArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_bicg<double>(int, const BicgArgs<double>&, int, int, cudaStream_t);

}  // namespace hom
