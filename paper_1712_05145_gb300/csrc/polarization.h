// Polarization scheme (polarization.cu): the pointwise steps of the fixed point
//   x <- (1 - g) x + g (r + W x - 2 Gamma0 * (C0 : W x)),   eps = (I - W) x,
// W = (C - C0) (C + C0)^-1, which solves A eps = r (Eq. cg_form) for compatible r: the scheme of
// Eyre-Milton / Monchiet-Bonnet (g = 1) and its averaged, augmented-Lagrangian form (g = 1/2),
// both cited in Sec. 1.  The transform step -Gamma0 * (C0 : W x) is an LS pass in FWD_TAU mode
// with the table below in place of the material table.
#pragma once
#include "internal.h"

namespace hom {

enum PolarStep { PO_UPDATE = 0, PO_FINISH = 1 };

template <typename Tf>
struct PolarArgs {
  Tf* x;                 // [rhs][6][M] the scheme's variable, updated in place (PO_UPDATE)
  const Tf* r;           // [rhs][6][M] right-hand side
  const Tf* eta;         // [rhs][6][M] -Gamma0 * (C0 : W x) of the current x
  Tf* d;                 // [rhs][6][M] PO_FINISH: d += (I - W) x
  const uint8_t* phase;  // [M]
  const Tf* wt;          // [n_phase][4] Kelvin: c0 w (hydrostatic, deviatoric), w (hydrostatic, deviatoric)
  int n_phase;
  double relax;          // g
  long long M;
  int rhs0;              // first load of the launch
  RhsState* st;          // [rhs]
  double* part;          // [rhs][2][pstride] partial sums
  int pstride;
  unsigned* cnt;         // [rhs] tickets
};

// PO_UPDATE: the x update of every active load with the FP64 Cauchy sum ||(I - W)(x_new - x)||^2;
// the last CTA of a load sets res = that norm / ||b||, counts the iteration and ends the load's
// sweep at its tolerance or iteration cap (NaN: status 2).  PO_FINISH: d += (I - W) x for loads
// rhs0 .. rhs0 + nrhs - 1, whatever their state.
template <typename Tf>
cudaError_t launch_polar(int step, const PolarArgs<Tf>& a, int nrhs, int nblk, cudaStream_t s);

}  // namespace hom
