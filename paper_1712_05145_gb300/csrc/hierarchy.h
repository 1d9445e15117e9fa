// Pointwise kernels of the order-alpha problems (Sec. 3) and stress fields.
#pragma once
#include "internal.h"

namespace hom {

// Builds, for every load of order `order` (1 or 2), the polarization p_alpha (Kelvin,
// components 0..5) and the body force g_alpha (Cartesian, components 6..8) into
// out9 [nload][9][M], and copies p_alpha into pf [nload][6][M].
//  order 1 (paper alpha = 2), load 3A+k:  p = C : sym(chi^A (x) e_k),  g = sigma^A e_k,
//          sigma^A = C : (E^A + eps^A)   from the order-0 correctors (disp0, eps0, EK).
//  order 2 (paper alpha = 3), load 6A+P, (k,l) the P-th Mandel pair, w = 1/(1+d_kl):
//          p = C : w [sym(u^(A,k) (x) e_l) + sym(u^(A,l) (x) e_k)],
//          g_i = w [s^(A,k)_il + s^(A,l)_ik],  s = C : eps_2 + p_2  from the order-1 correctors.
//  For order 1, map selects the loads: load L is the unit load u = map.unit[L] = 3A+k, and the
//  order-0 correctors of E^A are those of order-0 load map.a0[A].
//  For orders o >= 2 (the paper's alpha = o + 1) the unit loads are E^A m_K(Y), K a multiset
//  of o directions and m_K = Y^K / K!, load L = A * nK + (index of K); then
//      p = C : sum_j sym(u^(A, K - e_j) (x) e_j),   g = sum_j s^(A, K - e_j) e_j,
//  over the distinct directions j of K, with u and s = C : eps + p the displacement and stress
//  correctors of order o - 1 (table rec).
struct UnitMap {
  int unit[18];
  int a0[6];
};
constexpr int kMaxOrder = 6;     // orders 0..6 (the paper's alpha = 1..7)
constexpr int kMaxMultisets = 28; // multisets of 6 directions from 3: (6 + 1)(6 + 2) / 2
struct RecTable {
  int nK, nKprev;                  // multisets of this order and of the previous one
  int nterm[kMaxMultisets];
  int dir[kMaxMultisets][3];
  int src[kMaxMultisets][3];       // position of K - e_dir among the previous order's multisets
};
template <typename Tf>
cudaError_t launch_rhs_pointwise(int order, int nload, const UnitMap& map, const RecTable& rec, const Tf* disp,
                                 const Tf* eps, const Tf* pprev, const double* EK, const uint8_t* phase,
                                 const double* mat, long long M, Tf* out9, Tf* pf, cudaStream_t s);

// out[l][i] = sum_u W[l][u] in[u][i] for l < nout, u < nin, i < per (linear combinations of loads).
cudaError_t launch_combine_loads(const double* in, int nin, const double* W, int nout, long long per, double* out,
                                 cudaStream_t s);

// Mandel stress of one load: C : (eps + E) (EK non-null) or C : eps + p (pf non-null).
template <typename Tf>
cudaError_t launch_stress_field(const Tf* eps, const double* EK, const Tf* pf, const uint8_t* phase,
                                const double* mat, long long M, double* out, cudaStream_t s);

}  // namespace hom
