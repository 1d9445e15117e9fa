"""Pin of the higher-order problems (Sec. 3, Definition of the generalized problem of order alpha)
by a closed solution: a three-layer laminate.

Layers normal to y1 (fractions 1/4, 1/4, 1/2, three different isotropic phases, so the cell is not
centrosymmetric) make every corrector a function of y1 alone.  Take the unit load E^11 and the
monomial loads E^11 Y2^o / o! of order o.  Then each problem of the hierarchy is a scalar ODE on
the unit period, with a = lambda + 2 mu, a* = <1/a>^-1, zero-mean displacements and the body
force taken without its mean (the xi = 0 mode has no counterpart in the periodic problem):

* order 0: a (1 + chi') = a*, so the displacement is chi e1 and s22 = lambda a* / a;
* odd o: the displacement U_o runs along e2.  The polarization is mu U_{o-1} in the 12
  component, and the body force s22 of order o-1 acts along e2.  Then mu (U_o' + U_{o-1}) = C - J
  with J' = s22 - <s22>, and C = <J/mu> / <1/mu>.  The 12 stress is C - J, so
  D_o(12) = sqrt(2) C in Mandel form;
* even o: the displacement U_o runs along e1.  The polarization is lambda U_{o-1} (11),
  a U_{o-1} (22) and lambda U_{o-1} (33), and the body force C - J of order o-1 acts along e1.
  Then a U_o' + lambda U_{o-1} = K + F with K' = J and
  F = (<lambda U_{o-1}/a> - <K/a>) / <1/a>, so D_o(11) = F and s22 = lambda U_o' + a U_{o-1}.

These are integrals of piecewise polynomials, evaluated here by midpoint quadrature on 2^18 points
(error below 1e-10).  The oracle's voxel solutions (its FFT, Green operator, displacement recovery,
p_alpha, g_alpha and theta_alpha builders) must converge to them as the layers are resolved.  They
do at second order for orders 1 to 6, which fixes every sign, index and factor along the chain.
"""
import numpy as np
import pytest

from oracle.hierarchy import GeneralHierarchy, Hierarchy, multisets
from oracle.lippmann_schwinger import Problem

LAME = np.array([[1.0, 1.0], [6.0, 4.0], [0.3, 0.2]])
BOUNDS = (0.25, 0.5)          # layer interfaces in the unit period
MAX_ORDER = 6


def layer_fields(m):
    y = (np.arange(m) + 0.5) / m
    ph = np.where(y < BOUNDS[0], 0, np.where(y < BOUNDS[1], 1, 2))
    return LAME[ph, 0], LAME[ph, 1]


def closed_chain(max_order, m=1 << 18):
    """D_o of the chain E^11 Y2^o / o!: {o: value} (Mandel 12 for odd o, 11 for even o)."""
    lam, mu = layer_fields(m)
    a = lam + 2.0 * mu
    dy = 1.0 / m

    def antiderivative(f):            # zero-mean antiderivative on the period
        F = np.cumsum(f) * dy - 0.5 * f * dy
        return F - F.mean()

    a_star = 1.0 / np.mean(1.0 / a)
    U = antiderivative(a_star / a - 1.0)
    s22 = lam * a_star / a
    J = None
    out = {}
    for o in range(1, max_order + 1):
        if o % 2 == 1:
            J = antiderivative(s22 - s22.mean())
            C = np.mean(J / mu) / np.mean(1.0 / mu)
            U = antiderivative((C - J) / mu - U)
            out[o] = np.sqrt(2.0) * C
        else:
            K = antiderivative(J)
            F = (np.mean(lam * U / a) - np.mean(K / a)) / np.mean(1.0 / a)
            dU = (K + F - lam * U) / a
            s22 = lam * dU + a * U
            U = antiderivative(dU)
            out[o] = F
    return out


def oracle_chain(n):
    phase = np.zeros((2, 2, n), dtype=np.uint8)
    phase[:, :, int(BOUNDS[0] * n):int(BOUNDS[1] * n)] = 1
    phase[:, :, int(BOUNDS[1] * n):] = 2
    h = Hierarchy(Problem(phase, LAME, 3.0, 2.0), tol=1e-13)
    h.order1()
    h.order2()
    G = GeneralHierarchy(h)
    out = {1: h.d1[5, 1]}        # explicit alpha = 2 builder: load 3A + k, A = 11, k = y2
    for alpha in range(2, MAX_ORDER + 2):
        G.solve(alpha)
        o = alpha - 1
        col = multisets(o).index((1,) * o)
        out[o] = G.D[alpha][5 if o % 2 == 1 else 0, col]
    h.order3()
    out["explicit2"] = h.d2[0, 1]  # explicit alpha = 3 builder: load 6A + P, P = (2, 2)
    return out


@pytest.fixture(scope="module")
def chains():
    ref = closed_chain(MAX_ORDER)
    return ref, {n: oracle_chain(n) for n in (32, 64, 128)}


def test_closed_chain_is_resolved():
    """The quadrature itself has converged: halving the points changes nothing at 1e-9."""
    a, b = closed_chain(MAX_ORDER, 1 << 17), closed_chain(MAX_ORDER)
    for o in a:
        assert abs(a[o] - b[o]) < 1e-9 * abs(b[o])
        assert abs(b[o]) > 1e-4          # every order of the chain is a real test


@pytest.mark.parametrize("order", range(1, MAX_ORDER + 1))
def test_oracle_converges_to_the_laminate_solution(chains, order):
    ref, got = chains
    err = [abs(got[n][order] - ref[order]) / abs(ref[order]) for n in (32, 64, 128)]
    assert err[0] / err[1] > 3.0 and err[1] / err[2] > 3.0, err     # second order in h
    assert err[2] < 1e-3, err


def test_explicit_order2_builder_agrees_with_the_general_one(chains):
    _, got = chains
    for n in (32, 64, 128):
        assert abs(got[n]["explicit2"] - got[n][2]) < 1e-10 * abs(got[n][2])
