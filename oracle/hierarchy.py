"""Oracle for the generalized homogenization problems of order alpha (test infrastructure).

Sec. 3 of arXiv:1712.05145.  Orders are counted as in the paper: alpha = 1 is the
classical cell problem (solved by ``Problem.solve_order0``), alpha = 2 and alpha = 3
are the next two problems of the hierarchy.  (The C-ABI counts the same problems as
order 0, 1, 2.)

For a unit macroscopic load the separation ansatz u_alpha = X_alpha(y) . grad^(alpha-1) E(Y)
(Sec. 3) turns each problem into a cell problem

    div_y (C : e_y(u_alpha) + p_alpha) + g_alpha = 0,
    p_alpha = C : e_Y(u_{alpha-1}),  g_alpha = div_Y [C : (e_y(u_{alpha-1}) + e_Y(u_{alpha-2}))]

(Definition of the generalized problem; the divergence div_Y in g_alpha is the one of the
second-order problem, with u_0 = U and e_Y(U) = E).  It is solved with the same operator
A as alpha = 1 from eps_0 = -Gamma0 * (p_alpha + theta_alpha), where theta_alpha is the
closed-form symmetric field with i theta_hat xi = g_hat (Sec. 3, Eq. for theta_hat).

Unit loads:
* alpha = 2: E(Y) = E^A Y_k (A a Mandel unit strain, k a direction): 18 loads, index
  3*A + k.  Then p_2 = C : sym(chi^A (x) e_k) and g_2 = sigma^A e_k, the k-th column of the
  alpha = 1 stress sigma^A = C : (E^A + eps^A).
* alpha = 3: E(Y) = E^A Y_k Y_l / (1 + d_kl), so d_k d_l E = E^A: 36 loads, index 6*A + P
  with (k, l) the P-th Mandel pair.  Then
  p_3 = C : [sym(u_2^(A,k) (x) e_l) + sym(u_2^(A,l) (x) e_k)] / (1 + d_kl) and
  (g_3)_i = [s^(A,k)_il + s^(A,l)_ik] / (1 + d_kl),  s^(A,n) = C : eps_2^(A,n) + p_2^(A,n).

Readings (the paper is silent or garbled here):
* the mean of g_alpha is dropped (theta_hat(0) = 0), the corrector has zero mean;
* every spectral operator (theta_hat, displacement recovery, e_y, Gamma0_hat) uses the
  discrete wave vector of ``fourier.wavevectors``, whose Nyquist components are 0, and
  vanishes where that vector is 0;
* the higher-order effective tensor of order alpha is the mean order-alpha stress per
  unit load, D[:, load] = < C : eps_alpha + p_alpha > (Mandel), which the paper leaves
  for future work.

Any order alpha >= 2 (``GeneralHierarchy``): the unit loads are E^A m_K(Y) with m_K = Y^K / K!
for the multisets K of alpha - 1 directions; p_alpha and g_alpha are sums over the order
alpha - 1 correctors with the coefficients d_j d^J m_K, computed by differentiating the
monomial.

Pins (tests/test_oracle_hierarchy.py): i theta_hat xi = g_hat; the displacement /
strain round trip; linearity; D_1 = 0 for centrosymmetric cells; the general builder
reproduces the explicit alpha = 2 and alpha = 3 builders; D_3 = 0 (alpha = 4) for
centrosymmetric cells; zero correctors at every order for a homogeneous medium.
Values (tests/test_oracle_laminate_hierarchy.py): on a non-centrosymmetric three-layer laminate
the problems for the loads E^11 Y2^o / o! reduce to scalar ODEs whose solutions are integrals
of piecewise polynomials.  D_o for o = 1..6 (alpha = 2..7) converges to them at second order in
the voxel size.  That pins one component chain per order.  The other components share the same
builder code and are checked by the structural pins above.
"""
import numpy as np

from . import fourier
from .lippmann_schwinger import green_apply
from .tensors import tensor_to_mandel, unit_mandel_load, MANDEL_PAIRS


def _xi_stack(grid, shape):
    xi1, xi2, xi3 = fourier.wavevectors(grid)
    return np.stack(np.broadcast_arrays(xi1, xi2, xi3)).reshape((3,) + shape)


def displacement_from_strain(eps, grid):
    """Zero-mean displacement u with e_y(u) = eps for a compatible strain field.

    In Fourier space eps_hat = i sym(xi (x) u_hat), hence
    u_hat = -i (2 eps_hat xi - xi (xi . eps_hat xi)/|xi|^2) / |xi|^2.
    """
    shape = eps.shape[2:]
    xi = _xi_stack(grid, shape[-3:])
    eh = fourier.forward(eps)
    w = np.einsum("ij...,j...->i...", eh, xi)
    q = np.einsum("a...,a...->...", xi, xi)
    qs = np.where(q > 0, q, 1.0)
    s = np.einsum("i...,i...->...", xi, w)
    uh = -1j * (2.0 * w - xi * s / qs) / qs
    uh = np.where(q == 0, 0.0, uh)
    return fourier.inverse(uh).real


def strain_from_displacement(u, grid):
    """e_y(u) = sym grad_y u computed spectrally: i sym(xi (x) u_hat)."""
    shape = u.shape[1:]
    xi = _xi_stack(grid, shape[-3:])
    uh = fourier.forward(u)
    eh = 0.5j * (np.einsum("i...,j...->ij...", xi, uh) + np.einsum("i...,j...->ij...", uh, xi))
    return fourier.inverse(eh).real


def theta_hat(g_hat, grid):
    """theta_hat(xi) = i/|xi|^4 [ (xi (x) xi)(g_hat . xi) - (g_hat (x) xi + xi (x) g_hat)|xi|^2 ].

    Zero where the discrete wave vector vanishes.
    """
    shape = g_hat.shape[1:]
    xi = _xi_stack(grid, shape[-3:])
    q = np.einsum("a...,a...->...", xi, xi)
    qs = np.where(q > 0, q, 1.0)
    gx = np.einsum("i...,i...->...", g_hat, xi)
    xx = np.einsum("i...,j...->ij...", xi, xi)
    gxs = np.einsum("i...,j...->ij...", g_hat, xi) + np.einsum("i...,j...->ij...", xi, g_hat)
    th = 1j / qs ** 2 * (xx * gx - gxs * q)
    return np.where(q == 0, 0.0, th)


def rhs_order_alpha(problem, p, g):
    """eps_0 = -Gamma0 * (p_alpha + theta_alpha) (Sec. 3, modified initialization)."""
    ph = fourier.forward(p)
    th = theta_hat(fourier.forward(g), problem.grid)
    return fourier.inverse(green_apply(ph + th, problem.grid, problem.lam0, problem.mu0)).real


def sym_outer_vec_dir(v, k):
    """sym(v (x) e_k) for a vector field v (3, ...)."""
    t = np.zeros((3, 3) + v.shape[1:])
    for i in range(3):
        t[i, k] = t[i, k] + 0.5 * v[i]
        t[k, i] = t[k, i] + 0.5 * v[i]
    return t


class Hierarchy:
    """Solves alpha = 1, 2, 3 for all unit loads of one RVE with the oracle CG."""

    def __init__(self, problem, tol=1e-12):
        self.pb = problem
        self.tol = tol

    def _solve(self, b):
        eps, _, _ = self.pb.cg(b, self.tol)
        return eps

    def order1(self):
        """alpha = 1: strain, displacement and stress correctors; C_eff (6x6 Mandel)."""
        pb = self.pb
        self.eps1, self.chi, self.sig1 = [], [], []
        cols = []
        for a in range(6):
            E = unit_mandel_load(a)
            eps = self._solve(pb.rhs(E))
            ebig = np.broadcast_to(E[:, :, None, None, None], eps.shape)
            sig = pb.stress(eps + ebig)
            self.eps1.append(eps)
            self.chi.append(displacement_from_strain(eps, pb.grid))
            self.sig1.append(sig)
            cols.append(tensor_to_mandel(sig.reshape(3, 3, -1).mean(axis=-1)))
        self.c_eff = np.stack(cols, axis=1)
        return self.c_eff

    def p2_g2(self, a, k):
        pb = self.pb
        p = pb.stress(sym_outer_vec_dir(self.chi[a], k))
        g = self.sig1[a][:, k].copy()
        return p, g

    def order2(self):
        """alpha = 2 for the 18 loads E^A Y_k; returns D_1 (6 x 18 Mandel)."""
        pb = self.pb
        self.eps2, self.u2, self.s2 = {}, {}, {}
        cols = []
        for a in range(6):
            for k in range(3):
                p, g = self.p2_g2(a, k)
                eps = self._solve(rhs_order_alpha(pb, p, g))
                s = pb.stress(eps) + p
                self.eps2[(a, k)] = eps
                self.u2[(a, k)] = displacement_from_strain(eps, pb.grid)
                self.s2[(a, k)] = s
                cols.append(tensor_to_mandel(s.reshape(3, 3, -1).mean(axis=-1)))
        self.d1 = np.stack(cols, axis=1)
        return self.d1

    def p3_g3(self, a, pair):
        pb = self.pb
        k, l = MANDEL_PAIRS[pair]
        w = 1.0 / (1.0 + (k == l))
        e = sym_outer_vec_dir(self.u2[(a, k)], l) + sym_outer_vec_dir(self.u2[(a, l)], k)
        p = pb.stress(w * e)
        g = w * (self.s2[(a, k)][:, l] + self.s2[(a, l)][:, k])
        return p, g

    def order3(self):
        """alpha = 3 for the 36 loads E^A Y_k Y_l / (1 + d_kl); returns D_2 (6 x 36 Mandel)."""
        pb = self.pb
        self.eps3, self.u3, self.s3 = {}, {}, {}
        cols = []
        for a in range(6):
            for pair in range(6):
                p, g = self.p3_g3(a, pair)
                eps = self._solve(rhs_order_alpha(pb, p, g))
                self.eps3[(a, pair)] = eps
                s = pb.stress(eps) + p
                self.u3[(a, pair)] = displacement_from_strain(eps, pb.grid)
                self.s3[(a, pair)] = s
                cols.append(tensor_to_mandel(s.reshape(3, 3, -1).mean(axis=-1)))
        self.d2 = np.stack(cols, axis=1)
        return self.d2


# --- any order alpha >= 2, from the Definition with exact monomial loads -------------------
#
# A unit load of order alpha is E(Y) = E^A m_K(Y) with K a multiset of alpha - 1 directions and
# the monomial m_K = Y^K / K! (so that the derivative d^K m_K = 1).  With the separation ansatz
# u_beta(Y, y) = sum_J X_beta^(A,J)(y) d^J m(Y) (J over multisets of beta - 1 directions), the
# polarization and body force of the Definition,
#     p_alpha = C : e_Y(u_{alpha-1}),   g_alpha = div_Y [C : e_y(u_{alpha-1}) + p_{alpha-1}],
# become sums over the order-(alpha-1) correctors with the coefficients d_j d^J m_K, which are
# numbers because m_K has degree alpha - 1.  The coefficients are computed by differentiating
# the monomial, not from a table of which J and j pair up.

def multisets(size):
    """Multisets of `size` directions from {0, 1, 2} as sorted tuples, in lexicographic order
    (the unit-load order of alpha = size + 1 >= 4)."""
    out = []

    def rec(prefix, start):
        if len(prefix) == size:
            out.append(tuple(prefix))
            return
        for d in range(start, 3):
            rec(prefix + [d], d)

    rec([], 0)
    return out


def monomial(K):
    """m_K = Y^K / K! as (exponents, coefficient)."""
    e = [K.count(d) for d in range(3)]
    c = 1.0
    for n in e:
        for i in range(2, n + 1):
            c /= i
    return e, c


def derivative_value(mono, dirs):
    """d^dirs m as a number, for a monomial whose degree equals len(dirs) (else None if the
    result still depends on Y, 0.0 if it vanishes)."""
    e, c = list(mono[0]), mono[1]
    for d in dirs:
        if e[d] == 0:
            return 0.0
        c *= e[d]
        e[d] -= 1
    return c if sum(e) == 0 else None


def load_key(alpha, K):
    """Dictionary key of the unit load (A fixed) of order alpha for the sorted multiset K."""
    if alpha == 1:
        return ()
    return tuple(sorted(K))


class GeneralHierarchy:
    """Orders alpha >= 2 for all unit loads from the order-1 correctors of a ``Hierarchy``
    (paper numbering; the C-ABI's order is alpha - 1)."""

    def __init__(self, base):
        self.base = base
        pb = base.pb
        # order-1 displacement correctors and stresses, keyed by (A, ())
        self.U = {1: {(a, ()): base.chi[a] for a in range(6)}}
        self.S = {1: {(a, ()): base.sig1[a] for a in range(6)}}
        self.eps, self.D = {}, {}
        self.pb = pb

    def loads(self, alpha):
        return multisets(alpha - 1)

    def solve(self, alpha):
        """Solves order alpha (needs alpha - 1); returns D[alpha] (6 x 6 * n_K Mandel), columns
        ordered A-major over ``loads(alpha)``."""
        pb = self.pb
        U, S = self.U[alpha - 1], self.S[alpha - 1]
        Js = multisets(alpha - 2)
        self.U[alpha], self.S[alpha], self.eps[alpha] = {}, {}, {}
        cols = []
        for a in range(6):
            for K in self.loads(alpha):
                m = monomial(K)
                p = np.zeros((3, 3) + pb.phase.shape)
                g = np.zeros((3,) + pb.phase.shape)
                for J in Js:
                    for j in range(3):
                        c = derivative_value(m, list(J) + [j])
                        if not c:
                            continue
                        p += c * pb.stress(sym_outer_vec_dir(U[(a, J)], j))
                        g += c * S[(a, J)][:, j]
                eps = self.base._solve(rhs_order_alpha(pb, p, g))
                s = pb.stress(eps) + p
                self.eps[alpha][(a, K)] = eps
                self.U[alpha][(a, K)] = displacement_from_strain(eps, pb.grid)
                self.S[alpha][(a, K)] = s
                cols.append(tensor_to_mandel(s.reshape(3, 3, -1).mean(axis=-1)))
        self.D[alpha] = np.stack(cols, axis=1)
        return self.D[alpha]
