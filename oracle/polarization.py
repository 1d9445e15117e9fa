"""Oracle polarization scheme (test infrastructure; see ``oracle/__init__``).

The paper cites, besides the Basic Scheme, the polarization scheme of Monchiet and Bonnet and
the augmented-Lagrangian scheme of Michel, Moulinec and Suquet as FFT-based solvers of the same
cell problem (Sec. 1).  For linear elasticity both are fixed-point iterations on a
"polarization-like" variable built from the Lippmann-Schwinger data of Sec. 2; this module
derives them from the LS system A eps = b (Eq. cg_form) as follows.

For a zero-mean compatible eps, A eps = Gamma0 * (C : eps) (Gamma0 * C0 is the identity there),
so the problem reads: eps compatible with P(C0^-1 C : eps) = b, P = Gamma0 * C0 the
C0-orthogonal projection onto zero-mean compatible fields and b itself compatible.  Write
    x = 1/2 C0^-1 (C + C0) : eps,   y = 1/2 C0^-1 (C - C0) : eps,   so   eps = x - y,
    C0^-1 C : eps = x + y,   y = W x  with  W = (C - C0) (C + C0)^-1  (pointwise).
The two conditions P(x - y) = x - y and P(x + y) = b combine to
    x = b + Y W x,   Y = I - 2 P = I - 2 Gamma0 * C0,
a fixed point of T(x) = b + Y W x.  Y is an isometry and |W| <= max |(c - c0) / (c + c0)| < 1
in the C0 energy norm (C0 positive, every phase stiffness positive), so T contracts:
    relax = 1    x <- T(x)                          (the Eyre-Milton / Monchiet-Bonnet scheme)
    relax = 1/2  x <- (x + T(x)) / 2                (the averaged, augmented-Lagrangian form)
and eps = (I - W) x at the fixed point.  The stopping quantity is the Cauchy difference of the
strain, ||(I - W)(x_{n+1} - x_n)||_L2 / ||b||_L2.

W is formed per phase as the 6x6 Mandel product (C_p - C0) inv(C_p + C0) (numpy inverse), an
independent route from any eigenvalue formula.

Pins (tests/test_oracle_polarization.py): the fixed point equals the dense-LU solution of A on
tiny grids for both relaxations; each step contracts the C0-norm error by at most
max |(c - c0)/(c + c0)| (relax = 1); with the geometric-mean reference at contrast 100 the
scheme needs far fewer iterations than the Basic Scheme; the averaged form converges at
contrast 1e4.
"""
import numpy as np

from .tensors import iso_apply, iso_mandel_matrix, l2_norm, mandel_to_tensor, tensor_to_mandel

__all__ = ["phase_w_matrices", "apply_phase_matrix", "polarization_scheme", "contraction_factor"]


def phase_w_matrices(lame_table, lam0, mu0):
    """W_p = (C_p - C0) inv(C_p + C0) as 6x6 Mandel matrices, one per phase."""
    c0 = iso_mandel_matrix(lam0, mu0)
    out = []
    for lam, mu in np.asarray(lame_table, dtype=np.float64):
        cp = iso_mandel_matrix(lam, mu)
        out.append((cp - c0) @ np.linalg.inv(cp + c0))
    return np.stack(out)


def apply_phase_matrix(mats, phase, e):
    """(mats[phase] : e) for a (3, 3, N3, N2, N1) field, through Mandel vectors."""
    v = tensor_to_mandel(e)                          # (6, N3, N2, N1)
    per = mats[phase]                                # (N3, N2, N1, 6, 6)
    return mandel_to_tensor(np.einsum("...ab,b...->a...", per, v))


def contraction_factor(lame_table, lam0, mu0):
    """max over phases of the spectral radius of W_p (its largest |eigenvalue|)."""
    return float(max(np.max(np.abs(np.linalg.eigvals(w))) for w in phase_w_matrices(lame_table, lam0, mu0)))


def polarization_scheme(problem, lame_table, b, relax=1.0, tol=1e-12, max_iter=100000, record=None):
    """Fixed point x = b + (I - 2 Gamma0 * C0) W x, relaxed by `relax`; returns (eps, iterations,
    history of the Cauchy quantity).  `record`, if a list, receives every iterate x_n."""
    W = phase_w_matrices(lame_table, problem.lam0, problem.mu0)
    I_minus_W = np.eye(6)[None] - W
    nb = l2_norm(b)
    x = b.copy()
    hist = []
    if record is not None:
        record.append(x.copy())
    if nb == 0.0:
        return apply_phase_matrix(I_minus_W, problem.phase, x), 0, hist
    for it in range(1, max_iter + 1):
        y = apply_phase_matrix(W, problem.phase, x)                            # y = W x
        # Y y = y - 2 Gamma0 * (C0 : y); minus_gamma_conv gives -Gamma0 * (.)
        Yy = y + 2.0 * problem.minus_gamma_conv(iso_apply(problem.lam0, problem.mu0, y))
        x_new = (1.0 - relax) * x + relax * (b + Yy)
        crit = l2_norm(apply_phase_matrix(I_minus_W, problem.phase, x_new - x)) / nb
        hist.append(crit)
        x = x_new
        if record is not None:
            record.append(x.copy())
        if crit < tol:
            return apply_phase_matrix(I_minus_W, problem.phase, x), it, hist
    raise RuntimeError("polarization scheme did not converge: %g" % hist[-1])
