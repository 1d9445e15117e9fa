"""Oracle Lippmann-Schwinger operator and solvers (test infrastructure; see ``oracle/__init__``).

Follows Sec. 2 of arXiv:1712.05145 in its notation:

* polarization  tau = (C - C0) : eps + C : E                (Eq. auxiliary_problem)
* LS equation   eps = -Gamma0 * tau, a Fourier series over xi != 0 (Eq. strain_solution)
* Green operator, four-index closed form for xi != 0:
      Gamma0_hat_ijkl = (d_ki xi_l xi_j + d_li xi_k xi_j + d_kj xi_l xi_i + d_lj xi_k xi_i)
                        / (4 mu0 |xi|^2)
                        - (lam0 + mu0) / (mu0 (lam0 + 2 mu0)) xi_i xi_j xi_k xi_l / |xi|^4
* CG form  (Id + Gamma0 * (C - C0)) : eps = -Gamma0 * (C : E)   (Eq. cg_form), A eps = b
* Algorithm 1 (Basic Scheme, CG version) and the Cauchy criterion
  ||eps_{n+1} - eps_n||_L2 / ||eps_0||_L2 < TOL that follows it.

Readings of the paper taken here:

* Algorithm 1's loop body (polarization, transform, -Gamma0_hat contraction with the
  zero mode set to 0, inverse transform, eps_n - eta_n) is the application A eps_n.
  The Basic Scheme is the unit-step fixed point eps_{n+1} = eps_n + (b - A eps_n)
  (Moulinec-Suquet); for it eps_{n+1} - eps_n = b - A eps_n, so the paper's Cauchy
  quantity is the relative residual ||b - A eps||/||b||, used for every solver.
* The CG version runs CG on A eps = b.  A is self-adjoint on compatible fields in the
  C0-weighted product <a, b>_C0 = mean(a : C0 : b), which this CG uses (for lam0 = 0
  it is the plain L2 product up to the factor 2 mu0).

Pins (tests/test_oracle_ls.py): Gamma0_hat : C0 : Gamma0_hat = Gamma0_hat, major and
minor symmetry, mean annihilation, C = C0 and constant C give eps = 0, the exact
laminate stiffness, Voigt/Reuss bounds, the Hashin-Shtrikman bulk bounds, symmetry of
C_eff, and agreement of the Basic Scheme and CG with a dense LU solve of A.
"""
import numpy as np

from . import fourier
from .tensors import (iso_apply, lame_fields, mandel_to_tensor, tensor_to_mandel,
                      unit_mandel_load, c0_inner, l2_norm)


def gamma0_hat_slab(xi1, xi2, xi3, lam0, mu0):
    """Gamma0_hat_ijkl on a set of frequencies (arrays of equal shape); 0 where xi = 0."""
    xi = np.stack(np.broadcast_arrays(xi1, xi2, xi3)).astype(np.float64)
    q = np.einsum("a...,a...->...", xi, xi)
    nz = q > 0
    qs = np.where(nz, q, 1.0)
    d = np.eye(3)
    sym4 = (np.einsum("ki,l...,j...->ijkl...", d, xi, xi)
            + np.einsum("li,k...,j...->ijkl...", d, xi, xi)
            + np.einsum("kj,l...,i...->ijkl...", d, xi, xi)
            + np.einsum("lj,k...,i...->ijkl...", d, xi, xi))
    xxxx = np.einsum("i...,j...,k...,l...->ijkl...", xi, xi, xi, xi)
    c = (lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0))
    g = sym4 / (4.0 * mu0 * qs) - c * xxxx / qs ** 2
    return np.where(nz, g, 0.0)


def green_apply(tau_hat, grid, lam0, mu0):
    """eta_hat = -Gamma0_hat(xi) : tau_hat(xi) for xi != 0, eta_hat(0) = 0.

    xi is the discrete wave vector (Nyquist components 0, see ``fourier.wavevectors``),
    so the multiplier is Hermitian and Gamma0_hat : C0 : Gamma0_hat = Gamma0_hat holds at
    every frequency; it also vanishes at the pure-Nyquist frequencies.

    ``tau_hat`` has shape (3, 3, ..., N3, N2, N1); leading batch axes are allowed.
    """
    xi1, xi2, xi3 = fourier.wavevectors(grid)
    out = np.zeros_like(tau_hat)
    n3 = tau_hat.shape[-3]
    for z in range(n3):
        g = gamma0_hat_slab(xi1[0], xi2[0], xi3[z], lam0, mu0)       # (3,3,3,3,N2,N1)
        out[..., z, :, :] = -np.einsum("ijklyx,kl...yx->ij...yx", g, tau_hat[..., z, :, :])
    return out


class Problem:
    """A voxel RVE: grid (N1, N2, N3), per-voxel isotropic phases and reference C0."""

    def __init__(self, phase, lame_table, lam0, mu0):
        self.phase = np.asarray(phase)
        n3, n2, n1 = self.phase.shape
        self.grid = (n1, n2, n3)
        self.lam, self.mu = lame_fields(self.phase, lame_table)
        self.lam0 = float(lam0)
        self.mu0 = float(mu0)

    # --- Sec. 2 building blocks -------------------------------------------------
    def stress(self, e):
        """C : e, Hooke's law with the local stiffness (Eq. Hookes_law)."""
        return iso_apply(self.lam, self.mu, e)

    def polarization(self, eps, E):
        """tau = (C - C0) : eps + C : E (Eq. auxiliary_problem)."""
        tau = iso_apply(self.lam - self.lam0, self.mu - self.mu0, eps)
        if E is not None:
            ebig = np.broadcast_to(E.reshape(E.shape + (1,) * (eps.ndim - 2)), eps.shape)
            tau = tau + iso_apply(self.lam, self.mu, ebig)
        return tau

    def green(self, tau_hat):
        """eta_hat = -Gamma0_hat : tau_hat with eta_hat(0) = 0 (the Green operator of Sec. 2)."""
        return green_apply(tau_hat, self.grid, self.lam0, self.mu0)

    def minus_gamma_conv(self, tau):
        """-Gamma0 * tau as the Fourier series of Eq. strain_solution (real field)."""
        eta_hat = self.green(fourier.forward(tau))
        return fourier.inverse(eta_hat).real

    def ls_step(self, eps, E):
        """One Lippmann-Schwinger step: -Gamma0 * [(C - C0) : eps + C : E]."""
        return self.minus_gamma_conv(self.polarization(eps, E))

    def rhs(self, E):
        """b = -Gamma0 * (C : E), the right-hand side of Eq. cg_form (Algorithm 1 INIT)."""
        zero = np.zeros((3, 3) + self.phase.shape)
        return self.ls_step(zero, E)

    def apply_A(self, eps):
        """A eps = (Id + Gamma0 * (C - C0)) : eps, via Algorithm 1's loop body."""
        tau = iso_apply(self.lam - self.lam0, self.mu - self.mu0, eps)     # polarization
        tau_hat = fourier.forward(tau)                                      # transform
        eta_hat = self.green(tau_hat)                                       # -Gamma0_hat, eta(0)=0
        eta = fourier.inverse(eta_hat).real                                 # inverse transform
        return eps - eta                                                    # eps_n - eta_n

    def c0_inner(self, a, b):
        return c0_inner(a, b, self.lam0, self.mu0)

    # --- solvers ----------------------------------------------------------------
    def basic_scheme(self, b, tol=1e-12, max_iter=100000):
        """Unit-step fixed point on A eps = b from eps_0 = b (Algorithm 1 + Cauchy criterion).

        Returns (eps, iterations, history of the Cauchy quantity).
        """
        nb = l2_norm(b)
        eps = b.copy()
        hist = []
        if nb == 0.0:
            return eps, 0, hist
        for it in range(1, max_iter + 1):
            eps_new = eps + (b - self.apply_A(eps))
            crit = l2_norm(eps_new - eps) / nb
            hist.append(crit)
            eps = eps_new
            if crit < tol:
                return eps, it, hist
        raise RuntimeError("basic scheme did not converge: %g" % hist[-1])

    def cg(self, b, tol=1e-12, max_iter=100000, x0=None):
        """CG on A eps = b in the C0 inner product; stops at ||b - A eps||/||b|| < tol."""
        nb = l2_norm(b)
        x = np.zeros_like(b) if x0 is None else x0.copy()
        r = b - self.apply_A(x) if x0 is not None else b.copy()
        hist = []
        if nb == 0.0:
            return x, 0, hist
        p = r.copy()
        rho = self.c0_inner(r, r)
        for it in range(1, max_iter + 1):
            q = self.apply_A(p)
            alpha = rho / self.c0_inner(p, q)
            x = x + alpha * p
            r = r - alpha * q
            res = l2_norm(r) / nb
            hist.append(res)
            if res < tol:
                return x, it, hist
            rho_new = self.c0_inner(r, r)
            p = r + (rho_new / rho) * p
            rho = rho_new
        raise RuntimeError("cg did not converge: %g" % hist[-1])

    def residual(self, eps, b):
        """||b - A eps||_L2 / ||b||_L2."""
        return l2_norm(b - self.apply_A(eps)) / l2_norm(b)

    # --- effective quantities ---------------------------------------------------
    def mean_stress(self, eps, E):
        """<sigma> = <C : (eps + E)> as a Mandel 6-vector."""
        ebig = np.broadcast_to(E.reshape(E.shape + (1,) * (eps.ndim - 2)), eps.shape)
        sig = self.stress(eps + ebig)
        return tensor_to_mandel(sig.reshape(3, 3, -1).mean(axis=-1))

    def solve_order0(self, tol=1e-12, scheme="cg", loads=None):
        """Solve the 6 Mandel unit loads (or the given 3x3 loads); returns (eps list, C_eff)."""
        if loads is None:
            loads = [unit_mandel_load(a) for a in range(6)]
        sols = []
        cols = []
        for E in loads:
            b = self.rhs(E)
            if scheme == "cg":
                eps, _, _ = self.cg(b, tol)
            else:
                eps, _, _ = self.basic_scheme(b, tol)
            sols.append(eps)
            cols.append(self.mean_stress(eps, E))
        return sols, np.stack(cols, axis=1)


def assemble_A_mandel(problem):
    """Dense matrix of A acting on Mandel-vector fields, shape (6M, 6M), order [comp][voxel].

    Used only on tiny grids to obtain the exact discrete solution by LU.
    """
    shape = problem.phase.shape
    m = int(np.prod(shape))
    n = 6 * m
    eye = np.eye(n).reshape(n, 6, *shape)              # batch of unit Mandel fields
    t = mandel_to_tensor(np.moveaxis(eye, 0, 1))       # (3,3,n,N3,N2,N1)
    at = problem.apply_A(t)
    return tensor_to_mandel(at).reshape(6, n, m).transpose(1, 0, 2).reshape(n, n).T
