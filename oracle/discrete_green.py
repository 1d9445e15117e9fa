"""Oracle of a discrete Green operator: the rotated finite-difference scheme (test infrastructure;
see ``oracle/__init__``).

Sec. 1 of arXiv:1712.05145 places the method among the FFT-based schemes, among them the
variational scheme of Brisard and Dormieux, whose point is to replace the continuous Green
operator Gamma0_hat of Sec. 2 by one that belongs to a discretisation.  This module states one
such discretisation and derives its Green operator.

Discretisation.  Displacements live at the voxel corners (grid points n h), strains, stresses and
the material at the voxel centres (n + 1/2) h.  The derivative along y_j at a voxel centre is the
difference of u across the voxel along j, averaged over the four voxel edges parallel to y_j:

    (D_j u)(n) = 1/(4h) sum_{s in {0,1}^3, s_j = 0} [ u(n + s + e_j) - u(n + s) ],
    eps(u) = sym(D u)                                       (one strain per voxel)

and the discrete cell problem asks for periodic corner displacements u with

    D^T C : (E + eps(u)) = 0,

the stationarity of the voxel-summed energy of Sec. 2 over u.

Fourier symbol.  For a corner mode u(n) = u_hat exp(i xi . n h) the average of the edge
differences gives (D_j u)(n) = u_hat exp(i xi . (n + 1/2) h) (2 i / h) q_j(xi) with

    q_j(xi) = sin(xi_j h / 2) prod_{l != j} cos(xi_l h / 2)

(each edge pair contributes a factor 2 cos(xi_l h/2) exp(i xi_l h/2), the difference a factor
2 i sin(xi_j h/2) exp(i xi_j h/2)).  The factor (2 i / h) exp(i xi . h/2) is the same for every
j.  With the reference medium C0 and tau = (C - C0) : (E + eps), the problem reads
D^T C0 D u = -D^T tau, so eps = -Gamma^R * tau with

    Gamma^R_hat(xi) = D_hat (D_hat^* C0 D_hat)^-1 D_hat^* = Gamma0_hat(q(xi)),

the four-index formula of Sec. 2 evaluated at the real vector q instead of xi (it is homogeneous of
degree 0, so the common factor drops out), and Gamma^R_hat = 0 wherever q = 0 (the mean mode and,
on even grids, the frequencies with two or more Nyquist components, whose displacement modes
produce no strain).  q is odd in xi, so Gamma^R_hat is even and the operator is real; at a single
Nyquist component it is defined without any convention (q then points along that axis).

Pins (tests/test_oracle_discrete_green.py): the solution of the Lippmann-Schwinger equation with
Gamma^R equals the strain of a dense real-space solve of D^T C (E + D u) = 0 assembled from the
difference stencil above; Gamma^R_hat : C0 : Gamma^R_hat = Gamma^R_hat at every frequency; a voxel
laminate of any layer thicknesses gives the exact laminate stiffness; the solution does not depend
on C0.
"""
import numpy as np

from . import fourier
from .lippmann_schwinger import Problem, gamma0_hat_slab
from .tensors import MANDEL_PAIRS, MANDEL_W, iso_mandel_matrix, lame_fields


def rotated_vectors(grid):
    """(q1, q2, q3) of the rotated scheme, broadcastable to (N3, N2, N1) (h = 1/max N).

    theta_j = xi_j h / 2 = pi k_j / N_j with the signed integer frequency k_j (fourier.frequencies);
    the factor 2/h of the symbol is dropped (Gamma0_hat is homogeneous of degree 0 in its vector).
    """
    def sc(n):
        k = fourier.frequencies(n)
        t = np.pi * k / n
        c = np.where(2 * np.abs(k) == n, 0.0, np.cos(t))   # exactly 0 at the Nyquist index
        return np.sin(t), c

    (s1, c1), (s2, c2), (s3, c3) = sc(grid[0]), sc(grid[1]), sc(grid[2])
    s1, c1 = s1[None, None, :], c1[None, None, :]
    s2, c2 = s2[None, :, None], c2[None, :, None]
    s3, c3 = s3[:, None, None], c3[:, None, None]
    return s1 * c2 * c3, c1 * s2 * c3, c1 * c2 * s3


def green_apply_rotated(tau_hat, grid, lam0, mu0):
    """eta_hat = -Gamma^R_hat(xi) : tau_hat(xi), zero where q(xi) = 0.

    ``tau_hat`` has shape (3, 3, ..., N3, N2, N1); leading batch axes are allowed.
    """
    q1, q2, q3 = rotated_vectors(grid)
    q1, q2, q3 = np.broadcast_arrays(q1, q2, q3)
    out = np.zeros_like(tau_hat)
    n3 = tau_hat.shape[-3]
    for z in range(n3):
        g = gamma0_hat_slab(q1[z], q2[z], q3[z], lam0, mu0)          # (3,3,3,3,N2,N1)
        out[..., z, :, :] = -np.einsum("ijklyx,kl...yx->ij...yx", g, tau_hat[..., z, :, :])
    return out


class RotatedProblem(Problem):
    """The RVE of ``Problem`` with the rotated finite-difference Green operator in every LS step,
    so its Basic Scheme and CG solve the discrete cell problem of the rotated scheme."""

    def green(self, tau_hat):
        return green_apply_rotated(tau_hat, self.grid, self.lam0, self.mu0)


def difference_matrix(grid):
    """Dense matrix of the voxel-centre strain (Mandel, order [component][voxel]) of periodic corner
    displacements (order [direction][corner], corners indexed like the voxel at their + side),
    built stencil by stencil from the averaged edge differences: shape (6 M, 3 M), h = 1/max N."""
    n1, n2, n3 = grid
    m = n1 * n2 * n3
    h = 1.0 / max(grid)

    def vid(x, y, z):
        return (z % n3) * n2 * n1 + (y % n2) * n1 + (x % n1)

    # G[j][d] : derivative d/dy_j of displacement component d, shape (M, 3M)
    grad = np.zeros((3, 3, m, 3 * m))
    for z in range(n3):
        for y in range(n2):
            for x in range(n1):
                v = vid(x, y, z)
                for j in range(3):
                    for s in np.ndindex(2, 2, 2):
                        if s[j] != 0:
                            continue
                        a = [x + s[0], y + s[1], z + s[2]]
                        b = list(a)
                        b[j] += 1
                        for d in range(3):
                            grad[j, d, v, d * m + vid(*b)] += 1.0 / (4 * h)
                            grad[j, d, v, d * m + vid(*a)] -= 1.0 / (4 * h)
    D = np.zeros((6 * m, 3 * m))
    for comp, (i, j) in enumerate(MANDEL_PAIRS):
        sym = 0.5 * (grad[j, i] + grad[i, j])           # sym(D u)_ij
        D[comp * m:(comp + 1) * m] = MANDEL_W[comp] * sym
    return D


def real_space_solution(phase, lame_table, E_mandel):
    """Strain (Mandel, shape (6, N3, N2, N1)) of the discrete cell problem D^T C (E + D u) = 0,
    assembled in real space and solved densely (least squares: the displacement is defined up to
    translations and the strain-free corner modes, the strain is unique)."""
    phase = np.asarray(phase)
    n3, n2, n1 = phase.shape
    m = phase.size
    D = difference_matrix((n1, n2, n3))
    lam, mu = lame_fields(phase, lame_table)
    C = np.zeros((6 * m, 6 * m))
    lam, mu = lam.reshape(-1), mu.reshape(-1)
    for v in range(m):
        cv = iso_mandel_matrix(lam[v], mu[v])
        idx = np.arange(6) * m + v
        C[np.ix_(idx, idx)] = cv
    Ebig = np.repeat(np.asarray(E_mandel, dtype=float), m)
    K = D.T @ C @ D
    f = -D.T @ (C @ Ebig)
    u = np.linalg.lstsq(K, f, rcond=None)[0]
    return (D @ u).reshape(6, n3, n2, n1)
