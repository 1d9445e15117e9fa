"""Pins of the oracle's tensor algebra (oracle/tensors.py) against definitions written out
index by index and against textbook facts of isotropic elasticity (Sec. 2, Hooke's law and the
reference stiffness C0).  A consistent sqrt(2) slip shared by the Mandel conversions and the
6x6 matrix would survive a round trip; it fails the Frobenius and eigenvalue pins here."""
import numpy as np

from oracle.tensors import (c0_inner, ddot, iso_apply, iso_mandel_matrix, iso_stiffness_4, l2_norm,
                            mandel_to_tensor, tensor_to_mandel, unit_mandel_load)


def _random_sym(rng, extra=()):
    a = rng.uniform(-1, 1, size=(3, 3) + extra)
    return 0.5 * (a + np.swapaxes(a, 0, 1))


def _frobenius_loops(a, b):
    s = 0.0
    for i in range(3):
        for j in range(3):
            s += a[i, j] * b[i, j]
    return s


def _contract_loops(C, e):
    """sigma_ij = sum_kl C_ijkl e_kl, written out."""
    out = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    out[i, j] += C[i, j, k, l] * e[k, l]
    return out


def _hooke_explicit(lam, mu, e):
    """lambda tr(e) I + 2 mu e with the trace and the identity spelled out."""
    tr = e[0, 0] + e[1, 1] + e[2, 2]
    out = np.empty((3, 3))
    for i in range(3):
        for j in range(3):
            out[i, j] = 2.0 * mu * e[i, j] + (lam * tr if i == j else 0.0)
    return out


def test_mandel_round_trip_and_symmetric_part():
    rng = np.random.default_rng(0)
    v = rng.uniform(-1, 1, size=(6, 4, 3))
    assert np.allclose(tensor_to_mandel(mandel_to_tensor(v)), v, atol=1e-15)
    a = rng.uniform(-1, 1, size=(3, 3))             # not symmetric
    t = mandel_to_tensor(tensor_to_mandel(a))
    assert np.allclose(t, 0.5 * (a + a.T), atol=1e-15)


def test_mandel_vectors_carry_the_frobenius_product():
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = _random_sym(rng), _random_sym(rng)
        assert abs(float(tensor_to_mandel(a) @ tensor_to_mandel(b)) - _frobenius_loops(a, b)) < 1e-14
    # the off-diagonal entries: e12 = e21 = 1 has |e|^2 = 2, so its Mandel component is sqrt(2)
    e = np.zeros((3, 3))
    e[0, 1] = e[1, 0] = 1.0
    m = tensor_to_mandel(e)
    assert np.allclose(m, [0, 0, 0, 0, 0, np.sqrt(2.0)], atol=1e-15)


def test_unit_loads_are_orthonormal_tensors():
    loads = [unit_mandel_load(a) for a in range(6)]
    gram = np.array([[_frobenius_loops(p, q) for q in loads] for p in loads])
    assert np.allclose(gram, np.eye(6), atol=1e-15)
    for a, t in enumerate(loads):
        assert np.allclose(t, t.T)
        assert np.allclose(tensor_to_mandel(t), np.eye(6)[a], atol=1e-15)


def test_four_index_stiffness_is_hookes_law():
    rng = np.random.default_rng(2)
    lam, mu = 1.7, 0.6
    C = iso_stiffness_4(lam, mu)
    for _ in range(5):
        e = _random_sym(rng)
        assert np.allclose(_contract_loops(C, e), _hooke_explicit(lam, mu, e), atol=1e-14)
    # major and minor symmetries
    assert np.allclose(C, np.transpose(C, (1, 0, 2, 3)))
    assert np.allclose(C, np.transpose(C, (0, 1, 3, 2)))
    assert np.allclose(C, np.transpose(C, (2, 3, 0, 1)))


def test_iso_apply_matches_explicit_hooke_per_voxel():
    rng = np.random.default_rng(3)
    e = _random_sym(rng, (2, 3, 4))
    lam = rng.uniform(0.1, 5, size=(2, 3, 4))
    mu = rng.uniform(0.1, 5, size=(2, 3, 4))
    got = iso_apply(lam, mu, e.copy())
    for idx in np.ndindex(2, 3, 4):
        ref = _hooke_explicit(lam[idx], mu[idx], e[(slice(None), slice(None)) + idx])
        assert np.allclose(got[(slice(None), slice(None)) + idx], ref, atol=1e-14)


def test_mandel_matrix_acts_like_the_tensor_and_has_kelvin_moduli():
    rng = np.random.default_rng(4)
    lam, mu = 2.3, 0.9
    c = iso_mandel_matrix(lam, mu)
    for _ in range(5):
        e = _random_sym(rng)
        assert np.allclose(c @ tensor_to_mandel(e), tensor_to_mandel(_hooke_explicit(lam, mu, e)), atol=1e-14)
    # Kelvin's eigen-decomposition of an isotropic stiffness: 3K once (hydrostatic), 2 mu five times
    ev = np.sort(np.linalg.eigvalsh(c))
    K = lam + 2.0 * mu / 3.0
    assert np.allclose(ev, np.sort([3 * K, 2 * mu, 2 * mu, 2 * mu, 2 * mu, 2 * mu]), atol=1e-13)


def test_textbook_special_cases():
    lam, mu = 1.5, 0.75
    K = lam + 2.0 * mu / 3.0
    # hydrostatic strain eps I: stress 3 K eps I
    e = 0.01 * np.eye(3)
    assert np.allclose(iso_apply(lam, mu, e.copy()), 3 * K * e, atol=1e-15)
    # engineering shear gamma (e12 = e21 = gamma / 2): shear stress mu gamma
    g = 0.02
    e = np.zeros((3, 3))
    e[0, 1] = e[1, 0] = g / 2
    s = iso_apply(lam, mu, e.copy())
    assert abs(s[0, 1] - mu * g) < 1e-15 and abs(s[0, 0]) < 1e-15
    # uniaxial stress: with E = mu (3 lam + 2 mu) / (lam + mu) and nu = lam / (2 (lam + mu)),
    # eps = diag(1, -nu, -nu) / E gives sigma = diag(1, 0, 0)
    Ey = mu * (3 * lam + 2 * mu) / (lam + mu)
    nu = lam / (2 * (lam + mu))
    e = np.diag([1.0, -nu, -nu]) / Ey
    assert np.allclose(iso_apply(lam, mu, e.copy()), np.diag([1.0, 0.0, 0.0]), atol=1e-14)


def test_c0_inner_is_the_mean_of_a_C0_b():
    rng = np.random.default_rng(5)
    lam0, mu0 = 3.0, 1.25
    a = _random_sym(rng, (2, 2, 3))
    b = _random_sym(rng, (2, 2, 3))
    C0 = iso_stiffness_4(lam0, mu0)
    vals = []
    for idx in np.ndindex(2, 2, 3):
        sl = (slice(None), slice(None)) + idx
        vals.append(_frobenius_loops(a[sl], _contract_loops(C0, b[sl])))
    assert abs(c0_inner(a, b, lam0, mu0) - np.mean(vals)) < 1e-14
    # symmetric and positive on nonzero fields
    assert abs(c0_inner(a, b, lam0, mu0) - c0_inner(b, a, lam0, mu0)) < 1e-14
    assert c0_inner(a, a, lam0, mu0) > 0


def test_l2_norm_and_ddot():
    rng = np.random.default_rng(6)
    a = _random_sym(rng, (3, 2))
    vals = [_frobenius_loops(a[:, :, i, j], a[:, :, i, j]) for i in range(3) for j in range(2)]
    assert abs(l2_norm(a) - np.sqrt(np.mean(vals))) < 1e-14
    assert np.allclose(ddot(a, a), np.reshape(vals, (3, 2)), atol=1e-14)
