"""Seeded synthetic microstructures (input generators shared by tests, bench and oracle callers).

This module holds no arithmetic of the homogenization method: it only draws
geometries and material tables.  Both the CUDA path and the CPU oracle receive its
output as plain arrays.

Random numbers: SplitMix64 seeds a xoshiro256** stream (both from their published
definitions by Vigna and Blackman), written here so that the same seed gives the
same microstructure on every machine and numpy version.

Geometry lives in unit-cell coordinates: voxel centres y = (n + 1/2) h - 1/2 with
cubic voxels h = 1/max(N) (the unit torus [-1/2, 1/2)^3 for cubic grids, Sec. 2), so
two resolutions of the same seed discretise the same microstructure.

Each generator returns a ``Microstructure``: ``phase`` (uint8, shape (N3, N2, N1),
x fastest), ``lame`` ((n_phase, 2) float64 of Lame lambda, mu) and the reference
medium ``(lam0, mu0)``.
"""
from dataclasses import dataclass, field
import math

import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed):
        self.state = seed & MASK64

    def next(self):
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)


def _rotl(x, k):
    return ((x << k) | (x >> (64 - k))) & MASK64


class Xoshiro256ss:
    """xoshiro256** 1.0 seeded through SplitMix64."""

    def __init__(self, seed):
        sm = SplitMix64(seed)
        self.s = [sm.next() for _ in range(4)]

    def next(self):
        s = self.s
        result = (_rotl((s[1] * 5) & MASK64, 7) * 9) & MASK64
        t = (s[1] << 17) & MASK64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
        return result

    def uniform(self, lo=0.0, hi=1.0):
        return lo + (hi - lo) * ((self.next() >> 11) * (1.0 / (1 << 53)))

    def normal(self):
        """Standard normal by the Box-Muller transform."""
        u1 = self.uniform()
        while u1 <= 0.0:
            u1 = self.uniform()
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def lame_from_young(e, nu):
    """(lambda, mu) of an isotropic material from Young's modulus and Poisson's ratio."""
    lam = e * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = e / (2.0 * (1.0 + nu))
    return lam, mu


def midpoint_reference(lame):
    """Reference medium at the midpoint of the phases' min and max Lame parameters."""
    lame = np.asarray(lame, dtype=np.float64)
    return (0.5 * (lame[:, 0].min() + lame[:, 0].max()),
            0.5 * (lame[:, 1].min() + lame[:, 1].max()))


def geometric_reference(lame):
    """Reference medium whose Kelvin moduli 3K0 and 2mu0 are the geometric means of the phases'
    smallest and largest 3K and 2mu: the choice that minimises max |(c - c0) / (c + c0)|, the
    contraction factor of the polarization scheme."""
    lame = np.asarray(lame, dtype=np.float64)
    k3 = 3.0 * lame[:, 0] + 2.0 * lame[:, 1]
    m2 = 2.0 * lame[:, 1]
    k30 = np.sqrt(k3.min() * k3.max())
    m20 = np.sqrt(m2.min() * m2.max())
    return (k30 - m20) / 3.0, 0.5 * m20


@dataclass
class Microstructure:
    phase: np.ndarray
    lame: np.ndarray
    lam0: float
    mu0: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def grid(self):
        n3, n2, n1 = self.phase.shape
        return (n1, n2, n3)

    def volume_fractions(self):
        counts = np.bincount(self.phase.ravel(), minlength=len(self.lame))
        return counts / self.phase.size


def voxel_centres(grid):
    """Unit-cell coordinates of voxel centres along each axis, (y1, y2, y3)."""
    h = 1.0 / max(grid)
    return tuple((np.arange(n) + 0.5) * h - 0.5 for n in grid)


def _cell_lengths(grid):
    h = 1.0 / max(grid)
    return np.array([n * h for n in grid])


def centred_sphere(n=32, fraction=0.2, matrix=(1.0, 1.0), inclusion=(10.0, 10.0),
                   reference="mean"):
    """One centred spherical inclusion of target volume fraction in an n^3 cube."""
    r = (3.0 * fraction / (4.0 * math.pi)) ** (1.0 / 3.0)
    y1, y2, y3 = voxel_centres((n, n, n))
    d2 = y3[:, None, None] ** 2 + y2[None, :, None] ** 2 + y1[None, None, :] ** 2
    phase = (d2 < r * r).astype(np.uint8)
    lame = np.array([matrix, inclusion], dtype=np.float64)
    if reference == "mean":
        lam0, mu0 = float(lame[:, 0].mean()), float(lame[:, 1].mean())
    else:
        lam0, mu0 = midpoint_reference(lame)
    return Microstructure(phase, lame, lam0, mu0, "centred_sphere",
                          {"radius": r, "target_fraction": fraction})


def laminate(grid=(32, 32, 32), split=None, a=(1.0, 1.0), b=(10.0, 10.0), reference="mean"):
    """Layers normal to x1: voxels with n1 < split are phase 0, the rest phase 1."""
    n1, n2, n3 = grid
    split = n1 // 2 if split is None else split
    phase = np.zeros((n3, n2, n1), dtype=np.uint8)
    phase[:, :, split:] = 1
    lame = np.array([a, b], dtype=np.float64)
    if reference == "mean":
        lam0, mu0 = float(lame[:, 0].mean()), float(lame[:, 1].mean())
    else:
        lam0, mu0 = midpoint_reference(lame)
    return Microstructure(phase, lame, lam0, mu0, "laminate", {"split": split})


def _mark_sphere(mask, grid, centre, radius):
    """Set voxels whose centre lies within ``radius`` (periodic) of ``centre``."""
    h = 1.0 / max(grid)
    lengths = _cell_lengths(grid)
    sel = []
    for ax in range(3):
        n = grid[ax]
        lo = int(math.floor((centre[ax] - radius + 0.5 * lengths[ax]) / h - 0.5)) - 1
        hi = int(math.ceil((centre[ax] + radius + 0.5 * lengths[ax]) / h - 0.5)) + 1
        idx = np.arange(lo, hi + 1)
        pos = (idx + 0.5) * h - 0.5 * lengths[ax]
        d = pos - centre[ax]
        sel.append((np.mod(idx, n), d))
    (i1, d1), (i2, d2), (i3, d3) = sel
    dist2 = d3[:, None, None] ** 2 + d2[None, :, None] ** 2 + d1[None, None, :] ** 2
    inside = dist2 < radius * radius
    z, y, x = np.nonzero(inside)
    mask[i3[z], i2[y], i1[x]] = True


def _rsa_spheres(grid, rng, rmin, rmax, targets, gap=0.0, max_attempts=2000000):
    """Random sequential addition of non-overlapping spheres (periodic minimum image).

    ``targets`` lists the target voxel fraction of each inclusion type; the type with
    the largest remaining deficit gets the next sphere.  Returns (phase, spheres).
    """
    n1, n2, n3 = grid
    lengths = _cell_lengths(grid)
    phase = np.zeros((n3, n2, n1), dtype=np.uint8)
    centres = np.zeros((0, 3))
    radii = np.zeros(0)
    spheres = []
    counts = [0] * len(targets)
    total = n1 * n2 * n3
    attempts = 0
    while True:
        deficits = [t - c / total for t, c in zip(targets, counts)]
        kind = int(np.argmax(deficits))
        if deficits[kind] <= 0:
            break
        attempts += 1
        if attempts > max_attempts:
            raise RuntimeError("RSA could not reach the target fraction")
        r = rng.uniform(rmin, rmax)
        c = np.array([rng.uniform(-0.5 * lengths[a], 0.5 * lengths[a]) for a in range(3)])
        if len(radii):
            d = centres - c
            d -= lengths * np.round(d / lengths)
            if np.any(np.sqrt((d * d).sum(axis=1)) < radii + r + gap):
                continue
        centres = np.vstack([centres, c])
        radii = np.append(radii, r)
        spheres.append((kind + 1, c, r))
        mask = np.zeros_like(phase, dtype=bool)
        _mark_sphere(mask, (n1, n2, n3), c, r)
        mask &= phase == 0
        phase[mask] = kind + 1
        counts[kind] += int(mask.sum())
    return phase, spheres


def random_spheres(grid=(128, 128, 128), seed=1713, fraction=0.3, rmin_vox=4.0, rmax_vox=10.0,
                   matrix_e=1.0, inclusion_e=100.0, nu=0.3):
    """Non-overlapping random spheres, radii uniform in [4, 10] voxels of a 128 grid."""
    rng = Xoshiro256ss(seed)
    phase, spheres = _rsa_spheres(grid, rng, rmin_vox / 128.0, rmax_vox / 128.0, [fraction])
    lame = np.array([lame_from_young(matrix_e, nu), lame_from_young(inclusion_e, nu)])
    lam0, mu0 = midpoint_reference(lame)
    return Microstructure(phase, lame, lam0, mu0, "random_spheres",
                          {"seed": seed, "n_spheres": len(spheres)})


def three_phase_spheres(grid=(64, 64, 64), seed=1714, fractions=(0.15, 0.15),
                        youngs=(1.0, 10.0, 100.0), nu=0.3):
    """Two inclusion types (E = 10 and E = 100) in a matrix of E = 1, 15 % each."""
    rng = Xoshiro256ss(seed)
    phase, spheres = _rsa_spheres(grid, rng, 4.0 / 128.0, 10.0 / 128.0, list(fractions))
    lame = np.array([lame_from_young(e, nu) for e in youngs])
    lam0, mu0 = midpoint_reference(lame)
    return Microstructure(phase, lame, lam0, mu0, "three_phase_spheres",
                          {"seed": seed, "n_spheres": len(spheres)})


def voronoi(grid=(128, 128, 128), seed=1716, n_grains=256, sigma=1.0, nu_range=(0.2, 0.4)):
    """Periodic voxel Voronoi tessellation; each grain isotropic with lognormal E."""
    rng = Xoshiro256ss(seed)
    lengths = _cell_lengths(grid)
    seeds = np.array([[rng.uniform(-0.5 * lengths[a], 0.5 * lengths[a]) for a in range(3)]
                      for _ in range(n_grains)])
    lame = []
    for _ in range(n_grains):
        e = math.exp(sigma * rng.normal())
        nu = rng.uniform(*nu_range)
        lame.append(lame_from_young(e, nu))
    lame = np.array(lame)
    n1, n2, n3 = grid
    y1, y2, y3 = voxel_centres(grid)
    y1 = y1 - 0.5 * lengths[0] + 0.5
    y2 = y2 - 0.5 * lengths[1] + 0.5
    y3 = y3 - 0.5 * lengths[2] + 0.5
    phase = np.zeros((n3, n2, n1), dtype=np.uint8)
    best = np.full((n2, n1), np.inf)
    for z in range(n3):
        best[:] = np.inf
        lab = np.zeros((n2, n1), dtype=np.int64)
        for g in range(n_grains):
            d1 = y1 - seeds[g, 0]
            d1 -= lengths[0] * np.round(d1 / lengths[0])
            d2 = y2 - seeds[g, 1]
            d2 -= lengths[1] * np.round(d2 / lengths[1])
            d3 = y3[z] - seeds[g, 2]
            d3 -= lengths[2] * np.round(d3 / lengths[2])
            dist = d3 * d3 + d2[:, None] ** 2 + d1[None, :] ** 2
            better = dist < best
            best = np.where(better, dist, best)
            lab = np.where(better, g, lab)
        phase[z] = lab
    lam0, mu0 = midpoint_reference(lame)
    return Microstructure(phase, lame, lam0, mu0, "voronoi", {"seed": seed, "n_grains": n_grains})


def voronoi_seeds(grid, seed, n_grains, sigma=1.0, nu_range=(0.2, 0.4)):
    """Seeds (unit-cell coordinates) and Lame table of ``voronoi``, without voxelising."""
    rng = Xoshiro256ss(seed)
    lengths = _cell_lengths(grid)
    seeds = np.array([[rng.uniform(-0.5 * lengths[a], 0.5 * lengths[a]) for a in range(3)]
                      for _ in range(n_grains)])
    lame = []
    for _ in range(n_grains):
        e = math.exp(sigma * rng.normal())
        nu = rng.uniform(*nu_range)
        lame.append(lame_from_young(e, nu))
    return seeds, np.array(lame)


def voronoi_torch(grid=(512, 512, 512), seed=1716, n_grains=256, device="cuda"):
    """The tessellation of ``voronoi`` voxelised with torch (FP64, nearest seed under the periodic
    minimum image), for grids too large for the numpy loop.  Same seeds, tables and distance."""
    import torch
    seeds, lame = voronoi_seeds(grid, seed, n_grains)
    lengths = _cell_lengths(grid)
    n1, n2, n3 = grid
    y1, y2, y3 = voxel_centres(grid)
    c = [torch.tensor(y - (-0.5) - 0.5 * L, dtype=torch.float64, device=device)
         for y, L in zip((y1, y2, y3), lengths)]
    sd = torch.tensor(seeds, dtype=torch.float64, device=device)
    Lt = torch.tensor(lengths, dtype=torch.float64, device=device)
    phase = torch.empty((n3, n2, n1), dtype=torch.uint8, device=device)

    def wrap(d, L):
        return d - L * torch.round(d / L)
    d1 = wrap(c[0][None, :] - sd[:, 0:1], Lt[0]) ** 2          # (G, n1)
    d2 = wrap(c[1][None, :] - sd[:, 1:2], Lt[1]) ** 2          # (G, n2)
    for z0 in range(0, n3, 32):
        z1 = min(n3, z0 + 32)
        d3 = wrap(c[2][None, z0:z1] - sd[:, 2:3], Lt[2]) ** 2  # (G, nz)
        best = None
        for g in range(n_grains):
            dist = d3[g][:, None, None] + d2[g][None, :, None] + d1[g][None, None, :]
            if best is None:
                best = dist
                lab = torch.zeros_like(dist, dtype=torch.uint8)
            else:
                better = dist < best
                best = torch.where(better, dist, best)
                lab = torch.where(better, torch.tensor(g, dtype=torch.uint8, device=device), lab)
        phase[z0:z1] = lab
    lam0, mu0 = midpoint_reference(lame)
    return Microstructure(phase, lame, lam0, mu0, "voronoi", {"seed": seed, "n_grains": n_grains})


def coated_sphere(n=32, r1=0.25, r2=0.4, e_core=100.0, e_coat=1000.0, e_matrix=453.685, nu=0.3):
    """Centred coated sphere: core r < r1, coating r1 <= r < r2, matrix outside."""
    y1, y2, y3 = voxel_centres((n, n, n))
    d2 = y3[:, None, None] ** 2 + y2[None, :, None] ** 2 + y1[None, None, :] ** 2
    phase = np.full((n, n, n), 2, dtype=np.uint8)
    phase[d2 < r2 * r2] = 1
    phase[d2 < r1 * r1] = 0
    lame = np.array([lame_from_young(e, nu) for e in (e_core, e_coat, e_matrix)])
    lam0, mu0 = midpoint_reference(lame)
    return Microstructure(phase, lame, lam0, mu0, "coated_sphere", {"r1": r1, "r2": r2})


def plane_stress_lame(lam, mu):
    """(lambda*, mu) such that the three-dimensional isotropic law with lambda*, applied to
    in-plane strains (eps33 = eps13 = eps23 = 0), gives the in-plane stresses of the plane-stress
    law of (lambda, mu): lambda* = 2 lambda mu / (lambda + 2 mu)."""
    return 2.0 * lam * mu / (lam + 2.0 * mu), mu


def hashin_2d(n=128, r1=0.25, r2=0.4, e_core=100.0, e_coat=1000.0, e_matrix=453.685, nu=0.3,
              plane_stress=True):
    """Hashin's structure of Sec. 4 on an n x n grid (N3 = 1): a centred disk core r < r1
    (phase 0), a coating r1 <= r < r2 (phase 1) and the matrix outside (phase 2), with Young's
    moduli e_core, e_coat, e_matrix and a common Poisson ratio nu.  plane_stress=True stores
    plane-stress Lame parameters, else plane strain."""
    y1, y2, _ = voxel_centres((n, n, 1))
    d2 = y2[:, None] ** 2 + y1[None, :] ** 2
    phase = np.full((1, n, n), 2, dtype=np.uint8)
    phase[0][d2 < r2 * r2] = 1
    phase[0][d2 < r1 * r1] = 0
    lame = np.array([lame_from_young(e, nu) for e in (e_core, e_coat, e_matrix)])
    if plane_stress:
        lame = np.array([plane_stress_lame(l, m) for l, m in lame])
    lam0, mu0 = midpoint_reference(lame)
    return Microstructure(phase, lame, lam0, mu0, "hashin_2d",
                          {"r1": r1, "r2": r2, "E": (e_core, e_coat, e_matrix), "nu": nu,
                           "plane_stress": plane_stress})


def random_field_strain(grid, n_fields, seed, dtype=np.float64):
    """Seeded uniform(-1, 1) Mandel strain fields, shape (n_fields, 6, N3, N2, N1)."""
    n1, n2, n3 = grid
    rng = np.random.Generator(np.random.Philox(seed))
    return rng.uniform(-1.0, 1.0, size=(n_fields, 6, n3, n2, n1)).astype(dtype)
