"""Seeded input generators: determinism and geometry facts."""
import numpy as np

from paper_1712_05145_gb300 import synthetic


def test_splitmix64_reference_vector():
    s = synthetic.SplitMix64(1234567)
    assert [s.next() for _ in range(3)] == [6457827717110365317, 3203168211198807973,
                                            9817491932198370423]


def test_centred_sphere_fraction():
    ms = synthetic.centred_sphere(32)
    # r from f = 0.2 is 0.362783; counting voxel centres gives 6704 / 32768
    assert abs(ms.meta["radius"] - 0.3627831678) < 1e-9
    assert int(ms.phase.sum()) == 6704
    assert ms.lam0 == 5.5 and ms.mu0 == 5.5
    # centrosymmetric under n -> N-1-n
    assert np.array_equal(ms.phase, ms.phase[::-1, ::-1, ::-1])


def test_random_spheres_deterministic_and_fraction():
    a = synthetic.random_spheres((32, 32, 32), seed=5)
    b = synthetic.random_spheres((32, 32, 32), seed=5)
    assert np.array_equal(a.phase, b.phase)
    f = a.volume_fractions()[1]
    assert 0.3 <= f < 0.36
    lam, mu = synthetic.lame_from_young(1.0, 0.3)
    assert abs(lam - 0.576923076923) < 1e-11 and abs(mu - 0.384615384615) < 1e-11


def test_three_phase_and_voronoi():
    t = synthetic.three_phase_spheres((32, 32, 32), seed=3)
    f = t.volume_fractions()
    assert f[1] >= 0.15 and f[2] >= 0.15
    v = synthetic.voronoi((16, 16, 16), seed=2, n_grains=20)
    assert v.phase.max() < 20 and len(v.lame) == 20
