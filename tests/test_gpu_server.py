"""Request server: continuous batching gives every request the result it gets alone."""
import time

import numpy as np
import pytest

from paper_1712_05145_gb300 import synthetic
from tests.helpers import random_phase

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def requests():
    out = [(synthetic.centred_sphere(16), 1),
           (synthetic.random_spheres((24, 24, 24), seed=5, inclusion_e=10.0), 0),
           (synthetic.laminate((16, 16, 16)), 0),
           (synthetic.three_phase_spheres((16, 16, 16), seed=3), 1),
           (synthetic.Microstructure(random_phase((12, 16, 24), 3, 7), np.array([[1.0, 1.0], [5.0, 3.0], [0.3, 0.2]]),
                                     2.5, 1.6), 0),
           (synthetic.random_spheres((32, 16, 24), seed=8, inclusion_e=300.0), 1),
           (synthetic.centred_sphere(24, matrix=(0.6, 0.4), inclusion=(60.0, 40.0)), 0),
           (synthetic.random_spheres((16, 16, 16), seed=11, inclusion_e=1000.0), 0)]
    return out


def solo(ms, order, tol):
    from paper_1712_05145_gb300 import hom
    H = hom.Homogenization(ms, precision=hom.HOM_FP32_REFINE, scheme=hom.HOM_CG)
    info = H.solve(0, tol)
    c = H.effective(0)
    d = None
    if order >= 1:
        info += H.solve(1, tol)
        d = H.effective(1)
    H.close()
    assert all(i["status"] == 0 for i in info)
    return c, d


def test_mixed_requests_match_solo_solves():
    from paper_1712_05145_gb300 import hom
    tol = 1e-7
    reqs = requests()
    ref = [solo(ms, order, tol) for ms, order in reqs]
    s = hom.hom_server_create(0, 3)
    ids = [hom.hom_server_submit(s, ms, order, tol) for ms, order in reqs]
    res = [hom.hom_server_wait(s, i) for i in ids]
    hom.hom_server_destroy(s)
    for (c, d), r in zip(ref, res):
        assert r["done"] == 1 and r["status"] == 0
        assert r["latency_ms"] >= r["run_ms"] > 0
        np.testing.assert_allclose(r["c_eff"], c, rtol=0, atol=1e-12 * np.abs(c).max())
        if d is not None:
            np.testing.assert_allclose(r["d1"], d, rtol=0, atol=1e-12 * max(np.abs(d).max(), 1e-30))


def test_same_grid_requests_share_launches_and_handles():
    """Order-0 requests of one grid queued together run as one batch (one handle, every launch
    carrying all their loads); a later wave reuses the resident handle; results are the solo ones."""
    from paper_1712_05145_gb300 import hom
    tol = 1e-7
    reqs = [synthetic.random_spheres((16, 16, 16), seed=50 + k, inclusion_e=3.0 * 10 ** (k % 3)) for k in range(6)]
    ref = [solo(ms, 0, tol)[0] for ms in reqs]
    s = hom.hom_server_create(0, 1, 8)
    for wave in range(2):
        ids = [hom.hom_server_submit(s, ms, 0, tol) for ms in reqs]
        res = [hom.hom_server_wait(s, i) for i in ids]
        for c, r in zip(ref, res):
            assert r["status"] == 0, r["message"]
            np.testing.assert_allclose(r["c_eff"], c, rtol=0, atol=1e-12 * np.abs(c).max())
    cnt = hom.hom_server_counters(s)
    hom.hom_server_destroy(s)
    assert cnt["requests"] == 12
    assert cnt["batches"] < cnt["requests"]          # some requests shared a batch
    assert cnt["handles_created"] <= 2               # the second wave ran on resident handles


def test_admission_respects_the_memory_budget():
    from paper_1712_05145_gb300 import hom
    ms = synthetic.random_spheres((32, 32, 32), seed=4)
    est = hom.hom_estimate_bytes((32, 32, 32), 0)
    s = hom.hom_server_create(int(est * 1.5), 4)      # room for one request at a time
    ids = [hom.hom_server_submit(s, ms, 0, 1e-6) for _ in range(4)]
    seen = 0
    while True:
        st = hom.hom_server_stats(s)
        seen = max(seen, st["running"])
        assert st["bytes_in_use"] <= est * 1.5
        if st["queued"] == 0 and st["running"] == 0:
            break
        time.sleep(0.002)
    res = [hom.hom_server_wait(s, i) for i in ids]
    assert seen == 1 and all(r["status"] == 0 for r in res)
    big = synthetic.random_spheres((64, 64, 64), seed=4)
    with pytest.raises(hom.HomError) as e:
        hom.hom_server_submit(s, big, 1, 1e-6)
    assert e.value.status == hom.HOM_ERR_NOMEM
    hom.hom_server_destroy(s)


def test_concurrent_requests_with_different_plane_sizes():
    """Workers that run grids with different shared-memory needs at once (x-y planes of 64 KB and
    96 KB per CTA) all succeed and give the result of the solo solve."""
    from paper_1712_05145_gb300 import hom
    tol = 1e-6
    grids = [(128, 128, 8), (192, 128, 8), (128, 128, 12), (192, 128, 6)]
    reqs = [(synthetic.random_spheres(g, seed=20 + i, inclusion_e=50.0), i % 2) for i, g in enumerate(grids)]
    ref = [solo(ms, order, tol) for ms, order in reqs]
    s = hom.hom_server_create(0, 6)
    ids = [hom.hom_server_submit(s, ms, order, tol) for _ in range(3) for ms, order in reqs]
    res = [hom.hom_server_wait(s, i) for i in ids]
    hom.hom_server_destroy(s)
    for k, r in enumerate(res):
        assert r["status"] == 0, r["message"]
        c, d = ref[k % len(reqs)]
        np.testing.assert_allclose(r["c_eff"], c, rtol=0, atol=1e-12 * np.abs(c).max())
        if d is not None:
            np.testing.assert_allclose(r["d1"], d, rtol=0, atol=1e-12 * max(np.abs(d).max(), 1e-30))
