"""The stored oracle solutions (tests/golden/ceff_oracle_*.json, written by
tests/golden/make_ceff_golden.py from oracle/ alone) satisfy what the exact discrete solution must:
every load reached the oracle's tolerance, C_eff has major symmetry (Sec. 2: the energy form
<E_a : C : (E_b + eps_b)> is symmetric at the solution), is positive definite, and lies between the
Reuss and Voigt bounds of the microstructure's voxel phase fractions."""
import json
import os

import numpy as np
import pytest

from oracle import closed_forms
from paper_1712_05145_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASES = {"random_spheres_128": lambda: synthetic.random_spheres((128, 128, 128), seed=1713),
         "voronoi_128": lambda: synthetic.voronoi((128, 128, 128), seed=1716, n_grains=256)}


@pytest.mark.parametrize("name", sorted(CASES))
def test_stored_oracle_solution_is_a_converged_symmetric_bounded_stiffness(name):
    with open(os.path.join(GOLDEN, "ceff_oracle_%s.json" % name)) as f:
        d = json.load(f)
    c = np.array(d["c_eff"])
    assert d["tol"] <= 1e-10 and all(r < d["tol"] for r in d["final_residual"])
    assert np.abs(c - c.T).max() < 1e-10 * np.abs(c).max()
    assert np.linalg.eigvalsh(0.5 * (c + c.T)).min() > 0
    ms = CASES[name]()
    fr = ms.volume_fractions()
    lame = [tuple(x) for x in ms.lame]
    v, r = closed_forms.voigt(lame, fr), closed_forms.reuss(lame, fr)
    cs = 0.5 * (c + c.T)
    assert np.linalg.eigvalsh(cs - r).min() > -1e-9 * np.abs(v).max()
    assert np.linalg.eigvalsh(v - cs).min() > -1e-9 * np.abs(v).max()
