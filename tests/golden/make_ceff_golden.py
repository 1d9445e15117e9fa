"""Writes the oracle's effective stiffness of two 128^3 workloads to tests/golden/.

Calls only ``oracle/`` (and the seeded input generator ``synthetic``, which holds none of the
method's arithmetic).  For each workload the six Mandel unit loads are solved by the oracle's CG
on A eps = b (Eq. cg_form, Sec. 2) to a relative residual of 1e-10, one process per load, and
C_eff[:, a] = <C : (E_a + eps_a)> (the volume average of the stress, Sec. 2) is written with the
iteration counts and final residuals.  Run from the repository root:

    python tests/golden/make_ceff_golden.py [random_spheres_128|voronoi_128]

Each workload takes about 20-40 minutes of CPU time per load.
"""
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TOL = 1e-10
WORKLOADS = {
    # random non-overlapping spheres, radii 4-10 voxels, f = 0.3, E 1 / 100, nu 0.3, seed 1713
    "random_spheres_128": ("random_spheres", {"grid": (128, 128, 128), "seed": 1713}),
    # periodic Voronoi of 256 grains, E lognormal (sigma 1), nu U[0.2, 0.4], seed 1716, on 128^3
    "voronoi_128": ("voronoi", {"grid": (128, 128, 128), "seed": 1716, "n_grains": 256}),
}


def _microstructure(name):
    from paper_1712_05145_gb300 import synthetic
    fn, kw = WORKLOADS[name]
    return getattr(synthetic, fn)(**kw)


def _solve_load(args):
    name, a = args
    os.environ["OMP_NUM_THREADS"] = "1"
    import numpy as np
    from oracle.lippmann_schwinger import Problem
    from oracle.tensors import unit_mandel_load
    ms = _microstructure(name)
    pb = Problem(ms.phase, ms.lame, ms.lam0, ms.mu0)
    E = unit_mandel_load(a)
    b = pb.rhs(E)
    t = time.time()
    eps, it, hist = pb.cg(b, TOL)
    col = pb.mean_stress(eps, E)
    return a, col.tolist(), it, hist[-1], time.time() - t


def main():
    names = sys.argv[1:] or list(WORKLOADS)
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(os.cpu_count() or 1, 6 * len(names))) as pool:
        jobs = [(n, a) for n in names for a in range(6)]
        results = pool.map(_solve_load, jobs)
    for n in names:
        rows = sorted((r for (nn, _), r in zip(jobs, results) if nn == n), key=lambda r: r[0])
        ceff = [[rows[a][1][i] for a in range(6)] for i in range(6)]
        fn, kw = WORKLOADS[n]
        path = os.path.join(ROOT, "tests", "golden", "ceff_oracle_%s.json" % n)
        with open(path, "w") as f:
            json.dump({"what": "effective stiffness C_eff (6x6 Mandel, column a = mean stress of the unit "
                               "Mandel load e_a) of the discrete Lippmann-Schwinger problem (Sec. 2, Eq. cg_form "
                               "and the volume average of the stress), computed by the FP64 oracle's CG",
                       "generator": fn, "arguments": {k: list(v) if isinstance(v, tuple) else v
                                                       for k, v in kw.items()},
                       "tol": TOL, "iterations": [r[2] for r in rows], "final_residual": [r[3] for r in rows],
                       "cpu_seconds": [r[4] for r in rows], "c_eff": ceff}, f, indent=1)
        print("wrote", path)


if __name__ == "__main__":
    main()
