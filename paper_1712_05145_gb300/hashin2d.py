"""The numerical experiments of Sec. 4 on Hashin's structure, two-dimensional (N3 = 1), plane stress.

    python -m paper_1712_05145_gb300.hashin2d grid       # iterations and times against n (Fig. 3, Table 1)
    python -m paper_1712_05145_gb300.hashin2d contrast   # iterations against E2 / E1 at 64^2 (Fig. 4)
    python -m paper_1712_05145_gb300.hashin2d bulk       # in-plane bulk modulus against the matrix's
    python -m paper_1712_05145_gb300.hashin2d fields --out DIR   # the displacement fields of Fig. 2

Problems, as in Sec. 4 (the paper's numbering):
* first-order problem: the cell problem for E = Id (in-plane: E11 = E22 = 1);
* second-order problem: the alpha = 2 problem for (grad E)_111 = (grad E)_222 = 1.  It needs the
  first-order correctors of the unit strains e11 and e22, so its time includes that solve
  (both loads batched in one launch sequence) plus the alpha = 2 solve of the combined load.
The schemes run in FP64 with the paper's tolerance 1e-6: the Basic Scheme (FFTH), CG,
BiCGSTAB (the paper's CG-version ran MATLAB's BiCGSTAB; one BiCGSTAB iteration applies the
operator twice) and the polarization scheme of Sec. 1's references (Eyre-Milton, with the
geometric-mean reference medium).  Each line is one JSON object.
"""
import argparse
import json
import time

import numpy as np

TOL = 1e-6
E_ID = np.array([[1.0, 1.0, 0.0, 0.0, 0.0, 0.0]])
W_111_222 = np.zeros((1, 18))
W_111_222[0, 3 * 0 + 0] = 1.0   # E^(11) varying along Y1
W_111_222[0, 3 * 1 + 1] = 1.0   # E^(22) varying along Y2
SCHEMES = (("basic", 0), ("cg", 1), ("bicgstab", 2), ("polarization", 3))   # hom.HOM_* schemes


def _sync():
    import torch
    torch.cuda.synchronize()


def run_problems(ms, scheme, max_iter, repeat=1):
    """Iterations and device-synchronised wall times of the first- and second-order problems."""
    from paper_1712_05145_gb300 import hom, synthetic
    kw = {}
    if scheme == hom.HOM_POLARIZATION:   # its reference medium: geometric means of the phases
        kw["lam0"], kw["mu0"] = synthetic.geometric_reference(ms.lame)
    H = hom.Homogenization(ms, precision=hom.HOM_FP64, scheme=scheme, max_iter=max_iter, **kw)
    out = {}
    best1 = best2 = None
    for _ in range(repeat):
        _sync()
        t0 = time.perf_counter()
        i1 = H.solve(0, TOL, loads=E_ID)
        _sync()
        t1 = time.perf_counter() - t0
        t0 = time.perf_counter()
        i0 = H.solve(0, TOL, loads=np.eye(6)[[0, 1]])
        if all(i["status"] == 0 for i in i0):
            i2 = H.solve(1, TOL, loads=W_111_222)
        else:   # a prerequisite missed the tolerance within max_iter: no second-order solve
            i2 = [{"iterations": None, "status": hom.HOM_ERR_ORDER, "rel_residual_fp64": None}]
        _sync()
        t2 = time.perf_counter() - t0
        best1 = t1 if best1 is None else min(best1, t1)
        best2 = t2 if best2 is None else min(best2, t2)
    out["first_order"] = {"iterations": i1[0]["iterations"], "status": i1[0]["status"], "seconds": best1,
                          "rel_residual_fp64": i1[0]["rel_residual_fp64"]}
    out["second_order"] = {"iterations": i2[0]["iterations"], "status": i2[0]["status"],
                           "prerequisite_iterations": [i["iterations"] for i in i0], "seconds": best2,
                           "rel_residual_fp64": i2[0]["rel_residual_fp64"]}
    out["time_ratio"] = best2 / best1
    H.close()
    return out


def run_grid(sizes, max_iter):
    from paper_1712_05145_gb300 import hom, synthetic
    for n in sizes:
        ms = synthetic.hashin_2d(n)
        row = {"experiment": "Hashin 2-D plane stress, grid sweep (Fig. 3, Table 1)", "n": n}
        for name, scheme in SCHEMES:
            run_problems(ms, scheme, max_iter)                   # warm-up: kernel loads, tables
            row[name] = run_problems(ms, scheme, max_iter, repeat=2)
        print(json.dumps(row), flush=True)


def run_contrast(n, contrasts, max_iter):
    from paper_1712_05145_gb300 import hom, synthetic
    for q in contrasts:
        e2 = 100.0 * q
        ms = synthetic.hashin_2d(n, e_coat=e2)
        row = {"experiment": "Hashin 2-D plane stress, contrast sweep at %d^2 (Fig. 4)" % n,
               "E1": 100.0, "E2": e2, "contrast_E2_over_E1": q}
        for name, scheme in SCHEMES:
            row[name] = run_problems(ms, scheme, max_iter)
        print(json.dumps(row), flush=True)


def in_plane_bulk_modulus(sizes):
    """In-plane bulk modulus (sigma11 + sigma22) / 4 under E = Id against the matrix's
    E3 / (2 (1 - nu)): the coated inclusion is neutral, so they agree as the voxels shrink."""
    from paper_1712_05145_gb300 import hom, synthetic
    for n in sizes:
        ms = synthetic.hashin_2d(n)
        k3 = ms.meta["E"][2] / (2.0 * (1.0 - ms.meta["nu"]))
        H = hom.Homogenization(ms, precision=hom.HOM_FP32_REFINE, scheme=hom.HOM_CG)
        info = H.solve(0, 1e-8, loads=E_ID)
        s = H.effective(0)[:, 0]
        kap = 0.25 * (s[0] + s[1])
        print(json.dumps({"experiment": "Hashin 2-D plane stress, in-plane bulk modulus", "n": n,
                          "kappa_eff": kap, "kappa_matrix": k3, "rel_diff": (kap - k3) / k3,
                          "iterations": info[0]["iterations"], "status": info[0]["status"]}), flush=True)
        H.close()


def displacement_fields(n, out_dir):
    """The fields Fig. 2 shows, as arrays: the first displacement component of the first-order
    problem (E = Id) and of the second-order problem ((grad E)_111 = (grad E)_222 = 1) on the n x n
    Hashin structure, written to out_dir/hashin2d_fig2_n{n}.npz (arrays u1_first, u1_second, shape
    n x n, index [y2][y1])."""
    import os
    from paper_1712_05145_gb300 import hom, synthetic
    ms = synthetic.hashin_2d(n)
    H = hom.Homogenization(ms, precision=hom.HOM_FP64, scheme=hom.HOM_CG)
    H.solve(0, TOL, loads=E_ID)
    u_first = H.field(0, 0, hom.HOM_FIELD_DISPLACEMENT)[0, 0]
    H.solve(0, TOL, loads=np.eye(6)[[0, 1]])
    H.solve(1, TOL, loads=W_111_222)
    u_second = H.field(1, 0, hom.HOM_FIELD_DISPLACEMENT)[0, 0]
    H.close()
    os.makedirs(out_dir, exist_ok=True)
    path = os.path.join(out_dir, "hashin2d_fig2_n%d.npz" % n)
    np.savez(path, u1_first=u_first, u1_second=u_second)
    print(json.dumps({"experiment": "Hashin 2-D displacement fields (Fig. 2)", "n": n, "file": path,
                      "u1_first_range": [float(u_first.min()), float(u_first.max())],
                      "u1_second_range": [float(u_second.min()), float(u_second.max())]}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("experiment", choices=["grid", "contrast", "bulk", "fields"])
    ap.add_argument("--out", type=str, default="hashin2d_out")
    ap.add_argument("--sizes", type=str, default="8,16,32,64,128,256,512")
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--max-iter", type=int, default=100000)
    args = ap.parse_args()
    from paper_1712_05145_gb300 import build
    build.build()
    sizes = [int(s) for s in args.sizes.split(",")]
    if args.experiment == "grid":
        run_grid(sizes, args.max_iter)
    elif args.experiment == "contrast":
        run_contrast(args.n, [10.0 ** e for e in np.arange(-4.0, 4.01, 1.0)], args.max_iter)
    elif args.experiment == "fields":
        displacement_fields(128, args.out)
    else:
        in_plane_bulk_modulus(sizes)


if __name__ == "__main__":
    main()
