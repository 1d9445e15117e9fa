"""Timed runs of the workload configurations beside the benchmark's (which is C2).

    python -m paper_1712_05145_gb300.configs c1   # 32^3 sphere, FP64 Basic Scheme to 1e-8; 32^3 laminate
    python -m paper_1712_05145_gb300.configs c3   # 3-phase spheres, orders 0, 1, 2 at 64^3 and 128^3
    python -m paper_1712_05145_gb300.configs c5   # 512^3 periodic Voronoi of 256 grains, order 0
    python -m paper_1712_05145_gb300.configs schemes   # C2's RVE: CG, polarization, BiCGSTAB, Basic

Each prints one JSON line per case: iterations, device time per order, voxel-iterations per
second and the effective tensors.  Parity of these workloads with the CPU oracle is checked by
the test suite on sizes the oracle finishes.
"""
import argparse
import json
import time

import numpy as np


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t


def run_c1():
    from paper_1712_05145_gb300 import hom, synthetic
    import numpy as np
    ms = synthetic.centred_sphere(32)
    H = hom.Homogenization(ms, precision=hom.HOM_FP64, scheme=hom.HOM_BASIC, max_iter=10000)
    H.solve(0, 1e-8, loads=np.eye(6)[:1])
    info, dt = _timed(lambda: H.solve(0, 1e-8, loads=np.eye(6)[:1]))
    col = H.effective(0)[:, 0]
    print(json.dumps({"config": "C1 sphere 32^3 FP64 Basic Scheme, E = e11, tol 1e-8",
                      "iterations": info[0]["iterations"], "rel_residual_fp64": info[0]["rel_residual_fp64"],
                      "seconds": dt, "voxel_iters_per_s": 32 ** 3 * info[0]["iterations"] / dt,
                      "c_eff_column": col.tolist()}))
    H.close()
    lam = synthetic.laminate((32, 32, 32))
    H = hom.Homogenization(lam, precision=hom.HOM_FP64, scheme=hom.HOM_BASIC, max_iter=10000)
    info, dt = _timed(lambda: H.solve(0, 1e-8))
    print(json.dumps({"config": "C1 laminate 32^3 (16 + 16 layers) FP64 Basic Scheme, 6 unit loads, tol 1e-8",
                      "iterations": [i["iterations"] for i in info], "seconds": dt,
                      "c_eff": H.effective(0).tolist()}))
    H.close()


def run_c3(grids=(64, 128)):
    from paper_1712_05145_gb300 import hom, synthetic
    for n in grids:
        ms = synthetic.three_phase_spheres((n, n, n), seed=1714)
        H = hom.Homogenization(ms, precision=hom.HOM_FP32_REFINE, scheme=hom.HOM_CG)
        row = {"config": "C3 three-phase spheres %d^3 (E 1/10/100, 15 %% each), FP32 + FP64 refinement, tol 1e-6" % n}
        for order in (0, 1, 2):
            info, dt = _timed(lambda: H.solve(order, 1e-6))
            it = sum(i["iterations"] for i in info)
            row["order%d" % order] = {"loads": len(info), "iterations": it, "seconds": dt,
                                      "voxel_iters_per_s": n ** 3 * it / dt,
                                      "max_rel_residual_fp64": max(i["rel_residual_fp64"] for i in info),
                                      "ok": all(i["status"] == 0 for i in info)}
        row["time_ratio_order2_over_order1"] = row["order2"]["seconds"] / row["order1"]["seconds"]
        row["c_eff"] = H.effective(0).tolist()
        d1 = H.effective(1)
        row["d1_max_abs"] = float(abs(d1).max())
        print(json.dumps(row), flush=True)
        H.close()


def run_c5(n=512):
    import numpy as np
    import torch
    from paper_1712_05145_gb300 import hom, synthetic
    ms, tgen = _timed(lambda: synthetic.voronoi_torch((n, n, n), seed=1716, n_grains=256))
    H = hom.Homogenization(ms, precision=hom.HOM_FP32_REFINE, scheme=hom.HOM_CG)
    hom.hom_profile(H.h, 1)
    info, dt = _timed(lambda: H.solve(0, 1e-6))
    prof = hom.hom_profile_read(H.h)
    it = sum(i["iterations"] for i in info)
    ls = [p for p in prof if p["launches"]]
    print(json.dumps({"config": "C5 periodic Voronoi %d^3, 256 grains, E lognormal(sigma 1), nu U[0.2,0.4], order 0, "
                                "FP32 + FP64 refinement, tol 1e-6" % n,
                      "generate_seconds": tgen, "iterations": it, "seconds": dt,
                      "voxel_iters_per_s": n ** 3 * it / dt, "device_bytes": hom.hom_device_bytes(H.h),
                      "max_rel_residual_fp64": max(i["rel_residual_fp64"] for i in info),
                      "ok": all(i["status"] == 0 for i in info),
                      "kernels": [{"kernel": p["kernel"], "launches": p["launches"], "ms": p["ms"],
                                   "gbs": p["bytes"] / (p["ms"] / 1e3) / 1e9} for p in ls],
                      "c_eff": H.effective(0).tolist()}), flush=True)
    c512 = H.effective(0)
    H.close()
    # the same tessellation on a 128^3 grid: the difference is discretisation, not parity
    ms128 = synthetic.voronoi((128, 128, 128), seed=1716, n_grains=256)
    H = hom.Homogenization(ms128, precision=hom.HOM_FP32_REFINE, scheme=hom.HOM_CG)
    H.solve(0, 1e-6)
    c128 = H.effective(0)
    H.close()
    print(json.dumps({"config": "C5 Voronoi at 128^3 (same seeds) against 512^3",
                      "c_eff_128": c128.tolist(),
                      "max_rel_difference": float(np.abs(c512 - c128).max() / np.abs(c512).max())}), flush=True)


def run_schemes(n=128):
    """The C2 microstructure (random spheres, contrast 100, 6 unit loads, tol 1e-6) solved by each
    scheme in both precisions; the polarization scheme with the geometric-mean reference medium,
    the others with the midpoint reference."""
    from paper_1712_05145_gb300 import hom, synthetic
    ms = synthetic.random_spheres((n, n, n), seed=1713)
    geo = synthetic.geometric_reference(ms.lame)
    cases = [("CG", hom.HOM_CG, 0, None), ("BiCGSTAB", hom.HOM_BICGSTAB, 0, None),
             ("polarization (Eyre-Milton)", hom.HOM_POLARIZATION, 0, geo),
             ("polarization (augmented Lagrangian)", hom.HOM_POLARIZATION, 1, geo),
             ("Basic Scheme", hom.HOM_BASIC, 0, None)]
    for precision in (hom.HOM_FP32_REFINE, hom.HOM_FP64):
        for name, scheme, variant, ref in cases:
            if scheme == hom.HOM_BASIC and precision == hom.HOM_FP32_REFINE:
                continue   # the Basic Scheme does not refine: its FP32 result stops at FP32 accuracy
            kw = {} if ref is None else {"lam0": ref[0], "mu0": ref[1]}
            H = hom.Homogenization(ms, precision=precision, scheme=scheme, polarization_variant=variant,
                                   max_iter=20000, **kw)
            H.solve(0, 1e-6, loads=np.eye(6)[:1])        # warm-up (allocation, tables)
            info, dt = _timed(lambda: H.solve(0, 1e-6))
            it = sum(i["iterations"] for i in info)
            print(json.dumps({"config": "C2 RVE %d^3, 6 loads, tol 1e-6" % n, "scheme": name,
                              "precision": "fp32+refine" if precision == hom.HOM_FP32_REFINE else "fp64",
                              "iterations": it, "seconds": dt, "voxel_iters_per_s": n ** 3 * it / dt,
                              "max_rel_residual_fp64": max(i["rel_residual_fp64"] for i in info),
                              "ok": all(i["status"] == 0 for i in info),
                              "c11": float(H.effective(0)[0, 0])}), flush=True)
            H.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("config", choices=["c1", "c3", "c5", "schemes"])
    ap.add_argument("--grid", type=int, default=0)
    args = ap.parse_args()
    from paper_1712_05145_gb300 import build
    build.build()
    if args.config == "c1":
        run_c1()
    elif args.config == "c3":
        run_c3((args.grid,) if args.grid else (64, 128))
    elif args.config == "schemes":
        run_schemes(args.grid or 128)
    else:
        run_c5(args.grid or 512)


if __name__ == "__main__":
    main()
