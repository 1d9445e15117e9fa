"""Timed runs of the workload configurations beside the benchmark's (which is C2).

    python -m paper_1712_05145_gb300.configs c1   # 32^3 sphere, FP64 Basic Scheme to 1e-8; 32^3 laminate
    python -m paper_1712_05145_gb300.configs c3   # 3-phase spheres, orders 0, 1, 2 at 64^3 and 128^3
    python -m paper_1712_05145_gb300.configs c5   # 512^3 periodic Voronoi of 256 grains, order 0

Each prints one JSON line per case: iterations, device time per order, voxel-iterations per
second and the effective tensors.  Parity of these workloads with the CPU oracle is checked by
the test suite on sizes the oracle finishes.
"""
import argparse
import json
import time


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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("config", choices=["c1", "c3", "c5"])
    ap.add_argument("--grid", type=int, default=0)
    args = ap.parse_args()
    from paper_1712_05145_gb300 import build
    build.build()
    if args.config == "c1":
        run_c1()
    elif args.config == "c3":
        run_c3((args.grid,) if args.grid else (64, 128))
    else:
        run_c5(args.grid or 512)


if __name__ == "__main__":
    main()
