"""Bounded case for Nsight Compute captures of the Lippmann-Schwinger kernels.

Runs a few CG iterations of the order-0 problem and stops at the iteration cap, so a capture
sees every LS-step kernel kind with a small, fixed number of launches.  The default is the
benchmark microstructure (128^3 random spheres, 6 load cases, FP32 fields); --shape gives any
grid (the same generator, scaled to the grid), --loads the number of unit loads, and --pass-mode /
--z-mode / --y-mode select the plane, z and y passes (hom_options.pass_mode, z_mode, y_mode).  --autotune tunes the
launch shape in a first solve and profiles a second one:

    python -m paper_1712_05145_gb300.profile_case --grid 128 --iters 2
    python -m paper_1712_05145_gb300.profile_case --shape 512,512,64 --loads 1 --iters 2
"""
import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--shape", default="", help="N1,N2,N3 (overrides --grid)")
    ap.add_argument("--loads", type=int, default=6)
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--pass-mode", type=int, default=0)
    ap.add_argument("--z-mode", type=int, default=0)
    ap.add_argument("--y-mode", type=int, default=0)
    ap.add_argument("--seed", type=int, default=1713)
    ap.add_argument("--times", action="store_true", help="print per-kernel device times (CUDA events)")
    ap.add_argument("--autotune", action="store_true", help="tune the launch shape first (hom_options.autotune)")
    args = ap.parse_args()
    import numpy as np
    import torch
    from paper_1712_05145_gb300 import build, hom, synthetic

    build.build()
    grid = tuple(int(v) for v in args.shape.split(",")) if args.shape else (args.grid,) * 3
    ms = synthetic.random_spheres(grid, seed=args.seed)
    prec = hom.HOM_FP32_REFINE if args.precision == "fp32" else hom.HOM_FP64
    H = hom.Homogenization(ms, precision=prec, scheme=hom.HOM_CG, max_iter=args.iters,
                           check_every=args.iters, max_refine=0, pass_mode=args.pass_mode, z_mode=args.z_mode,
                           y_mode=args.y_mode, autotune=1 if args.autotune else 0)
    if args.autotune:
        H.solve(0, 1e-6, loads=np.eye(6)[: args.loads])
    if args.times:
        hom.hom_profile(H.h, 1)
    info = H.solve(0, 1e-6, loads=np.eye(6)[: args.loads])
    torch.cuda.synchronize()
    out = {"grid": list(grid), "iters": [i["iterations"] for i in info],
           "plane_cluster_ctas": hom.hom_plane_config(H.h), "zpass_cluster_tile": hom.hom_zpass_config(H.h),
           "ypass_tile_tma": hom.hom_ypass_config(H.h)}
    if args.times:
        out["kernels"] = [{"kernel": p["kernel"], "launches": p["launches"],
                           "ms_per_launch": p["ms"] / p["launches"], "gbs": p["bytes"] / (p["ms"] / 1e3) / 1e9}
                          for p in hom.hom_profile_read(H.h) if p["launches"]]
    print(json.dumps(out))
    H.close()


if __name__ == "__main__":
    main()
