"""Bounded case for Nsight Compute captures of the Lippmann-Schwinger kernels.

Runs a few CG iterations of the order-0 problem on the benchmark microstructure
(128^3 random spheres, 6 load cases, FP32 fields) and stops at the iteration cap, so a
capture sees every LS-step kernel kind with a small, fixed number of launches:

    python -m paper_1712_05145_gb300.profile_case --grid 128 --iters 2
"""
import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=128)
    ap.add_argument("--iters", type=int, default=2)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--seed", type=int, default=1713)
    args = ap.parse_args()
    import torch
    from paper_1712_05145_gb300 import build, hom, synthetic

    build.build()
    n = args.grid
    ms = synthetic.random_spheres((n, n, n), seed=args.seed)
    prec = hom.HOM_FP32_REFINE if args.precision == "fp32" else hom.HOM_FP64
    H = hom.Homogenization(ms, precision=prec, scheme=hom.HOM_CG, max_iter=args.iters,
                           check_every=args.iters, max_refine=0)
    info = H.solve(0, 1e-6)
    torch.cuda.synchronize()
    print(json.dumps({"grid": n, "iters": [i["iterations"] for i in info]}))
    H.close()


if __name__ == "__main__":
    main()
