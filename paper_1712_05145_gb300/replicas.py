"""Whole-job figures of a run with one process per GPU.

Loads and RVEs are independent, so the multi-GPU form of the solver is replicas: every rank
solves its own problems and no data crosses ranks on the solve path.  The only collective is the
one that turns per-rank measurements into the job's: the elapsed time is the maximum over ranks
(the job ends with its slowest rank) and the work is the sum of the ranks' work units.
"""


def env_rank():
    """(rank, world size, local rank) from the launcher's environment (single process: 0, 1, 0)."""
    import os
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def aggregate(elapsed_ms, units, device="cpu"):
    """Returns (max elapsed_ms over ranks, sum of units over ranks).  Without an initialised
    process group (or with one rank) the inputs come back unchanged.  `device` holds the two
    reduction tensors: "cuda" for NCCL, "cpu" for gloo."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_ms), float(units)
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def job_rate(elapsed_ms, units, device="cpu"):
    """Units per second of the whole job: the ranks' summed units over the slowest rank's time."""
    t, u = aggregate(elapsed_ms, units, device)
    return u / (t / 1e3) if t > 0 else 0.0
