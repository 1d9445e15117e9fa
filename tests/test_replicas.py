"""Multi-process path (replicas, one process per GPU) on CPU: gloo ranks, world size 2."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1712_05145_gb300 import replicas
    t, u = replicas.aggregate(10.0 + rank, 100.0 * (rank + 1))
    r = replicas.job_rate(10.0 + rank, 100.0 * (rank + 1))
    q.put((rank, t, u, r))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_is_max_time_and_summed_work_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u, r in res:
        assert t == 11.0 and u == 300.0
        assert abs(r - 300.0 / 0.011) < 1e-6


def test_single_process_passes_through():
    from paper_1712_05145_gb300 import replicas
    assert replicas.aggregate(5.0, 7.0) == (5.0, 7.0)
    assert abs(replicas.job_rate(500.0, 10.0) - 20.0) < 1e-12


def test_reference_arm_runs_on_rank_0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
