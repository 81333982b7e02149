"""The host side of a multi-GPU run, on the CPU: world_size-2 gloo process groups.

A replicas run (each rank solves its own copy; no collective on the data path) reports
the work of all ranks over the slowest rank's time.  bench.aggregate_ranks does that
reduction; here two gloo ranks feed it different figures and both must see the totals.
Under torchrun the reference arm runs on rank 0 only; the other ranks exit 0 silently.
"""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 10(r+1) units of work and 1 e2e unit; times 5 + r and 2 - r
        sums, maxes = bench.aggregate_ranks(dist, torch.device("cpu"), [10.0 * (rank + 1), 1.0],
                                            [5.0 + rank, 2.0 - rank])
        out.put((rank, sums, maxes))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_aggregate_ranks_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, sums, maxes in res:
        assert sums == [30.0, 2.0]       # work adds up over the ranks
        assert maxes == [6.0, 2.0]       # the slowest rank's time


def test_aggregate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(None, None, [3, 4], [5, 6]) == ([3.0, 4.0], [5.0, 6.0])


def test_reference_arm_other_ranks_exit_silently():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""
