"""The N>1 bench path on CPU: two gloo ranks (replicas, no collective on the data path).

Each rank times its own solves; the job's time is the max over ranks and `value` divides by the
solves of all ranks. The reference arm runs on rank 0 alone; other ranks exit 0 without work.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "took" (r + 1) seconds for its 3 solves
    mx = bench.reduce_max(float(rank + 1), dist)
    out[rank] = (mx, bench.per_solve_seconds(mx, 3, world))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_max_two_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        mx, v = out[r]
        assert mx == 2.0                  # the slowest rank sets the job's time
        assert v == pytest.approx(2.0 / 6)  # 3 solves on each of the 2 ranks


def test_reference_arm_other_ranks_exit_quietly(capsys):
    import bench

    class A:
        ref_iters, warmup, steps, gpus = 10, 0, 1, 2
    old = os.environ.get("RANK")
    os.environ["RANK"] = "1"
    try:
        assert bench.run_reference(A()) == 0
    finally:
        if old is None:
            del os.environ["RANK"]
        else:
            os.environ["RANK"] = old
    assert capsys.readouterr().out == ""
