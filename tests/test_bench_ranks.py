"""The replicas-only multi-GPU path of bench.py, on CPU: two gloo ranks
agree on the slowest rank's timings, and the whole-job value counts every
rank's problems over that time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5], "cpu")
        dist.barrier()
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    res = dict(q.get(timeout=5) for _ in range(2))
    assert res[0] == res[1] == [2.0, 10.0, 0.5]


def test_single_process_and_value_formula():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 1.5], "cpu") == [3.0, 1.5]
    # 2 ranks x 10 steps x 1e12 flops in 4 s: 5 TFLOP/s for the job
    assert bench.whole_job_tflops(1e12, 10, 2, 4.0) == pytest.approx(5.0)
