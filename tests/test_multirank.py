"""The multi-rank bench path on CPU: two gloo ranks, the job time is the
maximum over ranks and the value counts every rank's updates (weak scaling,
no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0 + 5.0 * rank, 20.0 - 3.0 * rank]  # rank-local kernel and end-to-end times
    out = bench.max_over_ranks(ms, dist, "cpu")
    val = bench.weak_scaling_value(world, 1e9, out[0])
    q.put((rank, out, val))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, out, val in res:
        assert out == [15.0, 20.0]
        assert val == pytest.approx(2 * 1e9 / 15e-3)


def test_single_rank_path_needs_no_process_group():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.weak_scaling_value(1, 5e8, 10.0) == pytest.approx(5e10)
