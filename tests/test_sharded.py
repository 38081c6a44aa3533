"""Algorithm 2 with the fine phase split over ranks as App. A (Algorithm 3)
prescribes, on CPU gloo ranks with the oracle's propagators: the iterates of
every level and the errors of Eq. 10 equal the single-process oracle run bit
for bit; and the partition arithmetic of App. A."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O
from paper_2502_02704_gb300 import sharded as S
from paper_2502_02704_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NX, NV, N, K, T = 16, 8, 5, 4, 0.04


def _problem():
    k = O.Kin(nx=NX, nv=NV, L=8.0, bc=O.BC_OUTFLOW, eps=1e-2, scheme=O.UPWIND)
    return O.Parareal(kin=k, T=T, N=N), W.sod(NX)


def test_partition_follows_app_a():
    # App. A: work = N_g - k, chunk = floor(work / N_p), remainder = work mod
    # N_p, start = rank chunk + min(remainder, rank) + 1, end = (rank + 1) chunk
    # + min(remainder, rank + 1) -- 10 positions over 3 ranks: 4 / 3 / 3.
    assert [S.slice_block(10, 1, 3, r) for r in range(3)] == [(1, 4), (5, 7), (8, 10)]
    for Ng in (1, 5, 8, 64, 65):
        for world in (1, 2, 3, 8):
            for k in range(1, Ng + 2):
                blocks = [S.slice_block(Ng, k, world, r) for r in range(world)]
                covered = [n for a, b in blocks for n in range(a, b + 1)]
                assert covered == list(range(k, Ng + 1)), (Ng, world, k)  # contiguous, in rank order
                sizes = [b - a + 1 for a, b in blocks]
                assert max(sizes) - min(sizes) <= 1
                assert max(sizes) <= S.block_capacity(Ng, world)


def test_single_process_run_equals_the_oracle_bitwise():
    p, U0 = _problem()
    Uo, errs_o, _ = O.parareal(p, U0, K=K)
    U, errs, hist = S.parareal_sharded(O.prim_to_cons(U0), N, K,
                                       lambda Vs: np.stack([O.fine_propagate(p, V) for V in Vs]),
                                       lambda V: O.coarse_propagate(p, V), history=True)
    assert np.array_equal(hist, Uo)
    assert errs == list(errs_o)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import oracle as O2
    from paper_2502_02704_gb300 import sharded as S2

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, U0 = _problem()
        calls = []

        def fine(Vs):
            calls.append(len(Vs))
            return np.stack([O2.fine_propagate(p, V) for V in Vs])

        U, errs, hist = S2.parareal_sharded(O2.prim_to_cons(U0), N, K, fine, lambda V: O2.coarse_propagate(p, V),
                                            group=S2.Group(dist.group.WORLD, "cpu"), history=True)
        q.put((rank, hist, errs, calls))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_equal_the_single_process_run_bitwise(world):
    p, U0 = _problem()
    Uo, errs_o, _ = O.parareal(p, U0, K=K)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr_ in procs:
        pr_.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for pr_ in procs:
        pr_.join(timeout=60)
        assert pr_.exitcode == 0
    for rank, hist, errs, calls in res:
        assert np.array_equal(hist, Uo), rank
        assert errs == list(errs_o), rank
        # each iteration the rank propagated exactly its App. A block
        want = [b - a + 1 for a, b in (S.slice_block(N, k, world, rank) for k in range(1, K + 1)) if b >= a]
        assert calls == want, (rank, calls, want)
