"""The sharded Algorithm 2 driver on the GPU with the library's propagators
(one rank: the fine block of an iteration is one persistent launch over a
sub-range of a batch), against the oracle and against the library's own
Algorithm 2; and the sub-range run it relies on."""
import os
import socket

import numpy as np
import pytest

import oracle as O
import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import sharded as S
from paper_2502_02704_gb300 import workloads as W
from helpers import TOL_FP64, f_rel_err, moment_rel_err

pytestmark = pytest.mark.gpu


def test_run_range_advances_only_its_instances():
    nx, nv = 40, 8
    dt = pr.fine_dt(nx, nv, 8.0)
    insts = [pr.instance(nx, nv, dt, bc=pr.PR_BC_PERIODIC, eps=e) for e in (1.0, 1e-2, 1e-4)]
    Us = [W.smooth_periodic(nx), W.sod(nx), W.density_modes(nx, 0.2, 0.1)]
    b = pr.pr_batch_create(insts, pr.PR_FP64)
    try:
        for i, U in enumerate(Us):
            pr.pr_batch_set_initial(b, i, U)
        f0 = [pr.pr_batch_get_f(b, i) for i in range(3)]
        pr.pr_batch_run_range(b, 1, 1, 5)
        f1 = [pr.pr_batch_get_f(b, i) for i in range(3)]
        with pytest.raises(pr.PrError):
            pr.pr_batch_run_range(b, 2, 2, 1)
    finally:
        pr.pr_batch_destroy(b)
    assert np.array_equal(f1[0], f0[0]) and np.array_equal(f1[2], f0[2])
    k = O.Kin(nx=nx, nv=nv, L=8.0, bc=O.BC_PERIODIC, eps=1e-2, scheme=O.UPWIND)
    assert f_rel_err(f1[1], O.fine_run(k, dt, 5, O.lift(k, Us[1]))) < TOL_FP64


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("nccl", [False, True])
def test_sharded_driver_with_library_propagators(nccl):
    nx, nv, N, K, T = 64, 16, 8, 3, 0.1
    U0 = W.sod(nx)
    k = O.Kin(nx=nx, nv=nv, L=8.0, bc=O.BC_OUTFLOW, eps=1e-2, scheme=O.UPWIND)
    Uo, errs_o, _ = O.parareal(O.Parareal(kin=k, T=T, N=N), U0, K=K)
    props = S.LibraryPropagators(nx, nv, 1e-2, T, N, S.block_capacity(N, 1))
    group = S.Group()
    if nccl:  # a one-rank NCCL group: the collectives move device tensors
        import torch.distributed as dist

        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(_free_port())
        dist.init_process_group("nccl", rank=0, world_size=1)
        group = S.Group(dist.group.WORLD, "cuda:0")
    try:
        U, errs, hist = S.parareal_sharded(O.prim_to_cons(U0), N, K, props.fine, props.coarse, group=group,
                                           history=True)
    finally:
        props.close()
        if nccl:
            dist.destroy_process_group()
    for kk in range(K + 1):
        for n in range(N + 1):
            assert moment_rel_err(hist[kk][n], Uo[kk][n]) < TOL_FP64, (kk, n)
    assert np.allclose(errs, errs_o, rtol=1e-9, atol=0)
    ctx = pr.pr_init(nx, 0.0, 1.0, pr.PR_BC_OUTFLOW, nv, 8.0, 1e-2, T, N, 0.5, 0.5, pr.PR_UPWIND, pr.PR_FP64)
    try:
        pr.pr_set_initial(ctx, U0)
        pr.pr_parareal_run(ctx, K)
        for n in range(N + 1):
            assert moment_rel_err(U[n], pr.pr_moments(ctx, n)) < TOL_FP64, n
    finally:
        pr.pr_destroy(ctx)
