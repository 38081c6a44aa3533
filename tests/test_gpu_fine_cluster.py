"""The cluster-resident fine run (one thread-block cluster per parareal slice,
the slice kept in shared memory for all its fine steps) against the CPU FP64
oracle's Algorithm 2, and its selection rules."""
import numpy as np
import pytest

import oracle as O
import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import workloads as W
from helpers import TOL_MIXED, moment_rel_err

pytestmark = pytest.mark.gpu

BC = {pr.PR_BC_PERIODIC: O.BC_PERIODIC, pr.PR_BC_OUTFLOW: O.BC_OUTFLOW, pr.PR_BC_REFLECT: O.BC_REFLECT}


def _run(nx, nv, bc, scheme, N, K, T, path, max_batch=0, U0=None, precision=pr.PR_MIXED):
    U0 = W.sod(nx) if U0 is None else U0
    ctx = pr.pr_init(nx, 0.0, 1.0, bc, nv, 8.0, 1e-2, T, N, 0.5, 0.5, scheme, precision, max_batch=max_batch)
    try:
        pr.pr_set_fine_path(ctx, path)
        used = pr.pr_get_fine_path(ctx)
        pr.pr_set_initial(ctx, U0)
        kd, errs = pr.pr_parareal_run(ctx, K)
        U = [pr.pr_moments(ctx, n, pr.PR_CONSERVED) for n in range(N + 1)]
    finally:
        pr.pr_destroy(ctx)
    return used, U, errs


def _oracle(nx, nv, bc, scheme, N, K, T, U0=None):
    U0 = W.sod(nx) if U0 is None else U0
    k = O.Kin(nx=nx, nv=nv, L=8.0, bc=BC[bc], eps=1e-2, scheme=scheme)
    p = O.Parareal(kin=k, T=T, N=N)
    Uo, errs, _ = O.parareal(p, U0, K=K)
    return Uo[K], errs


def test_sod_slices_take_the_cluster_run_and_match_the_oracle():
    # the Sod tube at the small size (64 x 16^3, N = 8, K = 3): the automatic
    # choice is the cluster run; both kernels agree with the oracle
    nx, nv, N, K, T = 64, 16, 8, 3, 0.1
    ref, errs_o = _oracle(nx, nv, pr.PR_BC_OUTFLOW, pr.PR_UPWIND, N, K, T)
    used, U, errs = _run(nx, nv, pr.PR_BC_OUTFLOW, pr.PR_UPWIND, N, K, T, pr.PR_FINE_AUTO)
    assert used == pr.PR_FINE_CLUSTER
    used_t, Ut, errs_t = _run(nx, nv, pr.PR_BC_OUTFLOW, pr.PR_UPWIND, N, K, T, pr.PR_FINE_TILED)
    assert used_t == pr.PR_FINE_TILED
    for n in range(N + 1):
        assert moment_rel_err(U[n], ref[n]) < TOL_MIXED, n
        assert moment_rel_err(Ut[n], ref[n]) < TOL_MIXED, n
    assert np.allclose(errs, errs_o, rtol=1e-2, atol=0)


@pytest.mark.parametrize("scheme", [pr.PR_UPWIND, pr.PR_MUSCL])
@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW, pr.PR_BC_REFLECT])
@pytest.mark.parametrize("nx,nv", [
    (37, 16),   # 13 CTAs of 3 cells, the last of 1
    (16, 16),   # 16 CTAs of one cell: every halo cell is a peer's or a ghost
    (2, 8),     # 2 CTAs of one cell, 64 threads
    (150, 8),   # 15 CTAs of 10 cells
])
def test_cluster_run_matches_oracle(nx, nv, bc, scheme):
    N, K, T = 3, 2, 0.02
    x = W.cell_centres(nx, 0.0, 1.0)
    w = 2 * np.pi * x
    U0 = np.stack([1 + 0.3 * np.sin(w) - 0.3 * (x > 0.6), 0.3 * np.cos(w), 0.1 * np.sin(2 * w),
                   -0.05 * np.cos(w), 1 + 0.2 * np.sin(w + 0.3)])
    ref, _ = _oracle(nx, nv, bc, scheme, N, K, T, U0)
    used, U, _ = _run(nx, nv, bc, scheme, N, K, T, pr.PR_FINE_CLUSTER, U0=U0)
    assert used == pr.PR_FINE_CLUSTER
    for n in range(N + 1):
        assert moment_rel_err(U[n], ref[n]) < TOL_MIXED, n


def test_cluster_run_in_waves_of_resident_slices():
    # max_batch < N: the iteration runs without a graph, in waves of 3 slices
    nx, nv, N, K, T = 48, 8, 7, 3, 0.06
    ref, errs_o = _oracle(nx, nv, pr.PR_BC_OUTFLOW, pr.PR_MUSCL, N, K, T)
    used, U, errs = _run(nx, nv, pr.PR_BC_OUTFLOW, pr.PR_MUSCL, N, K, T, pr.PR_FINE_CLUSTER, max_batch=3)
    assert used == pr.PR_FINE_CLUSTER
    for n in range(N + 1):
        assert moment_rel_err(U[n], ref[n]) < TOL_MIXED, n
    assert np.allclose(errs, errs_o, rtol=1e-2, atol=0)


def test_k_equals_n_on_the_cluster_run_is_its_serial_chain():
    # Sec. 2.2: N iterations reproduce the fine chain U^n = PFL(U^{n-1}) of the
    # propagator parareal runs, here the cluster kernel
    nx, nv, N, T = 40, 8, 4, 0.04
    used, U, errs = _run(nx, nv, pr.PR_BC_PERIODIC, pr.PR_UPWIND, N, N, T, pr.PR_FINE_CLUSTER,
                         U0=W.smooth_periodic(nx))
    assert used == pr.PR_FINE_CLUSTER
    k = O.Kin(nx=nx, nv=nv, L=8.0, bc=O.BC_PERIODIC, eps=1e-2, scheme=pr.PR_UPWIND)
    p = O.Parareal(kin=k, T=T, N=N)
    chain = [O.prim_to_cons(W.smooth_periodic(nx))]
    for _ in range(N):
        chain.append(O.fine_propagate(p, chain[-1]))
    for n in range(N + 1):
        assert moment_rel_err(U[n], chain[n]) < TOL_MIXED, n


def test_fine_path_selection_rules():
    # float64 slices, the first-order lifting and nv without an instantiation
    # stay on the tiled kernel; forcing the cluster run there is an error
    cases = [
        dict(precision=pr.PR_FP64, nv=16, lift=0),
        dict(precision=pr.PR_MIXED, nv=12, lift=0),
        dict(precision=pr.PR_MIXED, nv=16, lift=1),
    ]
    for cs in cases:
        ctx = pr.pr_init(32, 0.0, 1.0, pr.PR_BC_OUTFLOW, cs["nv"], 8.0, 1e-2, 0.05, 4,
                         precision=cs["precision"], lift_order=cs["lift"])
        try:
            assert pr.pr_get_fine_path(ctx) == pr.PR_FINE_TILED
            with pytest.raises(pr.PrError) as ei:
                pr.pr_set_fine_path(ctx, pr.PR_FINE_CLUSTER)
            assert ei.value.code == pr.PR_EINVAL
            assert pr.pr_get_fine_path(ctx) == pr.PR_FINE_TILED
            with pytest.raises(pr.PrError):
                pr.pr_set_fine_path(ctx, 7)
        finally:
            pr.pr_destroy(ctx)
    # a slice too large for one cluster's shared memory
    ctx = pr.pr_init(512, 0.0, 1.0, pr.PR_BC_PERIODIC, 16, 8.0, 1e-2, 0.01, 2, precision=pr.PR_MIXED)
    try:
        assert pr.pr_get_fine_path(ctx) == pr.PR_FINE_TILED
        with pytest.raises(pr.PrError):
            pr.pr_set_fine_path(ctx, pr.PR_FINE_CLUSTER)
    finally:
        pr.pr_destroy(ctx)
    # a force problem has no cluster run
    nx = 16
    ctx = pr.pr_init_force(nx, 0.0, 2.0, pr.PR_BC_PERIODIC, 8, 8, 8.0, 1e-2, 0.05, 2, W.test3_force(nx),
                           precision=pr.PR_MIXED)
    try:
        assert pr.pr_get_fine_path(ctx) == pr.PR_FINE_TILED
        with pytest.raises(pr.PrError):
            pr.pr_set_fine_path(ctx, pr.PR_FINE_CLUSTER)
        pr.pr_set_fine_path(ctx, pr.PR_FINE_TILED)
    finally:
        pr.pr_destroy(ctx)


def test_cluster_run_is_the_same_from_the_graph_and_in_waves():
    # each slice's cluster computes the same bits whether all slices run from
    # the captured iteration or in waves without a graph
    nx, nv, N, K, T = 48, 8, 7, 3, 0.06
    _, Ug, eg = _run(nx, nv, pr.PR_BC_PERIODIC, pr.PR_MUSCL, N, K, T, pr.PR_FINE_CLUSTER,
                     U0=W.smooth_periodic(nx))
    _, Uw, ew = _run(nx, nv, pr.PR_BC_PERIODIC, pr.PR_MUSCL, N, K, T, pr.PR_FINE_CLUSTER, max_batch=3,
                     U0=W.smooth_periodic(nx))
    for n in range(N + 1):
        assert np.array_equal(Ug[n], Uw[n]), n
    assert np.array_equal(eg, ew)
