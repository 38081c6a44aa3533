"""Parity of the higher-order coupling on the GPU (Eq. 8, Def. 3 with L = 1)
with the CPU FP64 oracle: the first-order lifting on both fine paths, the
compressible Navier-Stokes coarse step, and parareal with either."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import workloads as W
from helpers import TOL_FP64, TOL_MIXED, f_rel_err, moment_rel_err

pytestmark = pytest.mark.gpu

BC = {pr.PR_BC_PERIODIC: O.BC_PERIODIC, pr.PR_BC_OUTFLOW: O.BC_OUTFLOW, pr.PR_BC_REFLECT: O.BC_REFLECT}
TOL = {pr.PR_FP64: TOL_FP64, pr.PR_MIXED: TOL_MIXED}


def _prof(nx, x1=1.0):
    x = W.cell_centres(nx, 0.0, x1) / x1
    w = 2 * np.pi * x
    return np.stack([1 + 0.3 * np.sin(w), 0.2 * np.cos(w), 0.1 * np.sin(2 * w), -0.05 * np.cos(w),
                     1 + 0.25 * np.sin(w + 0.3)])


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW, pr.PR_BC_REFLECT])
def test_first_order_lift_and_run_match_oracle(precision, bc):
    nx, nv, L, eps, n = 40, 12, 7.0, 2e-2, 5
    U = _prof(nx)
    dt = pr.fine_dt(nx, nv, L)
    b = pr.pr_batch_create([pr.instance(nx, nv, dt, L=L, bc=bc, eps=eps, scheme=pr.PR_MUSCL)], precision)
    try:
        pr.pr_batch_set_lift_order(b, 1)
        pr.pr_batch_set_initial(b, 0, U)
        f0 = pr.pr_batch_get_f(b, 0)
        V0 = pr.pr_batch_moments(b, 0)
        pr.pr_batch_run(b, n)
        V = pr.pr_batch_moments(b, 0)
    finally:
        pr.pr_batch_destroy(b)
    k = O.Kin(nx=nx, nv=nv, L=L, bc=BC[bc], eps=eps, scheme=O.MUSCL)
    fo = O.lift_ce(k, U)
    assert f_rel_err(f0, fo) < (1e-13 if precision == pr.PR_FP64 else 1e-6)
    assert moment_rel_err(V0, O.project(k, fo, conserved=True)) < TOL[precision]
    Vo = O.project(k, O.fine_run(k, dt, n, fo), conserved=True)
    assert moment_rel_err(V, Vo) < TOL[precision]


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
def test_force_path_first_order_lift_matches_oracle(precision):
    nx, nvx, nvp, L, eps = 16, 24, 8, 8.0, 1e-2
    E = W.test3_force(nx)
    U = _prof(nx, 2.0)
    inst = pr.ForceInstance(nx, nvx, nvp, 1e-3, L=L, x0=0.0, x1=2.0, bc=pr.PR_BC_REFLECT, eps=eps, E=E)
    b = pr.pr_force_create([inst], pr.PR_UPWIND, precision)
    try:
        pr.pr_force_set_lift_order(b, 1)
        pr.pr_force_set_initial(b, 0, U)
        f0 = pr.pr_force_get_f(b, 0)
        pr.pr_force_run(b, 4)
        V = pr.pr_force_moments(b, 0)
    finally:
        pr.pr_force_destroy(b)
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, bc=O.BC_REFLECT, eps=eps, E=E)
    fo = O.v_lift_ce(k, U)
    assert f_rel_err(f0, fo) < (1e-13 if precision == pr.PR_FP64 else 1e-6)
    assert moment_rel_err(V, O.v_project(k, O.v_fine_run(k, 1e-3, 4, fo), conserved=True)) < TOL[precision]


@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW, pr.PR_BC_REFLECT])
def test_navier_stokes_coarse_step_matches_oracle(bc):
    nx, eps = 48, 2e-2
    V = O.prim_to_cons(_prof(nx))
    ctx = pr.pr_init(nx, 0.0, 1.0, bc, 8, 8.0, eps, 0.1, 4, coarse_model=pr.PR_COARSE_CNS)
    try:
        got = pr.pr_coarse_step(ctx, V, 0.04)
    finally:
        pr.pr_destroy(ctx)
    want, ns = O.coarse_run_cns(nx, BC[bc], 0.5, 0.04, V, eps)
    assert ns > 1
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
@pytest.mark.parametrize("coarse,lift", [(pr.PR_COARSE_CNS, 0), (pr.PR_COARSE_CNS, 1), (pr.PR_COARSE_EULER, 1)])
@pytest.mark.parametrize("max_batch", [0, 3])
def test_parareal_with_cns_and_first_order_lift_matches_oracle(precision, coarse, lift, max_batch):
    nx, nv, L, eps, T, N, K = 32, 8, 8.0, 2e-2, 0.05, 5, 3
    U0 = _prof(nx)
    k = O.Kin(nx=nx, nv=nv, L=L, eps=eps, scheme=O.UPWIND)
    p = O.Parareal(kin=k, T=T, N=N, coarse=coarse, lift=lift)
    Uo, errs_o, _ = O.parareal(p, U0, K=K)
    ctx = pr.pr_init(nx, 0.0, 1.0, pr.PR_BC_PERIODIC, nv, L, eps, T, N, precision=precision, max_batch=max_batch,
                     coarse_model=coarse, lift_order=lift)
    try:
        pr.pr_set_initial(ctx, U0)
        for n in range(N + 1):
            assert moment_rel_err(pr.pr_moments(ctx, n), Uo[0][n]) < TOL_FP64, n
        kd, errs = pr.pr_parareal_run(ctx, K)
        for n in range(N + 1):
            assert moment_rel_err(pr.pr_moments(ctx, n), Uo[K][n]) < TOL[precision], n
        assert np.all(np.abs(errs - errs_o) <= (1e-9 if precision == pr.PR_FP64 else 1e-3) * np.abs(errs_o))
    finally:
        pr.pr_destroy(ctx)


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
def test_force_parareal_with_cns_and_first_order_lift_matches_oracle(precision):
    nx, nvx, nvp, L, eps, T, N, K = 16, 16, 10, 6.0, 1e-2, 0.05, 4, 2
    E = W.test3_force(nx)
    U0 = _prof(nx, 2.0)
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, eps=eps, E=E)
    p = O.VParareal(kin=k, T=T, N=N, coarse=O.COARSE_CNS, lift=1)
    Uo, errs_o, _ = O.v_parareal(p, U0, K=K)
    ctx = pr.pr_init_force(nx, 0.0, 2.0, pr.PR_BC_PERIODIC, nvx, nvp, L, eps, T, N, E, precision=precision,
                           coarse_model=pr.PR_COARSE_CNS, lift_order=1)
    try:
        pr.pr_set_initial(ctx, U0)
        kd, errs = pr.pr_parareal_run(ctx, K)
        for n in range(N + 1):
            assert moment_rel_err(pr.pr_moments(ctx, n), Uo[K][n]) < TOL[precision], n
    finally:
        pr.pr_destroy(ctx)


def test_higher_order_options_need_collisions():
    with pytest.raises(pr.PrError) as ei:
        pr.pr_init(8, 0.0, 1.0, pr.PR_BC_PERIODIC, 4, 8.0, math.inf, 0.1, 2, coarse_model=pr.PR_COARSE_CNS)
    assert ei.value.code == pr.PR_EINVAL
    b = pr.pr_batch_create([pr.instance(8, 4, 1e-3, eps=math.inf)], pr.PR_FP64)
    try:
        with pytest.raises(pr.PrError) as ei:
            pr.pr_batch_set_lift_order(b, 1)
        assert ei.value.code == pr.PR_EINVAL
    finally:
        pr.pr_batch_destroy(b)


@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW, pr.PR_BC_REFLECT])
def test_first_order_lift_single_cell_and_two_cells(bc):
    # nx = 1: every gradient is zero (periodic, outflow) or comes from the
    # mirrored ghost (reflecting u_x); nx = 2 the smallest stencil
    for nx in (1, 2):
        U = _prof(max(nx, 2))[:, :nx].copy()
        nv, L, eps = 8, 6.0, 3e-2
        b = pr.pr_batch_create([pr.instance(nx, nv, 1e-3, L=L, bc=bc, eps=eps)], pr.PR_FP64)
        try:
            pr.pr_batch_set_lift_order(b, 1)
            pr.pr_batch_set_initial(b, 0, U)
            f = pr.pr_batch_get_f(b, 0)
        finally:
            pr.pr_batch_destroy(b)
        k = O.Kin(nx=nx, nv=nv, L=L, bc=BC[bc], eps=eps)
        assert f_rel_err(f, O.lift_ce(k, U)) < 1e-13, nx
