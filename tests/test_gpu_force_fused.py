"""The fused single-pass force step (k_force_fused: the moments of f* from
per-column sums of f^n, each cell read, relaxed and written once, a CTA
walking several x columns): parity with the CPU FP64 oracle (Eq. 11 with the
force term, the fluxes of Eq. 13), agreement with the clustered step, bit
equality across walk lengths and run splits, its selection rules, and the
staging-timeout check on it."""
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
FTOL = {pr.PR_FP64: 1e-12, pr.PR_MIXED: 2e-6}   # f against the oracle


def _profile(nx, phase=0.0):
    x = W.cell_centres(nx, 0.0, 2.0)
    return np.stack([1 + 0.3 * np.sin(np.pi * x + phase), 0.4 * np.cos(np.pi * x), 0.1 + 0 * x, -0.05 + 0 * x,
                     1 + 0.25 * np.cos(np.pi * x + phase)])


def _problem(nx, nvx, nvp, L, bc, eps, n_inst=2):
    insts, kins, initial = [], [], []
    for k in range(n_inst):
        E = W.test3_force(nx) * (1.0 + 0.5 * k)
        kin = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, bc=BC[bc], eps=eps, E=E)
        insts.append(pr.ForceInstance(nx, nvx, nvp, O.v_fine_dt_stab(kin, 0.5), L=L, x0=0.0, x1=2.0, bc=bc,
                                      eps=eps, E=E))
        kins.append(kin)
        initial.append(_profile(nx, 0.7 * k))
    return insts, kins, initial


def _run(insts, cluster, march, splits, initial, precision=pr.PR_MIXED, scheme=pr.PR_UPWIND, persistent=-1):
    """Run the step counts in `splits` one after the other; every instance's f
    and moments and the walk length in use."""
    b = pr.pr_force_create(insts, scheme, precision)
    try:
        pr.pr_force_set_cluster(b, cluster)
        pr.pr_force_set_march(b, march)
        pr.pr_force_set_persistent(b, persistent)
        used = pr.pr_force_get_march(b)
        for i, U in enumerate(initial):
            pr.pr_force_set_initial(b, i, U)
        for n in splits:
            pr.pr_force_run(b, n)
        out = [(pr.pr_force_get_f(b, i), pr.pr_force_moments(b, i)) for i in range(len(insts))]
    finally:
        pr.pr_force_destroy(b)
    return out, used


@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW, pr.PR_BC_REFLECT])
@pytest.mark.parametrize("nvx,nvp,cluster", [
    (64, 16, 2),   # 32 rows per CTA in 4 groups of 8
    (60, 16, 2),   # 30 rows: groups of 8, 8, 8, 6
    (48, 8, 6),    # 8 rows per CTA: 8 groups of one row on 128 threads
    (32, 4, 16),   # 2 rows per CTA, 32-thread CTAs
])
@pytest.mark.parametrize("eps", [1e-2, math.inf])
@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
def test_fused_step_matches_oracle_and_clustered_step(bc, nvx, nvp, cluster, eps, precision):
    nx, L, n = 20, 7.0, 5
    insts, kins, initial = _problem(nx, nvx, nvp, L, bc, eps)
    got, used = _run(insts, cluster, 7, (2, n - 2), initial, precision)
    ref, used0 = _run(insts, cluster, 0, (n,), initial, precision)
    assert used == 7 and used0 == 0
    for k, ((f, V), (fr, Vr)) in enumerate(zip(got, ref)):
        fo = O.v_fine_run(kins[k], insts[k].c.dt, n, O.v_lift(kins[k], initial[k]))
        assert f_rel_err(f, fo) < FTOL[precision]
        assert moment_rel_err(V, O.v_project(kins[k], fo, conserved=True)) < TOL[precision]
        assert f_rel_err(f, fr) < FTOL[precision]   # the clustered step sums f* itself
        assert moment_rel_err(V, Vr) < TOL[precision]


@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_REFLECT])
@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
def test_walk_length_and_run_splits_give_the_same_bits(bc, precision):
    # each column's arithmetic does not depend on how columns group into
    # walks, and the partials kernel sums in the step's order
    nx, nvx, nvp, L = 23, 64, 16, 7.0
    insts, _, initial = _problem(nx, nvx, nvp, L, bc, 1e-3, n_inst=3)
    ref, _ = _run(insts, 4, 1, (6,), initial, precision)
    for march, splits in ((3, (6,)), (8, (1, 1, 4)), (23, (2, 4)), (32, (6,))):
        got, used = _run(insts, 4, march, splits, initial, precision)
        assert used == min(march, nx) or (march, used) == (8, 8)
        for (f, V), (fr, Vr) in zip(got, ref):
            assert np.array_equal(f, fr)
            assert np.array_equal(V, Vr)
    # a new walk length drops the partials: the partials kernel recomputes
    # them from the stored f^n, bit for bit those the step wrote
    b = pr.pr_force_create(insts, pr.PR_UPWIND, precision)
    try:
        pr.pr_force_set_cluster(b, 4)
        pr.pr_force_set_march(b, 1)
        for i, U in enumerate(initial):
            pr.pr_force_set_initial(b, i, U)
        pr.pr_force_run(b, 2)
        pr.pr_force_set_march(b, 5)
        pr.pr_force_run(b, 4)
        for i, (fr, Vr) in enumerate(ref):
            assert np.array_equal(pr.pr_force_get_f(b, i), fr)
            assert np.array_equal(pr.pr_force_moments(b, i), Vr)
    finally:
        pr.pr_force_destroy(b)


def test_fused_step_from_a_loaded_state_matches_oracle():
    # set_f: the partials of the loaded state come from the partials kernel
    nx, nvx, nvp, L, n = 12, 64, 8, 8.0, 4
    E = W.test3_force(nx)
    kin = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, bc=O.BC_OUTFLOW, eps=1e-3, E=E)
    dt = O.v_fine_dt_stab(kin, 0.5)
    f0 = np.random.default_rng(7).random((nx, kin.ncol)) * O.v_lift(kin, _profile(nx))
    b = pr.pr_force_create([pr.ForceInstance(nx, nvx, nvp, dt, L=L, x0=0.0, x1=2.0, bc=pr.PR_BC_OUTFLOW, eps=1e-3,
                                             E=E)], pr.PR_UPWIND, pr.PR_MIXED)
    try:
        pr.pr_force_set_cluster(b, 2)   # one CTA's 64 rows would straddle v_x = 0
        pr.pr_force_set_march(b, 3)
        pr.pr_force_set_f(b, 0, f0)
        pr.pr_force_run(b, n)
        f = pr.pr_force_get_f(b, 0)
        V = pr.pr_force_moments(b, 0)
    finally:
        pr.pr_force_destroy(b)
    fo = O.v_fine_run(kin, dt, n, f0)
    assert f_rel_err(f, fo) < 2e-6
    assert moment_rel_err(V, O.v_project(kin, fo, conserved=True)) < TOL_MIXED


def test_fused_selection_rules():
    nx, nvx, nvp = 12, 64, 16
    E = W.test3_force(nx)
    inst = pr.ForceInstance(nx, nvx, nvp, 1e-3, L=8.0, x0=0.0, x1=2.0, E=E)
    b = pr.pr_force_create([inst], pr.PR_UPWIND, pr.PR_MIXED)
    try:
        # 12 columns, far fewer than the resident CTA groups: the clustered step
        assert pr.pr_force_config(b) == (2, 8192)
        assert pr.pr_force_get_march(b) == 0
        pr.pr_force_set_march(b, 5)
        assert pr.pr_force_get_march(b) == 4      # 3 equal walks
        pr.pr_force_set_march(b, 0)
        assert pr.pr_force_get_march(b) == 0      # the clustered step
        pr.pr_force_set_march(b, 100)
        assert pr.pr_force_get_march(b) == 12     # one walk over every column
        # 3 CTAs of 22 rows: the middle one straddles v_x = 0, so the explicit
        # walk falls back to the clustered step and a new walk is refused
        pr.pr_force_set_cluster(b, 3)
        assert pr.pr_force_get_march(b) == 0
        with pytest.raises(pr.PrError) as ei:
            pr.pr_force_set_march(b, 4)
        assert ei.value.code == pr.PR_EINVAL
        assert pr.pr_force_get_march(b) == 0
        with pytest.raises(pr.PrError):
            pr.pr_force_set_march(b, -2)
        pr.pr_force_set_cluster(b, 2)
        assert pr.pr_force_get_march(b) == 12     # the explicit walk applies again
        pr.pr_force_set_march(b, -1)
        assert pr.pr_force_get_march(b) == 0
        # more than 256 threads per CTA: the clustered step
        pr.pr_force_set_threads(b, 512)
        assert pr.pr_force_get_march(b) == 0
    finally:
        pr.pr_force_destroy(b)
    # FP64 upwind has the fused step too (16-byte lanes of two doubles)
    b = pr.pr_force_create([inst], pr.PR_UPWIND, pr.PR_FP64)
    try:
        pr.pr_force_set_cluster(b, 2)
        pr.pr_force_set_march(b, 4)
        assert pr.pr_force_get_march(b) == 4
    finally:
        pr.pr_force_destroy(b)
    for scheme, precision, nv in ((pr.PR_MUSCL, pr.PR_MIXED, nvp), (pr.PR_MUSCL, pr.PR_FP64, nvp),
                                  (pr.PR_UPWIND, pr.PR_MIXED, 5)):  # 25-float rows: no bulk copies
        b = pr.pr_force_create([pr.ForceInstance(nx, nvx, nv, 1e-3, L=8.0, x0=0.0, x1=2.0, E=E)], scheme, precision)
        try:
            assert pr.pr_force_get_march(b) == 0
            with pytest.raises(pr.PrError) as ei:
                pr.pr_force_set_march(b, 4)
            assert ei.value.code == pr.PR_EINVAL
        finally:
            pr.pr_force_destroy(b)


def test_test3_batch_uses_long_walks_by_default():
    # 64 Test 3 instances (100 x 256 x 16 x 16): 6400 columns
    nx = 100
    E = W.test3_force(nx)
    insts = [pr.ForceInstance(nx, 256, 16, 6.25e-4, L=8.0, x0=0.0, x1=2.0, eps=1e-5, E=E) for _ in range(64)]
    b = pr.pr_force_create(insts, pr.PR_UPWIND, pr.PR_MIXED)
    try:
        # 8 CTAs of 32 rows (two share an SM), walks of about 17 columns
        assert pr.pr_force_config(b) == (8, 8192)
        assert pr.pr_force_get_march(b) >= 8
    finally:
        pr.pr_force_destroy(b)


def test_fused_staging_wait_runs_out_and_object_stays_usable():
    nx = 16
    E = W.test3_force(nx)
    inst = pr.ForceInstance(nx, 32, 8, 1e-3, E=E)
    b = pr.pr_force_create([inst], pr.PR_UPWIND, pr.PR_MIXED)
    fresh = pr.pr_force_create([inst], pr.PR_UPWIND, pr.PR_MIXED)
    try:
        for o in (b, fresh):
            pr.pr_force_set_cluster(o, 2)
            pr.pr_force_set_march(o, 4)
        pr.pr_force_set_initial(b, 0, W.smooth_periodic(nx))
        assert pr.pr_force_inject_wait_timeout(b, 20) == pr.PR_ETIMEOUT
        assert "timed out" in pr.pr_force_last_error(b)
        runs = []
        for o in (b, fresh):
            pr.pr_force_set_initial(o, 0, W.smooth_periodic(nx))
            pr.pr_force_run(o, 3)
            runs.append(pr.pr_force_moments(o, 0))
        assert np.array_equal(runs[0], runs[1])
    finally:
        pr.pr_force_destroy(b)
        pr.pr_force_destroy(fresh)


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
def test_cluster_wider_than_its_ctas_threads(precision):
    # the clustered step with 16 CTAs of 2 rows of 16 cells: 32-thread CTAs
    # gather 80 partials
    nx, nvx, nvp, L, n = 6, 32, 4, 6.0, 3
    E = W.test3_force(nx)
    U = _profile(nx)
    kin = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, eps=1e-2, E=E)
    dt = O.v_fine_dt_stab(kin, 0.5)
    b = pr.pr_force_create([pr.ForceInstance(nx, nvx, nvp, dt, L=L, x0=0.0, x1=2.0, eps=1e-2, E=E)],
                           pr.PR_UPWIND, precision)
    try:
        pr.pr_force_set_march(b, 0)
        pr.pr_force_set_cluster(b, 16)
        pr.pr_force_set_initial(b, 0, U)
        pr.pr_force_run(b, n)
        V = pr.pr_force_moments(b, 0)
    finally:
        pr.pr_force_destroy(b)
    Vo = O.v_project(kin, O.v_fine_run(kin, dt, n, O.v_lift(kin, U)), conserved=True)
    assert moment_rel_err(V, Vo) < (1e-12 if precision == pr.PR_FP64 else TOL_MIXED)


@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW, pr.PR_BC_REFLECT])
@pytest.mark.parametrize("nvx,nvp,cluster,march", [(64, 16, 2, 1), (64, 16, 2, 6), (48, 8, 6, 4), (32, 4, 16, 23)])
@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
def test_persistent_run_is_bitwise_the_stepwise_run(bc, nvx, nvp, cluster, march, precision):
    # all steps of a run in one launch, items waiting on their neighbour
    # walks, against one launch per step
    nx, L, n = 23, 7.0, 7
    insts, _, initial = _problem(nx, nvx, nvp, L, bc, 1e-3, n_inst=3)
    out = []
    for mode in (0, 1):
        b = pr.pr_force_create(insts, pr.PR_UPWIND, precision)
        try:
            pr.pr_force_set_cluster(b, cluster)
            pr.pr_force_set_march(b, march)
            pr.pr_force_set_persistent(b, mode)
            for i, U in enumerate(initial):
                pr.pr_force_set_initial(b, i, U)
            pr.pr_force_run(b, 1)
            pr.pr_force_run(b, n - 1)
            out.append([(pr.pr_force_get_f(b, i), pr.pr_force_moments(b, i)) for i in range(3)])
        finally:
            pr.pr_force_destroy(b)
    for (f, V), (fr, Vr) in zip(out[1], out[0]):
        assert np.array_equal(f, fr)
        assert np.array_equal(V, Vr)


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
def test_force_parareal_on_the_fused_step_matches_oracle(persistent, precision):
    # Algorithm 2 with the fused step for the fine propagator (one launch per
    # slice run, or one persistent launch): the slices are the instances
    nx, nvx, nvp, L, eps, T, N, K = 16, 32, 8, 6.0, 1e-2, 0.05, 6, 3
    E = W.test3_force(nx)
    U0 = _profile(nx)
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, eps=eps, E=E)
    Uo, errs_o, _ = O.v_parareal(O.VParareal(kin=k, T=T, N=N), U0, K=K)
    ctx = pr.pr_init_force(nx, 0.0, 2.0, pr.PR_BC_PERIODIC, nvx, nvp, L, eps, T, N, E, precision=precision)
    try:
        pr.pr_set_force_step(ctx, 2, 4, persistent)
        pr.pr_set_initial(ctx, U0)
        kd, errs = pr.pr_parareal_run(ctx, K)
        for n in range(N + 1):
            assert moment_rel_err(pr.pr_moments(ctx, n), Uo[K][n]) < TOL[precision], n
    finally:
        pr.pr_destroy(ctx)


def test_persistent_dependency_wait_runs_out_and_object_stays_usable():
    nx = 16
    E = W.test3_force(nx)
    inst = pr.ForceInstance(nx, 32, 8, 1e-3, E=E)
    b = pr.pr_force_create([inst], pr.PR_UPWIND, pr.PR_MIXED)
    fresh = pr.pr_force_create([inst], pr.PR_UPWIND, pr.PR_MIXED)
    try:
        for o in (b, fresh):
            pr.pr_force_set_cluster(o, 2)
            pr.pr_force_set_march(o, 4)
            pr.pr_force_set_persistent(o, 1)
        pr.pr_force_set_initial(b, 0, W.smooth_periodic(nx))
        assert pr.pr_force_inject_wait_timeout(b, 20) == pr.PR_ETIMEOUT
        assert "timed out" in pr.pr_force_last_error(b)
        runs = []
        for o in (b, fresh):
            pr.pr_force_set_initial(o, 0, W.smooth_periodic(nx))
            pr.pr_force_run(o, 3)
            runs.append(pr.pr_force_moments(o, 0))
        assert np.array_equal(runs[0], runs[1])
    finally:
        pr.pr_force_destroy(b)
        pr.pr_force_destroy(fresh)


def test_force_step_setting_needs_a_force_problem():
    ctx = pr.pr_init(8, 0.0, 1.0, pr.PR_BC_PERIODIC, 4, 8.0, 1e-2, 0.1, 2)
    try:
        with pytest.raises(pr.PrError) as ei:
            pr.pr_set_force_step(ctx, 0, 4, 1)
        assert ei.value.code == pr.PR_EINVAL
    finally:
        pr.pr_destroy(ctx)


# ------------------------------------------------------------ MUSCL fused step
# Periodic and outflow boundaries; a CTA's rows per thread at most 4 (float)
# or 8 (double).
MU_GEOMS = [
    (64, 16, 4),   # 16 rows per CTA: float 4 groups of 4 rows, double 2 of 8
    (60, 16, 4),   # 15 rows: groups of 4, 4, 4, 3 (double 8, 7)
    (48, 8, 6),    # 8 rows per CTA, one row per thread
    (32, 4, 16),   # 2 rows per CTA, 32-thread CTAs
]


@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW])
@pytest.mark.parametrize("nvx,nvp,cluster", MU_GEOMS)
@pytest.mark.parametrize("eps", [1e-2, math.inf])
@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
def test_muscl_fused_step_matches_oracle_and_clustered_step(bc, nvx, nvp, cluster, eps, precision):
    nx, L, n = 20, 7.0, 5
    insts, kins, initial = _problem(nx, nvx, nvp, L, bc, eps)
    for k in kins:
        k.scheme = O.MUSCL
    got, used = _run(insts, cluster, 7, (2, n - 2), initial, precision, pr.PR_MUSCL)
    ref, used0 = _run(insts, cluster, 0, (n,), initial, precision, pr.PR_MUSCL)
    assert used == 7 and used0 == 0
    for k, ((f, V), (fr, Vr)) in enumerate(zip(got, ref)):
        fo = O.v_fine_run(kins[k], insts[k].c.dt, n, O.v_lift(kins[k], initial[k]))
        assert f_rel_err(f, fo) < FTOL[precision]
        assert moment_rel_err(V, O.v_project(kins[k], fo, conserved=True)) < TOL[precision]
        assert f_rel_err(f, fr) < FTOL[precision]
        assert moment_rel_err(V, Vr) < TOL[precision]


@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW])
@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
def test_muscl_walk_length_and_run_splits_give_the_same_bits(bc, precision):
    # a walk's neighbour columns are computed with the arithmetic of the walk
    # that owns them, and the partials kernel sums the limited values in the
    # step's order
    nx, nvx, nvp, L = 23, 64, 16, 7.0
    insts, _, initial = _problem(nx, nvx, nvp, L, bc, 1e-3, n_inst=3)
    ref, used = _run(insts, 4, 3, (6,), initial, precision, pr.PR_MUSCL)
    assert used == 4   # walks of 3 would leave a last walk of 2 columns
    for march, splits in ((1, (6,)), (5, (1, 1, 4)), (8, (2, 4)), (23, (6,)), (32, (3, 3))):
        got, used = _run(insts, 4, march, splits, initial, precision, pr.PR_MUSCL)
        assert used >= 3
        for (f, V), (fr, Vr) in zip(got, ref):
            assert np.array_equal(f, fr)
            assert np.array_equal(V, Vr)
    b = pr.pr_force_create(insts, pr.PR_MUSCL, precision)
    try:
        pr.pr_force_set_cluster(b, 4)
        pr.pr_force_set_march(b, 3)
        for i, U in enumerate(initial):
            pr.pr_force_set_initial(b, i, U)
        pr.pr_force_run(b, 2)
        pr.pr_force_set_march(b, 7)   # the partials kernel recomputes the limited sums
        pr.pr_force_run(b, 4)
        for i, (fr, Vr) in enumerate(ref):
            assert np.array_equal(pr.pr_force_get_f(b, i), fr)
            assert np.array_equal(pr.pr_force_moments(b, i), Vr)
    finally:
        pr.pr_force_destroy(b)


@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW])
@pytest.mark.parametrize("nvx,nvp,cluster,march", [(64, 16, 4, 3), (64, 16, 4, 6), (48, 8, 6, 4), (32, 4, 16, 23)])
@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
def test_muscl_persistent_run_is_bitwise_the_stepwise_run(bc, nvx, nvp, cluster, march, precision):
    nx, L, n = 23, 7.0, 7
    insts, _, initial = _problem(nx, nvx, nvp, L, bc, 1e-3, n_inst=3)
    out = [_run(insts, cluster, march, (1, n - 1), initial, precision, pr.PR_MUSCL, mode)[0] for mode in (0, 1)]
    for (f, V), (fr, Vr) in zip(out[1], out[0]):
        assert np.array_equal(f, fr)
        assert np.array_equal(V, Vr)


@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
def test_muscl_fused_step_from_a_loaded_state_matches_oracle(precision):
    # a rough state (the limiter active everywhere), outflow walls, and one
    # walk over all columns next to walks of three
    nx, nvx, nvp, L, n = 12, 64, 8, 8.0, 4
    E = W.test3_force(nx)
    kin = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, bc=O.BC_OUTFLOW, eps=1e-3, scheme=O.MUSCL, E=E)
    dt = O.v_fine_dt_stab(kin, 0.5)
    f0 = np.random.default_rng(7).random((nx, kin.ncol)) * O.v_lift(kin, _profile(nx))
    fo = O.v_fine_run(kin, dt, n, f0)
    for march in (3, 12):
        b = pr.pr_force_create([pr.ForceInstance(nx, nvx, nvp, dt, L=L, x0=0.0, x1=2.0, bc=pr.PR_BC_OUTFLOW,
                                                 eps=1e-3, E=E)], pr.PR_MUSCL, precision)
        try:
            pr.pr_force_set_cluster(b, 8)
            pr.pr_force_set_march(b, march)
            assert pr.pr_force_get_march(b) == march
            pr.pr_force_set_f(b, 0, f0)
            pr.pr_force_run(b, n)
            f = pr.pr_force_get_f(b, 0)
            V = pr.pr_force_moments(b, 0)
        finally:
            pr.pr_force_destroy(b)
        assert f_rel_err(f, fo) < FTOL[precision]
        assert moment_rel_err(V, O.v_project(kin, fo, conserved=True)) < TOL[precision]


def test_muscl_fused_selection_rules():
    nx, nvx, nvp = 12, 64, 16
    E = W.test3_force(nx)
    for precision in (pr.PR_MIXED, pr.PR_FP64):
        inst = pr.ForceInstance(nx, nvx, nvp, 1e-3, L=8.0, x0=0.0, x1=2.0, E=E)
        b = pr.pr_force_create([inst], pr.PR_MUSCL, precision)
        try:
            if precision == pr.PR_MIXED:
                # 2 CTAs of 32 rows: more rows per thread than the kernel
                # keeps (FP64 has no layout of 2 CTAs for this column at all)
                pr.pr_force_set_cluster(b, 2)
                with pytest.raises(pr.PrError) as ei:
                    pr.pr_force_set_march(b, 4)
                assert ei.value.code == pr.PR_EINVAL
            pr.pr_force_set_cluster(b, 4)
            pr.pr_force_set_march(b, 4)
            assert pr.pr_force_get_march(b) == 4
            pr.pr_force_set_march(b, 2)   # a walk reads three columns past its ends
            assert pr.pr_force_get_march(b) == 3
            pr.pr_force_set_march(b, 11)
            assert pr.pr_force_get_march(b) == 6    # two equal walks
        finally:
            pr.pr_force_destroy(b)
        # 10 columns: walks of 3 or 4 would leave a last walk of 1 or 2
        b = pr.pr_force_create([pr.ForceInstance(10, nvx, nvp, 1e-3, L=8.0, x0=0.0, x1=2.0, E=E[:10])],
                               pr.PR_MUSCL, precision)
        try:
            pr.pr_force_set_cluster(b, 4)
            pr.pr_force_set_march(b, 3)
            assert pr.pr_force_get_march(b) == 5
        finally:
            pr.pr_force_destroy(b)
    # a reflecting wall keeps the clustered step
    inst = pr.ForceInstance(nx, nvx, nvp, 1e-3, L=8.0, x0=0.0, x1=2.0, bc=pr.PR_BC_REFLECT, E=E)
    b = pr.pr_force_create([inst], pr.PR_MUSCL, pr.PR_MIXED)
    try:
        pr.pr_force_set_cluster(b, 4)
        assert pr.pr_force_get_march(b) == 0
        with pytest.raises(pr.PrError) as ei:
            pr.pr_force_set_march(b, 4)
        assert ei.value.code == pr.PR_EINVAL
    finally:
        pr.pr_force_destroy(b)


def test_muscl_test3_batch_uses_the_fused_step_by_default():
    nx = 100
    E = W.test3_force(nx)
    insts = [pr.ForceInstance(nx, 256, 16, 6.25e-4, L=8.0, x0=0.0, x1=2.0, eps=1e-5, E=E) for _ in range(64)]
    for precision in (pr.PR_MIXED, pr.PR_FP64):
        b = pr.pr_force_create(insts, pr.PR_MUSCL, precision)
        try:
            assert pr.pr_force_config(b) == (16, 4096)   # 16 CTAs of 16 rows
            assert pr.pr_force_get_march(b) >= 3
        finally:
            pr.pr_force_destroy(b)


@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
def test_muscl_force_parareal_on_the_fused_step_matches_oracle(precision):
    nx, nvx, nvp, L, eps, T, N, K = 16, 32, 8, 6.0, 1e-2, 0.05, 6, 3
    E = W.test3_force(nx)
    U0 = _profile(nx)
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, eps=eps, scheme=O.MUSCL, E=E)
    Uo, errs_o, _ = O.v_parareal(O.VParareal(kin=k, T=T, N=N), U0, K=K)
    ctx = pr.pr_init_force(nx, 0.0, 2.0, pr.PR_BC_PERIODIC, nvx, nvp, L, eps, T, N, E, scheme=pr.PR_MUSCL,
                           precision=precision)
    try:
        pr.pr_set_force_step(ctx, 4, 4, 1)
        pr.pr_set_initial(ctx, U0)
        kd, errs = pr.pr_parareal_run(ctx, K)
        for n in range(N + 1):
            assert moment_rel_err(pr.pr_moments(ctx, n), Uo[K][n]) < TOL[precision], n
    finally:
        pr.pr_destroy(ctx)


@pytest.mark.parametrize("scheme", [pr.PR_UPWIND, pr.PR_MUSCL])
@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
def test_autotune_keeps_the_states_and_picks_a_valid_layout(scheme, precision):
    nx, nvx, nvp, L = 40, 64, 16, 7.0
    insts, kins, initial = _problem(nx, nvx, nvp, L, pr.PR_BC_PERIODIC, 1e-2, n_inst=4)
    b = pr.pr_force_create(insts, scheme, precision)
    try:
        for i, U in enumerate(initial):
            pr.pr_force_set_initial(b, i, U)
        pr.pr_force_run(b, 2)
        before = [(pr.pr_force_get_f(b, i), pr.pr_force_moments(b, i)) for i in range(4)]
        cluster, walk = pr.pr_force_autotune(b, 3)
        after = [(pr.pr_force_get_f(b, i), pr.pr_force_moments(b, i)) for i in range(4)]
        for (f, V), (fa, Va) in zip(before, after):
            assert np.array_equal(f, fa) and np.array_equal(V, Va)
        assert pr.pr_force_config(b)[0] == cluster and pr.pr_force_get_march(b) == walk
        pr.pr_force_run(b, 3)
        tuned = [(pr.pr_force_get_f(b, i), pr.pr_force_moments(b, i)) for i in range(4)]
    finally:
        pr.pr_force_destroy(b)
    # the same sequence with the layout set by hand (2 steps on the default
    # layout, 3 on the chosen one) gives the same bits; the oracle agrees
    b = pr.pr_force_create(insts, scheme, precision)
    try:
        for i, U in enumerate(initial):
            pr.pr_force_set_initial(b, i, U)
        pr.pr_force_run(b, 2)
        pr.pr_force_set_cluster(b, cluster)
        pr.pr_force_set_march(b, walk)
        assert pr.pr_force_get_march(b) == walk
        pr.pr_force_run(b, 3)
        ref = [(pr.pr_force_get_f(b, i), pr.pr_force_moments(b, i)) for i in range(4)]
    finally:
        pr.pr_force_destroy(b)
    for k, ((f, V), (fr, Vr)) in enumerate(zip(tuned, ref)):
        assert np.array_equal(f, fr) and np.array_equal(V, Vr)
        kins[k].scheme = O.MUSCL if scheme == pr.PR_MUSCL else O.UPWIND
        fo = O.v_fine_run(kins[k], insts[k].c.dt, 5, O.v_lift(kins[k], initial[k]))
        assert f_rel_err(f, fo) < FTOL[precision]
