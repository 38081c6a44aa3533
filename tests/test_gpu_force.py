"""Parity of the exterior-force path (Eq. 11 with E != 0, the v_x Rusanov
flux of Eq. 13, the Euler source of Eq. 5; Test 3) with the CPU FP64 oracle,
through the C ABI: the clustered fine step, the lift, set_f / get_f, the
coarse solver with the source and the parareal iteration."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import workloads as W
from helpers import TOL_FP64, TOL_MIXED, f_rel_err, moment_rel_err

pytestmark = pytest.mark.gpu

BC = {pr.PR_BC_PERIODIC: O.BC_PERIODIC, pr.PR_BC_OUTFLOW: O.BC_OUTFLOW, pr.PR_BC_REFLECT: O.BC_REFLECT}
SCH = {pr.PR_UPWIND: O.UPWIND, pr.PR_MUSCL: O.MUSCL}
TOL = {pr.PR_FP64: TOL_FP64, pr.PR_MIXED: TOL_MIXED}


def _vkin(nx, nvx, nvp, L, bc, eps, scheme, E, x0=0.0, x1=2.0):
    return O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=x0, x1=x1, bc=BC[bc], eps=eps, scheme=SCH[scheme], E=E)


def _profile(nx):
    x = W.cell_centres(nx, 0.0, 2.0)
    return np.stack([1 + 0.3 * np.sin(np.pi * x), 0.4 * np.cos(np.pi * x), 0.1 + 0 * x, -0.05 + 0 * x,
                     1 + 0.25 * np.cos(np.pi * x)])


def _beams_f_oracle(k):
    b1, b2 = W.test3_beams(k.nx)
    return O.v_lift(k, b1) + O.v_lift(k, b2)


def _beams_f_gpu(nx, nvx, nvp, L, dt):
    # each beam lifted by the library, summed on the host
    insts = [pr.ForceInstance(nx, nvx, nvp, dt, L=L, x0=0.0, x1=2.0) for _ in range(2)]
    b = pr.pr_force_create(insts, pr.PR_UPWIND, pr.PR_FP64)
    try:
        for i, U in enumerate(W.test3_beams(nx)):
            pr.pr_force_set_initial(b, i, U)
        return pr.pr_force_get_f(b, 0) + pr.pr_force_get_f(b, 1)
    finally:
        pr.pr_force_destroy(b)


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
@pytest.mark.parametrize("scheme", [pr.PR_UPWIND, pr.PR_MUSCL])
@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW, pr.PR_BC_REFLECT])
@pytest.mark.parametrize("cluster", [1, 3, 7])
def test_fine_steps_match_oracle(precision, scheme, bc, cluster):
    # nvx = 25 (odd: a v_x = 0 node) split over 1, 3 or 7 CTAs (9/9/7 and
    # 4 x 6 + 1 rows: ragged last CTAs); nvp = 6: 36 (v_y, v_z) cells on a
    # 64-thread CTA, so 28 threads only join the reductions
    nx, nvx, nvp, L, n = 14, 25, 6, 7.0, 5
    E = W.test3_force(nx)
    U = _profile(nx)
    for eps in (1e-2, math.inf):
        k = _vkin(nx, nvx, nvp, L, bc, eps, scheme, E)
        dt = O.v_fine_dt_stab(k, 0.5)
        inst = pr.ForceInstance(nx, nvx, nvp, dt, L=L, x0=0.0, x1=2.0, bc=bc, eps=eps, E=E)
        b = pr.pr_force_create([inst], scheme, precision)
        try:
            pr.pr_force_set_cluster(b, cluster)
            assert pr.pr_force_config(b)[0] == cluster
            pr.pr_force_set_initial(b, 0, U)
            f0 = pr.pr_force_get_f(b, 0)
            pr.pr_force_run(b, 2)
            pr.pr_force_run(b, n - 2)
            f = pr.pr_force_get_f(b, 0)
            V = pr.pr_force_moments(b, 0)
        finally:
            pr.pr_force_destroy(b)
        fo0 = O.v_lift(k, U)
        fo = O.v_fine_run(k, dt, n, fo0)
        Vo = O.v_project(k, fo, conserved=True)
        tol = TOL[precision]
        assert f_rel_err(f0, fo0) < (1e-14 if precision == pr.PR_FP64 else 1e-6)
        assert f_rel_err(f, fo) < (1e-12 if precision == pr.PR_FP64 else 2e-6), (eps, f_rel_err(f, fo))
        assert moment_rel_err(V, Vo) < tol, (eps, moment_rel_err(V, Vo))


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
def test_wide_perpendicular_grid_and_several_instances(precision):
    # nvp = 20 (400 threads, 13 warps), three instances with different eps,
    # L, E and boundary in one launch
    nx, nvx, nvp, n = 9, 12, 20, 4
    specs = [(1e-3, 6.0, pr.PR_BC_PERIODIC, 1.0), (1.0, 7.0, pr.PR_BC_OUTFLOW, -0.5), (1e-5, 8.0, pr.PR_BC_REFLECT, 2.0)]
    insts, ks, dts = [], [], []
    for eps, L, bc, a in specs:
        E = a * W.test3_force(nx)
        k = _vkin(nx, nvx, nvp, L, bc, eps, pr.PR_MUSCL, E)
        dt = O.v_fine_dt_stab(k, 0.4)
        insts.append(pr.ForceInstance(nx, nvx, nvp, dt, L=L, x0=0.0, x1=2.0, bc=bc, eps=eps, E=E))
        ks.append(k)
        dts.append(dt)
    b = pr.pr_force_create(insts, pr.PR_MUSCL, precision)
    try:
        for i in range(3):
            pr.pr_force_set_initial(b, i, _profile(nx))
        pr.pr_force_run(b, n)
        got = [pr.pr_force_moments(b, i) for i in range(3)]
    finally:
        pr.pr_force_destroy(b)
    for i in range(3):
        Vo = O.v_project(ks[i], O.v_fine_run(ks[i], dts[i], n, O.v_lift(ks[i], _profile(nx))), conserved=True)
        assert moment_rel_err(got[i], Vo) < TOL[precision], i


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
def test_test3_full_size_beams_against_oracle(precision):
    # Test 3 at its full size: 100 x 256 x 16 x 16 on [0, 2] x [-8, 8]^3,
    # periodic, eps = 1e-5, the two beams loaded with set_f, 6 fine steps
    nx, nvx, nvp, L = 100, 256, 16, 8.0
    E = W.test3_force(nx)
    k = _vkin(nx, nvx, nvp, L, pr.PR_BC_PERIODIC, 1e-5, pr.PR_UPWIND, E)
    dt = O.v_fine_dt_stab(k, 0.5)
    f0 = _beams_f_oracle(k)
    inst = pr.ForceInstance(nx, nvx, nvp, dt, L=L, x0=0.0, x1=2.0, eps=1e-5, E=E)
    b = pr.pr_force_create([inst], pr.PR_UPWIND, precision)
    try:
        assert pr.pr_force_config(b) == (8, 8192)
        pr.pr_force_set_f(b, 0, f0)
        assert moment_rel_err(pr.pr_force_moments(b, 0), O.v_project(k, f0, conserved=True)) < TOL[precision]
        pr.pr_force_run(b, 6)
        V = pr.pr_force_moments(b, 0)
    finally:
        pr.pr_force_destroy(b)
    O.set_threads(16)
    try:
        Vo = O.v_project(k, O.v_fine_run(k, dt, 6, f0), conserved=True)
    finally:
        O.set_threads(1)
    assert moment_rel_err(V, Vo) < TOL[precision]
    # the library's own lift builds the same beams
    fg = _beams_f_gpu(nx, nvx, nvp, L, dt)
    assert f_rel_err(fg, f0) < 1e-14


@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
def test_test3_full_size_muscl_batch_on_the_fused_step_against_oracle(precision):
    # Test 3 at its full size with MUSCL-minmod x fluxes, four instances in
    # one persistent fused launch (16 CTAs of 16 rows, walks of at least three
    # columns), 5 steps from the beams: every instance's f and moments
    # against the oracle's
    nx, nvx, nvp, L = 100, 256, 16, 8.0
    E = W.test3_force(nx)
    k = _vkin(nx, nvx, nvp, L, pr.PR_BC_PERIODIC, 1e-5, pr.PR_MUSCL, E)
    dt = O.v_fine_dt_stab(k, 0.5)
    f0 = _beams_f_oracle(k)
    inst = pr.ForceInstance(nx, nvx, nvp, dt, L=L, x0=0.0, x1=2.0, eps=1e-5, E=E)
    b = pr.pr_force_create([inst] * 4, pr.PR_MUSCL, precision)
    try:
        assert pr.pr_force_config(b) == (16, 4096)
        assert pr.pr_force_get_march(b) >= 3 and pr.pr_force_get_persistent(b, 5) == 1
        for i in range(4):
            pr.pr_force_set_f(b, i, f0)
        pr.pr_force_run(b, 5)
        got = [(pr.pr_force_get_f(b, i), pr.pr_force_moments(b, i)) for i in range(4)]
    finally:
        pr.pr_force_destroy(b)
    O.set_threads(16)
    try:
        fo = O.v_fine_run(k, dt, 5, f0)
    finally:
        O.set_threads(1)
    Vo = O.v_project(k, fo, conserved=True)
    for f, V in got:
        assert f_rel_err(f, fo) < (1e-12 if precision == pr.PR_FP64 else 2e-6)
        assert moment_rel_err(V, Vo) < TOL[precision]


def test_coarse_step_with_source_matches_oracle():
    nx, N, T = 24, 4, 0.08
    E = W.test3_force(nx)
    ctx = pr.pr_init_force(nx, 0.0, 2.0, pr.PR_BC_PERIODIC, 12, 6, 8.0, 1e-3, T, N, E)
    try:
        V = O.prim_to_cons(_profile(nx))
        got = pr.pr_coarse_step(ctx, V, 0.05)
    finally:
        pr.pr_destroy(ctx)
    want, _ = O.coarse_run_force(nx, O.BC_PERIODIC, 0.5, 0.05, V, E, x0=0.0, x1=2.0)
    assert np.max(np.abs(got - want)) <= 1e-13 * np.max(np.abs(want))


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
@pytest.mark.parametrize("max_batch", [0, 3])
def test_parareal_with_force_matches_oracle(precision, max_batch):
    # Algorithm 2 with the force propagators: all slices resident (graph) or
    # in waves of 3; K = 3 of N = 5
    nx, nvx, nvp, L, N, K, T = 16, 16, 6, 8.0, 5, 3, 0.05
    E = W.test3_force(nx)
    k = _vkin(nx, nvx, nvp, L, pr.PR_BC_PERIODIC, 1e-3, pr.PR_UPWIND, E)
    U0 = O.v_project(k, _beams_f_oracle(k))
    p = O.VParareal(kin=k, T=T, N=N)
    Uo, errs_o, _ = O.v_parareal(p, U0, K=K)
    ctx = pr.pr_init_force(nx, 0.0, 2.0, pr.PR_BC_PERIODIC, nvx, nvp, L, 1e-3, T, N, E, precision=precision,
                           max_batch=max_batch)
    try:
        assert pr.pr_fine_steps_per_slice(ctx)[0] == O.v_fine_nsteps(p)[0]
        pr.pr_set_initial(ctx, U0)
        for n in range(N + 1):
            assert moment_rel_err(pr.pr_moments(ctx, n), Uo[0][n]) < TOL_FP64, n
        kd, errs = pr.pr_parareal_run(ctx, K)
        assert kd == K
        for n in range(N + 1):
            assert moment_rel_err(pr.pr_moments(ctx, n), Uo[K][n]) < TOL[precision], n
        rel = np.abs(errs - errs_o) / np.abs(errs_o)
        assert np.all(rel < (1e-9 if precision == pr.PR_FP64 else 1e-3)), (errs, errs_o)
    finally:
        pr.pr_destroy(ctx)


def test_free_running_slice_of_a_force_problem():
    nx, nvx, nvp, L, N, T = 12, 16, 6, 8.0, 3, 0.03
    E = W.test3_force(nx)
    k = _vkin(nx, nvx, nvp, L, pr.PR_BC_OUTFLOW, 1e-2, pr.PR_MUSCL, E)
    p = O.VParareal(kin=k, T=T, N=N)
    nf, dt = O.v_fine_nsteps(p)
    U0 = _profile(nx)
    ctx = pr.pr_init_force(nx, 0.0, 2.0, pr.PR_BC_OUTFLOW, nvx, nvp, L, 1e-2, T, N, E, scheme=pr.PR_MUSCL)
    try:
        pr.pr_set_initial(ctx, U0)
        pr.pr_fine_step(ctx, 1, 0)
        assert moment_rel_err(pr.pr_fine_moments(ctx, 1), O.v_project(k, O.v_lift(k, U0), conserved=True)) < TOL_FP64
        pr.pr_fine_step(ctx, 1, 3)
        f = pr.pr_fine_get_f(ctx, 1)
        V = pr.pr_fine_moments(ctx, 1)
    finally:
        pr.pr_destroy(ctx)
    fo = O.v_fine_run(k, dt, 3, O.v_lift(k, U0))
    assert f_rel_err(f, fo) < 1e-12
    assert moment_rel_err(V, O.v_project(k, fo, conserved=True)) < TOL_FP64


def test_force_path_errors_are_reported():
    nx, nvx, nvp = 8, 8, 4
    ok = pr.ForceInstance(nx, nvx, nvp, 1e-3, E=np.ones(nx))
    for bad in (pr.ForceInstance(nx, nvx, 33, 1e-3), pr.ForceInstance(nx, 1, nvp, 1e-3),
                pr.ForceInstance(nx, nvx, nvp, -1.0), pr.ForceInstance(nx, nvx, nvp, 1e-3, E=np.full(nx, np.nan))):
        with pytest.raises(pr.PrError) as ei:
            pr.pr_force_create([bad], pr.PR_UPWIND, pr.PR_FP64)
        assert ei.value.code == pr.PR_EINVAL
    with pytest.raises(pr.PrError):
        pr.pr_force_create([ok, pr.ForceInstance(nx + 1, nvx, nvp, 1e-3)])
    b = pr.pr_force_create([ok], pr.PR_UPWIND, pr.PR_FP64)
    try:
        for C in (17, 5):  # too many, or an empty CTA (8 rows over 5 CTAs of 2)
            with pytest.raises(pr.PrError) as ei:
                pr.pr_force_set_cluster(b, C)
            assert ei.value.code == pr.PR_EINVAL
        bad_U = _profile(nx)
        bad_U[4, 3] = -1.0
        with pytest.raises(pr.PrError) as ei:
            pr.pr_force_set_initial(b, 0, bad_U)
        assert ei.value.code == pr.PR_ENONPHYS
        # a negative distribution: the BGK step meets rho <= 0 and says so
        pr.pr_force_set_f(b, 0, -np.ones((nx, nvx * nvp * nvp)))
        pr.pr_force_run(b, 1)
        with pytest.raises(pr.PrError) as ei:
            pr.pr_force_sync(b)
        assert ei.value.code == pr.PR_ENONPHYS
        # the object stays usable
        pr.pr_force_set_initial(b, 0, _profile(nx))
        pr.pr_force_run(b, 2)
        pr.pr_force_sync(b)
    finally:
        pr.pr_force_destroy(b)


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
@pytest.mark.parametrize("threads", [32, 64, 512])
def test_thread_caps_give_the_same_step(precision, threads):
    # nvp = 8: 16 (float) / 32 (double) threads per v_x row, so the caps give
    # 1 to 32 row groups per CTA; 3 CTAs per column (rows 14 / 14 / 12)
    nx, nvx, nvp, L, n = 10, 40, 8, 7.0, 3
    E = W.test3_force(nx)
    U = _profile(nx)
    k = _vkin(nx, nvx, nvp, L, pr.PR_BC_PERIODIC, 1e-2, pr.PR_MUSCL, E)
    dt = O.v_fine_dt_stab(k, 0.5)
    b = pr.pr_force_create([pr.ForceInstance(nx, nvx, nvp, dt, L=L, x0=0.0, x1=2.0, eps=1e-2, E=E)], pr.PR_MUSCL,
                           precision)
    try:
        pr.pr_force_set_cluster(b, 3)
        pr.pr_force_set_threads(b, threads)
        pr.pr_force_set_initial(b, 0, U)
        pr.pr_force_run(b, n)
        V = pr.pr_force_moments(b, 0)
    finally:
        pr.pr_force_destroy(b)
    Vo = O.v_project(k, O.v_fine_run(k, dt, n, O.v_lift(k, U)), conserved=True)
    assert moment_rel_err(V, Vo) < TOL[precision]


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
@pytest.mark.parametrize("nx,nvx,nvp,bc,scheme", [
    (1, 8, 4, pr.PR_BC_PERIODIC, pr.PR_UPWIND),   # one x cell: every neighbour is itself
    (2, 8, 4, pr.PR_BC_REFLECT, pr.PR_MUSCL),     # the smallest reflecting MUSCL column pair
    (6, 2, 4, pr.PR_BC_OUTFLOW, pr.PR_MUSCL),     # two v_x rows: both are box ends
    (6, 10, 1, pr.PR_BC_PERIODIC, pr.PR_UPWIND),  # one (v_y, v_z) cell per row
    (6, 12, 5, pr.PR_BC_REFLECT, pr.PR_UPWIND),   # odd rows: staged by the threads, no bulk copies
])
def test_edge_geometries_match_oracle(precision, nx, nvx, nvp, bc, scheme):
    L, n = 6.0, 3
    E = np.linspace(-0.8, 0.6, nx)
    x = W.cell_centres(nx, 0.0, 2.0)
    U = np.stack([1 + 0.2 * np.cos(x), 0.1 * np.sin(x), 0 * x, 0 * x, 1 + 0.1 * x])
    k = _vkin(nx, nvx, nvp, L, bc, 5e-2, scheme, E)
    dt = O.v_fine_dt_stab(k, 0.5)
    b = pr.pr_force_create([pr.ForceInstance(nx, nvx, nvp, dt, L=L, x0=0.0, x1=2.0, bc=bc, eps=5e-2, E=E)], scheme,
                           precision)
    try:
        pr.pr_force_set_initial(b, 0, U)
        pr.pr_force_run(b, n)
        f = pr.pr_force_get_f(b, 0)
        V = pr.pr_force_moments(b, 0)
    finally:
        pr.pr_force_destroy(b)
    fo = O.v_fine_run(k, dt, n, O.v_lift(k, U))
    assert f_rel_err(f, fo) < (1e-12 if precision == pr.PR_FP64 else 2e-6)
    assert moment_rel_err(V, O.v_project(k, fo, conserved=True)) < TOL[precision]


@pytest.mark.parametrize("scheme", [pr.PR_UPWIND, pr.PR_MUSCL])
def test_zero_force_kernel_is_the_e0_kernel(scheme):
    # two independent GPU kernels for the same scheme when E = 0 and the grid
    # is isotropic: the clustered force step and the persistent E = 0 step
    nx, nv, L, n = 48, 16, 8.0, 7
    dt = pr.fine_dt(nx, nv, L)
    U = W.smooth_periodic(nx)
    a = pr.pr_batch_create([pr.instance(nx, nv, dt, L=L, eps=1e-2, scheme=scheme)], pr.PR_FP64)
    b = pr.pr_force_create([pr.ForceInstance(nx, nv, nv, dt, L=L, x0=0.0, x1=1.0, eps=1e-2)], scheme, pr.PR_FP64)
    try:
        pr.pr_batch_set_initial(a, 0, U)
        pr.pr_batch_run(a, n)
        pr.pr_force_set_initial(b, 0, U)
        pr.pr_force_run(b, n)
        assert f_rel_err(pr.pr_force_get_f(b, 0), pr.pr_batch_get_f(a, 0)) < 1e-12
        assert moment_rel_err(pr.pr_force_moments(b, 0), pr.pr_batch_moments(a, 0)) < 1e-12
    finally:
        pr.pr_batch_destroy(a)
        pr.pr_force_destroy(b)
