"""Parity of the CUDA fine propagator (fused transport + moments + Maxwellian +
implicit BGK, Eqs. 11-13) with the CPU FP64 oracle, through the C ABI."""
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


def _kin(nx, nv, L, bc, eps, scheme, x0=0.0, x1=1.0):
    return O.Kin(nx=nx, nv=nv, L=L, x0=x0, x1=x1, bc=BC[bc], eps=eps, scheme=SCH[scheme])


def _profile(bc, nx):
    if bc == pr.PR_BC_PERIODIC:
        return W.smooth_periodic(nx)
    if bc == pr.PR_BC_OUTFLOW:
        return W.sod(nx)
    return W.thirds(nx)


def _run_gpu(insts, Us, nsteps, precision, chunks=None):
    b = pr.pr_batch_create(insts, precision)
    try:
        for i, U in enumerate(Us):
            pr.pr_batch_set_initial(b, i, U)
        for n in (chunks or [nsteps]):
            pr.pr_batch_run(b, n)
        pr.pr_batch_sync(b)
        return ([pr.pr_batch_get_f(b, i) for i in range(len(insts))],
                [pr.pr_batch_moments(b, i) for i in range(len(insts))])
    finally:
        pr.pr_batch_destroy(b)


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
@pytest.mark.parametrize("scheme", [pr.PR_UPWIND, pr.PR_MUSCL])
@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW, pr.PR_BC_REFLECT])
def test_fine_run_matches_oracle(precision, scheme, bc):
    # nx = 70: three x tiles of 32 (last one ragged); nv = 12: 1728 velocities,
    # two v chunks of 1024 (last one ragged)
    nx, nv, L, eps, nsteps = 70, 12, 8.0, 1e-2, 9
    dt = pr.fine_dt(nx, nv, L)
    U = _profile(bc, nx)
    f, V = _run_gpu([pr.instance(nx, nv, dt, L=L, bc=bc, eps=eps, scheme=scheme)], [U], nsteps, precision)
    k = _kin(nx, nv, L, bc, eps, scheme)
    fo = O.fine_run(k, dt, nsteps, O.lift(k, U))
    Vo = O.project(k, fo, conserved=True)
    tol = TOL_FP64 if precision == pr.PR_FP64 else TOL_MIXED
    assert moment_rel_err(V[0], Vo) < tol
    assert f_rel_err(f[0], fo) < tol
    # the run moved the state: the comparison is not against the initial data
    assert f_rel_err(O.lift(k, U), fo) > 1e-3


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
def test_lift_matches_oracle(precision):
    nx, nv, L = 33, 16, 8.0
    U = W.sod(nx)
    b = pr.pr_batch_create([pr.instance(nx, nv, 1e-3, L=L, bc=pr.PR_BC_OUTFLOW)], precision)
    try:
        pr.pr_batch_set_initial(b, 0, U)
        f = pr.pr_batch_get_f(b, 0)
        V = pr.pr_batch_moments(b, 0)
    finally:
        pr.pr_batch_destroy(b)
    k = _kin(nx, nv, L, pr.PR_BC_OUTFLOW, 1e-2, pr.PR_UPWIND)
    fo = O.lift(k, U)
    tol = 1e-13 if precision == pr.PR_FP64 else 1e-6
    assert f_rel_err(f, fo) < tol
    assert moment_rel_err(V, O.project(k, fo, conserved=True)) < tol


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
def test_arbitrary_initial_f_and_collisionless(precision):
    # a loaded non-Maxwellian f (set_f path) and eps = inf (pure transport)
    nx, nv, L = 45, 8, 6.0
    dt = pr.fine_dt(nx, nv, L)
    f0 = W.random_positive_f(nx, nv, seed=5)
    for eps in (3e-3, math.inf):
        b = pr.pr_batch_create([pr.instance(nx, nv, dt, L=L, bc=pr.PR_BC_PERIODIC, eps=eps, scheme=pr.PR_MUSCL)],
                               precision)
        try:
            pr.pr_batch_set_f(b, 0, f0)
            V0 = pr.pr_batch_moments(b, 0)
            pr.pr_batch_run(b, 6)
            f = pr.pr_batch_get_f(b, 0)
            V = pr.pr_batch_moments(b, 0)
        finally:
            pr.pr_batch_destroy(b)
        k = _kin(nx, nv, L, pr.PR_BC_PERIODIC, eps, pr.PR_MUSCL)
        fo = O.fine_run(k, dt, 6, f0)
        tol = TOL_FP64 if precision == pr.PR_FP64 else TOL_MIXED
        assert moment_rel_err(V0, O.project(k, f0, conserved=True)) < tol
        assert moment_rel_err(V, O.project(k, fo, conserved=True)) < tol
        assert f_rel_err(f, fo) < tol


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
def test_ragged_batch_each_instance_matches_its_oracle(precision):
    # uneven nx / nv / eps / dt in one persistent launch
    specs = [(37, 8, 1e-1, pr.PR_BC_PERIODIC), (64, 12, 1e-4, pr.PR_BC_OUTFLOW), (5, 16, 1.0, pr.PR_BC_REFLECT),
             (1, 4, 1e-2, pr.PR_BC_PERIODIC), (90, 8, 1e-3, pr.PR_BC_REFLECT)]
    insts, Us, kins, dts = [], [], [], []
    for nx, nv, eps, bc in specs:
        dt = pr.fine_dt(nx, nv, 8.0)
        insts.append(pr.instance(nx, nv, dt, L=8.0, bc=bc, eps=eps, scheme=pr.PR_MUSCL if nx > 1 else pr.PR_MUSCL))
        Us.append(W.sod(nx) if bc != pr.PR_BC_PERIODIC else W.smooth_periodic(nx))
        kins.append(_kin(nx, nv, 8.0, bc, eps, pr.PR_MUSCL))
        dts.append(dt)
    f, V = _run_gpu(insts, Us, 7, precision)
    tol = TOL_FP64 if precision == pr.PR_FP64 else TOL_MIXED
    for i in range(len(specs)):
        fo = O.fine_run(kins[i], dts[i], 7, O.lift(kins[i], Us[i]))
        assert moment_rel_err(V[i], O.project(kins[i], fo, conserved=True)) < tol, i
        assert f_rel_err(f[i], fo) < tol, i


def test_persistent_multistep_equals_repeated_single_steps():
    # one launch of 8 steps (dependency waits between steps) gives the same
    # bits as 8 launches of one step (kernel boundaries between steps)
    nx, nv = 100, 8
    dt = pr.fine_dt(nx, nv, 8.0)
    inst = [pr.instance(nx, nv, dt, bc=pr.PR_BC_PERIODIC, eps=1e-2, scheme=pr.PR_MUSCL)]
    U = [W.smooth_periodic(nx)]
    fa, Va = _run_gpu(inst, U, 8, pr.PR_MIXED)
    fb, Vb = _run_gpu(inst, U, 8, pr.PR_MIXED, chunks=[1] * 8)
    assert np.array_equal(fa[0], fb[0]) and np.array_equal(Va[0], Vb[0])


def test_autotuned_tiles_keep_results():
    nx, nv = 200, 12
    dt = pr.fine_dt(nx, nv, 8.0)
    inst = [pr.instance(nx, nv, dt, bc=pr.PR_BC_OUTFLOW, eps=1e-3, scheme=pr.PR_MUSCL)]
    b = pr.pr_batch_create(inst, pr.PR_FP64)
    try:
        pr.pr_batch_set_initial(b, 0, W.sod(nx))
        pr.pr_batch_autotune(b)
        tx, tuned = pr.pr_batch_tile(b, 0)
        assert tuned and tx in (8, 16, 32, 64)
        pr.pr_batch_run(b, 5)
        V = pr.pr_batch_moments(b, 0)
    finally:
        pr.pr_batch_destroy(b)
    k = _kin(nx, nv, 8.0, pr.PR_BC_OUTFLOW, 1e-3, pr.PR_MUSCL)
    Vo = O.project(k, O.fine_run(k, dt, 5, O.lift(k, W.sod(nx))), conserved=True)
    assert moment_rel_err(V, Vo) < TOL_FP64


@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
def test_full_size_smooth_periodic_three_knudsen_numbers(precision):
    # the measured workload: Nx = 512, 32^3 on [-8, 8]^3, MUSCL, periodic,
    # eps in {1, 1e-2, 1e-4}, all three in one batched persistent launch.
    nx, nv, L = 512, 32, 8.0
    dt = pr.fine_dt(nx, nv, L)
    epss = (1.0, 1e-2, 1e-4)
    insts = [pr.instance(nx, nv, dt, L=L, bc=pr.PR_BC_PERIODIC, eps=e, scheme=pr.PR_MUSCL) for e in epss]
    U = W.smooth_periodic(nx)
    b = pr.pr_batch_create(insts, precision)
    try:
        for i in range(3):
            pr.pr_batch_set_initial(b, i, U)
        pr.pr_batch_run(b, 3)
        V3 = [pr.pr_batch_moments(b, i) for i in range(3)]
        f3 = pr.pr_batch_get_f(b, 1)
        pr.pr_batch_run(b, 197)
        V200 = [pr.pr_batch_moments(b, i) for i in range(3)]
    finally:
        pr.pr_batch_destroy(b)
    tol = TOL_FP64 if precision == pr.PR_FP64 else TOL_MIXED
    O.set_threads(8)
    for i, e in enumerate(epss):
        k = _kin(nx, nv, L, pr.PR_BC_PERIODIC, e, pr.PR_MUSCL)
        fo = O.fine_run(k, dt, 3, O.lift(k, U))
        assert moment_rel_err(V3[i], O.project(k, fo, conserved=True)) < tol
        if i == 1:
            assert f_rel_err(f3, fo) < tol
        # 200 steps: mass is conserved exactly by the flux form and up to the
        # quadrature defect of M by BGK; the state stays physical
        m0 = O.project(k, O.lift(k, U), conserved=True)[0].sum()
        assert abs(V200[i][0].sum() - m0) < (1e-11 if precision == pr.PR_FP64 else 1e-5) * m0
        assert np.all(V200[i][0] > 0)
    O.set_threads(1)


def test_default_tile_width_follows_batch_size():
    # a batch with fewer items than resident CTAs takes narrower tiles; one
    # that fills the GPU keeps 32 columns; widths never exceed nx
    def default_tiles(insts):
        b = pr.pr_batch_create(insts, pr.PR_MIXED)
        try:
            return [pr.pr_batch_tile(b, i) for i in range(len(insts))]
        finally:
            pr.pr_batch_destroy(b)

    small = default_tiles([pr.instance(64, 16, pr.fine_dt(64, 16, 8.0), eps=1e-2)])
    assert small == [(8, False)]
    tiny = default_tiles([pr.instance(5, 8, pr.fine_dt(5, 8, 8.0), eps=1e-2)])
    assert tiny == [(5, False)]
    big = default_tiles([pr.instance(512, 32, pr.fine_dt(512, 32, 8.0), eps=e, scheme=pr.PR_MUSCL)
                         for e in (1.0, 1e-2, 1e-4)])
    assert big == [(32, False)] * 3


@pytest.mark.parametrize("tx", [8, 13, 64])
def test_manual_tile_widths_keep_results(tx):
    # tile width 13 leaves a ragged last tile; widths below 8 are raised to 8
    nx, nv = 90, 8
    dt = pr.fine_dt(nx, nv, 8.0)
    inst = [pr.instance(nx, nv, dt, bc=pr.PR_BC_PERIODIC, eps=1e-2, scheme=pr.PR_MUSCL)]
    b = pr.pr_batch_create(inst, pr.PR_FP64)
    try:
        pr.pr_batch_set_tile(b, tx)
        assert pr.pr_batch_tile(b, 0) == (tx, False)
        pr.pr_batch_set_initial(b, 0, W.smooth_periodic(nx))
        pr.pr_batch_run(b, 6)
        V = pr.pr_batch_moments(b, 0)
        with pytest.raises(pr.PrError):
            pr.pr_batch_set_tile(b, 65)
    finally:
        pr.pr_batch_destroy(b)
    k = _kin(nx, nv, 8.0, pr.PR_BC_PERIODIC, 1e-2, pr.PR_MUSCL)
    Vo = O.project(k, O.fine_run(k, dt, 6, O.lift(k, W.smooth_periodic(nx))), conserved=True)
    assert moment_rel_err(V, Vo) < TOL_FP64


@pytest.mark.parametrize("precision", [pr.PR_MIXED, pr.PR_FP64])
@pytest.mark.parametrize("bc,scheme,nv", [
    (pr.PR_BC_PERIODIC, pr.PR_MUSCL, 16),
    (pr.PR_BC_OUTFLOW, pr.PR_MUSCL, 16),
    (pr.PR_BC_REFLECT, pr.PR_MUSCL, 16),
    (pr.PR_BC_OUTFLOW, pr.PR_MUSCL, 24),
    (pr.PR_BC_PERIODIC, pr.PR_UPWIND, 16),
    (pr.PR_BC_OUTFLOW, pr.PR_MUSCL, 12),   # four velocities per thread
])
def test_tile_width_and_march_direction_give_the_same_bits(precision, bc, scheme, nv):
    # odd tiles march right to left, so a column changes direction with the
    # tile width: each column's f* and moment sums must come out the same
    # whatever the width (the upwind side's code paths round alike)
    nx = 100
    dt = pr.fine_dt(nx, nv, 8.0)
    U = _profile(bc, nx)
    ref = None
    for tx in (32, 16, 8):
        b = pr.pr_batch_create([pr.instance(nx, nv, dt, bc=bc, eps=1e-2, scheme=scheme)], precision)
        try:
            pr.pr_batch_set_tile(b, tx)
            pr.pr_batch_set_initial(b, 0, U)
            pr.pr_batch_run(b, 3)
            got = (pr.pr_batch_get_f(b, 0), pr.pr_batch_moments(b, 0))
        finally:
            pr.pr_batch_destroy(b)
        if ref is None:
            ref = got
        else:
            assert np.array_equal(got[0], ref[0]), tx
            assert np.array_equal(got[1], ref[1]), tx


def test_autotuned_layout_in_float32_keeps_results():
    # nv = 16: the search covers 8 and 4 velocities per thread in float32
    nx, nv = 160, 16
    dt = pr.fine_dt(nx, nv, 8.0)
    inst = [pr.instance(nx, nv, dt, bc=pr.PR_BC_PERIODIC, eps=1e-2, scheme=pr.PR_MUSCL),
            pr.instance(96, nv, dt, bc=pr.PR_BC_OUTFLOW, eps=1e-4, scheme=pr.PR_MUSCL)]
    U = [W.smooth_periodic(nx), W.sod(96)]
    b = pr.pr_batch_create(inst, pr.PR_MIXED)
    try:
        assert pr.pr_batch_vpt(b) == 8      # the default where every nv allows it
        for i, u in enumerate(U):
            pr.pr_batch_set_initial(b, i, u)
        pr.pr_batch_autotune(b)
        assert pr.pr_batch_vpt(b) in (4, 8)
        assert all(pr.pr_batch_tile(b, i)[1] for i in range(2))
        pr.pr_batch_run(b, 6)
        V = [pr.pr_batch_moments(b, i) for i in range(2)]
    finally:
        pr.pr_batch_destroy(b)
    for i, d in enumerate(inst):
        k = _kin(d.nx, nv, 8.0, d.bc, d.eps, pr.PR_MUSCL)
        Vo = O.project(k, O.fine_run(k, dt, 6, O.lift(k, U[i])), conserved=True)
        assert moment_rel_err(V[i], Vo) < TOL_MIXED
    # with nv = 12 only 4 velocities per thread exist
    b = pr.pr_batch_create([pr.instance(64, 12, dt, eps=1e-2)], pr.PR_MIXED)
    try:
        pr.pr_batch_set_initial(b, 0, W.smooth_periodic(64))
        pr.pr_batch_autotune(b)
        assert pr.pr_batch_vpt(b) == 4
    finally:
        pr.pr_batch_destroy(b)


@pytest.mark.parametrize("precision,nv", [(pr.PR_MIXED, 16), (pr.PR_MIXED, 24), (pr.PR_FP64, 16)])
def test_propagate_is_the_fine_propagator(precision, nv):
    # P F L of three instances of one shape: cluster-resident for mixed
    # 64 x 16^3 slices, the tiled run otherwise; from device states, then
    # again from the stored lift sources
    import torch

    nx, nf = 64, 12
    dt = pr.fine_dt(nx, nv, 8.0)
    epss = (1e-2, 1e-3, 1.0)
    insts = [pr.instance(nx, nv, dt, bc=pr.PR_BC_OUTFLOW, eps=e) for e in epss]
    Us = [W.sod(nx), W.sod(nx, split=0.3), W.smooth_periodic(nx)]
    Vs = np.concatenate([O.prim_to_cons(U) for U in Us])
    b = pr.pr_batch_create(insts, precision)
    try:
        pr.pr_batch_propagate(b, nf, torch.tensor(Vs, device="cuda"))
        got = [pr.pr_batch_moments(b, i) for i in range(3)]
        pr.pr_batch_propagate(b, nf)
        again = [pr.pr_batch_moments(b, i) for i in range(3)]
    finally:
        pr.pr_batch_destroy(b)
    for i, e in enumerate(epss):
        k = _kin(nx, nv, 8.0, pr.PR_BC_OUTFLOW, e, pr.PR_UPWIND)
        Vo = O.project(k, O.fine_run(k, dt, nf, O.lift(k, Us[i])), conserved=True)
        tol = TOL_FP64 if precision == pr.PR_FP64 else TOL_MIXED
        assert moment_rel_err(got[i], Vo) < tol, i
        assert np.array_equal(got[i], again[i])
