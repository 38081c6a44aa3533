"""Parity of the device coarse propagator and of the parareal driver
(Algorithm 2) with the CPU FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import workloads as W
from helpers import TOL_FP64, TOL_MIXED, moment_rel_err

pytestmark = pytest.mark.gpu

BC = {pr.PR_BC_PERIODIC: O.BC_PERIODIC, pr.PR_BC_OUTFLOW: O.BC_OUTFLOW, pr.PR_BC_REFLECT: O.BC_REFLECT}


def _ctx(nx=64, nv=16, L=8.0, eps=1e-2, T=0.1, N=8, bc=pr.PR_BC_OUTFLOW, scheme=pr.PR_UPWIND,
         precision=pr.PR_FP64, max_batch=0, sound=pr.PR_SOUND_GAMMA53):
    return pr.pr_init(nx, 0.0, 1.0, bc, nv, L, eps, T, N, 0.5, 0.5, scheme, precision, sound, max_batch, 0)


def _oracle_pr(nx=64, nv=16, L=8.0, eps=1e-2, T=0.1, N=8, bc=pr.PR_BC_OUTFLOW, scheme=pr.PR_UPWIND,
               sound=pr.PR_SOUND_GAMMA53):
    k = O.Kin(nx=nx, nv=nv, L=L, bc=BC[bc], eps=eps, scheme=scheme)
    return O.Parareal(kin=k, T=T, N=N, sound=sound)


@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW, pr.PR_BC_REFLECT])
@pytest.mark.parametrize("sound", [pr.PR_SOUND_GAMMA53, pr.PR_SOUND_SQRT_THETA])
def test_coarse_step_matches_oracle(bc, sound):
    nx = 77
    U = W.thirds(nx) if bc != pr.PR_BC_PERIODIC else W.smooth_periodic(nx)
    V = O.prim_to_cons(U)
    ctx = _ctx(nx=nx, bc=bc, sound=sound)
    try:
        for dT in (0.0, 0.013, 0.05):
            out = pr.pr_coarse_step(ctx, V, dT)
            ref, _ = O.coarse_run(nx, BC[bc], 0.5, dT, V, sound=sound)
            assert moment_rel_err(out, ref) < 1e-14
    finally:
        pr.pr_destroy(ctx)


def _block_profile(nx):
    # smooth part plus a jump at x = 0.4: every component moves, so the
    # reflecting ghost's flip of rho u_x and the viscous terms all matter
    x = W.cell_centres(nx, 0.0, 1.0)
    w = 2 * np.pi * x
    jump = np.where(x < 0.4, 0.0, 1.0)
    return np.stack([1 + 0.3 * np.sin(w) - 0.4 * jump, 0.2 * np.cos(w) + 0.1 * jump, 0.1 * np.sin(2 * w),
                     -0.05 * np.cos(w), 1 + 0.25 * np.sin(w + 0.3) - 0.2 * jump])


@pytest.mark.parametrize("model", ["euler", "cns", "euler+E", "cns+E"])
@pytest.mark.parametrize("bc", [pr.PR_BC_PERIODIC, pr.PR_BC_OUTFLOW, pr.PR_BC_REFLECT])
@pytest.mark.parametrize("nx", [
    1, 2, 17,      # one CTA
    97,            # 4 CTAs of 25 cells, the last of 22
    130,           # 5 CTAs of 26 cells
    3000,          # 16 CTAs, blocks in shared memory, the last ragged
    40000,         # 16 CTAs, blocks in the global workspace
])
def test_coarse_step_on_cluster_blocks_matches_oracle(nx, bc, model):
    # the coarse step runs on a cluster of CTAs owning contiguous blocks of
    # cells: faces across blocks and the boundary ghosts come from the
    # owners' regions; the Navier-Stokes terms and the force source ride on
    # the same face and update passes
    eps = 1e-4
    cns = model.startswith("cns")
    V = O.prim_to_cons(_block_profile(nx))
    dT = 2.0 / nx  # about six hyperbolic local steps (more where the viscous limit binds)
    cm = pr.PR_COARSE_CNS if cns else pr.PR_COARSE_EULER
    E = 0.5 * np.sin(2 * np.pi * W.cell_centres(nx, 0.0, 1.0)) if model.endswith("+E") else None
    if E is None:
        ctx = pr.pr_init(nx, 0.0, 1.0, bc, 4, 8.0, eps, 0.1, 1, coarse_model=cm)
    else:
        ctx = pr.pr_init_force(nx, 0.0, 1.0, bc, 4, 4, 8.0, eps, 0.1, 1, E, coarse_model=cm)
    try:
        out = pr.pr_coarse_step(ctx, V, dT)
    finally:
        pr.pr_destroy(ctx)
    if cns:
        ref, ns = O.coarse_run_cns(nx, BC[bc], 0.5, dT, V, eps, E=E)
    elif E is not None:
        ref, ns = O.coarse_run_force(nx, BC[bc], 0.5, dT, V, E)
    else:
        ref, ns = O.coarse_run(nx, BC[bc], 0.5, dT, V)
    assert ns >= 2
    assert moment_rel_err(out, ref) < 1e-13


@pytest.mark.parametrize("precision,tol", [(pr.PR_FP64, TOL_FP64), (pr.PR_MIXED, TOL_MIXED)])
def test_sod_parareal_matches_oracle(precision, tol):
    # Test 1 setup at the small size: Nx = 64, 16^3, eps = 1e-2, outflow,
    # upwind, T = 0.1, N = 8, K = 3 (12 fine steps per slice)
    U0 = W.sod(64)
    p = _oracle_pr()
    Uo, errs_o, _ = O.parareal(p, U0, K=3)
    ctx = _ctx(precision=precision)
    try:
        assert pr.pr_fine_steps_per_slice(ctx)[0] == 12
        pr.pr_set_initial(ctx, U0)
        for n in range(9):
            assert moment_rel_err(pr.pr_moments(ctx, n), Uo[0][n]) < 1e-14
        errs = []
        for k in range(1, 4):
            errs.append(pr.pr_parareal_iter(ctx))
            for n in range(9):
                assert moment_rel_err(pr.pr_moments(ctx, n), Uo[k][n]) < tol, (k, n)
        assert np.allclose(errs, errs_o, rtol=1e-6 if precision == pr.PR_FP64 else 1e-2, atol=0)
    finally:
        pr.pr_destroy(ctx)


def test_graph_replayed_run_equals_step_by_step():
    U0 = W.sod(64)
    a = _ctx(precision=pr.PR_MIXED)
    b = _ctx(precision=pr.PR_MIXED)
    try:
        pr.pr_set_initial(a, U0)
        pr.pr_set_initial(b, U0)
        kd, errs = pr.pr_parareal_run(a, 4)
        e2 = [pr.pr_parareal_iter(b) for _ in range(4)]
        assert kd == 4 and np.array_equal(errs, e2)
        for n in range(9):
            assert np.array_equal(pr.pr_moments(a, n), pr.pr_moments(b, n))
    finally:
        pr.pr_destroy(a)
        pr.pr_destroy(b)


@pytest.mark.parametrize("scheme", [pr.PR_UPWIND, pr.PR_MUSCL])
def test_k_equals_n_is_the_serial_fine_chain(scheme):
    # Sec. 2.2: N iterations reproduce the fine propagation chain U^n = PFL(U^{n-1})
    N, nx = 5, 40
    U0 = W.sod(nx)
    p = _oracle_pr(nx=nx, nv=8, T=0.05, N=N, scheme=scheme)
    chain = [O.prim_to_cons(U0)]
    for _ in range(N):
        chain.append(O.fine_propagate(p, chain[-1]))
    ctx = _ctx(nx=nx, nv=8, T=0.05, N=N, scheme=scheme)
    try:
        pr.pr_set_initial(ctx, U0)
        kd, errs = pr.pr_parareal_run(ctx, N)
        for n in range(N + 1):
            assert moment_rel_err(pr.pr_moments(ctx, n), chain[n]) < TOL_FP64
        # iterations past N change nothing
        e = pr.pr_parareal_iter(ctx)
        assert e == 0.0
    finally:
        pr.pr_destroy(ctx)


def test_waves_when_slices_exceed_resident_states():
    # max_batch < N: the fine phase runs in waves of resident slices
    U0 = W.sod(48)
    p = _oracle_pr(nx=48, nv=8, T=0.06, N=7, scheme=pr.PR_MUSCL)
    Uo, errs_o, _ = O.parareal(p, U0, K=3)
    ctx = _ctx(nx=48, nv=8, T=0.06, N=7, scheme=pr.PR_MUSCL, max_batch=3)
    try:
        pr.pr_set_initial(ctx, U0)
        kd, errs = pr.pr_parareal_run(ctx, 3)
        for n in range(8):
            assert moment_rel_err(pr.pr_moments(ctx, n), Uo[3][n]) < TOL_FP64
        assert np.allclose(errs, errs_o, rtol=1e-6)
    finally:
        pr.pr_destroy(ctx)


def test_tolerance_stop_and_notconv():
    U0 = W.sod(32)
    ctx = _ctx(nx=32, nv=8, T=0.05, N=6)
    try:
        pr.pr_set_initial(ctx, U0)
        kd, errs = pr.pr_parareal_run(ctx, 6, tol=1e-300)
        assert kd == 6
        with pytest.raises(pr.PrError) as ei:
            pr.pr_set_initial(ctx, U0)
            pr.pr_parareal_run(ctx, 2, tol=1e-300, allow_notconv=False)
        assert ei.value.code == pr.PR_ENOTCONV
        pr.pr_set_initial(ctx, U0)
        kd, errs2 = pr.pr_parareal_run(ctx, 6, tol=0.5 * (errs[1] + errs[2]))
        assert kd == 3 and np.allclose(errs2, errs[:3], rtol=1e-12)
    finally:
        pr.pr_destroy(ctx)


def test_fine_step_api_advances_a_slice():
    nx, nv = 30, 8
    U0 = W.sod(nx)
    ctx = _ctx(nx=nx, nv=nv, T=0.04, N=4)
    p = _oracle_pr(nx=nx, nv=nv, T=0.04, N=4)
    try:
        pr.pr_set_initial(ctx, U0)
        nf, dt = pr.pr_fine_steps_per_slice(ctx)
        pr.pr_fine_step(ctx, 2, 3)
        pr.pr_fine_step(ctx, 2, nf - 3)
        V = pr.pr_fine_moments(ctx, 2)
        ref = O.fine_propagate(p, pr.pr_moments(ctx, 1))
        assert moment_rel_err(V, ref) < TOL_FP64
    finally:
        pr.pr_destroy(ctx)


def test_errors_are_reported_not_raised_on_device():
    ctx = _ctx(nx=16, nv=4, N=2)
    try:
        with pytest.raises(pr.PrError) as ei:
            pr.pr_parareal_iter(ctx)  # before pr_set_initial
        assert ei.value.code == pr.PR_EINVAL
        bad = W.sod(16)
        bad[4, 3] = -1.0
        with pytest.raises(pr.PrError) as ei:
            pr.pr_set_initial(ctx, bad)
        assert ei.value.code == pr.PR_ENONPHYS
    finally:
        pr.pr_destroy(ctx)
    with pytest.raises(pr.PrError) as ei:
        pr.pr_batch_create([pr.instance(10, 6, 1e-3)])
    assert ei.value.code == pr.PR_EINVAL


def test_parareal_on_a_grid_larger_than_the_sweep_threads():
    # 5000 cells: 16 sweep CTAs of 313 cells, more cells than threads, so the
    # sweep's correction loads its inputs after G instead of prefetching them,
    # and the face and update passes loop over their items
    nx, nv, T, N, K = 5000, 4, 0.002, 2, 2
    U0 = W.sod(nx)
    p = _oracle_pr(nx=nx, nv=nv, T=T, N=N)
    Uo, errs_o, _ = O.parareal(p, U0, K=K)
    ctx = _ctx(nx=nx, nv=nv, T=T, N=N)
    try:
        pr.pr_set_initial(ctx, U0)
        kd, errs = pr.pr_parareal_run(ctx, K)
        for n in range(N + 1):
            assert moment_rel_err(pr.pr_moments(ctx, n), Uo[K][n]) < TOL_FP64, n
        assert np.allclose(errs, errs_o, rtol=1e-6, atol=0)
    finally:
        pr.pr_destroy(ctx)
