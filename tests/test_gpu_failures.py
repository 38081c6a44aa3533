"""Failure detection on the device without a GPU fault: a dependency wait of
the persistent launch that runs out (a flag nothing sets), a staging wait of
the force path that runs out (an mbarrier no copy completes), non-physical
states, and that each object stays usable afterwards."""
import math

import numpy as np
import pytest

import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch(precision=pr.PR_MIXED):
    nx, nv = 64, 8
    dt = pr.fine_dt(nx, nv, 8.0)
    return pr.pr_batch_create([pr.instance(nx, nv, dt, bc=pr.PR_BC_PERIODIC, eps=1e-2, scheme=pr.PR_MUSCL)],
                              precision)


def _reference_run(steps):
    b = _batch()
    try:
        pr.pr_batch_set_initial(b, 0, W.smooth_periodic(64))
        pr.pr_batch_run(b, steps)
        return pr.pr_batch_moments(b, 0)
    finally:
        pr.pr_batch_destroy(b)


def test_dependency_wait_runs_out_and_batch_stays_usable():
    b = _batch()
    try:
        pr.pr_batch_set_initial(b, 0, W.smooth_periodic(64))
        for wait_ms in (20, 50):
            assert pr.pr_batch_inject_wait_timeout(b, 3, wait_ms) == pr.PR_ETIMEOUT
            assert "timed out" in pr.pr_batch_last_error(b)
        # the status was cleared: a normal run afterwards gives the normal bits
        pr.pr_batch_set_initial(b, 0, W.smooth_periodic(64))
        pr.pr_batch_run(b, 5)
        V = pr.pr_batch_moments(b, 0)
    finally:
        pr.pr_batch_destroy(b)
    assert np.array_equal(V, _reference_run(5))


def _force_run(b, steps):
    pr.pr_force_set_initial(b, 0, W.smooth_periodic(8))
    pr.pr_force_run(b, steps)
    return pr.pr_force_moments(b, 0)


def test_force_staging_wait_runs_out_and_object_stays_usable():
    E = W.test3_force(8)
    inst = pr.ForceInstance(8, 16, 4, 1e-3, E=E)  # 16 floats per row: bulk-copy staging
    b = pr.pr_force_create([inst], pr.PR_UPWIND, pr.PR_MIXED)
    fresh = pr.pr_force_create([inst], pr.PR_UPWIND, pr.PR_MIXED)
    try:
        pr.pr_force_set_initial(b, 0, W.smooth_periodic(8))
        for wait_ms in (20, 50):
            assert pr.pr_force_inject_wait_timeout(b, wait_ms) == pr.PR_ETIMEOUT
            assert "timed out" in pr.pr_force_last_error(b)
        assert np.array_equal(_force_run(b, 3), _force_run(fresh, 3))
    finally:
        pr.pr_force_destroy(b)
        pr.pr_force_destroy(fresh)
    # rows of 25 floats are staged by the threads: no staging wait to poison
    b = pr.pr_force_create([pr.ForceInstance(8, 16, 5, 1e-3, E=E)], pr.PR_UPWIND, pr.PR_MIXED)
    try:
        assert pr.pr_force_inject_wait_timeout(b, 20) == pr.PR_EINVAL
    finally:
        pr.pr_force_destroy(b)


def test_nonphysical_state_is_reported_and_cleared():
    b = _batch(pr.PR_FP64)
    try:
        f = W.random_positive_f(64, 8, seed=2)
        f[10] *= -1.0  # negative density in x cell 10
        pr.pr_batch_set_f(b, 0, f)
        pr.pr_batch_run(b, 2)
        with pytest.raises(pr.PrError) as ei:
            pr.pr_batch_sync(b)
        assert ei.value.code == pr.PR_ENONPHYS
        pr.pr_batch_set_initial(b, 0, W.smooth_periodic(64))
        pr.pr_batch_run(b, 2)
        pr.pr_batch_sync(b)
        assert np.all(pr.pr_batch_moments(b, 0, pr.PR_PRIMITIVE)[4] > 0)
    finally:
        pr.pr_batch_destroy(b)


def test_coarse_solver_reports_negative_temperature():
    nx = 32
    ctx = pr.pr_init(nx, 0.0, 1.0, pr.PR_BC_OUTFLOW, 4, 8.0, 1e-2, 0.1, 2)
    try:
        V = np.zeros((5, nx))
        V[0] = 1.0
        V[4] = 1.0
        V[4, 7] = -0.5  # energy below the kinetic part: theta < 0
        with pytest.raises(pr.PrError) as ei:
            pr.pr_coarse_step(ctx, V, 0.01)
        assert ei.value.code == pr.PR_ENONPHYS
        V[4, 7] = 1.0
        out = pr.pr_coarse_step(ctx, V, 0.01)
        assert np.all(np.isfinite(out))
    finally:
        pr.pr_destroy(ctx)


def test_coarse_step_rejects_non_finite_inputs():
    # G's local-step loop must end: a non-finite interval or state is refused
    # on the host before any launch, and the object stays usable.
    nx = 32
    ctx = pr.pr_init(nx, 0.0, 1.0, pr.PR_BC_OUTFLOW, 4, 8.0, 1e-2, 0.1, 2)
    try:
        V = np.zeros((5, nx))
        V[0] = 1.0
        V[4] = 1.5
        for dT in (math.inf, math.nan, -1.0):
            with pytest.raises(pr.PrError) as ei:
                pr.pr_coarse_step(ctx, V, dT)
            assert ei.value.code == pr.PR_EINVAL
        for q, bad in ((0, math.inf), (4, math.inf), (1, math.nan), (0, 0.0)):
            W2 = V.copy()
            W2[q, 5] = bad
            with pytest.raises(pr.PrError) as ei:
                pr.pr_coarse_step(ctx, W2, 0.01)
            assert ei.value.code == pr.PR_ENONPHYS, (q, bad)
        out = pr.pr_coarse_step(ctx, V, 0.01)
        assert np.allclose(out, V, rtol=0, atol=1e-15)  # a constant state stays
    finally:
        pr.pr_destroy(ctx)
    with pytest.raises(pr.PrError) as ei:
        pr.pr_init(nx, 0.0, 1.0, pr.PR_BC_OUTFLOW, 4, 8.0, 1e-2, math.inf, 2)
    assert ei.value.code == pr.PR_EINVAL
