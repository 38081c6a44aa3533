"""Parareal resume (pr_save / pr_load): the state Algorithm 2 carries from
one iteration to the next (the iterates U^{n,k}, the coarse values
G(U^{n-1,k}) the next correction reuses, k and the errors), written to a
file and read into a new problem, continues the run bit for bit; files of
another problem, truncated files and non-physical iterates are refused."""
import os

import numpy as np
import pytest

import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ctx(precision, nx=48, N=6, eps=1e-2, max_batch=0, force=False, scheme=pr.PR_UPWIND):
    if force:
        return pr.pr_init_force(nx, 0.0, 2.0, pr.PR_BC_PERIODIC, 32, 8, 6.0, eps, 0.05, N, W.test3_force(nx),
                                scheme=scheme, precision=precision, max_batch=max_batch)
    return pr.pr_init(nx, 0.0, 1.0, pr.PR_BC_OUTFLOW, 8, 8.0, eps, 0.1, N, scheme=scheme, precision=precision,
                      max_batch=max_batch)


def _initial(nx, force):
    return W.smooth_periodic(nx) if force else W.sod(nx)


def _levels(ctx, N):
    return np.stack([pr.pr_moments(ctx, n) for n in range(N + 1)])


@pytest.mark.parametrize("force", [False, True])
@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
def test_resumed_run_continues_bit_for_bit(tmp_path, force, precision):
    nx, N, K, k1 = 48, 6, 5, 2
    U0 = _initial(nx, force)
    ref = _ctx(precision, nx, N, force=force)
    try:
        pr.pr_set_initial(ref, U0)
        _, errs_ref = pr.pr_parareal_run(ref, K)
        U_ref = _levels(ref, N)
    finally:
        pr.pr_destroy(ref)
    path = os.fspath(tmp_path / "state.bin")
    first = _ctx(precision, nx, N, force=force)
    try:
        pr.pr_set_initial(first, U0)
        _, errs1 = pr.pr_parareal_run(first, k1)
        pr.pr_save(first, path)
    finally:
        pr.pr_destroy(first)
    assert os.path.getsize(path) == 8 + 16 * 4 + 12 * 8 + (nx if force else 0) * 8 + (N + 2) * 8 \
        + 2 * (N + 1) * 5 * nx * 8
    # a new problem with the same settings (its fine phase in waves of 4)
    second = _ctx(precision, nx, N, max_batch=4, force=force)
    try:
        pr.pr_load(second, path)
        assert pr.pr_iterations(second) == k1
        errs2 = [pr.pr_parareal_iter(second) for _ in range(K - k1)]
        assert np.array_equal(_levels(second, N), U_ref)
        assert pr.pr_iterations(second) == K
    finally:
        pr.pr_destroy(second)
    assert np.array_equal(np.concatenate([errs1, errs2]), errs_ref)


def test_resume_from_the_coarse_guess(tmp_path):
    # k = 0: the file holds U^{n,0} = G(U^{n-1,0}) and its coarse values
    nx, N, K = 48, 6, 3
    U0 = _initial(nx, False)
    path = os.fspath(tmp_path / "k0.bin")
    a = _ctx(pr.PR_FP64, nx, N)
    b = _ctx(pr.PR_FP64, nx, N)
    try:
        pr.pr_set_initial(a, U0)
        pr.pr_save(a, path)
        pr.pr_parareal_run(a, K)
        pr.pr_load(b, path)
        assert pr.pr_iterations(b) == 0
        pr.pr_parareal_run(b, K)
        assert np.array_equal(_levels(a, N), _levels(b, N))
    finally:
        pr.pr_destroy(a)
        pr.pr_destroy(b)


def test_foreign_truncated_and_nonphysical_files_are_refused(tmp_path):
    nx, N = 48, 6
    path = os.fspath(tmp_path / "s.bin")
    a = _ctx(pr.PR_FP64, nx, N)
    try:
        with pytest.raises(pr.PrError) as ei:
            pr.pr_save(a, path)              # before pr_set_initial
        assert ei.value.code == pr.PR_EINVAL
        pr.pr_set_initial(a, _initial(nx, False))
        pr.pr_parareal_run(a, 2)
        pr.pr_save(a, path)
        U_a = _levels(a, N)
    finally:
        pr.pr_destroy(a)
    raw = open(path, "rb").read()
    for kw in ({"nx": 40}, {"N": 5}, {"eps": 1e-3}, {"precision": pr.PR_MIXED}, {"scheme": pr.PR_MUSCL}):
        args = dict(precision=pr.PR_FP64, nx=nx, N=N)
        args.update(kw)
        other = _ctx(**args)
        try:
            with pytest.raises(pr.PrError) as ei:
                pr.pr_load(other, path)
            assert ei.value.code == pr.PR_EINVAL and "not a state of this problem" in pr.pr_last_error(other)
        finally:
            pr.pr_destroy(other)
    b = _ctx(pr.PR_FP64, nx, N)
    try:
        pr.pr_set_initial(b, _initial(nx, False))
        U_b = _levels(b, N)
        for bad in (raw[:-8], raw + b"\0", raw[:4]):
            bp = os.fspath(tmp_path / "bad.bin")
            open(bp, "wb").write(bad)
            with pytest.raises(pr.PrError) as ei:
                pr.pr_load(b, bp)
            assert ei.value.code == pr.PR_EINVAL
        # a negative density in slice 3's iterate
        hdr = 8 + 16 * 4 + 12 * 8 + (N + 2) * 8
        arr = bytearray(raw)
        off = hdr + (3 * 5 * nx + 7) * 8
        arr[off:off + 8] = np.float64(-1.0).tobytes()
        bp = os.fspath(tmp_path / "neg.bin")
        open(bp, "wb").write(bytes(arr))
        with pytest.raises(pr.PrError) as ei:
            pr.pr_load(b, bp)
        assert ei.value.code == pr.PR_ENONPHYS
        # nothing changed: b still holds its own coarse guess
        assert pr.pr_iterations(b) == 0
        assert np.array_equal(_levels(b, N), U_b)
        # and the intact file loads
        pr.pr_load(b, path)
        assert np.array_equal(_levels(b, N), U_a)
    finally:
        pr.pr_destroy(b)
    with pytest.raises(pr.PrError):
        c = _ctx(pr.PR_FP64, nx, N)
        try:
            pr.pr_load(c, os.fspath(tmp_path / "missing.bin"))
        finally:
            pr.pr_destroy(c)
