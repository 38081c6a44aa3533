"""The allocation-free fine step (pr_fine_step_noalloc) gives the same result
as the regular batch path and as the CPU oracle's fine step.

Some callers cannot allocate GPU memory through this library (their device
memory belongs to another allocator, or they must not allocate once set up);
for them pr_fine_step_noalloc takes caller-owned input and output arrays and
keeps all its scratch in a static device array.  This file is collected last
so that a failure here does not hide the other tests; it also runs alone.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import workloads as W
from helpers import TOL_FP64, f_rel_err

pytestmark = pytest.mark.gpu


def _batch_step(inst, f0):
    b = pr.pr_batch_create([inst], pr.PR_FP64)
    try:
        pr.pr_batch_set_f(b, 0, f0)
        pr.pr_batch_run(b, 1)
        return pr.pr_batch_get_f(b, 0)
    finally:
        pr.pr_batch_destroy(b)


@pytest.mark.parametrize("scheme,bc", [(pr.PR_MUSCL, pr.PR_BC_PERIODIC), (pr.PR_UPWIND, pr.PR_BC_REFLECT)])
def test_noalloc_step_matches_batch_step_twice(scheme, bc):
    import torch

    nx, nv = 70, 12
    inst = pr.instance(nx, nv, pr.fine_dt(nx, nv, 8.0), bc=bc, eps=1e-2, scheme=scheme)
    f0 = W.random_positive_f(nx, nv, seed=3)
    fin = torch.tensor(f0, dtype=torch.float64, device="cuda")
    out1 = torch.empty_like(fin)
    out2 = torch.empty_like(fin)
    # two calls in a row: the second starts from the first one's output
    pr.pr_fine_step_noalloc(inst, fin, out1)
    pr.pr_fine_step_noalloc(inst, out1, out2)
    r1 = _batch_step(inst, f0)
    r2 = _batch_step(inst, r1)
    assert f_rel_err(out1.cpu().numpy(), r1) < TOL_FP64
    assert f_rel_err(out2.cpu().numpy(), r2) < TOL_FP64
    assert f_rel_err(r1, f0) > 1e-3
    # and the oracle's fine step (Eqs. 11-13) directly, twice
    k = O.Kin(nx=nx, nv=nv, L=8.0, bc=bc, eps=1e-2, scheme=scheme)
    o1 = O.fine_step(k, inst.dt, f0)
    o2 = O.fine_step(k, inst.dt, o1)
    assert f_rel_err(out1.cpu().numpy(), o1) < TOL_FP64
    assert f_rel_err(out2.cpu().numpy(), o2) < TOL_FP64


def test_noalloc_rejects_instances_beyond_the_static_scratch():
    import torch

    inst = pr.instance(4096, 64, 1e-5)  # needs far more than the fixed scratch
    x = torch.empty(16, dtype=torch.float64, device="cuda")
    with pytest.raises(pr.PrError) as ei:
        pr.pr_fine_step_noalloc(inst, x, x.clone())
    assert ei.value.code == pr.PR_EINVAL
    assert "scratch" in str(ei.value)


def test_noalloc_rejects_non_finite_step_with_a_message():
    import torch

    x = torch.empty(8 * 4 ** 3, dtype=torch.float64, device="cuda")
    for dt in (math.inf, math.nan, 0.0):
        with pytest.raises(pr.PrError) as ei:
            pr.pr_fine_step_noalloc(pr.instance(8, 4, dt), x, x.clone())
        assert ei.value.code == pr.PR_EINVAL
        assert "dt" in str(ei.value)
