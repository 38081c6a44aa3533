"""The paper's Test 1 (Sod) and Test 2 (blast waves) at the paper's own size
(Sec. 5: 200 x 32^3 cells, T = 0.5, N_g = 200, N_f = 800), checked against
what the paper states about them, and the blast-wave data at a size the oracle
finishes, against the oracle."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import workloads as W
from helpers import TOL_FP64, TOL_MIXED, moment_rel_err

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_statements.json")))


def _paper_ctx(precision):
    # x in [0, 2], 200 cells, 32^3 on [-8, 8]^3, eps = 1e-2, outflow, T = 0.5, N = 200
    return pr.pr_init(200, 0.0, 2.0, pr.PR_BC_OUTFLOW, 32, 8.0, 1e-2, 0.5, 200, 0.5, 0.5, pr.PR_UPWIND, precision)


def test_blast_waves_paper_scale_error_after_ten_iterations():
    g = GOLD["test2_blast_waves"]
    errs = {}
    for prec in (pr.PR_MIXED, pr.PR_FP64):
        ctx = _paper_ctx(prec)
        try:
            assert pr.pr_fine_steps_per_slice(ctx)[0] == 4  # N_f / N_g = 800 / 200
            pr.pr_set_initial(ctx, W.blast(200))
            kd, e = pr.pr_parareal_run(ctx, g["K"])
            errs[prec] = e
        finally:
            pr.pr_destroy(ctx)
    e = errs[pr.PR_MIXED]
    order = g["successive_error_order_of_magnitude"]
    assert order / 10 < e[-1] < order * 10, e
    assert all(b < a for a, b in zip(e[1:], e[2:])), e
    assert np.allclose(errs[pr.PR_MIXED], errs[pr.PR_FP64], rtol=1e-3)


def test_sod_paper_scale_converges_exponentially_in_fp64():
    g = GOLD["test1_sod"]
    ctx = _paper_ctx(pr.PR_FP64)
    try:
        pr.pr_set_initial(ctx, W.sod(200, 0.0, 2.0))
        kd, e = pr.pr_parareal_run(ctx, g["K_max"], g["tol"])
    finally:
        pr.pr_destroy(ctx)
    assert kd < g["K_max"] and e[-1] < g["tol"]
    # exponential decay: a log-linear fit over the iterations has slope < 0
    # and every later error is below the earlier ones
    k = np.arange(1, kd + 1)
    slope = np.polyfit(k[5:], np.log(e[5:]), 1)[0]
    assert slope < -0.2, slope
    assert all(b < a for a, b in zip(e[5:], e[6:]))


@pytest.mark.parametrize("precision,tol", [(pr.PR_FP64, TOL_FP64), (pr.PR_MIXED, TOL_MIXED)])
def test_blast_waves_scaled_matches_oracle(precision, tol):
    nx, nv, L, N, K, T = 64, 16, 8.0, 8, 3, 0.1
    U0 = W.blast(nx)
    k = O.Kin(nx=nx, nv=nv, L=L, x0=0.0, x1=2.0, bc=O.BC_OUTFLOW, eps=1e-2, scheme=O.UPWIND)
    O.set_threads(8)
    Uo, errs_o, _ = O.parareal(O.Parareal(kin=k, T=T, N=N), U0, K=K)
    O.set_threads(1)
    ctx = pr.pr_init(nx, 0.0, 2.0, pr.PR_BC_OUTFLOW, nv, L, 1e-2, T, N, 0.5, 0.5, pr.PR_UPWIND, precision)
    try:
        pr.pr_set_initial(ctx, U0)
        kd, errs = pr.pr_parareal_run(ctx, K)
        for n in range(N + 1):
            assert moment_rel_err(pr.pr_moments(ctx, n), Uo[K][n]) < tol, n
        assert np.allclose(errs, errs_o, rtol=1e-6 if precision == pr.PR_FP64 else 1e-2)
    finally:
        pr.pr_destroy(ctx)
