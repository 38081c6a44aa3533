"""Several parareal problems and independent instances in one launch per
iteration (pr_multi: the batching of Sec. 2.2 across problems): each
problem's Algorithm 2 iterates against the oracle's and against the same
problem run alone, the independent instances against their own batch run,
and the lockstep and set-up rules."""
import numpy as np
import pytest

import oracle as O
import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import workloads as W
from helpers import TOL_FP64, TOL_MIXED, f_rel_err, moment_rel_err

pytestmark = pytest.mark.gpu

TOL = {pr.PR_FP64: TOL_FP64, pr.PR_MIXED: TOL_MIXED}
FTOL = {pr.PR_FP64: 1e-12, pr.PR_MIXED: 2e-6}
NF = 6
# (nx, nv, L, eps, T, N, bc, initial state)
PROBLEMS = [
    (64, 8, 8.0, 1e-2, 0.03, 6, pr.PR_BC_OUTFLOW, lambda nx: W.sod(nx)),
    (40, 12, 6.0, 1e-3, 0.04, 4, pr.PR_BC_PERIODIC, lambda nx: W.smooth_periodic(nx)),
    (33, 8, 7.0, 1.0, 0.02, 5, pr.PR_BC_REFLECT, lambda nx: W.smooth_periodic(nx)),
]
OBC = {pr.PR_BC_PERIODIC: O.BC_PERIODIC, pr.PR_BC_OUTFLOW: O.BC_OUTFLOW, pr.PR_BC_REFLECT: O.BC_REFLECT}


def _ctx(spec, scheme, precision, nf=NF):
    nx, nv, L, eps, T, N, bc, _ = spec
    return pr.pr_init(nx, 0.0, 1.0, bc, nv, L, eps, T, N, scheme=scheme, precision=precision, nf=nf)


def _extras(scheme):
    return [pr.instance(24, 8, 1e-3, L=8.0, bc=pr.PR_BC_PERIODIC, eps=1e-2, scheme=scheme),
            pr.instance(50, 16, 5e-4, L=8.0, bc=pr.PR_BC_OUTFLOW, eps=1e-4, scheme=scheme),
            pr.instance(17, 4, 2e-3, L=6.0, bc=pr.PR_BC_REFLECT, eps=1.0, scheme=scheme)]


def _levels(ctx):
    return np.stack([pr.pr_moments(ctx, n) for n in range(ctx.N + 1)])


@pytest.mark.parametrize("scheme", [pr.PR_UPWIND, pr.PR_MUSCL])
@pytest.mark.parametrize("precision", [pr.PR_FP64, pr.PR_MIXED])
def test_problems_and_instances_in_one_launch_match_oracle_and_single_runs(scheme, precision):
    K = 3
    ctxs = [_ctx(sp, scheme, precision) for sp in PROBLEMS]
    extras = _extras(scheme)
    ext_U = [W.smooth_periodic(d.nx) for d in extras]
    m = None
    try:
        for c, sp in zip(ctxs, PROBLEMS):
            pr.pr_set_initial(c, sp[7](sp[0]))
        m = pr.pr_multi_create(ctxs, extras)
        assert m.first_independent == sum(sp[5] for sp in PROBLEMS)
        for j, U in enumerate(ext_U):
            pr.pr_batch_set_initial(m.batch, m.first_independent + j, U, pr.PR_PRIMITIVE)
        errs = np.concatenate([pr.pr_multi_iterate(m, 1), pr.pr_multi_iterate(m, K - 1)])
        assert errs.shape == (K, len(PROBLEMS))
        got = [_levels(c) for c in ctxs]
        f_ext = [pr.pr_batch_get_f(m.batch, m.first_independent + j) for j in range(len(extras))]
        assert all(pr.pr_iterations(c) == K for c in ctxs)
    finally:
        pr.pr_multi_destroy(m)
        for c in ctxs:
            pr.pr_destroy(c)
    for p, sp in enumerate(PROBLEMS):
        nx, nv, L, eps, T, N, bc, init = sp
        # the oracle's Algorithm 2 with the same n_f
        kin = O.Kin(nx=nx, nv=nv, L=L, bc=OBC[bc], eps=eps, scheme=scheme)
        Uo, errs_o, _ = O.parareal(O.Parareal(kin=kin, T=T, N=N, nf=NF), init(nx), K)
        for n in range(N + 1):
            assert moment_rel_err(got[p][n], Uo[K][n]) < TOL[precision], (p, n)
        # the same problem alone
        c = _ctx(sp, scheme, precision)
        try:
            pr.pr_set_initial(c, init(nx))
            _, errs1 = pr.pr_parareal_run(c, K)
            alone = _levels(c)
        finally:
            pr.pr_destroy(c)
        for n in range(N + 1):
            assert moment_rel_err(got[p][n], alone[n]) < TOL[precision], (p, n)
        assert np.allclose(errs[:, p], errs1, rtol=1e-6 if precision == pr.PR_FP64 else 1e-2, atol=1e-14)
    # the independent instances advanced K n_f steps, as in a batch of their own
    b = pr.pr_batch_create(extras, precision)
    try:
        for j, U in enumerate(ext_U):
            pr.pr_batch_set_initial(b, j, U, pr.PR_PRIMITIVE)
        pr.pr_batch_run(b, K * NF)
        for j in range(len(extras)):
            assert f_rel_err(f_ext[j], pr.pr_batch_get_f(b, j)) < FTOL[precision], j
    finally:
        pr.pr_batch_destroy(b)


def test_lockstep_and_iteration_limits():
    ctxs = [_ctx(sp, pr.PR_UPWIND, pr.PR_FP64) for sp in PROBLEMS[:2]]
    m = None
    try:
        for c, sp in zip(ctxs, PROBLEMS):
            pr.pr_set_initial(c, sp[7](sp[0]))
        m = pr.pr_multi_create(ctxs)
        assert m.first_independent == PROBLEMS[0][5] + PROBLEMS[1][5]
        pr.pr_multi_iterate(m, 2)
        pr.pr_parareal_iter(ctxs[1])     # one problem alone: no longer in lockstep
        with pytest.raises(pr.PrError) as ei:
            pr.pr_multi_iterate(m, 1)
        assert ei.value.code == pr.PR_EINVAL and "same iteration" in pr.pr_multi_last_error(m)
        pr.pr_parareal_iter(ctxs[0])     # both at k = 3 again
        pr.pr_multi_iterate(m, 1)
        assert [pr.pr_iterations(c) for c in ctxs] == [4, 4]
        with pytest.raises(pr.PrError) as ei:
            pr.pr_multi_iterate(m, 1)    # k = 5 > the smaller N = 4
        assert ei.value.code == pr.PR_EINVAL
        assert len(pr.pr_multi_iterate(m, 0)) == 0
    finally:
        pr.pr_multi_destroy(m)
        for c in ctxs:
            pr.pr_destroy(c)


def test_multi_set_up_rules():
    a = _ctx(PROBLEMS[0], pr.PR_UPWIND, pr.PR_FP64)
    b = _ctx(PROBLEMS[1], pr.PR_UPWIND, pr.PR_FP64, nf=NF + 1)
    c = _ctx(PROBLEMS[1], pr.PR_UPWIND, pr.PR_MIXED)
    nx = 16
    f = pr.pr_init_force(nx, 0.0, 2.0, pr.PR_BC_PERIODIC, 32, 8, 6.0, 1e-2, 0.05, 4, W.test3_force(nx), nf=NF)
    try:
        for bad, extra, what in (([a, b], [], "fine steps"), ([a, c], [], "precision"), ([a, a], [], "twice"),
                                 ([a, f], [], "exterior force"),
                                 ([a], _extras(pr.PR_MUSCL)[:1], "scheme")):
            with pytest.raises(pr.PrError) as ei:
                pr.pr_multi_create(bad, extra)
            assert ei.value.code == pr.PR_EINVAL and what in pr.pr_multi_last_error(None), what
        m = pr.pr_multi_create([a])
        try:
            with pytest.raises(pr.PrError) as ei:
                pr.pr_multi_iterate(m, 1)    # not initialised
            assert "pr_set_initial" in pr.pr_multi_last_error(m)
        finally:
            pr.pr_multi_destroy(m)
    finally:
        for x in (a, b, c, f):
            pr.pr_destroy(x)
