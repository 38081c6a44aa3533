"""The hand-written adjoint of the float64 upwind fine run (pr_batch_adjoint)
against the oracle's reference gradient and against central differences of
the GPU forward run; the torch.autograd wrapper on the density-misfit workload."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import workloads as W
from paper_2502_02704_gb300.autograd import density_misfit, density_modes_state, fine_run_moments

pytestmark = pytest.mark.gpu


def _gpu_grad(nx, nv, L, bc, eps, dt, n, U0, lamV, ckpt):
    b = pr.pr_batch_create([pr.instance(nx, nv, dt, L=L, bc=bc, eps=eps, scheme=pr.PR_UPWIND)], pr.PR_FP64)
    try:
        pr.pr_batch_set_initial(b, 0, U0)
        return pr.pr_batch_adjoint(b, 0, n, lamV, ckpt)
    finally:
        pr.pr_batch_destroy(b)


@pytest.mark.parametrize("bc,ckpt", [(pr.PR_BC_PERIODIC, 4), (pr.PR_BC_OUTFLOW, 5), (pr.PR_BC_PERIODIC, 100)])
def test_adjoint_matches_oracle_gradient(bc, ckpt):
    # nx = 40 (two x tiles), nv = 12 (two v chunks, the last ragged), 13 steps
    nx, nv, L, eps, n = 40, 12, 6.0, 3e-2, 13
    dt = pr.fine_dt(nx, nv, L)
    U0 = W.density_modes(nx, 0.2, 0.1)
    U0[1] = 0.1 * np.sin(2 * np.pi * W.cell_centres(nx))
    U0[4] = 1.0 + 0.2 * np.cos(2 * np.pi * W.cell_centres(nx))
    lamV = np.random.default_rng(1).normal(size=(5, nx))
    dU, de = _gpu_grad(nx, nv, L, bc, eps, dt, n, U0, lamV, ckpt)
    k = O.Kin(nx=nx, nv=nv, L=L, bc={pr.PR_BC_PERIODIC: O.BC_PERIODIC, pr.PR_BC_OUTFLOW: O.BC_OUTFLOW}[bc],
              eps=eps, scheme=O.UPWIND)
    dUo, deo = O.adjoint(k, dt, n, U0, lamV)
    scale = np.max(np.abs(dUo), axis=1, keepdims=True)
    assert np.max(np.abs(dU - dUo) / scale) < 1e-10
    assert abs(de - deo) <= 1e-10 * abs(deo)


def test_adjoint_rejects_unsupported_setups():
    for prec, scheme, bc in [(pr.PR_MIXED, pr.PR_UPWIND, pr.PR_BC_PERIODIC),
                             (pr.PR_FP64, pr.PR_MUSCL, pr.PR_BC_PERIODIC),
                             (pr.PR_FP64, pr.PR_UPWIND, pr.PR_BC_REFLECT)]:
        b = pr.pr_batch_create([pr.instance(8, 4, 1e-3, bc=bc, scheme=scheme)], prec)
        try:
            pr.pr_batch_set_initial(b, 0, W.density_modes(8, 0.1, 0.1))
            with pytest.raises(pr.PrError) as ei:
                pr.pr_batch_adjoint(b, 0, 3, np.zeros((5, 8)))
            assert ei.value.code == pr.PR_EINVAL
        finally:
            pr.pr_batch_destroy(b)


def test_autograd_matches_central_differences_small():
    nx, nv, L, n = 24, 8, 6.0, 11
    dt = pr.fine_dt(nx, nv, L)
    target = torch.as_tensor(W.density_modes(nx, 0.05, 0.25)[0])
    a = torch.tensor([0.2, 0.1, math.log(2e-2)], dtype=torch.float64, requires_grad=True)
    J = density_misfit(a[0], a[1], a[2], target, nx, nv, dt, n, L=L, checkpoint=4)
    J.backward()
    g = a.grad.numpy()

    def Jf(p):
        with torch.no_grad():
            return float(density_misfit(torch.tensor(p[0]), torch.tensor(p[1]), torch.tensor(p[2]), target, nx, nv,
                                        dt, n, L=L))

    p0 = a.detach().numpy()
    for k in range(3):
        h = 1e-5
        e = np.zeros(3)
        e[k] = h
        fd = (Jf(p0 + e) - Jf(p0 - e)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-8), (k, fd, g[k])


def test_density_misfit_gradient_full_size_with_checkpoints():
    # the misfit workload: Nx = 256, 24^3, eps = 1e-3, T = 0.05 (197 steps of
    # 0.05/197), seeded (a1, a2) and target modes, checkpoint every 16 steps;
    # gradient w.r.t. (a1, a2, log eps) against central differences in FP64
    nx, nv, L, T = 256, 24, 8.0, 0.05
    n = math.ceil(T / pr.fine_dt(nx, nv, L) * (1 - 1e-9))
    dt = T / n
    assert n == 197
    a1, a2 = W.draw_modes(1)
    t1, t2 = W.draw_modes(2)
    target = torch.as_tensor(W.density_modes(nx, t1, t2)[0])
    p = torch.tensor([a1, a2, math.log(1e-3)], dtype=torch.float64, requires_grad=True)
    J = density_misfit(p[0], p[1], p[2], target, nx, nv, dt, n, L=L, checkpoint=16)
    J.backward()
    g = p.grad.numpy()

    def Jf(q):
        with torch.no_grad():
            return float(density_misfit(torch.tensor(q[0]), torch.tensor(q[1]), torch.tensor(q[2]), target, nx, nv,
                                        dt, n, L=L))

    q0 = p.detach().numpy()
    for k in range(3):
        fds = []
        for h in (1e-4, 1e-5, 1e-6):
            e = np.zeros(3)
            e[k] = h
            fds.append((Jf(q0 + e) - Jf(q0 - e)) / (2 * h))
        best = min(abs(fd - g[k]) for fd in fds)
        assert best <= 1e-6 * abs(g[k]), (k, fds, g[k])
