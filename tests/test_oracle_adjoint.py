"""Pins of the oracle's reference gradient (hand-derived adjoint of the upwind
fine run) against central finite differences of the oracle's own forward run
-- the definition of the derivative, evaluated at several step sizes."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2502_02704_gb300 import workloads as W


def _J(k, dt, n, U, lamV):
    return float((O.project(k, O.fine_run(k, dt, n, O.lift(k, U)), conserved=True) * lamV).sum())


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_OUTFLOW, O.BC_REFLECT])
def test_adjoint_matches_central_differences(bc):
    nx, nv, L, dt, n, eps = 10, 8, 6.0, 0.004, 8, 2e-2
    k = O.Kin(nx=nx, nv=nv, L=L, bc=bc, eps=eps, scheme=O.UPWIND)
    U0 = W.density_modes(nx, 0.2, 0.1)
    U0[1] = 0.1 * np.sin(2 * np.pi * W.cell_centres(nx))
    U0[4] = 1.0 + 0.1 * np.cos(2 * np.pi * W.cell_centres(nx))
    lamV = np.random.default_rng(bc + 3).normal(size=(5, nx))
    dU, de = O.adjoint(k, dt, n, U0, lamV)
    h = 1e-5
    for q, i in [(0, 0), (0, 6), (1, 3), (2, 9), (3, 4), (4, 1), (4, 8)]:
        Up, Um = U0.copy(), U0.copy()
        Up[q, i] += h
        Um[q, i] -= h
        fd = (_J(k, dt, n, Up, lamV) - _J(k, dt, n, Um, lamV)) / (2 * h)
        assert abs(fd - dU[q, i]) <= 1e-6 * max(abs(dU[q, i]), 1e-3), (q, i, fd, dU[q, i])
    he = 1e-4
    kp = O.Kin(nx=nx, nv=nv, L=L, bc=bc, eps=eps * math.exp(he), scheme=O.UPWIND)
    km = O.Kin(nx=nx, nv=nv, L=L, bc=bc, eps=eps * math.exp(-he), scheme=O.UPWIND)
    fd = (_J(kp, dt, n, U0, lamV) - _J(km, dt, n, U0, lamV)) / (2 * he)
    assert abs(fd - de) <= 1e-5 * abs(de), (fd, de)


def test_adjoint_of_collisionless_run_has_no_eps_gradient():
    k = O.Kin(nx=6, nv=4, L=4.0, bc=O.BC_PERIODIC, eps=math.inf, scheme=O.UPWIND)
    U0 = W.density_modes(6, 0.1, 0.2)
    lamV = np.random.default_rng(0).normal(size=(5, 6))
    dU, de = O.adjoint(k, 0.01, 5, U0, lamV)
    assert de == 0.0
    # free transport conserves total mass: the gradient of total mass is 1 per unit rho0 dx
    dU2, _ = O.adjoint(k, 0.01, 5, U0, np.vstack([np.ones(6), np.zeros((4, 6))]))
    m = O.project(k, O.lift(k, U0))[0] / U0[0]  # discrete mass of a unit Maxwellian
    assert np.allclose(dU2[0], m, rtol=1e-12)
