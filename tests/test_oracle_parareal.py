"""Pins of the CPU oracle's parareal driver (Algorithms 1-2, Sec. 2) and of the
Euler limit of the kinetic model (Sec. 1, Eq. 5)."""
import math

import numpy as np
import pytest

import oracle as O
from exact_riemann import density_profile


def _sod_U(nx, split=0.5):
    x = (np.arange(nx) + 0.5) / nx
    left = x < split
    return np.stack([np.where(left, 1.0, 0.125), 0 * x, 0 * x, 0 * x, np.where(left, 1.0, 0.8)])


def _small_problem(N=5, scheme=O.UPWIND, bc=O.BC_OUTFLOW):
    k = O.Kin(nx=24, nv=8, L=8.0, bc=bc, eps=1e-2, scheme=scheme)
    return O.Parareal(kin=k, T=0.05, N=N)


def _serial_chain(p, V0, propagate):
    out = [V0]
    for _ in range(p.N):
        out.append(propagate(p, out[-1]))
    return np.stack(out)


def _close(a, b, rel):
    scale = np.max(np.abs(b), axis=(0, 2), keepdims=True) if b.ndim == 3 else np.max(np.abs(b))
    scale = np.maximum(scale, 1e-300)
    return np.max(np.abs(a - b) / scale) <= rel


def test_fine_step_count_for_sod_setup():
    # Sec. 2.2 with the CFL reading: dx = 1/64, max|v_x| = 7.5, dt_stab = cfl dx / 7.5,
    # dT_g = 0.1/8 -> exactly 12 steps of 1/960.
    p = O.Parareal(kin=O.Kin(nx=64, nv=16, L=8.0), T=0.1, N=8)
    n, dt = O.fine_nsteps(p)
    assert n == 12 and abs(dt - 0.1 / 8 / 12) < 1e-18


def test_iteration_zero_is_the_coarse_chain():
    p = _small_problem()
    V0 = O.prim_to_cons(_sod_U(24))
    U, errs, kd = O.parareal(p, _sod_U(24), K=0)
    chain = _serial_chain(p, V0, O.coarse_propagate)
    assert np.array_equal(U[0], chain)


@pytest.mark.parametrize("scheme", [O.UPWIND, O.MUSCL])
def test_k_equals_n_reproduces_serial_fine_chain(scheme):
    # Sec. 2.2: after N_g iterations the outcome is the fully fine solution,
    # here the chain U^n = P F L(U^{n-1}) (re-lifted at every T^n); the form
    # G(a) + (F(a) - G(a)) equals F(a) up to rounding only.
    p = _small_problem(N=4, scheme=scheme)
    V0 = O.prim_to_cons(_sod_U(24))
    chain = _serial_chain(p, V0, O.fine_propagate)
    U, errs, kd = O.parareal(p, _sod_U(24), K=4)
    assert kd == 4
    assert _close(U[4], chain, 1e-13)
    # and the first k slices are exact after k iterations
    for k in range(1, 5):
        assert _close(U[k][: k + 1], chain[: k + 1], 1e-13)
    # while the later ones still differ before convergence
    assert np.max(np.abs(U[1][4] - chain[4])) > 1e-6


def test_algorithm_1_and_2_agree_bitwise():
    # Algorithm 2 only skips work whose result Algorithm 1 would reproduce.
    p = _small_problem(N=4)
    U1, e1, _ = O.parareal(p, _sod_U(24), K=3, alg=1)
    U2, e2, _ = O.parareal(p, _sod_U(24), K=3, alg=2)
    assert np.array_equal(U1, U2) and np.array_equal(e1, e2)


def test_successive_error_definition_and_decay():
    # Eq. (10): error = max_n |U^{n,k} - U^{n,k-1}|; it decays with k (Sec. 5.1).
    p = _small_problem(N=6)
    U, errs, _ = O.parareal(p, _sod_U(24), K=4)
    for k in range(1, 5):
        assert errs[k - 1] == np.max(np.abs(U[k] - U[k - 1]))
    assert all(b < a for a, b in zip(errs, errs[1:]))


def test_tolerance_stops_the_iteration():
    p = _small_problem(N=6)
    _, errs, _ = O.parareal(p, _sod_U(24), K=4)
    tol = 0.5 * (errs[1] + errs[2])
    U, errs2, kd = O.parareal(p, _sod_U(24), K=4, tol=tol)
    assert kd == 3 and np.array_equal(errs2[:3], errs[:3])
    assert np.array_equal(U[4], U[3])


def test_fine_propagator_is_lift_run_project():
    p = _small_problem(N=3)
    V0 = O.prim_to_cons(_sod_U(24))
    n, dt = O.fine_nsteps(p)
    f = O.fine_run(p.kin, dt, n, O.lift(p.kin, O.cons_to_prim(V0)))
    assert np.array_equal(O.fine_propagate(p, V0), O.project(p.kin, f, conserved=True))


def test_kinetic_moments_approach_euler_as_eps_goes_to_zero():
    # Sec. 1: as eps -> 0 the moments of f solve the Euler equations (Eq. 5).
    # Kinetic Sod at eps = 1e-1 vs 1e-5 against the exact Riemann solution.
    nx, T = 100, 0.1
    errs = []
    x = (np.arange(nx) + 0.5) / nx
    exact = density_profile((1.0, 0.0, 1.0), (0.125, 0.0, 0.1), 5.0 / 3.0, x, 0.5, T)
    for eps in (1e-1, 1e-5):
        k = O.Kin(nx=nx, nv=12, L=7.0, bc=O.BC_OUTFLOW, eps=eps, scheme=O.MUSCL)
        n = math.ceil(T / O.fine_dt_stab(k, 0.5))
        f = O.fine_run(k, T / n, n, O.lift(k, _sod_U(nx)))
        errs.append(np.mean(np.abs(O.project(k, f)[0] - exact)))
    assert errs[1] < 0.5 * errs[0], errs
    assert errs[1] < 0.015, errs


def test_one_iteration_carries_a_constant_fine_drift_through_the_coarse_chain():
    # Parareal correction of Sec. 1 / Algorithm 1 in the case where F = G + d
    # with d almost constant: a uniform gas (G is then the identity) on a
    # coarse velocity grid, whose quadrature defect makes P F L drift by a
    # small d(U).  One iteration gives U^{n,1} = U^{n-1,1} + d(U^0), i.e. the
    # fine chain S^n = S^{n-1} + d(S^{n-1}) up to O(n^2 d d'), whereas a
    # correction that used the previous iterate would stay at U^0 + d(U^0).
    nx, N = 4, 6
    k = O.Kin(nx=nx, nv=12, L=6.0, bc=O.BC_PERIODIC, eps=1e-2)
    p = O.Parareal(kin=k, T=0.06, N=N)
    U0 = np.tile(np.array([[1.0], [0.2], [0.0], [0.0], [0.7]]), (1, nx))
    V0 = O.prim_to_cons(U0)
    chain = _serial_chain(p, V0, O.fine_propagate)
    U, errs, _ = O.parareal(p, U0, K=1)
    assert np.array_equal(U[0][N], V0)  # G is the identity on a uniform state
    drift = np.max(np.abs(chain[N] - V0))
    assert drift > 1e-4
    assert np.max(np.abs(U[1] - chain)) < 1e-2 * drift
