"""Pins of the oracle's higher-order coupling (Eq. 8, Remark 1 / Def. 3 with
L = 1): the first-order Chapman-Enskog lifting against a finite-difference
construction of -(d_t + v d_x) M, its zero moments and its stress and heat
flux; the compressible Navier-Stokes coarse model against the analytic shear
decay, against the kinetic model's own decay rates, against the stress of the
lifting, and its conservation; parareal with both at K = N."""
import math

import numpy as np
import pytest

import oracle as O


def _nodes(n, L):
    dv = 2 * L / n
    return -L + (np.arange(n) + 0.5) * dv, dv


def _grid(nv, L):
    v, dv = _nodes(nv, L)
    VX, VY, VZ = np.meshgrid(v, v, v, indexing="ij")
    return VX.ravel(), VY.ravel(), VZ.ravel(), dv ** 3


def _maxwell(rho, u, th, VX, VY, VZ):
    c2 = (VX - u[0]) ** 2 + (VY - u[1]) ** 2 + (VZ - u[2]) ** 2
    return rho / (2 * math.pi * th) ** 1.5 * np.exp(-c2 / (2 * th))


# a smooth analytic primitive profile on the periodic unit interval
def _prof(x):
    w = 2 * np.pi * x
    return np.array([1 + 0.3 * np.sin(w), 0.2 * np.cos(w), 0.1 * np.sin(2 * w), -0.05 * np.cos(w),
                     1 + 0.25 * np.sin(w + 0.3)])


def _mode(a, nx):
    return 2 * np.abs(np.fft.rfft(a)[1]) / nx


# ------------------------------------------------------------------ first-order lifting


def test_first_order_lift_matches_finite_difference_of_the_maxwellian():
    # g1 = -(d_t + v_x d_x) M with d_t M from the Euler equations (Eq. 5),
    # built here from the analytic profile by finite differences in x and in
    # the Maxwellian's parameters -- a different route from the oracle's
    # closed polynomial form.  The oracle's gradients are central differences
    # of cell values (O(dx^2)); nx = 400 makes that 1e-4.
    nx, nv, L, eps = 400, 10, 7.0, 1e-2
    x = (np.arange(nx) + 0.5) / nx
    U = _prof(x)
    k = O.Kin(nx=nx, nv=nv, L=L, eps=eps)
    f1 = O.lift_ce(k, U)
    VX, VY, VZ, _ = _grid(nv, L)
    h = 1e-5
    for i in (37, 180, 333):
        xi = x[i]
        r, ux, uy, uz, th = _prof(np.array(xi))
        P = lambda p: _maxwell(p[0], p[1:4], p[4], VX, VY, VZ)
        p0 = np.array([r, ux, uy, uz, th])
        dU = (_prof(np.array(xi + h)) - _prof(np.array(xi - h))) / (2 * h)  # d/dx of (rho, u, theta)
        dM_dx = (P(_prof(np.array(xi + h))) - P(_prof(np.array(xi - h)))) / (2 * h)
        # Euler (Eq. 5, E = 0) in primitive form: time derivatives of (rho, u, theta)
        drho, dux, duy, duz, dth = dU
        dt_p = np.array([-(ux * drho + r * dux), -(ux * dux + (r * dth + th * drho) / r), -ux * duy, -ux * duz,
                         -(ux * dth + 2.0 / 3.0 * th * dux)])
        dM_dt = np.zeros_like(dM_dx)
        for q in range(5):
            e = np.zeros(5)
            e[q] = h
            dM_dt += dt_p[q] * (P(p0 + e) - P(p0 - e)) / (2 * h)
        g_ref = -(dM_dt + VX * dM_dx)
        g = (f1[i] - O.lift(k, U)[i]) / eps
        assert np.max(np.abs(g - g_ref)) <= 2e-4 * np.max(np.abs(g_ref)), i


def test_first_order_lift_has_the_maxwellian_moments_and_bgk_transport_coefficients():
    # on a fine velocity grid: P(L1 U) = P(L0 U) (g1 carries no mass, momentum
    # or energy); its stress and heat flux are -eps (4/3) rho theta du_x,
    # -eps rho theta du_y, -eps rho theta du_z and -eps (5/2) rho theta dtheta
    # (mu = rho theta, kappa = 5 rho theta / 2), the gradients taken here as
    # central differences of the cell values
    nx, nv, L, eps = 24, 40, 10.0, 1e-2
    x = (np.arange(nx) + 0.5) / nx
    U = _prof(x)
    k = O.Kin(nx=nx, nv=nv, L=L, eps=eps)
    f1, f0 = O.lift_ce(k, U), O.lift(k, U)
    assert np.max(np.abs(O.project(k, f1, conserved=True) - O.project(k, f0, conserved=True))) < 1e-11
    VX, VY, VZ, dv3 = _grid(nv, L)
    dx = 1.0 / nx
    d = (np.roll(U, -1, axis=1) - np.roll(U, 1, axis=1)) / (2 * dx)
    for i in range(nx):
        r, ux, uy, uz, th = U[:, i]
        g = f1[i] - f0[i]
        cx, cy, cz = VX - ux, VY - uy, VZ - uz
        c2 = cx * cx + cy * cy + cz * cz
        mu = r * th
        assert abs((cx * cx * g).sum() * dv3 - (-eps * mu * 4 / 3 * d[1, i])) < 1e-11
        assert abs((cx * cy * g).sum() * dv3 - (-eps * mu * d[2, i])) < 1e-11
        assert abs((cx * cz * g).sum() * dv3 - (-eps * mu * d[3, i])) < 1e-11
        assert abs((0.5 * cx * c2 * g).sum() * dv3 - (-eps * 2.5 * mu * d[4, i])) < 1e-11


def test_force_grid_first_order_lift_is_the_isotropic_one():
    nx, nv = 10, 8
    x = (np.arange(nx) + 0.5) / nx
    U = _prof(x)
    for bc in (O.BC_PERIODIC, O.BC_OUTFLOW, O.BC_REFLECT):
        k = O.Kin(nx=nx, nv=nv, L=6.0, bc=bc, eps=3e-2)
        kv = O.VKin(nx=nx, nvx=nv, nvp=nv, L=6.0, bc=bc, eps=3e-2, E=np.ones(nx))
        assert np.array_equal(O.v_lift_ce(kv, U), O.lift_ce(k, U))


# ------------------------------------------------------------------ Navier-Stokes coarse model


def test_vanishing_viscosity_is_the_euler_solver_bit_for_bit():
    nx = 32
    x = (np.arange(nx) + 0.5) / nx
    V = O.prim_to_cons(_prof(x))
    for bc in (O.BC_PERIODIC, O.BC_OUTFLOW, O.BC_REFLECT):
        a, na = O.coarse_run(nx, bc, 0.5, 0.05, V)
        b, nb = O.coarse_run_cns(nx, bc, 0.5, 0.05, V, 1e-300)
        assert na == nb and np.array_equal(a, b)


def test_shear_wave_decays_at_the_analytic_viscous_rate():
    # u_y = A sin(2 pi x) on a uniform state: the viscous term adds the decay
    # exp(-eps (mu/rho) k_d^2 T), mu/rho = theta = 1, k_d^2 the eigenvalue of
    # the discrete second difference; the Rusanov part is shared with the
    # Euler run, whose amplitude divides it out
    nx, eps, T, A = 128, 1e-2, 0.2, 1e-4
    x = (np.arange(nx) + 0.5) / nx
    V = O.prim_to_cons(np.stack([1 + 0 * x, 0 * x, A * np.sin(2 * np.pi * x), 0 * x, 1 + 0 * x]))
    a, _ = O.coarse_run(nx, O.BC_PERIODIC, 0.5, T, V)
    b, _ = O.coarse_run_cns(nx, O.BC_PERIODIC, 0.5, T, V, eps)
    dx = 1.0 / nx
    kd2 = 4 / dx ** 2 * math.sin(math.pi * dx) ** 2
    rate = math.log(_mode(b[2], nx) / _mode(a[2], nx))
    assert abs(rate - (-eps * kd2 * T)) <= 1e-3 * eps * kd2 * T


@pytest.mark.parametrize("kind", ["shear", "heat"])
def test_viscous_decay_matches_the_kinetic_model(kind):
    # the BGK model itself (Eq. 7, tau = 1) damps a shear wave through
    # mu = rho theta and a temperature wave through kappa = 5 rho theta / 2
    # (and the acoustic coupling); the CNS decay in excess of the Euler
    # solver's own numerical damping must match the kinetic decay, which is
    # free of a coarse-scheme dissipation (MUSCL, 24^3)
    nx, eps, T = 48, 2e-2, 0.1
    x = (np.arange(nx) + 0.5) / nx
    if kind == "shear":
        U = np.stack([1 + 0 * x, 0 * x, 1e-3 * np.sin(2 * np.pi * x), 0 * x, 1 + 0 * x])
        q, off = 2, 0.0
    else:
        th = 1 + 1e-3 * np.cos(2 * np.pi * x)
        U = np.stack([1 / th, 0 * x, 0 * x, 0 * x, th])
        q, off = 4, 1.0
    k = O.Kin(nx=nx, nv=24, L=8.0, eps=eps, scheme=O.MUSCL)
    n = math.ceil(T / O.fine_dt_stab(k, 0.5))
    O.set_threads(8)
    try:
        f0 = O.lift_ce(k, U)
        U0, U1 = O.project(k, f0), O.project(k, O.fine_run(k, T / n, n, f0))
    finally:
        O.set_threads(1)
    rk = math.log(_mode(U1[q] - off, nx) / _mode(U0[q] - off, nx)) / T
    V0 = O.prim_to_cons(U0)
    Uc = O.cons_to_prim(O.coarse_run_cns(nx, O.BC_PERIODIC, 0.5, T, V0, eps)[0])
    Ue = O.cons_to_prim(O.coarse_run(nx, O.BC_PERIODIC, 0.5, T, V0)[0])
    rc = math.log(_mode(Uc[q] - off, nx) / _mode(Ue[q] - off, nx)) / T
    assert abs(rc - rk) <= 0.05 * abs(rk), (rc, rk)


def test_one_step_viscous_increment_is_the_stress_of_the_first_order_lift():
    # one local step: (CNS - Euler) / dt = -d/dx of the viscous flux; the flux
    # is the stress and heat flux of the first-order lifting (their moments,
    # by quadrature on a fine velocity grid), differentiated by central
    # differences -- pins mu, kappa, the 4/3 and the energy flux u . Pi + q
    nx, nv, L, eps, dT = 256, 28, 9.0, 1e-2, 1e-6
    x = (np.arange(nx) + 0.5) / nx
    U = _prof(x)
    V = O.prim_to_cons(U)
    a, na = O.coarse_run(nx, O.BC_PERIODIC, 0.5, dT, V)
    b, nb = O.coarse_run_cns(nx, O.BC_PERIODIC, 0.5, dT, V, eps)
    assert na == nb == 1
    inc = (b - a) / dT
    k = O.Kin(nx=nx, nv=nv, L=L, eps=eps)
    g = O.lift_ce(k, U) - O.lift(k, U)
    VX, VY, VZ, dv3 = _grid(nv, L)
    flux = np.zeros((5, nx))
    for i in range(nx):
        ux, uy, uz = U[1:4, i]
        cx, cy, cz = VX - ux, VY - uy, VZ - uz
        c2 = cx * cx + cy * cy + cz * cz
        P = [(cx * c * g[i]).sum() * dv3 for c in (cx, cy, cz)]
        qx = (0.5 * cx * c2 * g[i]).sum() * dv3
        flux[1:4, i] = P
        flux[4, i] = ux * P[0] + uy * P[1] + uz * P[2] + qx
    dx = 1.0 / nx
    want = -(np.roll(flux, -1, axis=1) - np.roll(flux, 1, axis=1)) / (2 * dx)
    for q in range(1, 5):
        assert np.max(np.abs(inc[q] - want[q])) <= 2e-3 * np.max(np.abs(want[q])), q
    assert np.max(np.abs(inc[0])) == 0.0


def test_navier_stokes_conserves_on_a_periodic_domain():
    nx = 40
    x = (np.arange(nx) + 0.5) / nx
    V = O.prim_to_cons(_prof(x))
    b, ns = O.coarse_run_cns(nx, O.BC_PERIODIC, 0.5, 0.1, V, 3e-2)
    assert ns > 1
    assert np.allclose(b.sum(axis=1), V.sum(axis=1), rtol=0, atol=1e-12)
    assert np.max(np.abs(b - V)) > 1e-2


# ------------------------------------------------------------------ parareal


@pytest.mark.parametrize("coarse,lift", [(O.COARSE_CNS, 0), (O.COARSE_CNS, 1), (O.COARSE_EULER, 1)])
def test_parareal_with_cns_or_first_order_lift_reaches_the_serial_chain(coarse, lift):
    nx, N = 20, 4
    x = (np.arange(nx) + 0.5) / nx
    k = O.Kin(nx=nx, nv=8, L=8.0, eps=2e-2, scheme=O.UPWIND)
    p = O.Parareal(kin=k, T=0.04, N=N, coarse=coarse, lift=lift)
    U0 = _prof(x)
    chain = [O.prim_to_cons(U0)]
    for _ in range(N):
        chain.append(O.fine_propagate(p, chain[-1]))
    chain = np.stack(chain)
    Uall, errs, _ = O.parareal(p, U0, K=N)
    scale = np.max(np.abs(chain), axis=(0, 2), keepdims=True)
    assert np.max(np.abs(Uall[N] - chain) / scale) < 1e-13
    c = [chain[0]]
    for _ in range(N):
        c.append(O.coarse_propagate(p, c[-1]))
    assert np.array_equal(Uall[0], np.stack(c))
    if coarse == O.COARSE_CNS:
        G, _ = O.coarse_run_cns(nx, O.BC_PERIODIC, 0.5, 0.01, chain[0], 2e-2)
        assert np.array_equal(c[1], G)


def test_fine_propagator_with_first_order_lift_is_lift_run_project():
    nx = 12
    x = (np.arange(nx) + 0.5) / nx
    k = O.Kin(nx=nx, nv=8, L=8.0, eps=2e-2, scheme=O.MUSCL)
    p = O.Parareal(kin=k, T=0.03, N=3, lift=1)
    V = O.prim_to_cons(_prof(x))
    n, dt = O.fine_nsteps(p)
    f = O.fine_run(k, dt, n, O.lift_ce(k, O.cons_to_prim(V)))
    assert np.array_equal(O.fine_propagate(p, V), O.project(k, f, conserved=True))
    kv = O.VKin(nx=nx, nvx=8, nvp=8, L=8.0, eps=2e-2, scheme=O.MUSCL, E=0.5 * np.ones(nx))
    pv = O.VParareal(kin=kv, T=0.03, N=3, lift=1, coarse=O.COARSE_CNS)
    n, dt = O.v_fine_nsteps(pv)
    f = O.v_fine_run(kv, dt, n, O.v_lift_ce(kv, O.cons_to_prim(V)))
    assert np.array_equal(O.v_fine_propagate(pv, V), O.v_project(kv, f, conserved=True))
    G, _ = O.coarse_run_cns(nx, O.BC_PERIODIC, 0.5, 0.01, V, 2e-2, E=kv.E)
    assert np.array_equal(O.v_coarse_propagate(pv, V), G)
