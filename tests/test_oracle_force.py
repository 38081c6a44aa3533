"""Pins of the oracle's exterior-force path (Eq. 11 with E != 0, the v_x
Rusanov flux of Eq. 13, the Euler source of Eq. 5, Test 3) against closed
forms, summation-by-parts identities, an equilibrium in a potential and the
Euler limit, none of which restates the flux formula."""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _nodes(n, L):
    dv = 2 * L / n
    return -L + (np.arange(n) + 0.5) * dv, dv


def _homogeneous_f(nx, nvx, nvp, L, U1):
    """nx identical columns, the Maxwellian of primitive U1 (5 numbers)."""
    k = O.VKin(nx=1, nvx=nvx, nvp=nvp, L=L)
    f1 = O.v_lift(k, np.array(U1, dtype=float).reshape(5, 1))
    return np.repeat(f1, nx, axis=0)


def _moments(f, nvx, nvp, L):
    """Conserved sums (rho, rho u, E) of every column by plain numpy quadrature."""
    vx, dvx = _nodes(nvx, L)
    vp, dvp = _nodes(nvp, L)
    dv3 = dvx * dvp * dvp
    F = f.reshape(f.shape[0], nvx, nvp, nvp)
    VX, VY, VZ = np.meshgrid(vx, vp, vp, indexing="ij")
    return np.stack([(F * w).sum(axis=(1, 2, 3)) * dv3
                     for w in (1.0, VX, VY, VZ, 0.5 * (VX ** 2 + VY ** 2 + VZ ** 2))])


# ------------------------------------------------------------------ reduction to E = 0


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_OUTFLOW, O.BC_REFLECT])
@pytest.mark.parametrize("scheme", [O.UPWIND, O.MUSCL])
def test_zero_force_isotropic_grid_is_the_pinned_e0_oracle(bc, scheme):
    # with E = 0 and nvx = nvp the force path must be the E = 0 scheme, bit for bit
    nx, nv = 9, 6
    x = (np.arange(nx) + 0.5) / nx
    U = np.stack([1 + 0.3 * np.sin(2 * np.pi * x), 0.2 * np.cos(2 * np.pi * x), 0.05 + 0 * x, -0.1 + 0 * x,
                  1 + 0.2 * x])
    for eps in (1e-2, math.inf):
        k = O.Kin(nx=nx, nv=nv, L=6.0, bc=bc, eps=eps, scheme=scheme)
        for E in (None, np.zeros(nx)):
            kv = O.VKin(nx=nx, nvx=nv, nvp=nv, L=6.0, bc=bc, eps=eps, scheme=scheme, E=E)
            f = O.lift(k, U)
            assert np.array_equal(O.v_lift(kv, U), f)
            g = O.fine_step(k, 1e-3, f)
            assert np.array_equal(O.v_fine_step(kv, 1e-3, f), g)
            assert np.array_equal(O.v_project(kv, g), O.project(k, g))
            assert O.v_fine_dt_stab(kv, 0.5) == O.fine_dt_stab(k, 0.5)


def test_zero_force_coarse_source_is_the_plain_coarse_solver():
    nx = 16
    x = (np.arange(nx) + 0.5) / nx
    V = O.prim_to_cons(np.stack([1 + 0.3 * np.sin(2 * np.pi * x), 0.1 + 0 * x, 0 * x, 0 * x, 1 + 0 * x]))
    a, na = O.coarse_run(nx, O.BC_PERIODIC, 0.5, 0.05, V)
    b, nb = O.coarse_run_force(nx, O.BC_PERIODIC, 0.5, 0.05, V, np.zeros(nx))
    assert na == nb and np.array_equal(a, b)


# ------------------------------------------------------------------ homogeneous closed forms


@pytest.mark.parametrize("E", [0.8, -0.8])
def test_unit_courant_number_shifts_by_one_velocity_cell(E):
    # collisionless, x-homogeneous, constant E, dt |E| / dv_x = 1: the v_x
    # Rusanov flux is then the exact upwind shift by one cell, the outermost
    # cell keeps what arrives (closed box) and the first one empties
    nx, nvx, nvp, L = 3, 10, 3, 5.0
    rng = np.random.default_rng(7)
    f1 = rng.uniform(0.1, 1.0, size=(1, nvx * nvp * nvp))
    f = np.repeat(f1, nx, axis=0)
    dvx = 2 * L / nvx
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, eps=math.inf, E=np.full(nx, E))
    g = O.v_fine_step(k, dvx / abs(E), f).reshape(nx, nvx, nvp * nvp)
    F = f.reshape(nx, nvx, nvp * nvp)
    want = np.zeros_like(F)
    if E > 0:
        want[:, 1:] = F[:, :-1]
        want[:, -1] += F[:, -1]
    else:
        want[:, :-1] = F[:, 1:]
        want[:, 0] += F[:, 0]
    assert np.max(np.abs(g - want)) <= 1e-15 * np.max(F) * 4


@pytest.mark.parametrize("eps", [math.inf, 1e-2])
def test_homogeneous_momentum_grows_as_rho_E_t(eps):
    # Eq. (5): d_t(rho u_x) = rho E, rho, u_y, u_z unchanged.  The closed
    # velocity box adds only the tail values at |v_x| = L (the mean moves from
    # 0.2 to 1.0 and the upwind diffusion widens the profile a little, leaving
    # ~1e-15 of f at v_x = 10).
    # (v_y, v_z cells fine enough that the discrete Maxwellian of the BGK step
    # carries the moments to rounding)
    nx, nvx, nvp, L, E = 2, 60, 32, 10.0, 0.7
    U1 = [1.3, 0.2, -0.1, 0.05, 0.9]
    f = _homogeneous_f(nx, nvx, nvp, L, U1)
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, eps=eps, E=np.full(nx, E))
    dt = 0.3 * (2 * L / nvx) / E
    m0 = _moments(f, nvx, nvp, L)
    n = 8
    g = O.v_fine_run(k, dt, n, f)
    m = _moments(g, nvx, nvp, L)
    rho = m0[0]
    # (collisionless 4e-16; the BGK step's discrete Maxwellian adds ~2e-13)
    assert np.max(np.abs(m[0] - rho)) <= 1e-12 * rho[0]
    assert np.max(np.abs(m[1] - (m0[1] + rho * E * n * dt))) <= 1e-12
    assert np.max(np.abs(m[2:4] - m0[2:4])) <= 1e-12


def test_one_step_energy_gain_closed_form():
    # Summation by parts of one collisionless step on x-homogeneous data with a
    # cell-wise force E_i (columns identical, so the x fluxes cancel):
    #   d(rho u_x)_i = dt E_i rho,
    #   dE_i = dt (E_i rho u_x + E_max dv_x rho / 2),
    # the second term being the numerical heating of the Rusanov viscosity,
    # with E_max = max_i |E_i| the same for every column (also where E_i = 0).
    nx, nvx, nvp, L = 4, 50, 10, 10.0
    E = np.array([0.9, -0.4, 0.0, 1.3])
    U1 = [0.8, 0.3, 0.1, -0.2, 1.1]
    f = _homogeneous_f(nx, nvx, nvp, L, U1)
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, eps=math.inf, E=E)
    dvx = 2 * L / nvx
    dt = 0.4 * dvx / 1.3
    m0 = _moments(f, nvx, nvp, L)
    m1 = _moments(O.v_fine_step(k, dt, f), nvx, nvp, L)
    rho, mx = m0[0], m0[1]
    assert np.max(np.abs((m1[1] - m0[1]) - dt * E * rho)) <= 1e-13
    gain = dt * (E * mx + 1.3 * dvx * rho / 2)
    assert np.max(np.abs((m1[4] - m0[4]) - gain)) <= 1e-13 * np.max(np.abs(gain))


# ------------------------------------------------------------------ conservation with x-dependent E


def _test3_E(x):
    return -5 * x ** 4 * (x - 2) ** 4 * (x - 1)


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_REFLECT])
@pytest.mark.parametrize("scheme", [O.UPWIND, O.MUSCL])
def test_mass_is_conserved_exactly_by_the_closed_velocity_box(bc, scheme):
    nx, nvx, nvp, L = 12, 16, 4, 8.0
    x = 2 * (np.arange(nx) + 0.5) / nx
    rng = np.random.default_rng(11)
    f = rng.uniform(0.0, 1.0, size=(nx, nvx * nvp * nvp))
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, bc=bc, eps=math.inf, scheme=scheme, E=_test3_E(x))
    g = O.v_fine_run(k, O.v_fine_dt_stab(k, 0.5), 3, f)
    assert abs(g.sum() - f.sum()) <= 1e-13 * f.sum()


def test_global_momentum_balance_uses_each_cells_own_force():
    # periodic, collisionless: the x fluxes telescope, so
    # sum_i d(rho u_x)_i = dt sum_i E_i rho_i (up to the v_x = +-L tails)
    nx, nvx, nvp, L = 20, 50, 8, 10.0
    x = 2 * (np.arange(nx) + 0.5) / nx
    U = np.stack([1 + 0.4 * np.sin(np.pi * x), 0.3 * np.cos(np.pi * x), 0 * x, 0 * x, 1 + 0.3 * np.cos(np.pi * x)])
    E = _test3_E(x)
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, eps=math.inf, scheme=O.MUSCL, E=E)
    f = O.v_lift(k, U)
    dt = O.v_fine_dt_stab(k, 0.5)
    m0 = _moments(f, nvx, nvp, L)
    m1 = _moments(O.v_fine_step(k, dt, f), nvx, nvp, L)
    lhs = (m1[1] - m0[1]).sum()
    rhs = dt * (E * m0[0]).sum()
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)
    # a force read one cell off would break the balance
    assert abs(dt * (np.roll(E, 1) * m0[0]).sum() - rhs) > 1e-3 * abs(rhs)


# ------------------------------------------------------------------ equilibrium in a potential


@pytest.mark.parametrize("scheme", [O.UPWIND, O.MUSCL])
def test_equilibrium_in_a_potential_is_kept_to_first_order(scheme):
    # f = exp(-phi(x)/theta) M_{0,theta}(v) with E = -phi' solves
    # v d_x f + E d_v f = 0 (and is Maxwellian, so BGK keeps it); the scheme's
    # residual |f* - f| / dt must fall at first order as x and v_x are refined
    # together.  The opposite sign of the force term leaves an O(1) residual.
    def resid(n, sign):
        x = (np.arange(n) + 0.5) / n
        phi = 0.1 * np.cos(2 * np.pi * x)
        E = sign * 0.2 * np.pi * np.sin(2 * np.pi * x)
        U = np.stack([np.exp(-phi), 0 * x, 0 * x, 0 * x, 1 + 0 * x])
        k = O.VKin(nx=n, nvx=n, nvp=6, L=8.0, eps=math.inf, scheme=scheme, E=E)
        f = O.v_lift(k, U)
        dt = O.v_fine_dt_stab(k, 0.5)
        return np.max(np.abs(O.v_fine_step(k, dt, f) - f)) / (dt * np.max(f))

    r = [resid(n, 1.0) for n in (16, 32, 64)]
    assert r[0] / r[1] > 1.8 and r[1] / r[2] > 1.8, r
    assert r[2] < 0.1, r
    assert resid(32, -1.0) > 0.5


# ------------------------------------------------------------------ coarse source


def test_coarse_source_single_local_step_closed_form():
    # x-homogeneous Euler state: the Rusanov fluxes cancel, and a coarse
    # interval shorter than one CFL step is one forward-Euler step of
    # d_t(rho u_x) = rho E, d_t E = rho u_x E (Eq. 5).
    nx = 5
    E = np.array([0.5, -1.0, 0.0, 2.0, 0.25])
    U1 = np.array([1.2, 0.3, -0.2, 0.1, 0.8])
    V = O.prim_to_cons(np.repeat(U1.reshape(5, 1), nx, axis=1))
    dT = 1e-4
    out, ns = O.coarse_run_force(nx, O.BC_PERIODIC, 0.5, dT, V, E)
    assert ns == 1
    want = V.copy()
    want[1] += dT * V[0] * E
    want[4] += dT * V[1] * E
    assert np.max(np.abs(out - want)) <= 1e-15
    # several local steps under a uniform force: the state stays homogeneous
    # and rho u_x grows exactly linearly (rho constant)
    out, ns = O.coarse_run_force(nx, O.BC_PERIODIC, 0.5, 0.3, V, np.full(nx, 0.7))
    assert ns > 1
    assert np.max(np.abs(out[0] - V[0])) == 0.0
    assert np.max(np.abs(out[1] - (V[1] + 0.3 * V[0] * 0.7))) <= 1e-14


def test_coarse_source_is_forward_euler_on_the_old_state():
    # one local step on a non-uniform state: the force adds dT S(V^n) to the
    # plain Rusanov update (pinned separately), S evaluated on the old state
    nx = 12
    x = (np.arange(nx) + 0.5) / nx
    V = O.prim_to_cons(np.stack([1 + 0.3 * np.sin(2 * np.pi * x), 0.4 * np.cos(2 * np.pi * x), 0 * x, 0 * x,
                                 1 + 0.2 * np.sin(4 * np.pi * x)]))
    E = 1.5 * np.cos(2 * np.pi * x) + 0.3
    dT = 1e-4
    a, na = O.coarse_run_force(nx, O.BC_PERIODIC, 0.5, dT, V, E)
    b, nb = O.coarse_run(nx, O.BC_PERIODIC, 0.5, dT, V)
    assert na == nb == 1
    S = np.zeros_like(V)
    S[1] = V[0] * E
    S[4] = V[1] * E
    assert np.max(np.abs((a - b) - dT * S)) <= 1e-15


def test_force_propagators_are_their_definitions():
    nx = 10
    x = 2 * (np.arange(nx) + 0.5) / nx
    k = O.VKin(nx=nx, nvx=12, nvp=6, L=8.0, x0=0.0, x1=2.0, bc=O.BC_PERIODIC, eps=1e-3, E=_test3_E(x))
    p = O.VParareal(kin=k, T=0.04, N=2, cfl_g=0.4)
    V = O.prim_to_cons(np.stack([1 + 0.2 * np.sin(np.pi * x), 0.1 + 0 * x, 0 * x, 0 * x, 1 + 0 * x]))
    n, dt = O.v_fine_nsteps(p)
    f = O.v_fine_run(k, dt, n, O.v_lift(k, O.cons_to_prim(V)))
    assert np.array_equal(O.v_fine_propagate(p, V), O.v_project(k, f, conserved=True))
    G, _ = O.coarse_run_force(nx, O.BC_PERIODIC, 0.4, 0.02, V, k.E, x0=0.0, x1=2.0)
    assert np.array_equal(O.v_coarse_propagate(p, V), G)


def test_stable_step_is_the_positivity_limit():
    # R19: at cfl = 1 the worst cell (v_x = -max|v_x| where E = +E_max, so it
    # empties through its left x face and its upper v_x face at once) keeps
    # exactly nothing of itself, at cfl = 1/2 half; random positive data stay
    # positive at cfl = 1
    nx, nvx, nvp, L = 6, 12, 3, 6.0
    x = (np.arange(nx) + 0.5) / nx
    E = np.array([0.2, 1.7, -0.9, 0.0, 1.1, -1.7 + 1e-3])
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, bc=O.BC_OUTFLOW, eps=math.inf, E=E)
    f = np.zeros((nx, nvx * nvp * nvp))
    f[1, 0] = 1.0  # jx = 0, jy = jz = 0 in column 1 (E = E_max > 0)
    for cfl, keep in ((1.0, 0.0), (0.5, 0.5)):
        g = O.v_fine_step(k, O.v_fine_dt_stab(k, cfl), f)
        assert abs(g[1, 0] - keep) <= 1e-14
    rng = np.random.default_rng(3)
    h = rng.uniform(0.0, 1.0, size=f.shape)
    assert np.min(O.v_fine_step(k, O.v_fine_dt_stab(k, 1.0), h)) >= -1e-14


def test_force_effect_matches_the_euler_limit():
    # Sec. 1: as eps -> 0 the moments follow Eq. (5) with its force terms.  The
    # change the force makes to the kinetic moments (eps = 1e-6) must match the
    # change it makes to the Euler solution; a flipped or missing force term on
    # either side would be off by 100 % or more.
    nx, nvx, nvp, T = 64, 48, 12, 0.1
    x = (np.arange(nx) + 0.5) / nx
    E = np.sin(2 * np.pi * x)
    U = np.stack([1 + 0.2 * np.sin(2 * np.pi * x), 0 * x, 0 * x, 0 * x, 1 + 0 * x])
    O.set_threads(8)
    try:
        res = []
        for EE in (E, None):
            k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=8.0, eps=1e-6, scheme=O.MUSCL, E=EE)
            n = math.ceil(T / O.v_fine_dt_stab(k, 0.5))
            res.append(O.v_project(k, O.v_fine_run(k, T / n, n, O.v_lift(k, U)), conserved=True))
    finally:
        O.set_threads(1)
    V = O.prim_to_cons(U)
    de = O.coarse_run_force(nx, O.BC_PERIODIC, 0.5, T, V, E)[0] - O.coarse_run(nx, O.BC_PERIODIC, 0.5, T, V)[0]
    dk = res[0] - res[1]
    rel = [np.max(np.abs(dk[q] - de[q])) / np.max(np.abs(de[q])) for q in (0, 1)]
    assert rel[0] < 0.15 and rel[1] < 0.03, rel


# ------------------------------------------------------------------ parareal with the force


def _beams(nx, L, nvx, nvp, x0=0.0, x1=2.0):
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=x0, x1=x1)
    one = np.ones(nx)
    z = np.zeros(nx)
    return O.v_lift(k, np.stack([one, one, z, z, one])) + O.v_lift(k, np.stack([one, -one, z, z, one]))


def test_parareal_with_force_reaches_the_serial_fine_chain_at_k_equals_n():
    nx, N = 16, 4
    x = 2 * (np.arange(nx) + 0.5) / nx
    k = O.VKin(nx=nx, nvx=16, nvp=6, L=8.0, x0=0.0, x1=2.0, eps=1e-3, scheme=O.UPWIND, E=_test3_E(x))
    p = O.VParareal(kin=k, T=0.05, N=N)
    U0 = O.v_project(k, _beams(nx, 8.0, 16, 6))
    chain = [O.prim_to_cons(U0)]
    for _ in range(N):
        chain.append(O.v_fine_propagate(p, chain[-1]))
    chain = np.stack(chain)
    Uall, errs, kd = O.v_parareal(p, U0, K=N)
    scale = np.max(np.abs(chain), axis=(0, 2), keepdims=True)
    assert np.max(np.abs(Uall[N] - chain) / scale) < 1e-13
    assert errs[0] > 1e-6 and errs[-1] < errs[0]
    # iteration 0 is the coarse chain with the source
    c = [chain[0]]
    for _ in range(N):
        c.append(O.v_coarse_propagate(p, c[-1]))
    assert np.array_equal(Uall[0], np.stack(c))


def test_test3_force_concentrates_mass_towards_the_centre():
    # Sec. 5.3 (Test 3): the force E(x) = -5 x^4 (x-2)^4 (x-1) pushes the gas
    # towards x = 1 (printed statement in tests/golden/paper_statements.json).
    st = json.load(open(os.path.join(HERE, "golden", "paper_statements.json")))["test3_exterior_force"]
    # (v_y, v_z as in the paper, 16 cells on [-8, 8]; v_x and x coarsened)
    nx, nvx, nvp, L = 40, 64, 16, 8.0
    x = 2 * (np.arange(nx) + 0.5) / nx
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, eps=st["eps"], scheme=O.UPWIND, E=_test3_E(x))
    f0 = _beams(nx, L, nvx, nvp)
    T = 0.1
    n = math.ceil(T / O.v_fine_dt_stab(k, 0.5))
    O.set_threads(8)
    try:
        U = O.v_project(k, O.v_fine_run(k, T / n, n, f0))
    finally:
        O.set_threads(1)
    rho0 = O.v_project(k, f0)[0]
    centre = np.abs(x - 1.0) < 0.2
    edges = np.abs(x - 1.0) > 0.8
    assert np.all(U[0][centre] > rho0[centre]) and np.all(U[0][edges] < rho0[edges] + 1e-12)
    # the flow points towards x = 1 on both sides
    assert np.all(U[1][(x > 0.2) & (x < 0.9)] > 0) and np.all(U[1][(x > 1.1) & (x < 1.8)] < 0)


# ------------------------------------------------- moments of f* from column sums
def _column_sums(f, nvx, nvp, L):
    """Per column: the five moments M, the upwind half sums A+ (v_x > 0) and
    A- (v_x <= 0) of v_x f times each moment weight, and the densities of the
    first and last v_x rows (plain numpy)."""
    vx, _ = _nodes(nvx, L)
    vp, _ = _nodes(nvp, L)
    F = f.reshape(f.shape[0], nvx, nvp, nvp)
    VX, VY, VZ = np.meshgrid(vx, vp, vp, indexing="ij")
    phis = (np.ones_like(VX), VX, VY, VZ, VX ** 2 + VY ** 2 + VZ ** 2)
    pos = VX > 0
    M = np.stack([(F * p).sum(axis=(1, 2, 3)) for p in phis], axis=1)
    Ap = np.stack([(F * np.where(pos, VX * p, 0)).sum(axis=(1, 2, 3)) for p in phis], axis=1)
    An = np.stack([(F * np.where(pos, 0, VX * p)).sum(axis=(1, 2, 3)) for p in phis], axis=1)
    return M, Ap, An, F[:, 0].sum(axis=(1, 2)), F[:, -1].sum(axis=(1, 2))


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_OUTFLOW, O.BC_REFLECT])
@pytest.mark.parametrize("nvx", [8, 9])
def test_transport_moments_follow_from_column_sums(bc, nvx):
    # With upwind x fluxes the sums of phi f* over a column are M - nu (A+_c -
    # A+_{c-1} + A-_{c+1} - A-_c) - nuv Q, where the v_x Rusanov fluxes
    # telescope (summation by parts, zero flux through +-L): Q vanishes for
    # phi = 1, v_y, v_z and needs only the column density, sum v_x f and the
    # end-row densities for phi = v_x, |v|^2.  A reflecting wall's ghost
    # swaps A+ and A- with the sign of the even weights.
    nx, nvp, L = 7, 4, 5.0
    E = np.linspace(-0.6, 0.9, nx)
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, bc=bc, eps=math.inf, E=E)
    f = np.random.default_rng(3).random((nx, k.ncol)) + 0.1
    dt = O.v_fine_dt_stab(k, 0.5)
    want = _column_sums(O.v_fine_run(k, dt, 1, f), nvx, nvp, L)[0]
    M, Ap, An, r0, rn = _column_sums(f, nvx, nvp, L)
    dvx, nu = 2 * L / nvx, dt / (2.0 / nx)
    nuv, Em = dt / dvx, np.max(np.abs(E))
    s = np.array([-1.0, 1.0, -1.0, -1.0, -1.0])
    if bc == O.BC_PERIODIC:
        Apg, Ang = Ap[nx - 1], An[0]
    elif bc == O.BC_OUTFLOW:
        Apg, Ang = Ap[0], An[nx - 1]
    else:
        Apg, Ang = s * An[0], s * Ap[nx - 1]
    Ap_m = np.vstack([Apg, Ap[:-1]])   # A+ of column c-1
    An_p = np.vstack([An[1:], Ang])    # A- of column c+1
    Q = np.zeros((nx, 5))
    Q[:, 1] = -dvx * (E * (M[:, 0] - 0.5 * (r0 + rn)) - Em * 0.5 * (rn - r0))
    Q[:, 4] = -dvx * (E * (2 * M[:, 1] - L * (rn - r0)) - Em * (L * (r0 + rn) - dvx * M[:, 0]))
    got = M - nu * (Ap - Ap_m + An_p - An) - nuv * Q
    assert np.max(np.abs(got - want)) < 1e-13 * np.max(np.abs(want))


def _ghost_x(f, c, bc, nvx, nvp):
    """Column c of f [nx, ncol] through the boundary rule (a reflecting wall
    mirrors the column and reverses v_x)."""
    nx = f.shape[0]
    if 0 <= c < nx:
        return f[c]
    if bc == O.BC_PERIODIC:
        return f[c % nx]
    if bc == O.BC_OUTFLOW:
        return f[0 if c < 0 else nx - 1]
    m = -1 - c if c < 0 else 2 * nx - 1 - c
    return f[m].reshape(nvx, nvp * nvp)[::-1].reshape(-1)


def _minmod(a, b):
    return np.where(a * b <= 0, 0.0, np.where(np.abs(a) < np.abs(b), a, b))


@pytest.mark.parametrize("bc", [O.BC_PERIODIC, O.BC_OUTFLOW, O.BC_REFLECT])
@pytest.mark.parametrize("nvx", [8, 9])
def test_muscl_transport_moments_follow_from_limited_column_sums(bc, nvx):
    # With MUSCL-minmod x fluxes the interface value on the upwind side of
    # face c+1/2 is f_c + s_c/2 (v_x > 0) or f_{c+1} - s_{c+1}/2 (v_x <= 0),
    # s_c = minmod(f_c - f_{c-1}, f_{c+1} - f_c), so the upwind identity holds
    # with A+ and A- taken of f + s/2 and f - s/2: each column's limited sums
    # need only that column and its two neighbours.  Ghosts: an outflow edge
    # column has s = 0 (its ghost repeats it), so the ghost's sums are the
    # edge column's; a reflecting ghost has s_ghost(v) = -s_edge(-v) (minmod
    # is odd), so it swaps A+ and A- with the sign of the even weights as
    # the upwind sums do.
    nx, nvp, L = 7, 4, 5.0
    E = np.linspace(-0.6, 0.9, nx)
    k = O.VKin(nx=nx, nvx=nvx, nvp=nvp, L=L, x0=0.0, x1=2.0, bc=bc, eps=math.inf, scheme=O.MUSCL, E=E)
    f = np.random.default_rng(5).random((nx, k.ncol)) + 0.1
    dt = O.v_fine_dt_stab(k, 0.5)
    want = _column_sums(O.v_fine_run(k, dt, 1, f), nvx, nvp, L)[0]
    ext = np.stack([_ghost_x(f, c, bc, nvx, nvp) for c in range(-1, nx + 1)])  # columns -1 .. nx
    s = _minmod(ext[1:-1] - ext[:-2], ext[2:] - ext[1:-1])                     # slopes of columns 0 .. nx-1
    M, _, _, r0, rn = _column_sums(f, nvx, nvp, L)
    _, Ap, _, _, _ = _column_sums(f + 0.5 * s, nvx, nvp, L)
    _, _, An, _, _ = _column_sums(f - 0.5 * s, nvx, nvp, L)
    dvx, nu = 2 * L / nvx, dt / (2.0 / nx)
    nuv, Em = dt / dvx, np.max(np.abs(E))
    if bc == O.BC_OUTFLOW:  # the edge columns' slopes vanish
        assert np.all(s[0] == 0) and np.all(s[nx - 1] == 0)
    Q = np.zeros((nx, 5))
    Q[:, 1] = -dvx * (E * (M[:, 0] - 0.5 * (r0 + rn)) - Em * 0.5 * (rn - r0))
    Q[:, 4] = -dvx * (E * (2 * M[:, 1] - L * (rn - r0)) - Em * (L * (r0 + rn) - dvx * M[:, 0]))

    def predict(Ap, An):
        sg = np.array([-1.0, 1.0, -1.0, -1.0, -1.0])
        if bc == O.BC_PERIODIC:
            Apg, Ang = Ap[nx - 1], An[0]
        elif bc == O.BC_OUTFLOW:
            Apg, Ang = Ap[0], An[nx - 1]
        else:
            Apg, Ang = sg * An[0], sg * Ap[nx - 1]
        return M - nu * (Ap - np.vstack([Apg, Ap[:-1]]) + np.vstack([An[1:], Ang]) - An) - nuv * Q

    assert np.max(np.abs(predict(Ap, An) - want)) < 1e-13 * np.max(np.abs(want))
    # the limiter matters here: the unlimited (upwind) sums give another answer
    _, Ap0, An0, _, _ = _column_sums(f, nvx, nvp, L)
    assert np.max(np.abs(predict(Ap0, An0) - want)) > 1e-6 * np.max(np.abs(want))
