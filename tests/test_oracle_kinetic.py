"""Pins of the CPU oracle's kinetic parts against facts fixed outside the oracle:
library routines, closed forms, hand-derived values and invariants.

Each test names the passage of the paper whose statement it checks.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.stats import multivariate_normal

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_velocity_nodes_are_cube_centres():
    # Sec. 3: uniform velocity cubes on [-L, L]^3; nodes at the cube centres.
    v = O.velocity_nodes(16, 8.0)
    assert np.allclose(np.diff(v), 1.0, rtol=0, atol=1e-15)
    assert v[0] == -7.5 and v[-1] == 7.5
    assert np.allclose(v + v[::-1], 0.0, atol=0)


def test_lift_matches_library_gaussian_density():
    # Eq. (17): the discrete lifting is the Maxwellian of Eq. (4) at the nodes,
    # i.e. rho times the N(u, theta I) density (scipy's routine).
    k = O.Kin(nx=3, nv=6, L=3.0)
    rng = np.random.default_rng(7)
    U = np.stack([rng.uniform(0.5, 2, 3), rng.uniform(-0.5, 0.5, 3), rng.uniform(-0.5, 0.5, 3),
                  rng.uniform(-0.5, 0.5, 3), rng.uniform(0.4, 2, 3)])
    f = O.lift(k, U)
    v = O.velocity_nodes(6, 3.0)
    grid = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1).reshape(-1, 3)
    for i in range(3):
        ref = U[0, i] * multivariate_normal(mean=U[1:4, i], cov=U[4, i] * np.eye(3)).pdf(grid)
        assert np.allclose(f[i], ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("nv,L,theta,u", [(16, 8.0, 0.8, 0.0), (16, 8.0, 1.0, 0.3), (12, 6.0, 0.6, -0.2)])
def test_projected_density_equals_poisson_summation_defect(nv, L, theta, u):
    # Eq. (18) applied to Eq. (17): the midpoint sum of a Gaussian over the
    # half-integer lattice is, by Poisson summation,
    #   h sum_j g((j+1/2)h) = 1 + 2 sum_m (-1)^m exp(-2 pi^2 theta m^2/h^2) cos(2 pi m u/h)
    # per direction (truncation at |v| = L is below 1e-13 here).
    k = O.Kin(nx=1, nv=nv, L=L)
    U = np.array([[1.3], [u], [0.0], [0.0], [theta]])
    rho = O.project(k, O.lift(k, U))[0, 0]
    h = 2 * L / nv

    def factor(ud):
        return 1 + 2 * sum((-1) ** m * math.exp(-2 * math.pi ** 2 * theta * m * m / h ** 2)
                           * math.cos(2 * math.pi * m * ud / h) for m in range(1, 6))

    expect = 1.3 * factor(u) * factor(0.0) ** 2
    assert abs(rho - expect) < 2e-14
    assert abs(rho - 1.3) > 1e-9  # the defect is real on these grids


def test_lift_project_roundtrip_resolved_grid():
    # Def. 1 o Def. 2 is the identity on moments; on a resolved and wide
    # enough grid the quadrature defect (Poisson summation, h = 1/2) and the
    # truncation at |v| = L = 10 are both below 1e-12.
    k = O.Kin(nx=4, nv=40, L=10.0)
    rng = np.random.default_rng(3)
    U = np.stack([rng.uniform(0.2, 2, 4), rng.uniform(-0.5, 0.5, 4), rng.uniform(-0.5, 0.5, 4),
                  rng.uniform(-0.5, 0.5, 4), rng.uniform(0.7, 1.5, 4)])
    Up = O.project(k, O.lift(k, U))
    assert np.allclose(Up, U, rtol=0, atol=1e-12)


def test_projection_sums_are_exact_to_rounding():
    # Eq. (18) defines the moments as exact sums over the nv^3 velocity cells.
    # math.fsum gives the correctly rounded sum of the same terms, so the
    # oracle's projection (which is then converted to conserved variables)
    # must agree with the exact sums to a few ulps, at a grid with as many
    # cells as the batched parareal workload (24^3) and at 32^3.
    for nv, nx in ((24, 3), (32, 2)):
        k = O.Kin(nx=nx, nv=nv, L=8.0)
        rng = np.random.default_rng(nv)
        f = rng.uniform(0.1, 1.0, (nx, nv ** 3)) * O.lift(k, np.tile([[1.0], [0.3], [0.0], [-0.2], [0.9]], (1, nx)))
        V = O.project(k, f, conserved=True)
        v = O.velocity_nodes(nv, 8.0)
        dv3 = (16.0 / nv) ** 3
        vx, vy, vz = (g.ravel() for g in np.meshgrid(v, v, v, indexing="ij"))
        for i in range(nx):
            fc = f[i]
            ex = [math.fsum(fc * dv3), math.fsum(vx * fc * dv3), math.fsum(vy * fc * dv3),
                  math.fsum(vz * fc * dv3), 0.5 * math.fsum((vx * vx + vy * vy + vz * vz) * fc * dv3)]
            scale = [ex[0], ex[0], ex[0], ex[0], ex[4]]
            for q in range(5):
                assert abs(V[q, i] - ex[q]) <= 4e-16 * scale[q], (nv, i, q, V[q, i], ex[q])


def _beams(k, rng):
    """x-uniform, far-from-equilibrium f0: two drifting Maxwellians (as in Test 3)."""
    nx = k.nx
    U1 = np.tile(np.array([[0.7], [1.0], [0.2], [0.0], [0.6]]), (1, nx))
    U2 = np.tile(np.array([[0.5], [-1.0], [0.0], [-0.3], [0.8]]), (1, nx))
    return O.lift(k, U1) + O.lift(k, U2)


def test_homogeneous_bgk_closed_form():
    # Spatially homogeneous data: the transport of Eq. (12) vanishes and the
    # implicit BGK step (eps f* + dt M)/(eps + dt) with tau = 1 keeps the
    # moments, so f^n - M = (eps/(eps+dt))^n (f^0 - M) exactly (the grid below
    # resolves M to 1e-15, so the discrete moments of M equal those of f).
    k = O.Kin(nx=2, nv=40, L=10.0, bc=O.BC_PERIODIC, eps=1e-2)
    f0 = _beams(k, np.random.default_rng(0))
    dt, n = 1e-3, 7
    f = O.fine_run(k, dt, n, f0)
    v = O.velocity_nodes(40, 10.0)
    grid = np.stack(np.meshgrid(v, v, v, indexing="ij"), -1).reshape(-1, 3)
    dv3 = (20.0 / 40) ** 3
    rho = f0[0].sum() * dv3
    u = (grid * f0[0][:, None]).sum(0) * dv3 / rho
    th = (((grid - u) ** 2).sum(1) * f0[0]).sum() * dv3 / (3 * rho)
    M = rho * multivariate_normal(mean=u, cov=th * np.eye(3)).pdf(grid)
    a = k.eps / (k.eps + dt)
    expect = M + a ** n * (f0[0] - M)
    assert np.max(np.abs(f[0] - expect)) < 1e-13 * np.max(f0)
    assert np.max(np.abs(f[1] - f[0])) == 0.0


def test_homogeneous_bgk_entropy_decreases():
    # Eq. (3): BGK dissipates the Boltzmann entropy sum f log f.
    k = O.Kin(nx=1, nv=24, L=8.0, eps=1e-2)
    f = _beams(k, None)
    H = []
    for _ in range(6):
        pos = f[0] > 1e-300
        H.append(np.sum(f[0][pos] * np.log(f[0][pos])))
        f = O.fine_run(k, 2e-3, 1, f)
    assert all(b < a for a, b in zip(H, H[1:]))


@pytest.mark.parametrize("scheme", [O.UPWIND, O.MUSCL])
def test_global_maxwellian_is_invariant(scheme):
    # Eq. (4): Maxwellians are BGK equilibria, and a global (x-uniform)
    # Maxwellian is not moved by the transport.  On a resolved, wide grid
    # (h = 2/3, L = 10) M[P(M)] = M to rounding, so f stays put.
    k = O.Kin(nx=5, nv=30, L=10.0, bc=O.BC_PERIODIC, eps=1e-3, scheme=scheme)
    U = np.tile(np.array([[0.9], [0.3], [-0.1], [0.2], [1.1]]), (1, 5))
    f0 = O.lift(k, U)
    f = O.fine_run(k, 5e-4, 10, f0)
    assert np.max(np.abs(f - f0)) < 1e-13 * np.max(f0)


def test_upwind_transport_matches_dft_closed_form():
    # Collisionless, periodic upwind transport (Eq. 12-13, sign reading of the
    # upwind flux) is circulant: each Fourier mode of each velocity is
    # multiplied per step by 1 - nu (1 - e^{-i k dx}) for v_x > 0 and by
    # 1 - nu (e^{i k dx} - 1) for v_x < 0, with nu = v_x dt/dx.
    nx, nv, L = 16, 4, 4.0
    k = O.Kin(nx=nx, nv=nv, L=L, bc=O.BC_PERIODIC, eps=math.inf, scheme=O.UPWIND)
    rng = np.random.default_rng(11)
    f0 = rng.uniform(0.1, 1.0, (nx, nv ** 3))
    dt, n = 0.004, 9
    f = O.fine_run(k, dt, n, f0)
    v = O.velocity_nodes(nv, L)
    kk = 2 * np.pi * np.fft.fftfreq(nx)  # k dx
    for j in range(nv ** 3):
        vx = v[j // (nv * nv)]
        nu = vx * dt / k.dx
        g = 1 - nu * (1 - np.exp(-1j * kk)) if vx > 0 else 1 - nu * (np.exp(1j * kk) - 1)
        expect = np.real(np.fft.ifft(np.fft.fft(f0[:, j]) * g ** n))
        assert np.allclose(f[:, j], expect, rtol=0, atol=1e-13)


def _tiny_case(case):
    nx, nv, L = 4, 2, 2.0
    bc = {"periodic": O.BC_PERIODIC, "outflow": O.BC_OUTFLOW, "reflect": O.BC_REFLECT}[case["bc"]]
    sch = O.MUSCL if case["scheme"] == "muscl" else O.UPWIND
    k = O.Kin(nx=nx, nv=nv, L=L, bc=bc, eps=math.inf, scheme=sch)
    f = np.zeros((nx, nv ** 3))
    jpos = (1 * nv + 0) * nv + 0  # v = (+1, -1, -1)
    jneg = (0 * nv + 0) * nv + 0  # v = (-1, -1, -1)
    f[:, jpos] = case["f_pos"]
    f[:, jneg] = case["f_neg"]
    out = O.fine_step(k, 1.0 / 16, f)
    return out, jpos, jneg


def test_transport_hand_derived_cases():
    data = json.load(open(os.path.join(GOLD, "transport_tiny.json")))
    for case in data["cases"]:
        out, jp, jn = _tiny_case(case)
        assert np.allclose(out[:, jp], case["expect_pos"], rtol=0, atol=1e-15), case["name"]
        assert np.allclose(out[:, jn], case["expect_neg"], rtol=0, atol=1e-15), case["name"]
        others = [j for j in range(8) if j not in (jp, jn)]
        assert np.all(out[:, others] == 0.0)


def _smooth_transport_error(nx, scheme):
    # dt = 2 dx^2 makes the forward-Euler time error O(dx^2), so the observed
    # order is the spatial order of the flux.
    k = O.Kin(nx=nx, nv=2, L=2.0, bc=O.BC_PERIODIC, eps=math.inf, scheme=scheme)
    x = (np.arange(nx) + 0.5) / nx
    f0 = np.zeros((nx, 8))
    prof = lambda s: 1.0 + 0.5 * np.sin(2 * np.pi * s)
    f0[:, :] = prof(x)[:, None]
    T = 0.25
    nsteps = nx * nx // 8
    f = O.fine_run(k, T / nsteps, nsteps, f0)
    err = 0.0
    for j, vx in ((7, 1.0), (0, -1.0)):  # (jx, jy, jz) = (1,1,1) and (0,0,0)
        err = max(err, np.mean(np.abs(f[:, j] - prof(x - vx * T))))
    return err


@pytest.mark.parametrize("scheme,order", [(O.UPWIND, 1.0), (O.MUSCL, 2.0)])
def test_transport_convergence_order(scheme, order):
    # Upwind is first order in x (Sec. 3.1); with the minmod-limited slopes
    # (the flux limiter of Sec. 3.1) the flux is second order on smooth data.
    errs = [_smooth_transport_error(nx, scheme) for nx in (32, 64, 128)]
    rates = [math.log2(a / b) for a, b in zip(errs, errs[1:])]
    assert all(r > order - 0.35 for r in rates), (errs, rates)
    assert all(r < order + 0.5 for r in rates), (errs, rates)


def test_muscl_is_tvd_and_conservative():
    # minmod-limited transport with CFL <= 1/2 adds no total variation and, in
    # flux form, keeps the sum of f exactly (periodic).
    nx = 40
    k = O.Kin(nx=nx, nv=2, L=2.0, bc=O.BC_PERIODIC, eps=math.inf, scheme=O.MUSCL)
    f = np.zeros((nx, 8))
    f[10:25, :] = 1.0
    f[25:30, :] = 0.3
    tv0 = np.abs(np.diff(np.r_[f[:, 7], f[0, 7]])).sum()
    for _ in range(30):
        f = O.fine_step(k, 0.5 / nx, f)
        tv = np.abs(np.diff(np.r_[f[:, 7], f[0, 7]])).sum()
        assert tv <= tv0 + 1e-13
        tv0 = tv
        assert f.min() >= -1e-15 and f.max() <= 1.0 + 1e-15
    assert abs(f.sum() - (15 + 5 * 0.3) * 8) < 1e-12


@pytest.mark.parametrize("scheme", [O.UPWIND, O.MUSCL])
def test_periodic_conservation_of_mass_momentum_energy(scheme):
    # Eq. (2): BGK conserves mass, momentum and energy; transport in flux form
    # conserves them in sum over x (periodic).  The discrete BGK step keeps
    # them up to the quadrature defect of M, below 1e-12 on this grid.
    nx, nv, L = 12, 40, 10.0
    k = O.Kin(nx=nx, nv=nv, L=L, bc=O.BC_PERIODIC, eps=1e-2, scheme=scheme)
    x = (np.arange(nx) + 0.5) / nx
    U = np.stack([1 + 0.5 * np.sin(2 * np.pi * x), 0.2 * np.sin(2 * np.pi * x), 0 * x,
                  0.1 * np.cos(2 * np.pi * x), 1 + 0.2 * np.cos(2 * np.pi * x)])
    f0 = O.lift(k, U)
    f = O.fine_run(k, 1.26e-3, 8, f0)
    V0 = O.project(k, f0, conserved=True).sum(1)
    V1 = O.project(k, f, conserved=True).sum(1)
    assert abs(V1[0] - V0[0]) < 1e-13 * abs(V0[0])
    assert np.all(np.abs(V1[1:4] - V0[1:4]) < 1e-12 * V0[0])
    assert abs(V1[4] - V0[4]) < 1e-12 * abs(V0[4])
    # the moments did change locally, so the test is not vacuous
    assert np.max(np.abs(O.project(k, f) - O.project(k, f0))) > 1e-3


@pytest.mark.parametrize("scheme", [O.UPWIND, O.MUSCL])
def test_reflecting_walls_keep_mirror_symmetry_and_mass(scheme):
    # Specular walls: data symmetric under (x -> 1-x, v_x -> -v_x) stays so,
    # and no mass crosses the walls (exactly, in the collisionless case).
    nx, nv = 10, 8
    x = (np.arange(nx) + 0.5) / nx
    U = np.stack([1 + 0.3 * np.cos(2 * np.pi * x) + 0.2 * np.cos(6 * np.pi * x), 0.4 * np.sin(2 * np.pi * x),
                  0 * x, 0 * x, 1 + 0.1 * np.cos(4 * np.pi * x)])
    for eps in (1e-2, math.inf):
        k = O.Kin(nx=nx, nv=nv, L=6.0, bc=O.BC_REFLECT, eps=eps, scheme=scheme)
        f0 = O.lift(k, U)
        f = O.fine_run(k, 2e-3, 12, f0)
        g = f.reshape(nx, nv, nv, nv)
        assert np.allclose(g, g[::-1, ::-1, :, :], rtol=0, atol=1e-15)
        if eps == math.inf:
            assert abs(f.sum() - f0.sum()) < 1e-13 * f0.sum()
            assert np.max(np.abs(f - f0)) > 1e-3


def test_outflow_keeps_uniform_state():
    # Zero-gradient ghosts: an x-uniform state sees no boundary flux, so it
    # stays exactly x-uniform; on a resolved grid it also stays at M.
    k = O.Kin(nx=6, nv=30, L=10.0, bc=O.BC_OUTFLOW, eps=1e-1, scheme=O.MUSCL)
    U = np.tile(np.array([[0.7], [0.5], [0.0], [0.0], [0.9]]), (1, 6))
    f0 = O.lift(k, U)
    f = O.fine_run(k, 1e-3, 5, f0)
    assert np.max(np.abs(f - f0)) < 1e-13 * np.max(f0)
    assert np.max(np.abs(f[1:] - f[:-1])) == 0.0


def test_collisionless_limit_and_stiff_limit_of_bgk():
    # eps = inf leaves f* untouched; eps -> 0 projects f* onto M[P f*]
    # (the implicit step is stable for any eps, Sec. 3.1 AP property).
    k_inf = O.Kin(nx=1, nv=24, L=8.0, eps=math.inf)
    f0 = _beams(k_inf, None)
    assert np.array_equal(O.fine_step(k_inf, 1e-3, f0), f0)
    k0 = O.Kin(nx=1, nv=24, L=8.0, eps=1e-14)
    f1 = O.fine_step(k0, 1e-3, f0)
    M = O.lift(k0, O.project(k0, f0))
    assert np.max(np.abs(f1 - M)) < 1e-10 * np.max(M)
