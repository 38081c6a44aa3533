"""Seeded synthetic inputs for the kinetic-fluid parareal workloads.

This module only draws and tabulates initial macroscopic profiles
(rho, u, theta) -- primitive variables, shape [5, nx] -- and instance
parameters.  It holds none of the method's arithmetic (no lifting, moments,
transport or coarse solver), so the CUDA path and the CPU oracle can both be
fed from it.  The profiles are the paper's test cases (Sec. 5) and their
variants used for measurement:

* ``sod``: Test 1 Riemann data, (1, 0, 1) left / (0.125, 0, 0.8) right.
* ``blast``: Test 2 three-state data (1, 1, 2) / (1, 0, 0.25) / (1, -1, 2).
* ``smooth_periodic``: rho = 1 + 0.5 sin 2 pi x, u_x = 0.2 sin 2 pi x,
  theta = 1 + 0.2 cos 2 pi x on [0, 1).
* ``thirds``: two interacting shocks, rho = 1 / 0.2 / 1, theta = 2 / 0.5 / 2.
* ``density_modes``: rho = 1 + a1 sin 2 pi x + a2 cos 4 pi x, u = 0, theta = 1.
* ``ragged_instances``: Sod-type instances of uneven size and Knudsen number.
* ``test3_force`` / ``test3_beams``: Test 3, the force E(x) = -5 x^4 (x-2)^4 (x-1)
  sampled at the cell centres of [0, 2] and the two beams (1, +-1, 0, 0, 1)
  whose Maxwellians sum to the initial distribution.
"""
from __future__ import annotations

import numpy as np


def cell_centres(nx: int, x0: float = 0.0, x1: float = 1.0) -> np.ndarray:
    return x0 + (np.arange(nx) + 0.5) * (x1 - x0) / nx


def _stack(rho, ux, th, uy=None, uz=None) -> np.ndarray:
    z = np.zeros_like(rho)
    return np.stack([rho, ux, z if uy is None else uy, z if uz is None else uz, th]).astype(np.float64)


def sod(nx: int, x0: float = 0.0, x1: float = 1.0, split: float | None = None,
        left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.8)) -> np.ndarray:
    x = cell_centres(nx, x0, x1)
    split = 0.5 * (x0 + x1) if split is None else split
    L = x < split
    rho = np.where(L, left[0], right[0])
    ux = np.where(L, left[1], right[1])
    th = np.where(L, left[2], right[2])
    return _stack(rho, ux, th)


def blast(nx: int, x0: float = 0.0, x1: float = 2.0) -> np.ndarray:
    x = cell_centres(nx, x0, x1)
    a, b = x0 + 0.2 * (x1 - x0), x0 + 0.8 * (x1 - x0)
    rho = np.ones(nx)
    ux = np.where(x < a, 1.0, np.where(x < b, 0.0, -1.0))
    th = np.where(x < a, 2.0, np.where(x < b, 0.25, 2.0))
    return _stack(rho, ux, th)


def smooth_periodic(nx: int) -> np.ndarray:
    x = cell_centres(nx)
    return _stack(1 + 0.5 * np.sin(2 * np.pi * x), 0.2 * np.sin(2 * np.pi * x), 1 + 0.2 * np.cos(2 * np.pi * x))


def thirds(nx: int) -> np.ndarray:
    x = cell_centres(nx)
    mid = (x >= 1 / 3) & (x < 2 / 3)
    return _stack(np.where(mid, 0.2, 1.0), np.zeros(nx), np.where(mid, 0.5, 2.0))


def density_modes(nx: int, a1: float, a2: float) -> np.ndarray:
    x = cell_centres(nx)
    return _stack(1 + a1 * np.sin(2 * np.pi * x) + a2 * np.cos(4 * np.pi * x), np.zeros(nx), np.ones(nx))


def draw_modes(seed: int) -> tuple[float, float]:
    """(a1, a2) uniform in [0, 0.3], as in the density-misfit workload."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 0.3, 2)
    return float(a[0]), float(a[1])


def ragged_instances(count: int = 32, seed: int = 2502027040, nx_range=(128, 1024), nvs=(16, 24, 32),
                     log_eps=(-5.0, 0.0)) -> list[dict]:
    """Independent Sod-type instances: instance i uses seed + i.

    nx ~ U{nx_range}, nv from ``nvs``, log10 eps ~ U[log_eps], left/right
    rho ~ U[0.1, 1], theta ~ U[0.5, 1.5], u = 0, velocity box [-8, 8]^3.
    """
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        nv = int(nvs[int(rng.integers(0, len(nvs)))])
        eps = float(10.0 ** rng.uniform(*log_eps))
        rl, rr = rng.uniform(0.1, 1.0, 2)
        tl, tr = rng.uniform(0.5, 1.5, 2)
        out.append({"nx": nx, "nv": nv, "eps": eps, "L": 8.0,
                    "U": sod(nx, left=(float(rl), 0.0, float(tl)), right=(float(rr), 0.0, float(tr)))})
    return out


def random_positive_f(nx: int, nv: int, seed: int, lo: float = 0.05, hi: float = 1.0) -> np.ndarray:
    """Arbitrary positive distribution [nx, nv^3] (not a Maxwellian)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, (nx, nv ** 3))


def test3_force(nx: int, x0: float = 0.0, x1: float = 2.0) -> np.ndarray:
    """Test 3's exterior force E(x) = -5 x^4 (x-2)^4 (x-1) at the cell centres."""
    x = cell_centres(nx, x0, x1)
    return -5.0 * x ** 4 * (x - 2.0) ** 4 * (x - 1.0)


def test3_beams(nx: int) -> tuple[np.ndarray, np.ndarray]:
    """The two beams of Test 3 as primitive states: (1, 1, 0, 0, 1) and (1, -1, 0, 0, 1)."""
    one, z = np.ones(nx), np.zeros(nx)
    return np.stack([one, one, z, z, one]), np.stack([one, -one, z, z, one])
