"""Plain CPU FP64 oracle for the kinetic-fluid parareal method (Laidin & Rey).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package.  The
product path (``paper_2502_02704_gb300``) never imports it; the two share no
code.  The arithmetic lives in ``pr_oracle.c`` (plain C, double precision,
naive loops); this module compiles it with gcc and marshals numpy arrays.

Shapes: primitive ``U`` and conserved ``V`` are ``[5, nx]`` float64;
``f`` is ``[nx, nv**3]`` float64 with velocity index ``(jx*nv + jy)*nv + jz``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pr_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "pr_oracle_force.c")]
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

BC_PERIODIC, BC_OUTFLOW, BC_REFLECT = 0, 1, 2
UPWIND, MUSCL = 0, 1
SOUND_GAMMA53, SOUND_SQRT_THETA = 0, 1
COARSE_EULER, COARSE_CNS = 0, 1


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile ``pr_oracle.c`` and ``pr_oracle_force.c`` into ``_build/liboracle.so``
    (gcc, -O2, OpenMP).

    ``-ffp-contract=off`` keeps gcc from fusing multiply-adds, so the oracle
    gives the same bits on x86-64 and aarch64.
    """
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        [os.path.getmtime(x) for x in _SRCS] + [os.path.getmtime(os.path.join(_HERE, "pr_oracle.h"))]
    ):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", *_SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Kin(C.Structure):
    _fields_ = [("nx", C.c_int), ("x0", C.c_double), ("x1", C.c_double), ("bc", C.c_int),
                ("nv", C.c_int), ("L", C.c_double), ("eps", C.c_double), ("scheme", C.c_int)]


class _Pr(C.Structure):
    _fields_ = [("kin", _Kin), ("T", C.c_double), ("N", C.c_int), ("cfl_f", C.c_double),
                ("cfl_g", C.c_double), ("sound", C.c_int), ("nf", C.c_int), ("coarse", C.c_int), ("lift", C.c_int)]


_D = C.POINTER(C.c_double)


class _VKin(C.Structure):
    _fields_ = [("nx", C.c_int), ("x0", C.c_double), ("x1", C.c_double), ("bc", C.c_int),
                ("nvx", C.c_int), ("nvp", C.c_int), ("L", C.c_double), ("eps", C.c_double),
                ("scheme", C.c_int), ("E", _D)]


class _VPr(C.Structure):
    _fields_ = [("kin", _VKin), ("T", C.c_double), ("N", C.c_int), ("cfl_f", C.c_double),
                ("cfl_g", C.c_double), ("sound", C.c_int), ("nf", C.c_int), ("coarse", C.c_int), ("lift", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            pk, pp = C.POINTER(_Kin), C.POINTER(_Pr)
            pvk, pvp = C.POINTER(_VKin), C.POINTER(_VPr)
            sig = {
                "or_set_threads": (None, [C.c_int]),
                "or_get_threads": (C.c_int, []),
                "or_velocity_nodes": (None, [C.c_int, C.c_double, _D]),
                "or_prim_to_cons": (None, [C.c_int, _D, _D]),
                "or_cons_to_prim": (C.c_int, [C.c_int, _D, _D]),
                "or_lift": (C.c_int, [pk, _D, _D]),
                "or_project": (C.c_int, [pk, _D, _D]),
                "or_project_cons": (C.c_int, [pk, _D, _D]),
                "or_fine_dt_stab": (C.c_double, [pk, C.c_double]),
                "or_fine_nsteps": (C.c_int, [pp, _D]),
                "or_fine_step": (C.c_int, [pk, C.c_double, _D, _D]),
                "or_fine_run": (C.c_int, [pk, C.c_double, C.c_int, _D]),
                "or_coarse_run": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, C.c_double,
                                            C.c_int, C.c_double, _D, _D, C.POINTER(C.c_int)]),
                "or_fine_propagate": (C.c_int, [pp, _D, _D]),
                "or_coarse_propagate": (C.c_int, [pp, _D, _D]),
                "or_parareal": (C.c_int, [pp, _D, C.c_int, C.c_double, C.c_int, _D, _D,
                                          C.POINTER(C.c_int)]),
                "or_adjoint": (C.c_int, [pk, C.c_double, C.c_int, _D, _D, _D, _D]),
                "or_coarse_run_force": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, C.c_double,
                                                  C.c_int, C.c_double, _D, _D, _D, C.POINTER(C.c_int)]),
                "or_v_lift": (C.c_int, [pvk, _D, _D]),
                "or_v_lift_ce": (C.c_int, [pvk, _D, _D]),
                "or_lift_ce": (C.c_int, [pk, _D, _D]),
                "or_coarse_run_cns": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_int, C.c_double, C.c_int,
                                                C.c_double, C.c_double, _D, _D, _D, C.POINTER(C.c_int)]),
                "or_v_project": (C.c_int, [pvk, _D, _D]),
                "or_v_project_cons": (C.c_int, [pvk, _D, _D]),
                "or_v_fine_dt_stab": (C.c_double, [pvk, C.c_double]),
                "or_v_fine_nsteps": (C.c_int, [pvp, _D]),
                "or_v_fine_step": (C.c_int, [pvk, C.c_double, _D, _D]),
                "or_v_fine_run": (C.c_int, [pvk, C.c_double, C.c_int, _D]),
                "or_v_fine_propagate": (C.c_int, [pvp, _D, _D]),
                "or_v_coarse_propagate": (C.c_int, [pvp, _D, _D]),
                "or_v_parareal": (C.c_int, [pvp, _D, C.c_int, C.c_double, C.c_int, _D, _D,
                                            C.POINTER(C.c_int)]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


@dataclass
class Kin:
    """Kinetic problem: x grid, boundary, velocity grid, Knudsen number, scheme."""
    nx: int
    nv: int
    L: float = 8.0
    x0: float = 0.0
    x1: float = 1.0
    bc: int = BC_PERIODIC
    eps: float = 1e-2
    scheme: int = UPWIND

    def c(self) -> _Kin:
        return _Kin(self.nx, self.x0, self.x1, self.bc, self.nv, self.L, self.eps, self.scheme)

    @property
    def dx(self) -> float:
        return (self.x1 - self.x0) / self.nx

    @property
    def nv3(self) -> int:
        return self.nv ** 3


@dataclass
class Parareal:
    """Parareal problem: kinetic setup plus time grid and coarse parameters."""
    kin: Kin
    T: float
    N: int
    cfl_f: float = 0.5
    cfl_g: float = 0.5
    sound: int = SOUND_GAMMA53
    nf: int = 0
    coarse: int = COARSE_EULER
    lift: int = 0

    def c(self) -> _Pr:
        return _Pr(self.kin.c(), self.T, self.N, self.cfl_f, self.cfl_g, self.sound, self.nf, self.coarse, self.lift)


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def velocity_nodes(nv: int, L: float) -> np.ndarray:
    v = np.empty(nv)
    lib().or_velocity_nodes(nv, L, _ptr(v))
    return v


def prim_to_cons(U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    V = np.empty_like(U)
    lib().or_prim_to_cons(U.shape[1], _ptr(U), _ptr(V))
    return V


def cons_to_prim(V: np.ndarray) -> np.ndarray:
    V = np.ascontiguousarray(V, dtype=np.float64)
    U = np.empty_like(V)
    _check(lib().or_cons_to_prim(V.shape[1], _ptr(V), _ptr(U)), "cons_to_prim")
    return U


def lift(k: Kin, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    f = np.empty((k.nx, k.nv3))
    kc = k.c()
    _check(lib().or_lift(C.byref(kc), _ptr(U), _ptr(f)), "lift")
    return f


def lift_ce(k: Kin, U: np.ndarray) -> np.ndarray:
    """First-order (Chapman-Enskog) lifting L^(1) of Def. 3."""
    U = np.ascontiguousarray(U, dtype=np.float64)
    f = np.empty((k.nx, k.nv3))
    kc = k.c()
    _check(lib().or_lift_ce(C.byref(kc), _ptr(U), _ptr(f)), "lift_ce")
    return f


def coarse_run_cns(nx: int, bc: int, cfl: float, dT: float, V: np.ndarray, eps: float, E=None, x0: float = 0.0,
                   x1: float = 1.0, sound: int = SOUND_GAMMA53) -> tuple[np.ndarray, int]:
    """Compressible Navier-Stokes coarse model (Eq. 8) over dT."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty_like(V)
    ns = C.c_int()
    Ep = _ptr(np.ascontiguousarray(E, dtype=np.float64)) if E is not None else C.cast(None, _D)
    Ekeep = E
    _check(lib().or_coarse_run_cns(nx, x0, x1, bc, cfl, sound, dT, eps, Ep, _ptr(V), _ptr(out), C.byref(ns)),
           "coarse_run_cns")
    del Ekeep
    return out, ns.value


def project(k: Kin, f: np.ndarray, conserved: bool = False) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty((5, k.nx))
    kc = k.c()
    fn = lib().or_project_cons if conserved else lib().or_project
    _check(fn(C.byref(kc), _ptr(f), _ptr(out)), "project")
    return out


def fine_dt_stab(k: Kin, cfl: float) -> float:
    kc = k.c()
    return lib().or_fine_dt_stab(C.byref(kc), cfl)


def fine_nsteps(p: Parareal) -> tuple[int, float]:
    pc = p.c()
    dt = C.c_double()
    n = lib().or_fine_nsteps(C.byref(pc), C.byref(dt))
    return n, dt.value


def fine_step(k: Kin, dt: float, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    kc = k.c()
    _check(lib().or_fine_step(C.byref(kc), dt, _ptr(f), _ptr(out)), "fine_step")
    return out


def fine_run(k: Kin, dt: float, nsteps: int, f: np.ndarray) -> np.ndarray:
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    kc = k.c()
    _check(lib().or_fine_run(C.byref(kc), dt, nsteps, _ptr(f)), "fine_run")
    return f


def coarse_run(nx: int, bc: int, cfl: float, dT: float, V: np.ndarray, x0: float = 0.0,
               x1: float = 1.0, sound: int = SOUND_GAMMA53) -> tuple[np.ndarray, int]:
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty_like(V)
    ns = C.c_int()
    _check(lib().or_coarse_run(nx, x0, x1, bc, cfl, sound, dT, _ptr(V), _ptr(out), C.byref(ns)),
           "coarse_run")
    return out, ns.value


def fine_propagate(p: Parareal, V: np.ndarray) -> np.ndarray:
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty_like(V)
    pc = p.c()
    _check(lib().or_fine_propagate(C.byref(pc), _ptr(V), _ptr(out)), "fine_propagate")
    return out


def coarse_propagate(p: Parareal, V: np.ndarray) -> np.ndarray:
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty_like(V)
    pc = p.c()
    _check(lib().or_coarse_propagate(C.byref(pc), _ptr(V), _ptr(out)), "coarse_propagate")
    return out


def parareal(p: Parareal, U0: np.ndarray, K: int, tol: float = 0.0, alg: int = 2):
    """Run Algorithm 1 or 2.  Returns (U[K+1, N+1, 5, nx] conserved, errs[K], k_done)."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    nx = p.kin.nx
    Uall = np.zeros((K + 1, p.N + 1, 5, nx))
    errs = np.zeros(max(K, 1))
    kd = C.c_int()
    pc = p.c()
    _check(lib().or_parareal(C.byref(pc), _ptr(U0), K, tol, alg, _ptr(Uall), _ptr(errs),
                             C.byref(kd)), "parareal")
    return Uall, errs[:K], kd.value


def adjoint(k: Kin, dt: float, nsteps: int, U0: np.ndarray, lamV: np.ndarray):
    """(dJ/dU0 [5, nx] primitive, dJ/dlog eps) for a scalar J of the final
    conserved moments with dJ/dV(T) = lamV [5, nx] (upwind fine run)."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    lamV = np.ascontiguousarray(lamV, dtype=np.float64)
    dU0 = np.empty_like(U0)
    de = C.c_double()
    kc = k.c()
    _check(lib().or_adjoint(C.byref(kc), dt, nsteps, _ptr(U0), _ptr(lamV), _ptr(dU0), C.byref(de)), "adjoint")
    return dU0, de.value


# ---------------------------------------------------------------- exterior force


@dataclass
class VKin:
    """Kinetic problem with an exterior force E (one value per x cell) on an
    anisotropic velocity grid: nvx cells along v_x, nvp along v_y and v_z."""
    nx: int
    nvx: int
    nvp: int
    L: float = 8.0
    x0: float = 0.0
    x1: float = 1.0
    bc: int = BC_PERIODIC
    eps: float = 1e-2
    scheme: int = UPWIND
    E: np.ndarray | None = None

    def __post_init__(self):
        if self.E is not None:
            self.E = np.ascontiguousarray(self.E, dtype=np.float64)
            assert self.E.shape == (self.nx,)

    def c(self) -> _VKin:
        e = _ptr(self.E) if self.E is not None else C.cast(None, _D)
        return _VKin(self.nx, self.x0, self.x1, self.bc, self.nvx, self.nvp, self.L, self.eps, self.scheme, e)

    @property
    def ncol(self) -> int:
        return self.nvx * self.nvp * self.nvp


@dataclass
class VParareal:
    kin: VKin
    T: float
    N: int
    cfl_f: float = 0.5
    cfl_g: float = 0.5
    sound: int = SOUND_GAMMA53
    nf: int = 0
    coarse: int = COARSE_EULER
    lift: int = 0

    def c(self) -> _VPr:
        return _VPr(self.kin.c(), self.T, self.N, self.cfl_f, self.cfl_g, self.sound, self.nf, self.coarse,
                    self.lift)


def v_lift(k: VKin, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    f = np.empty((k.nx, k.ncol))
    kc = k.c()
    _check(lib().or_v_lift(C.byref(kc), _ptr(U), _ptr(f)), "v_lift")
    return f


def v_lift_ce(k: VKin, U: np.ndarray) -> np.ndarray:
    U = np.ascontiguousarray(U, dtype=np.float64)
    f = np.empty((k.nx, k.ncol))
    kc = k.c()
    _check(lib().or_v_lift_ce(C.byref(kc), _ptr(U), _ptr(f)), "v_lift_ce")
    return f


def v_project(k: VKin, f: np.ndarray, conserved: bool = False) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty((5, k.nx))
    kc = k.c()
    fn = lib().or_v_project_cons if conserved else lib().or_v_project
    _check(fn(C.byref(kc), _ptr(f), _ptr(out)), "v_project")
    return out


def v_fine_dt_stab(k: VKin, cfl: float) -> float:
    kc = k.c()
    return lib().or_v_fine_dt_stab(C.byref(kc), cfl)


def v_fine_nsteps(p: VParareal) -> tuple[int, float]:
    pc = p.c()
    dt = C.c_double()
    n = lib().or_v_fine_nsteps(C.byref(pc), C.byref(dt))
    return n, dt.value


def v_fine_step(k: VKin, dt: float, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty_like(f)
    kc = k.c()
    _check(lib().or_v_fine_step(C.byref(kc), dt, _ptr(f), _ptr(out)), "v_fine_step")
    return out


def v_fine_run(k: VKin, dt: float, nsteps: int, f: np.ndarray) -> np.ndarray:
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    kc = k.c()
    _check(lib().or_v_fine_run(C.byref(kc), dt, nsteps, _ptr(f)), "v_fine_run")
    return f


def coarse_run_force(nx: int, bc: int, cfl: float, dT: float, V: np.ndarray, E: np.ndarray, x0: float = 0.0,
                     x1: float = 1.0, sound: int = SOUND_GAMMA53) -> tuple[np.ndarray, int]:
    V = np.ascontiguousarray(V, dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    assert E.shape == (nx,)
    out = np.empty_like(V)
    ns = C.c_int()
    _check(lib().or_coarse_run_force(nx, x0, x1, bc, cfl, sound, dT, _ptr(E), _ptr(V), _ptr(out), C.byref(ns)),
           "coarse_run_force")
    return out, ns.value


def v_fine_propagate(p: VParareal, V: np.ndarray) -> np.ndarray:
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty_like(V)
    pc = p.c()
    _check(lib().or_v_fine_propagate(C.byref(pc), _ptr(V), _ptr(out)), "v_fine_propagate")
    return out


def v_coarse_propagate(p: VParareal, V: np.ndarray) -> np.ndarray:
    V = np.ascontiguousarray(V, dtype=np.float64)
    out = np.empty_like(V)
    pc = p.c()
    _check(lib().or_v_coarse_propagate(C.byref(pc), _ptr(V), _ptr(out)), "v_coarse_propagate")
    return out


def v_parareal(p: VParareal, U0: np.ndarray, K: int, tol: float = 0.0, alg: int = 2):
    """Algorithm 1 or 2 with the force propagators; same returns as ``parareal``."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    nx = p.kin.nx
    Uall = np.zeros((K + 1, p.N + 1, 5, nx))
    errs = np.zeros(max(K, 1))
    kd = C.c_int()
    pc = p.c()
    _check(lib().or_v_parareal(C.byref(pc), _ptr(U0), K, tol, alg, _ptr(Uall), _ptr(errs), C.byref(kd)),
           "v_parareal")
    return Uall, errs[:K], kd.value


INF = math.inf
