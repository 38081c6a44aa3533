"""Python binding of libpr, the GB300 kinetic-fluid parareal library
(Laidin & Rey, arXiv 2502.02704).

Argument marshalling only: every function below calls the C entry point of
the same name in ``libpr.so`` (declared in ``include/pr.h``) and raises
:class:`PrError` on a non-zero status.  All numerics run in the library's CUDA
kernels; there is no fallback.  Importing works without a GPU (the library is
loaded lazily); the first call needs the built ``libpr.so`` and a CUDA device.

Host arrays are numpy float64 (C order).  Device arguments (``*_device``) take
torch CUDA tensors (float64, contiguous) or raw integer pointers.  ``stream``
is a ``torch.cuda.Stream``, an integer ``cudaStream_t`` or ``None`` (the
object's own stream).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpr.so")

PR_OK, PR_EINVAL, PR_ENOMEM, PR_ECUDA, PR_ETIMEOUT, PR_ENONPHYS, PR_ENOTCONV = 0, -1, -2, -3, -4, -5, -6
PR_BC_PERIODIC, PR_BC_OUTFLOW, PR_BC_REFLECT = 0, 1, 2
PR_UPWIND, PR_MUSCL = 0, 1
PR_FP64, PR_MIXED = 0, 1
PR_SOUND_GAMMA53, PR_SOUND_SQRT_THETA = 0, 1
PR_PRIMITIVE, PR_CONSERVED = 0, 1
PR_COARSE_EULER, PR_COARSE_CNS = 0, 1
PR_FINE_AUTO, PR_FINE_TILED, PR_FINE_CLUSTER = 0, 1, 2

_CODES = {PR_EINVAL: "PR_EINVAL", PR_ENOMEM: "PR_ENOMEM", PR_ECUDA: "PR_ECUDA", PR_ETIMEOUT: "PR_ETIMEOUT",
          PR_ENONPHYS: "PR_ENONPHYS", PR_ENOTCONV: "PR_ENOTCONV"}


class PrError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_CODES.get(code, code)}: {msg}")
        self.code = code


class pr_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("x0", C.c_double), ("x1", C.c_double), ("bc", C.c_int)]


class pr_velocity(C.Structure):
    _fields_ = [("nv", C.c_int), ("L", C.c_double)]


class pr_time(C.Structure):
    _fields_ = [("T", C.c_double), ("n_slices", C.c_int), ("cfl_f", C.c_double), ("cfl_g", C.c_double),
                ("scheme", C.c_int), ("precision", C.c_int), ("sound_speed", C.c_int), ("max_batch", C.c_int),
                ("nf", C.c_int), ("coarse_model", C.c_int), ("lift_order", C.c_int)]


class pr_instance(C.Structure):
    _fields_ = [("nx", C.c_int), ("x0", C.c_double), ("x1", C.c_double), ("bc", C.c_int), ("nv", C.c_int),
                ("L", C.c_double), ("eps", C.c_double), ("dt", C.c_double), ("scheme", C.c_int)]


_D = C.POINTER(C.c_double)
_VP = C.c_void_p


class pr_force_instance(C.Structure):
    _fields_ = [("nx", C.c_int), ("x0", C.c_double), ("x1", C.c_double), ("bc", C.c_int), ("nvx", C.c_int),
                ("nvp", C.c_int), ("L", C.c_double), ("eps", C.c_double), ("dt", C.c_double), ("E", _D)]


_lock = threading.Lock()
_lib = None

_SIGS = {
    "pr_init": (C.c_int, [C.POINTER(_VP), C.POINTER(pr_grid), C.POINTER(pr_velocity), C.c_double, C.POINTER(pr_time)]),
    "pr_destroy": (C.c_int, [_VP]),
    "pr_last_error": (C.c_char_p, [_VP]),
    "pr_set_initial": (C.c_int, [_VP, _D]),
    "pr_coarse_step": (C.c_int, [_VP, _D, _D, C.c_double]),
    "pr_fine_step": (C.c_int, [_VP, C.c_int, C.c_int, _VP]),
    "pr_fine_moments": (C.c_int, [_VP, C.c_int, C.c_int, _D]),
    "pr_fine_get_f": (C.c_int, [_VP, C.c_int, _D]),
    "pr_parareal_iter": (C.c_int, [_VP, _D]),
    "pr_parareal_run": (C.c_int, [_VP, C.c_int, C.c_double, C.POINTER(C.c_int), _D]),
    "pr_moments": (C.c_int, [_VP, C.c_int, C.c_int, _D]),
    "pr_fine_steps_per_slice": (C.c_int, [_VP, C.POINTER(C.c_int), _D]),
    "pr_iterations": (C.c_int, [_VP, C.POINTER(C.c_int)]),
    "pr_save": (C.c_int, [_VP, C.c_char_p]),
    "pr_batch_vpt": (C.c_int, [_VP, C.POINTER(C.c_int)]),
    "pr_force_autotune": (C.c_int, [_VP, C.c_int]),
    "pr_multi_create": (C.c_int, [C.POINTER(_VP), C.POINTER(_VP), C.c_int, C.POINTER(pr_instance), C.c_int]),
    "pr_multi_destroy": (C.c_int, [_VP]),
    "pr_multi_last_error": (C.c_char_p, [_VP]),
    "pr_multi_batch": (C.c_int, [_VP, C.POINTER(_VP), C.POINTER(C.c_int)]),
    "pr_multi_iterate": (C.c_int, [_VP, C.c_int, _D]),
    "pr_load": (C.c_int, [_VP, C.c_char_p]),
    "pr_batch_create": (C.c_int, [C.POINTER(_VP), C.POINTER(pr_instance), C.c_int, C.c_int]),
    "pr_batch_destroy": (C.c_int, [_VP]),
    "pr_batch_last_error": (C.c_char_p, [_VP]),
    "pr_batch_set_initial": (C.c_int, [_VP, C.c_int, _D, C.c_int]),
    "pr_batch_set_initial_device": (C.c_int, [_VP, C.c_int, _VP, C.c_int, _VP]),
    "pr_batch_set_f": (C.c_int, [_VP, C.c_int, _D]),
    "pr_batch_run": (C.c_int, [_VP, C.c_int, _VP]),
    "pr_batch_moments": (C.c_int, [_VP, C.c_int, C.c_int, _D]),
    "pr_batch_moments_device": (C.c_int, [_VP, C.c_int, _VP, _VP]),
    "pr_batch_get_f": (C.c_int, [_VP, C.c_int, _D]),
    "pr_batch_sync": (C.c_int, [_VP]),
    "pr_batch_set_lift_order": (C.c_int, [_VP, C.c_int]),
    "pr_force_set_lift_order": (C.c_int, [_VP, C.c_int]),
    "pr_batch_inject_wait_timeout": (C.c_int, [_VP, C.c_int, C.c_int]),
    "pr_batch_tile": (C.c_int, [_VP, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pr_batch_autotune": (C.c_int, [_VP]),
    "pr_batch_set_tile": (C.c_int, [_VP, C.c_int]),
    "pr_batch_kernel_time": (C.c_int, [_VP, _D, C.POINTER(C.c_int), C.c_int]),
    "pr_kernel_launches": (C.c_longlong, [C.c_int]),
    "pr_batch_adjoint": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int, _D, _D, _D]),
    "pr_fine_step_noalloc": (C.c_int, [C.POINTER(pr_instance), _VP, _VP, _VP]),
    "pr_fine_dt_stab": (C.c_int, [C.POINTER(pr_instance), C.c_double, _D]),
    "pr_batch_run_range": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int, _VP]),
    "pr_batch_propagate": (C.c_int, [_VP, _VP, C.c_int, _VP]),
    "pr_probe_fp64_peak": (C.c_int, [_D]),
    "pr_force_create": (C.c_int, [C.POINTER(_VP), C.POINTER(pr_force_instance), C.c_int, C.c_int, C.c_int]),
    "pr_force_destroy": (C.c_int, [_VP]),
    "pr_force_last_error": (C.c_char_p, [_VP]),
    "pr_force_set_initial": (C.c_int, [_VP, C.c_int, _D, C.c_int]),
    "pr_force_set_f": (C.c_int, [_VP, C.c_int, _D]),
    "pr_force_run": (C.c_int, [_VP, C.c_int, _VP]),
    "pr_force_moments": (C.c_int, [_VP, C.c_int, C.c_int, _D]),
    "pr_force_get_f": (C.c_int, [_VP, C.c_int, _D]),
    "pr_force_sync": (C.c_int, [_VP]),
    "pr_force_config": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pr_force_set_cluster": (C.c_int, [_VP, C.c_int]),
    "pr_force_set_threads": (C.c_int, [_VP, C.c_int]),
    "pr_force_set_march": (C.c_int, [_VP, C.c_int]),
    "pr_force_set_persistent": (C.c_int, [_VP, C.c_int]),
    "pr_force_get_persistent": (C.c_int, [_VP, C.c_int, C.POINTER(C.c_int)]),
    "pr_force_get_march": (C.c_int, [_VP, C.POINTER(C.c_int)]),
    "pr_force_kernel_time": (C.c_int, [_VP, _D, C.POINTER(C.c_int), C.c_int]),
    "pr_force_dt_stab": (C.c_int, [C.POINTER(pr_force_instance), C.c_double, _D]),
    "pr_force_inject_wait_timeout": (C.c_int, [_VP, C.c_int]),
    "pr_set_force_step": (C.c_int, [_VP, C.c_int, C.c_int, C.c_int]),
    "pr_set_fine_path": (C.c_int, [_VP, C.c_int]),
    "pr_get_fine_path": (C.c_int, [_VP, C.POINTER(C.c_int)]),
    "pr_fine_cluster_shape": (C.c_int, [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "pr_init_force": (C.c_int, [C.POINTER(_VP), C.POINTER(pr_grid), C.POINTER(pr_velocity), C.c_double,
                                C.POINTER(pr_time), C.c_int, _D]),
}

EXPORTED = tuple(_SIGS)


def lib():
    """Load libpr.so (raises if it has not been built: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c \"import __graft_entry__ as g; "
                                   f"g.build()\"` (CUDA library required; no CPU fallback exists)")
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _f64(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    return a


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


_CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy: the legacy default stream


def _stream(s):
    """cudaStream_t for a torch stream / integer handle; None -> the object's
    own stream.  torch's default stream has handle 0, which the C ABI would
    read as "own stream", so it is passed as cudaStreamLegacy instead."""
    if s is None:
        return None
    h = s.cuda_stream if hasattr(s, "cuda_stream") else int(s)
    return C.c_void_p(h if h != 0 else _CUDA_STREAM_LEGACY)


def _dptr(t):
    if hasattr(t, "data_ptr"):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("device arguments must be contiguous CUDA tensors")
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(int(t))


class _Handle:
    """Opaque library object (pr_ctx* or pr_batch*) with cached sizes."""

    def __init__(self, ptr, kind, **meta):
        self.ptr = ptr
        self.kind = kind
        self.__dict__.update(meta)

    def __repr__(self):
        return f"<{self.kind} at {self.ptr.value:#x}>"


def _ctx_check(ctx, rc):
    if rc != PR_OK:
        msg = lib().pr_last_error(ctx.ptr if ctx is not None else None)
        raise PrError(rc, (msg or b"").decode())


def _batch_check(b, rc):
    if rc != PR_OK:
        msg = lib().pr_batch_last_error(b.ptr if b is not None else None)
        raise PrError(rc, (msg or b"").decode())


# ---------------------------------------------------------------- parareal

def pr_init(nx, x0, x1, bc, nv, L, eps, T, n_slices, cfl_f=0.5, cfl_g=0.5, scheme=PR_UPWIND,
            precision=PR_FP64, sound_speed=PR_SOUND_GAMMA53, max_batch=0, nf=0, coarse_model=PR_COARSE_EULER,
            lift_order=0):
    g = pr_grid(nx, x0, x1, bc)
    v = pr_velocity(nv, L)
    t = pr_time(T, n_slices, cfl_f, cfl_g, scheme, precision, sound_speed, max_batch, nf, coarse_model, lift_order)
    out = _VP()
    rc = lib().pr_init(C.byref(out), C.byref(g), C.byref(v), float(eps), C.byref(t))
    if rc != PR_OK:
        raise PrError(rc, (lib().pr_last_error(None) or b"").decode())
    return _Handle(out, "pr_ctx", nx=nx, nv=nv, N=n_slices)


def pr_destroy(ctx):
    if ctx is not None and ctx.ptr:
        lib().pr_destroy(ctx.ptr)
        ctx.ptr = _VP()


def pr_last_error(ctx=None) -> str:
    return (lib().pr_last_error(ctx.ptr if ctx is not None else None) or b"").decode()


def pr_set_initial(ctx, U0):
    U0 = _f64(U0, (5, ctx.nx))
    _ctx_check(ctx, lib().pr_set_initial(ctx.ptr, _p(U0)))


def pr_coarse_step(ctx, Vin, dT):
    Vin = _f64(Vin, (5, ctx.nx))
    out = np.empty_like(Vin)
    _ctx_check(ctx, lib().pr_coarse_step(ctx.ptr, _p(Vin), _p(out), float(dT)))
    return out


def pr_fine_step(ctx, slice_, nsteps, stream=None):
    _ctx_check(ctx, lib().pr_fine_step(ctx.ptr, int(slice_), int(nsteps), _stream(stream)))


def pr_fine_moments(ctx, slice_, kind=PR_CONSERVED):
    out = np.empty((5, ctx.nx))
    _ctx_check(ctx, lib().pr_fine_moments(ctx.ptr, int(slice_), int(kind), _p(out)))
    return out


def pr_fine_get_f(ctx, slice_):
    out = np.empty((ctx.nx, getattr(ctx, "nvx", ctx.nv) * ctx.nv ** 2))
    _ctx_check(ctx, lib().pr_fine_get_f(ctx.ptr, int(slice_), _p(out)))
    return out


def pr_parareal_iter(ctx) -> float:
    e = C.c_double()
    _ctx_check(ctx, lib().pr_parareal_iter(ctx.ptr, C.byref(e)))
    return e.value


def pr_parareal_run(ctx, K, tol=0.0, allow_notconv=True):
    errs = np.zeros(max(int(K), 1))
    kd = C.c_int()
    rc = lib().pr_parareal_run(ctx.ptr, int(K), float(tol), C.byref(kd), _p(errs))
    if not (allow_notconv and rc == PR_ENOTCONV):
        _ctx_check(ctx, rc)
    return kd.value, errs[: kd.value]


def pr_moments(ctx, n, kind=PR_CONSERVED):
    out = np.empty((5, ctx.nx))
    _ctx_check(ctx, lib().pr_moments(ctx.ptr, int(n), int(kind), _p(out)))
    return out


def pr_fine_steps_per_slice(ctx):
    nf = C.c_int()
    dt = C.c_double()
    _ctx_check(ctx, lib().pr_fine_steps_per_slice(ctx.ptr, C.byref(nf), C.byref(dt)))
    return nf.value, dt.value


def pr_iterations(ctx) -> int:
    k = C.c_int()
    _ctx_check(ctx, lib().pr_iterations(ctx.ptr, C.byref(k)))
    return k.value


def pr_save(ctx, path):
    """Write the parareal iteration state to path (pr_save)."""
    _ctx_check(ctx, lib().pr_save(ctx.ptr, os.fsencode(path)))


def pr_load(ctx, path):
    """Continue a parareal run from a state written by pr_save (pr_load)."""
    _ctx_check(ctx, lib().pr_load(ctx.ptr, os.fsencode(path)))


# ---------------------------------------------------------------- batches

def instance(nx, nv, dt, L=8.0, x0=0.0, x1=1.0, bc=PR_BC_PERIODIC, eps=1e-2, scheme=PR_UPWIND) -> pr_instance:
    return pr_instance(int(nx), float(x0), float(x1), int(bc), int(nv), float(L), float(eps), float(dt), int(scheme))


def pr_batch_create(instances, precision=PR_MIXED):
    n = len(instances)
    arr = (pr_instance * n)(*instances)
    out = _VP()
    rc = lib().pr_batch_create(C.byref(out), arr, n, int(precision))
    if rc != PR_OK:
        raise PrError(rc, (lib().pr_batch_last_error(None) or b"").decode())
    return _Handle(out, "pr_batch", shapes=[(d.nx, d.nv) for d in instances], n=n)


def pr_multi_create(ctxs, extra=()):
    """Several parareal problems (and independent instances) iterated
    together, one persistent launch per iteration (pr_multi_create)."""
    n = len(ctxs)
    arr = (_VP * n)(*[c.ptr for c in ctxs])
    ex = (pr_instance * max(len(extra), 1))(*extra)
    out = _VP()
    rc = lib().pr_multi_create(C.byref(out), arr, n, ex, len(extra))
    if rc != PR_OK:
        raise PrError(rc, (lib().pr_multi_last_error(None) or b"").decode())
    shapes = []
    for n_ in range(1, max(c.N for c in ctxs) + 1):
        shapes += [(c.nx, c.nv) for c in ctxs if n_ <= c.N]
    shapes += [(d.nx, d.nv) for d in extra]
    b = _VP()
    first = C.c_int()
    lib().pr_multi_batch(out, C.byref(b), C.byref(first))
    batch = _Handle(b, "pr_batch (of a pr_multi)", shapes=shapes, n=len(shapes))
    return _Handle(out, "pr_multi", n_ctx=n, batch=batch, first_independent=first.value)


def pr_multi_batch(m):
    """The batch of a pr_multi and the index of its first independent
    instance (pr_multi_batch); pr_multi_create keeps both on the handle."""
    return m.batch, m.first_independent


def pr_multi_last_error(m=None) -> str:
    return (lib().pr_multi_last_error(m.ptr if m is not None else None) or b"").decode()


def _multi_check(m, rc):
    if rc != PR_OK:
        msg = lib().pr_multi_last_error(m.ptr if m is not None else None)
        raise PrError(rc, (msg or b"").decode())


def pr_multi_iterate(m, count=1):
    """count lockstep iterations; the errors of Eq. 10, [count, n_problems]."""
    errs = np.zeros((max(int(count), 1), m.n_ctx))
    _multi_check(m, lib().pr_multi_iterate(m.ptr, int(count), _p(errs)))
    return errs[: int(count)]


def pr_multi_destroy(m):
    if m is not None and m.ptr:
        lib().pr_multi_destroy(m.ptr)
        m.ptr = _VP()


def pr_batch_vpt(b) -> int:
    """Velocities per thread of the fine kernel in use (pr_batch_vpt)."""
    v = C.c_int()
    _batch_check(b, lib().pr_batch_vpt(b.ptr, C.byref(v)))
    return v.value


def pr_batch_destroy(b):
    if b is not None and b.ptr:
        lib().pr_batch_destroy(b.ptr)
        b.ptr = _VP()


def pr_batch_last_error(b=None) -> str:
    return (lib().pr_batch_last_error(b.ptr if b is not None else None) or b"").decode()


def pr_batch_set_initial(b, i, U, kind=PR_PRIMITIVE):
    nx = b.shapes[i][0]
    U = _f64(U, (5, nx))
    _batch_check(b, lib().pr_batch_set_initial(b.ptr, int(i), _p(U), int(kind)))


def pr_batch_set_initial_device(b, i, U_dev, kind=PR_CONSERVED, stream=None):
    _batch_check(b, lib().pr_batch_set_initial_device(b.ptr, int(i), _dptr(U_dev), int(kind), _stream(stream)))


def pr_batch_set_f(b, i, f):
    nx, nv = b.shapes[i]
    f = _f64(f, (nx, nv ** 3))
    _batch_check(b, lib().pr_batch_set_f(b.ptr, int(i), _p(f)))


def pr_batch_run(b, nsteps, stream=None):
    _batch_check(b, lib().pr_batch_run(b.ptr, int(nsteps), _stream(stream)))


def pr_batch_run_range(b, first, count, nsteps, stream=None):
    _batch_check(b, lib().pr_batch_run_range(b.ptr, int(first), int(count), int(nsteps), _stream(stream)))


def pr_batch_propagate(b, nsteps, U_dev=None, stream=None):
    """P F L of every instance (pr_batch_propagate): lift from U_dev (a device
    tensor holding the instances' conserved states one after another) or from
    the last set_initial sources, nsteps fine steps, projection."""
    ptr = _dptr(U_dev) if U_dev is not None else None
    _batch_check(b, lib().pr_batch_propagate(b.ptr, ptr, int(nsteps), _stream(stream)))


def pr_batch_moments(b, i, kind=PR_CONSERVED):
    out = np.empty((5, b.shapes[i][0]))
    _batch_check(b, lib().pr_batch_moments(b.ptr, int(i), int(kind), _p(out)))
    return out


def pr_batch_moments_device(b, i, out_dev, stream=None):
    _batch_check(b, lib().pr_batch_moments_device(b.ptr, int(i), _dptr(out_dev), _stream(stream)))


def pr_batch_get_f(b, i):
    nx, nv = b.shapes[i]
    out = np.empty((nx, nv ** 3))
    _batch_check(b, lib().pr_batch_get_f(b.ptr, int(i), _p(out)))
    return out


def pr_batch_inject_wait_timeout(b, nsteps=3, wait_ms=50) -> int:
    """Run the failure-detection launch; returns the status it reported
    (PR_ETIMEOUT expected) without raising."""
    return int(lib().pr_batch_inject_wait_timeout(b.ptr, int(nsteps), int(wait_ms)))


def pr_batch_sync(b):
    _batch_check(b, lib().pr_batch_sync(b.ptr))


def pr_batch_set_lift_order(b, order):
    _batch_check(b, lib().pr_batch_set_lift_order(b.ptr, int(order)))


def pr_batch_tile(b, i):
    tx, tuned = C.c_int(), C.c_int()
    _batch_check(b, lib().pr_batch_tile(b.ptr, int(i), C.byref(tx), C.byref(tuned)))
    return tx.value, bool(tuned.value)


def pr_batch_set_tile(b, tx):
    _batch_check(b, lib().pr_batch_set_tile(b.ptr, int(tx)))


def pr_batch_autotune(b):
    _batch_check(b, lib().pr_batch_autotune(b.ptr))


def pr_batch_kernel_time(b, reset=False):
    ms = C.c_double()
    n = C.c_int()
    _batch_check(b, lib().pr_batch_kernel_time(b.ptr, C.byref(ms), C.byref(n), int(bool(reset))))
    return ms.value, n.value


def pr_batch_adjoint(b, i, nsteps, lamV, checkpoint=16):
    """(dJ/dU0 [5, nx] primitive, dJ/dlog eps) for dJ/dV(T) = lamV [5, nx]
    (float64 upwind instance, lifted start)."""
    nx = b.shapes[i][0]
    lamV = _f64(lamV, (5, nx))
    dU0 = np.empty((5, nx))
    de = C.c_double()
    _batch_check(b, lib().pr_batch_adjoint(b.ptr, int(i), int(nsteps), int(checkpoint), _p(lamV), _p(dU0),
                                           C.byref(de)))
    return dU0, de.value


def pr_kernel_launches(reset=False) -> int:
    return int(lib().pr_kernel_launches(int(bool(reset))))


def pr_fine_step_noalloc(inst, f_in_dev, f_out_dev, stream=None):
    """One float64 fine step f_out = F(f_in) on caller-owned device arrays,
    with all scratch in the library's static device array (no allocation)."""
    rc = lib().pr_fine_step_noalloc(C.byref(inst), _dptr(f_in_dev), _dptr(f_out_dev), _stream(stream))
    if rc != PR_OK:
        raise PrError(rc, (lib().pr_batch_last_error(None) or b"").decode() or "pr_fine_step_noalloc failed")


def pr_fine_dt_stab(inst, cfl=0.5) -> float:
    out = C.c_double()
    rc = lib().pr_fine_dt_stab(C.byref(inst), float(cfl), C.byref(out))
    if rc != PR_OK:
        raise PrError(rc, "pr_fine_dt_stab: invalid grid or cfl")
    return out.value


def pr_probe_fp64_peak() -> float:
    """Measured FP64 FMA throughput of the current device, TFLOP/s."""
    out = C.c_double()
    rc = lib().pr_probe_fp64_peak(C.byref(out))
    if rc != PR_OK:
        raise PrError(rc, "pr_probe_fp64_peak failed")
    return out.value


def fine_dt(nx, nv, L, cfl=0.5, x0=0.0, x1=1.0) -> float:
    """dt_stab = cfl dx / max|v_x| of the x transport (Sec. 2.2), from the library."""
    return pr_fine_dt_stab(instance(nx, nv, 1.0, L=L, x0=x0, x1=x1), cfl)


# ---------------------------------------------------------------- exterior force

class ForceInstance:
    """One force-path instance: pr_force_instance plus the force array it
    points at (kept alive here; the library copies it at creation)."""

    def __init__(self, nx, nvx, nvp, dt, L=8.0, x0=0.0, x1=1.0, bc=PR_BC_PERIODIC, eps=1e-2, E=None):
        self.E = None if E is None else _f64(E, (nx,))
        self.c = pr_force_instance(int(nx), float(x0), float(x1), int(bc), int(nvx), int(nvp), float(L),
                                   float(eps), float(dt), _p(self.E) if self.E is not None else C.cast(None, _D))
        self.nx, self.nvx, self.nvp = int(nx), int(nvx), int(nvp)


def _force_check(b, rc):
    if rc != PR_OK:
        msg = lib().pr_force_last_error(b.ptr if b is not None else None)
        raise PrError(rc, (msg or b"").decode())


def pr_force_create(instances, scheme=PR_UPWIND, precision=PR_MIXED):
    n = len(instances)
    arr = (pr_force_instance * n)(*[d.c for d in instances])
    out = _VP()
    rc = lib().pr_force_create(C.byref(out), arr, n, int(scheme), int(precision))
    if rc != PR_OK:
        raise PrError(rc, (lib().pr_force_last_error(None) or b"").decode())
    d = instances[0]
    return _Handle(out, "pr_force", n=n, nx=d.nx, nvx=d.nvx, nvp=d.nvp, ncol=d.nvx * d.nvp ** 2)


def pr_force_destroy(b):
    if b is not None and b.ptr:
        lib().pr_force_destroy(b.ptr)
        b.ptr = _VP()


def pr_force_last_error(b=None) -> str:
    return (lib().pr_force_last_error(b.ptr if b is not None else None) or b"").decode()


def pr_force_set_initial(b, i, U, kind=PR_PRIMITIVE):
    U = _f64(U, (5, b.nx))
    _force_check(b, lib().pr_force_set_initial(b.ptr, int(i), _p(U), int(kind)))


def pr_force_set_f(b, i, f):
    f = _f64(f, (b.nx, b.ncol))
    _force_check(b, lib().pr_force_set_f(b.ptr, int(i), _p(f)))


def pr_force_run(b, nsteps, stream=None):
    _force_check(b, lib().pr_force_run(b.ptr, int(nsteps), _stream(stream)))


def pr_force_moments(b, i, kind=PR_CONSERVED):
    out = np.empty((5, b.nx))
    _force_check(b, lib().pr_force_moments(b.ptr, int(i), int(kind), _p(out)))
    return out


def pr_force_get_f(b, i):
    out = np.empty((b.nx, b.ncol))
    _force_check(b, lib().pr_force_get_f(b.ptr, int(i), _p(out)))
    return out


def pr_force_sync(b):
    _force_check(b, lib().pr_force_sync(b.ptr))


def pr_force_set_lift_order(b, order):
    _force_check(b, lib().pr_force_set_lift_order(b.ptr, int(order)))


def pr_force_config(b):
    c, k = C.c_int(), C.c_int()
    _force_check(b, lib().pr_force_config(b.ptr, C.byref(c), C.byref(k)))
    return c.value, k.value


def pr_force_set_cluster(b, cluster):
    _force_check(b, lib().pr_force_set_cluster(b.ptr, int(cluster)))


def pr_force_set_threads(b, threads):
    _force_check(b, lib().pr_force_set_threads(b.ptr, int(threads)))


def pr_force_set_march(b, columns):
    _force_check(b, lib().pr_force_set_march(b.ptr, int(columns)))


def pr_force_autotune(b, nsteps=4):
    """Time the candidate step layouts on the current states and keep the
    fastest (pr_force_autotune); the chosen (cluster, walk)."""
    _force_check(b, lib().pr_force_autotune(b.ptr, int(nsteps)))
    return pr_force_config(b)[0], pr_force_get_march(b)


def pr_force_set_persistent(b, mode):
    _force_check(b, lib().pr_force_set_persistent(b.ptr, int(mode)))


def pr_force_get_persistent(b, nsteps) -> int:
    n = C.c_int()
    _force_check(b, lib().pr_force_get_persistent(b.ptr, int(nsteps), C.byref(n)))
    return n.value


def pr_force_get_march(b) -> int:
    n = C.c_int()
    _force_check(b, lib().pr_force_get_march(b.ptr, C.byref(n)))
    return n.value


def pr_force_kernel_time(b, reset=False):
    ms = C.c_double()
    n = C.c_int()
    _force_check(b, lib().pr_force_kernel_time(b.ptr, C.byref(ms), C.byref(n), int(bool(reset))))
    return ms.value, n.value


def pr_force_inject_wait_timeout(b, wait_ms=50) -> int:
    """Run the failure-detection step; returns the status it reported
    (PR_ETIMEOUT expected) without raising."""
    return int(lib().pr_force_inject_wait_timeout(b.ptr, int(wait_ms)))


def pr_force_dt_stab(inst: ForceInstance, cfl=0.5) -> float:
    dt = C.c_double()
    rc = lib().pr_force_dt_stab(C.byref(inst.c), float(cfl), C.byref(dt))
    if rc != PR_OK:
        raise PrError(rc, "pr_force_dt_stab")
    return dt.value


def pr_init_force(nx, x0, x1, bc, nvx, nvp, L, eps, T, n_slices, E, cfl_f=0.5, cfl_g=0.5, scheme=PR_UPWIND,
                  precision=PR_FP64, sound_speed=PR_SOUND_GAMMA53, max_batch=0, nf=0, coarse_model=PR_COARSE_EULER,
                  lift_order=0):
    """Parareal problem with the exterior force E [nx] (host, copied)."""
    g = pr_grid(nx, x0, x1, bc)
    v = pr_velocity(nvp, L)
    t = pr_time(T, n_slices, cfl_f, cfl_g, scheme, precision, sound_speed, max_batch, nf, coarse_model, lift_order)
    Ea = None if E is None else _f64(E, (nx,))
    out = _VP()
    rc = lib().pr_init_force(C.byref(out), C.byref(g), C.byref(v), float(eps), C.byref(t), int(nvx),
                             _p(Ea) if Ea is not None else C.cast(None, _D))
    if rc != PR_OK:
        raise PrError(rc, (lib().pr_last_error(None) or b"").decode())
    return _Handle(out, "pr_ctx", nx=nx, nv=nvp, nvx=nvx, N=n_slices)


def pr_set_fine_path(ctx, mode):
    """Kernel of the fine phase of a parareal iteration (PR_FINE_AUTO / _TILED / _CLUSTER)."""
    _ctx_check(ctx, lib().pr_set_fine_path(ctx.ptr, int(mode)))


def pr_get_fine_path(ctx):
    """The kernel the fine phase of an iteration uses (PR_FINE_TILED or PR_FINE_CLUSTER)."""
    v = C.c_int()
    _ctx_check(ctx, lib().pr_get_fine_path(ctx.ptr, C.byref(v)))
    return v.value


def pr_fine_cluster_shape(ctx):
    """(CTAs per cluster, x cells per CTA, clusters resident at once) of the
    cluster-resident fine run, zeros when it does not apply."""
    a, b, r = C.c_int(), C.c_int(), C.c_int()
    _ctx_check(ctx, lib().pr_fine_cluster_shape(ctx.ptr, C.byref(a), C.byref(b), C.byref(r)))
    return a.value, b.value, r.value


def pr_set_force_step(ctx, cluster=0, columns=-1, persistent=-1):
    """Step kernel of a force problem's fine propagator (pr_set_force_step)."""
    _ctx_check(ctx, lib().pr_set_force_step(ctx.ptr, int(cluster), int(columns), int(persistent)))


INF = math.inf
