"""The C ABI library builds, loads and exports every entry point that
include/pr.h declares; the Python binding wraps each of them (no GPU needed)."""
import os
import re

import paper_2502_02704_gb300 as pr
from paper_2502_02704_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(pr_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_declared_entry_point():
    B.build()
    L = pr.lib()
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name


def test_binding_covers_the_abi():
    declared = set(_declared())
    assert declared == set(pr.EXPORTED)
    for name in declared:
        assert callable(getattr(pr, name)), name


def test_null_problem_is_rejected_without_a_device():
    # entry points validate their handle before any CUDA call
    import ctypes as C
    L = pr.lib()
    v = C.c_int()
    assert L.pr_set_fine_path(None, pr.PR_FINE_CLUSTER) == pr.PR_EINVAL
    assert L.pr_get_fine_path(None, C.byref(v)) == pr.PR_EINVAL
    assert L.pr_fine_cluster_shape(None, C.byref(v), C.byref(v), C.byref(v)) == pr.PR_EINVAL
    assert L.pr_set_force_step(None, 0, -1, -1) == pr.PR_EINVAL
    assert L.pr_parareal_iter(None, None) == pr.PR_EINVAL


def test_fine_dt_stab_needs_no_device():
    # Sec. 2.2: dt_stab = cfl dx / max|v_x|, max|v_x| the outermost node
    # L - dv/2 (cube centres); computed by the library, not by the binding.
    dt = pr.pr_fine_dt_stab(pr.instance(64, 16, 1.0, L=8.0), 0.5)
    assert dt == 0.5 * (1.0 / 64) / 7.5
    assert pr.fine_dt(256, 24, 8.0) == pr.pr_fine_dt_stab(pr.instance(256, 24, 1.0), 0.5)
    for bad in (pr.instance(0, 16, 1.0), pr.instance(8, 16, 1.0, L=-1.0), pr.instance(8, 16, 1.0, x0=1.0, x1=1.0)):
        try:
            pr.pr_fine_dt_stab(bad, 0.5)
            raise AssertionError("accepted an invalid grid")
        except pr.PrError as e:
            assert e.code == pr.PR_EINVAL
    for cfl in (0.0, float("inf"), float("nan")):
        try:
            pr.pr_fine_dt_stab(pr.instance(8, 16, 1.0), cfl)
            raise AssertionError("accepted an invalid cfl")
        except pr.PrError as e:
            assert e.code == pr.PR_EINVAL
