"""The C-ABI library loads and exports every function include/pf.h declares (no GPU needed:
only host-side entry points are called)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(pf_\w+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1511_08463_gb300 import _build, binding

    _build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_1511_08463_gb300 import binding

    assert set(_declared()) == set(binding._SIGS)


def test_host_entry_points(lib):
    import workloads as W
    from paper_1511_08463_gb300 import binding as B
    from paper_1511_08463_gb300.sim import mesh_desc

    assert lib.pf_version().decode().startswith("libpf")
    o = B.pf_solver_opts()
    assert lib.pf_default_opts(C.byref(o)) == B.PF_OK
    assert o.algo == B.PF_ALGO_ORAM and o.am_tol == 1e-6
    d = mesh_desc(W.notched_square(n=64))
    nb = lib.pf_workspace_bytes(C.byref(d), B.PF_FP64)
    d2 = mesh_desc(W.notched_square(n=128))
    nb2 = lib.pf_workspace_bytes(C.byref(d2), B.PF_FP64)
    assert 0 < nb < nb2 < 5 * nb
    bad = mesh_desc(W.notched_square(n=64))
    bad.nx = 0
    assert lib.pf_workspace_bytes(C.byref(bad), B.PF_FP64) == 0
    conflict = mesh_desc(W.bar(nx=16, ny=2))
    conflict.fixed[2][0] = 1  # bottom u_x clashes with the right edge value at a corner
    conflict.load[2][0] = 0.0
    assert lib.pf_workspace_bytes(C.byref(conflict), B.PF_FP64) == 0
    assert "corner" in lib.pf_last_error().decode()
    pinbad = mesh_desc(W.bar(nx=16, ny=2))
    pinbad.pin_x2[0] = 1  # not a node of a right mesh
    assert lib.pf_workspace_bytes(C.byref(pinbad), B.PF_FP64) == 0
