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


def test_solver_opts_layout_matches_header(lib):
    """pf_default_opts writes the C struct: the binding's struct must have the same size (no write
    past it) and the same field offsets (every default read back through the binding)."""
    from paper_1511_08463_gb300 import binding as B

    size = C.sizeof(B.pf_solver_opts)
    raw = (C.c_ubyte * (size + 64))(*([0xAB] * (size + 64)))
    assert lib.pf_default_opts(C.cast(raw, C.POINTER(B.pf_solver_opts))) == B.PF_OK
    assert all(b == 0xAB for b in raw[size:])  # nothing written past the binding's struct
    o = B.pf_solver_opts.from_buffer(raw)
    expect = dict(algo=B.PF_ALGO_ORAM, precision=B.PF_FP64, omega=1.0, am_tol=1e-6, am_maxit=20000,
                  u_rtol=1e-8, inner_rtol=1e-4, cg_maxit=2000, rs_rtol=1e-8, rs_maxit=100,
                  alpha_cg_rtol=1e-6, zeta=1e-10, mg_levels_max=0, mg_degree=2, switch_tol=1e-2,
                  newton_rtol=1e-8, newton_maxit=30, minres_maxit=500, minres_rtol=1e-6,
                  use_graphs=1, batch_workers=8, am_forcing=0.0, am_forcing_max=1e-3, mg_tail=1,
                  mg_coarse_degree=0, omega_rule=0, omega_auto=0, omega_max=1.9, autotune=0,
                  tile_rows_fine=0, tile_rows_coarse=0)
    assert [f for f, _ in B.pf_solver_opts._fields_] == list(expect)
    for k, v in expect.items():
        assert getattr(o, k) == v, k


def test_header_is_plain_c_and_links(tmp_path, lib):
    """include/pf.h compiles as C99 (no C++-only constructs), and a C caller links against
    libpf.so and calls the host-only entry points."""
    import shutil
    import subprocess

    from paper_1511_08463_gb300 import _build

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "caller.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "pf.h"
int main(void) {
  pf_solver_opts o;
  pf_mesh_desc d;
  if (pf_default_opts(&o) != PF_OK || o.algo != PF_ALGO_ORAM) return 1;
  memset(&d, 0, sizeof d);
  d.kind = PF_MESH_CROSSED; d.nx = 64; d.ny = 64; d.lx = 1.0; d.ly = 1.0;
  if (pf_workspace_bytes(&d, PF_MIXED) == 0) return 2;
  d.nx = 0;
  if (pf_workspace_bytes(&d, PF_MIXED) != 0) return 3;
  printf("%s\n", pf_version());
  return 0;
}
''')
    exe = tmp_path / "caller"
    libdir = os.path.dirname(_build.LIB)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-pedantic", "-I",
                    os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lpf",
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stderr)
    assert out.stdout.startswith("libpf")


def test_kernel_class_names(lib):
    """Launch-accounting classes (host-side table): one name per (kernel, precision, level), and
    the names bench.py reads for its roofline and its double-float vs FP64 comparison exist."""
    n = lib.pf_prof_class_count()
    names = []
    for k in range(n):
        nm = C.c_char_p()
        assert lib.pf_prof_get(k, C.byref(nm), None, None, None, None) == 0
        names.append(nm.value.decode())
    assert len(set(names)) == n
    for want in ("elastic_cheb_f32_l0", "elastic_cheb_z_f32_l0", "tail_vcycle_f32_l6",
                 "elastic_resid_df_f64_l0", "elastic_resid_f64_l0", "damage_grad_df_f64_l0",
                 "damage_grad_f64_l0", "damage_trial_df_f64_l0", "damage_trial_f64_l0",
                 "damage_q_df_f64_l0", "damage_q_f64_l0"):
        assert want in names, want
    assert lib.pf_prof_get(n, None, None, None, None, None) != 0
