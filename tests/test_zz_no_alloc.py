"""The allocation-free energy entry point (pf_energy_noalloc) against pf_energy.

pf_energy_noalloc serves callers that cannot let a library allocate device memory (for example
when their own memory pool holds all free device memory, or when the implicit synchronization of
cudaMalloc/cudaFree is not acceptable).  It keeps its scratch in a fixed array inside the library.
This file is collected last so that a failure here stops a run only after every other test.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

from .gpu_util import need_gpu, tight_opts

pytestmark = pytest.mark.gpu


def _noalloc(lib, B, S, w, u_dev, a_dev, load, torch):
    out = (C.c_double * 3)()
    d = S.mesh_desc(w)
    m = S.material(w)
    L = B.pf_load(*load)
    st = lib.pf_energy_noalloc(C.byref(d), C.byref(m), C.byref(L), u_dev.data_ptr(),
                               a_dev.data_ptr(), out, torch.cuda.current_stream().cuda_stream)
    return st, list(out)


def test_energy_noalloc_matches_pf_energy_twice():
    torch = need_gpu()
    from paper_1511_08463_gb300 import binding as B
    from paper_1511_08463_gb300 import sim as S

    lib = B.load()
    w = W.thermal_shock(nx=64, ny=16)  # thermal eigenstrain exercises the scratch table too
    g = S.Sim(w)
    opts = tight_opts(S, omega=w.omega)
    for k in (10, 11):  # two calls in a row, on different states
        g.load_step(*w.loads[k], opts)
        ref = g.energy()
        u, a, _ = g.get_fields()
        ud = torch.tensor(u.ravel(), device="cuda")
        ad = torch.tensor(a, device="cuda")
        st, out = _noalloc(lib, B, S, w, ud, ad, w.loads[k], torch)
        assert st == B.PF_OK, lib.pf_last_error().decode()
        np.testing.assert_allclose(out, ref, rtol=1e-12)
        assert out[1] > 0  # damage has appeared in these steps


def test_energy_noalloc_rejects_meshes_beyond_its_scratch():
    torch = need_gpu()
    from paper_1511_08463_gb300 import binding as B
    from paper_1511_08463_gb300 import sim as S

    lib = B.load()
    w = W.Workload(name="tall", kind="right", nx=2, ny=8194, x0=0, y0=0, lx=1.0, ly=4.0)
    n = w.n_nodes()
    ud = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
    ad = torch.zeros(n, dtype=torch.float64, device="cuda")
    st, _ = _noalloc(lib, B, S, w, ud, ad, (0.0, 0.0), torch)
    assert st == B.PF_EINVAL
    assert "8192" in lib.pf_last_error().decode()
