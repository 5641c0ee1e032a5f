"""Autotuner: smoother degrees and FP32 stencil tile heights picked by timing whole PCG solves on
the sim's own state, cached per (mesh, precision).  The choice changes only the speed: load steps
with the tuned configuration converge to the same states as with the defaults."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import need_gpu, rel_max

pytestmark = pytest.mark.gpu


def test_autotune_reports_a_valid_configuration_and_keeps_results():
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.notched_square(n=64, n_steps=10, t_max=1.0)
    g = S.Sim(w)
    o = S.make_opts(omega=w.omega, precision="mixed")
    g.load_step(*w.loads[0], o)
    rep = g.autotune(o)
    assert rep["trials"] == 20
    assert 1 <= rep["mg_degree"] <= 4 and 1 <= rep["mg_coarse_degree"] <= 3
    assert rep["tile_rows_fine"] in (4, 8, 16) and rep["tile_rows_coarse"] in (4, 8, 16)
    assert 0 < rep["ms_best"] <= rep["ms_default"]
    snap = g.get_fields()
    res = []
    for tune in (0, 1):
        g.set_fields(*snap)
        ot = S.make_opts(omega=w.omega, precision="mixed", autotune=tune, am_tol=1e-9,
                         u_rtol=1e-11, rs_rtol=1e-11)
        r = g.load_step(*w.loads[1], ot)
        assert r["status"] == 0
        res.append((r, g.get_fields()))
    (r0, f0), (r1, f1) = res
    assert abs(r0["energy"][2] - r1["energy"][2]) <= 1e-9 * abs(r0["energy"][2])
    assert rel_max(f1[0], f0[0]) <= 1e-6 and np.abs(f1[1] - f0[1]).max() <= 1e-6


def test_tile_heights_change_only_the_speed():
    """The FP32 stencil kernels compute every element record the same way and gather each node's
    records in a fixed order whatever the tile height; only the block partial sums of the
    reductions change.  Load steps with 4- and 16-row tiles agree with the 8-row default."""
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.notched_square(n=64, n_steps=10, t_max=1.0)
    out = []
    for tf, tc in ((0, 0), (4, 16), (16, 4)):
        g = S.Sim(w)
        o = S.make_opts(omega=w.omega, precision="mixed", tile_rows_fine=tf, tile_rows_coarse=tc,
                        am_tol=1e-9, u_rtol=1e-11, rs_rtol=1e-11)
        r = g.load_step(*w.loads[0], o)
        assert r["status"] == 0
        out.append((r["energy"][2], g.get_fields()))
    for e, f in out[1:]:
        assert abs(e - out[0][0]) <= 1e-9 * abs(out[0][0])
        assert rel_max(f[0], out[0][1][0]) <= 1e-6
