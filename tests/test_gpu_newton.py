"""GPU parity of the coupled (ORAM-N) path against the oracle: the off-diagonal Jacobian block B
of Section 3.3 (eq. offdiag) and whole load steps of Algorithm 3."""
import numpy as np
import pytest

import workloads as W
from oracle import am, fe
from oracle.problem import Problem

from .gpu_util import need_gpu, rel_max, tight_opts

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["notched", "thermal", "at2"])
def test_coupling_apply(case):
    torch = need_gpu()
    from paper_1511_08463_gb300 import sim as S

    if case == "notched":
        w, (t, dT) = W.notched_square(n=32), (0.3, 0.0)
    elif case == "at2":
        w, (t, dT) = W.notched_square(n=24, model="AT2"), (0.3, 0.0)
    else:
        w = W.thermal_shock(nx=48, ny=12)
        t, dT = w.loads[10]
    p = Problem(w)
    rng = np.random.default_rng(11)
    n = p.mesh.n_nodes
    u = 0.02 * rng.normal(size=(n, 2))
    alpha = rng.uniform(0.0, 0.8, n)
    g = S.Sim(w)
    g.set_fields(u=u, alpha=alpha, alpha_prev=np.zeros(n))
    g.set_load(t, dT)
    ug, _, _ = g.get_fields()  # u after the Dirichlet lift of set_load
    Bm = fe.coupling(p.mat, p.geo, ug, alpha, dT).tocsr()
    free = ~p.u_fixed
    xa = rng.normal(size=n)
    xu = rng.normal(size=2 * n)
    dev = torch.device("cuda:0")
    y = g.coupling_apply(torch.tensor(xa, device=dev)).cpu().numpy()
    yref = np.where(free, Bm @ xa, 0.0)
    assert rel_max(y, yref) <= 1e-12
    yt = g.coupling_apply(torch.tensor(xu, device=dev), transpose=True).cpu().numpy()
    ytref = Bm.T @ np.where(free, xu, 0.0)
    assert rel_max(yt, ytref) <= 1e-12


def _oramn_pair(w, steps, omega, precision="fp64", **kw):
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    g = S.Sim(w)
    p = Problem(w)
    opts = tight_opts(S, algo="ORAM_N", omega=omega, precision=precision, newton_rtol=1e-9,
                      switch_tol=1e-2, **kw)
    out = []
    for (t, dT) in steps:
        rep = g.load_step(t, dT, opts)
        r = am.load_step_oramn(p, t, dT, omega=omega, switch_tol=1e-2, rtol=1e-9)
        out.append((rep, r))
    return g, p, out


def test_notched_oramn_load_steps():
    """Algorithm 3 on the notched square through crack growth: both reach ||Phi|| <= 1e-9
    ||Phi_start||, so they agree on the energies and fields of each step."""
    w = W.notched_square(n=32, n_steps=10, t_max=1.0)
    g, p, out = _oramn_pair(w, w.loads[:7], omega=1.5)
    newton = 0
    for rep, r in out:
        assert rep["status"] == 0 and r["status"] == "converged"
        assert rep["phi_norm"] <= 1e-9 * rep["phi_start"] * 1.0001
        np.testing.assert_allclose(rep["energy"], r["energy"], rtol=1e-8, atol=1e-14)
        newton += rep["newton_iters"]
    assert newton > 0  # the Newton phase ran
    u, a, ap = g.get_fields()
    assert np.abs(a - p.alpha).max() <= 1e-6
    assert rel_max(u, p.u) <= 1e-6
    assert p.alpha[p.alpha_prev < 1].max() > 0.1


def test_thermal_oramn_load_steps():
    w = W.thermal_shock(nx=64, ny=16, n_steps=40)
    g, p, out = _oramn_pair(w, w.loads[8:11], omega=1.6)
    for rep, r in out:
        assert rep["status"] == 0
        np.testing.assert_allclose(rep["energy"], r["energy"], rtol=1e-8, atol=1e-14)
    u, a, _ = g.get_fields()
    assert np.abs(a - p.alpha).max() <= 1e-6


def test_oramn_matches_oram_solution():
    """ORAM and ORAM-N solve the same load step: same energies at tight tolerances."""
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.notched_square(n=32, n_steps=10, t_max=1.0)
    ga, gb = S.Sim(w), S.Sim(w)
    oa = tight_opts(S, algo="ORAM", omega=1.5)
    ob = tight_opts(S, algo="ORAM_N", omega=1.5, newton_rtol=1e-10)
    for (t, dT) in w.loads[:6]:
        ra = ga.load_step(t, dT, oa)
        rb = gb.load_step(t, dT, ob)
        np.testing.assert_allclose(ra["energy"], rb["energy"], rtol=1e-7, atol=1e-14)
