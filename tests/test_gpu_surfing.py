"""Surfing (Section 4.1, eq. surfingloading): the asymptotic Mode-I displacement prescribed on
the whole boundary of the slab [0, 2] x [-1/2, 1/2], its tip moving at speed v.  GPU against the
oracle for the boundary data and for ORAM load steps (AT1 and AT2), and the Griffith check of
the section: with K_I = sqrt(Gc E) the dissipated energy grows at Gc v whatever ell is (h = ell/5)."""
import numpy as np
import pytest

import workloads as W
from oracle import am
from oracle.problem import Problem
from tests.gpu_util import need_gpu, rel_max, tight_opts

pytestmark = pytest.mark.gpu


def test_mode_I_boundary_data_matches_oracle():
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    for kind in ("crossed", "right"):
        w = W.surfing(nx=40, ny=20, ell=0.2, kind=kind)
        g = S.Sim(w)
        p = Problem(w)
        for t in (0.0, 0.37, 1.1):
            g.set_load(t, 0.0)
            u, _, _ = g.get_fields()
            p.lift(t)
            fx = p.u_fixed.reshape(-1, 2)
            assert fx.any()
            np.testing.assert_allclose(u[fx], p.u[fx], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("model", ["AT1", "AT2"])
def test_surfing_oram_load_steps(model):
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.surfing(nx=52, ny=26, ell=0.2, n_steps=8, t_max=1.2, model=model)
    g = S.Sim(w)
    p = Problem(w)
    opts = tight_opts(S, omega=w.omega)
    for (t, dT) in w.loads[:4]:
        rep = g.load_step(t, dT, opts)
        r = am.load_step(p, t, dT, omega=w.omega, tol=1e-10)
        assert rep["status"] == 0 and r["status"] == "converged"
        np.testing.assert_allclose(rep["energy"], r["energy"], rtol=1e-8, atol=1e-14)
    u, a, _ = g.get_fields()
    assert rel_max(u, p.u) <= 1e-6 and np.abs(a - p.alpha).max() <= 1e-6
    assert p.alpha[p.alpha_prev < 1].max() > 0.5  # the crack has started to move


def test_surfing_dissipation_rate_griffith_independent_of_ell():
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    rates = []
    for n, ell in ((104, 0.1), (208, 0.05)):
        w = W.surfing(nx=n, ny=n // 2, ell=ell, n_steps=8, t_max=1.2)
        g = S.Sim(w)
        opts = S.make_opts(omega=w.omega, precision="mixed")
        es = []
        for (t, dT) in w.loads:
            rep = g.load_step(t, dT, opts)
            assert rep["status"] == 0
            es.append(rep["energy"][1])
        ts = [t for t, _ in w.loads]
        rates.append((es[-1] - es[3]) / (ts[-1] - ts[3]))
        g.close()
    gv = 1.0 * 1.0  # Gc v
    for r in rates:
        assert abs(r - gv) <= 0.1 * gv, rates
    assert abs(rates[0] - rates[1]) <= 0.05 * gv, rates


def test_automated_omega_matches_oracle_and_beats_plain_am():
    """Automated omega (two-block SOR optimum from the observed contraction) on the surfing
    steps: the GPU and the oracle apply the same rule and reach the same stationary points, and
    it needs fewer alternate-minimization iterations than omega = 1 (Table 1's trend)."""
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.surfing(nx=52, ny=26, ell=0.2, n_steps=8, t_max=1.2)
    g = S.Sim(w)
    g1 = S.Sim(w)
    p = Problem(w)
    auto = tight_opts(S, omega=1.0, omega_auto=1, omega_max=1.9)
    plain = tight_opts(S, omega=1.0)
    its_auto = its_plain = 0
    for (t, dT) in w.loads[:4]:
        rep = g.load_step(t, dT, auto)
        r = am.load_step(p, t, dT, omega=1.0, tol=1e-10, omega_auto=True, omega_max=1.9)
        assert rep["status"] == 0 and r["status"] == "converged"
        np.testing.assert_allclose(rep["energy"], r["energy"], rtol=1e-8, atol=1e-14)
        its_auto += rep["am_iters"]
        its_plain += g1.load_step(t, dT, plain)["am_iters"]
    u, a, _ = g.get_fields()
    assert rel_max(u, p.u) <= 1e-6 and np.abs(a - p.alpha).max() <= 1e-6
    assert its_auto < its_plain, (its_auto, its_plain)
