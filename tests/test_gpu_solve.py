"""GPU parity of the subproblem solves and of whole load steps (Algorithms 1, 2 and 4) against
the oracle: fields within 1e-6 relative in the max norm, energies within 1e-8 relative (FP64);
the mixed-precision path within 1e-6 relative energy."""
import numpy as np
import pytest

import workloads as W
from oracle import am, fe
from oracle.problem import Problem

from .gpu_util import need_gpu, rel_max, tight_opts

pytestmark = pytest.mark.gpu


def _fields_close(g, p, tol=1e-6):
    u, a, ap = g.get_fields()
    assert np.abs(a - p.alpha).max() <= tol, np.abs(a - p.alpha).max()
    assert rel_max(u, p.u) <= tol, rel_max(u, p.u)
    assert np.abs(ap - p.alpha_prev).max() <= tol


@pytest.mark.parametrize("w", [W.notched_square(n=32), W.bar(nx=64, ny=8),
                               W.thermal_shock(nx=64, ny=16)], ids=["notched", "bar", "thermal"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_u_solve(w, precision):
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    p = Problem(w)
    rng = np.random.default_rng(3)
    alpha = rng.uniform(0, 0.9, p.mesh.n_nodes)
    alpha[p.a_fixed] = p.a_value[p.a_fixed]
    t, dT = w.loads[10]
    g = S.Sim(w)
    g.set_fields(alpha=alpha)
    g.set_load(t, dT)
    p.alpha = alpha
    p.lift(t)
    g.u_solve(tight_opts(S, precision=precision))
    uref = am.solve_u(p, alpha, dT)
    u, _, _ = g.get_fields()
    assert rel_max(u, uref) <= 1e-9


@pytest.mark.parametrize("model", ["AT1", "AT2"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_alpha_solve(model, precision):
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.notched_square(n=32, model=model)
    p = Problem(w)
    rng = np.random.default_rng(4)
    G = np.array([[0.6, 0.2], [0.1, 1.4]]) * (4.0 if model == "AT1" else 1.0)
    u = p.mesh.xy @ G.T + 0.05 * rng.normal(size=(p.mesh.n_nodes, 2))
    ap = np.where(p.alpha == 1.0, 1.0, rng.uniform(0, 0.2, p.mesh.n_nodes))
    g = S.Sim(w)
    g.set_fields(u=u, alpha=ap, alpha_prev=ap)
    g.set_load(0.0, 0.0)
    rep = g.alpha_solve(tight_opts(S, precision=precision))
    p.u, p.alpha, p.alpha_prev = u.copy(), ap.copy(), ap.copy()
    p.lift(0.0)  # the same Dirichlet lift the GPU applied in set_load
    aref, info = am.solve_alpha(p, p.u, ap.copy(), 0.0)
    _, a, _ = g.get_fields()
    assert np.abs(a - aref).max() <= 1e-8
    assert 0 < np.sum((aref > ap + 1e-12)) < aref.size  # a genuine box-constrained solve
    assert rep["rs_iters"] >= 1


def _run_steps(w, steps, omega, precision="fp64", **kw):
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    g = S.Sim(w)
    p = Problem(w)
    opts = tight_opts(S, omega=omega, precision=precision, **kw)
    reps = []
    for (t, dT) in steps:
        rep = g.load_step(t, dT, opts)
        r = am.load_step(p, t, dT, omega=omega, tol=1e-10)
        reps.append((rep, r))
    return g, p, reps


def test_notched_oram_load_steps():
    w = W.notched_square(n=32, n_steps=10, t_max=1.0)
    g, p, reps = _run_steps(w, w.loads[:7], omega=1.5)
    for rep, r in reps:
        np.testing.assert_allclose(rep["energy"], r["energy"], rtol=1e-8, atol=1e-14)
        assert rep["status"] == 0
    _fields_close(g, p)
    assert p.alpha[p.alpha_prev < 1].max() > 0.1  # damage has developed beyond the notch


def test_bar_am_through_nucleation():
    """Bar (Section 4.2) with a symmetry-breaking seed column near x = L/2 (at nucleation the
    branch would otherwise be chosen by round-off); AM (omega = 1)."""
    w = W.bar(nx=64, ny=8, n_steps=20, seed_column=True)
    g, p, reps = _run_steps(w, w.loads[11:16], omega=1.0)
    for rep, r in reps:
        np.testing.assert_allclose(rep["energy"], r["energy"], rtol=1e-8, atol=1e-14)
    _fields_close(g, p)
    assert p.alpha.max() > 0.9


def test_thermal_onset():
    w = W.thermal_shock(nx=64, ny=16, n_steps=40)
    g, p, reps = _run_steps(w, w.loads[8:12], omega=1.6)
    for rep, r in reps:
        np.testing.assert_allclose(rep["energy"], r["energy"], rtol=1e-8, atol=1e-14)
    _fields_close(g, p)


def test_at2_notched():
    w = W.notched_square(n=16, n_steps=10, t_max=1.0, model="AT2")
    g, p, reps = _run_steps(w, w.loads[:5], omega=1.3)
    for rep, r in reps:
        np.testing.assert_allclose(rep["energy"], r["energy"], rtol=1e-8, atol=1e-14)
    _fields_close(g, p)


def test_mixed_precision_energy_error():
    w = W.notched_square(n=32, n_steps=10, t_max=1.0)
    g, p, reps = _run_steps(w, w.loads[:6], omega=1.5, precision="mixed", inner_rtol=1e-4)
    for rep, r in reps:
        assert abs(rep["energy"][2] - r["energy"][2]) <= 1e-6 * abs(r["energy"][2])
    _fields_close(g, p, tol=1e-5)


def test_single_level_and_jacobi_paths():
    """Odd mesh sizes have no coarse level: the solver runs Chebyshev-preconditioned CG."""
    w = W.notched_square(n=18, n_steps=10, t_max=1.0)
    w.nx = w.ny = 17
    w.alpha_boxes = [(0, 17, 15, 19, 1.0)]
    g, p, reps = _run_steps(w, w.loads[:4], omega=1.5)
    assert g.levels == 1
    for rep, r in reps:
        np.testing.assert_allclose(rep["energy"], r["energy"], rtol=1e-8, atol=1e-14)
    _fields_close(g, p)


def test_graph_and_host_loops_agree_bitwise():
    """The CUDA-graph PCG (device-side loop) runs the same kernels in the same order as the
    host-driven loop, so the load steps agree bit for bit."""
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.notched_square(n=32, n_steps=10, t_max=1.0)
    out = []
    for graphs in (0, 1):
        g = S.Sim(w)
        opts = tight_opts(S, omega=1.5, precision="mixed", use_graphs=graphs)
        reps = [g.load_step(t, dT, opts) for (t, dT) in w.loads[:4]]
        out.append((g.get_fields(), reps))
    for a, b in zip(out[0][0], out[1][0]):
        np.testing.assert_array_equal(a, b)
    for ra, rb in zip(out[0][1], out[1][1]):
        assert ra["cg_iters_u"] == rb["cg_iters_u"] and ra["cg_iters_alpha"] == rb["cg_iters_alpha"]


@pytest.mark.parametrize("n", [32, 64])
def test_single_block_tail_matches_grid_vcycle(n):
    """The coarse levels run as one thread block (mg_tail=1) or one grid per step (mg_tail=0):
    the same V-cycle up to summation order, so the same solutions and iteration counts."""
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.notched_square(n=n, n_steps=10, t_max=1.0)
    out = []
    for tail in (1, 0):
        g = S.Sim(w)
        opts = tight_opts(S, omega=1.5, precision="mixed", mg_tail=tail)
        reps = [g.load_step(t, dT, opts) for (t, dT) in w.loads[:5]]
        out.append((g.get_fields(), reps))
    (u1, a1, _), r1 = out[0]
    (u0, a0, _), r0 = out[1]
    assert rel_max(u1, u0) <= 1e-8 and np.abs(a1 - a0).max() <= 1e-8
    for x, y in zip(r1, r0):
        np.testing.assert_allclose(x["energy"], y["energy"], rtol=1e-10, atol=1e-15)
        assert abs(x["cg_iters_u"] - y["cg_iters_u"]) <= max(2, 0.05 * y["cg_iters_u"])


def test_bar_config_full_schedule_against_oracle():
    """The 128 x 16 bar (Section 4.2) over its whole 20-step schedule, AM, FP64: every step's
    energies at 1e-8 and the final fields at 1e-6 against the oracle.  The nucleation step picks
    its branch by round-off in a perfectly symmetric bar, so both sides carry the same seed
    column (alpha_prev = 1e-3 next to the middle)."""
    w = W.bar(seed_column=True)
    g, p, reps = _run_steps(w, w.loads, omega=1.0)
    for rep, r in reps:
        np.testing.assert_allclose(rep["energy"], r["energy"], rtol=1e-8, atol=1e-14)
        assert rep["status"] == 0
    _fields_close(g, p)
    # elastic phase below t_c (no damage beyond the seed), then at step 14 a crack whose surface
    # energy is about Gc H = 0.1 (Section 4.2)
    assert reps[12][1]["energy"][1] < 1e-3 and p.alpha.max() > 0.99
    assert abs(reps[13][0]["energy"][1] - 0.1) < 0.01


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_load_exactly_at_damage_threshold_converges(precision):
    """A load step exactly at the AT1 critical load of the bar (t = t_c: the linear term of the
    damage gradient cancels, so what is left of it is the u-solve's error): the damage solve's
    tolerance follows the size of the gradient's terms, and the step converges like its
    neighbours; the bar is still undamaged (elastic energy 1/2 E' (t/L)^2 L H = 0.375)."""
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.bar(nx=128, ny=16, n_steps=30)  # t_20 = 1.5 t_c 20 / 30 = t_c
    g = S.Sim(w)
    o = S.make_opts(omega=1.0, precision=precision, am_maxit=500)
    for (t, dT) in w.loads[:20]:
        rep = g.load_step(t, dT, o)
        assert rep["status"] == 0 and rep["am_iters"] < 50
        assert rep["alpha_notconv"] == 0
    assert abs(rep["energy"][0] - 0.375) < 1e-4 and rep["energy"][1] < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_smoother_degree_one_matches_default(precision):
    """With one pre-smoothing step per level, the step from zero is formed inside the residual
    launch (grid levels) or pointwise (single-block tail): the multigrid changes, the converged load
    steps do not.  Degree 1 on every level, with and without the tail, against the default."""
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.notched_square(n=48, n_steps=6, t_max=1.5)
    out = []
    for deg, cdeg, tail in ((2, 0, 1), (1, 1, 1), (1, 1, 0)):
        g = S.Sim(w)
        o = tight_opts(S, omega=w.omega, precision=precision, mg_degree=deg, mg_coarse_degree=cdeg,
                       mg_tail=tail)
        for (t, dT) in w.loads:
            r = g.load_step(t, dT, o)
            assert r["status"] == 0
        out.append((r["energy"][2], g.get_fields()))
    for e, f in out[1:]:
        assert abs(e - out[0][0]) <= 1e-8 * abs(out[0][0])
        assert rel_max(f[0], out[0][1][0]) <= 1e-6
        assert np.abs(f[1] - out[0][1][1]).max() <= 1e-6
