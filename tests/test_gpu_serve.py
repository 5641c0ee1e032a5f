"""Serving loop and concurrent batch: a job's result is the same alone, in a mix of jobs and
through a plain resident Sim (the kernels and reductions are deterministic, so bit for bit);
admission respects the arena; arrival times and per-step latencies are consistent."""
import numpy as np
import pytest

import workloads as W

from .gpu_util import need_gpu

pytestmark = pytest.mark.gpu


def _mix():
    return [W.notched_square(n=32, n_steps=6, t_max=1.6),
            W.bar(nx=64, ny=8, n_steps=6),
            W.notched_square(n=48, n_steps=5, t_max=1.6, model="AT2"),
            W.thermal_shock(nx=64, ny=16, n_steps=6),
            W.notched_square(n=16, n_steps=8, t_max=1.6)]


def _opts(S, w):
    return S.make_opts(omega=w.omega, precision="mixed")


def _direct(S, w):
    g = S.Sim(w)
    reps = [g.load_step(t, dT, _opts(S, w), allow_notconv=True) for (t, dT) in w.loads]
    u, a, _ = g.get_fields()
    return u, a, reps


def test_serve_alone_equals_mix_equals_direct():
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    jobs = _mix()
    arena = 4 * sum(S.Server.footprint(w) for w in jobs)
    alone = S.Server(arena, workers=1)
    r0 = alone.wait(alone.submit(jobs[0], opts=_opts(S, jobs[0])))
    alone.close()
    srv = S.Server(arena, workers=4)
    ids = [srv.submit(w, opts=_opts(S, w), arrival=0.0) for w in jobs]
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["jobs_done"] == len(jobs) and st["max_active"] >= 2
    np.testing.assert_array_equal(res[0]["u"], r0["u"])
    np.testing.assert_array_equal(res[0]["alpha"], r0["alpha"])
    for w, r in zip(jobs, res):
        assert r["status"] in (0, 3) and r["steps_done"] == len(w.loads)
        u, a, reps = _direct(S, w)
        np.testing.assert_array_equal(r["u"], u)
        np.testing.assert_array_equal(r["alpha"], a)
        for x, y in zip(r["reports"], reps):
            assert x["energy"] == y["energy"] and x["am_iters"] == y["am_iters"]
        assert np.all(r["latency"] > 0)
    assert any(r["alpha"].max() > 0.5 for r in res)  # cracks grew in the mix


def test_admission_by_footprint():
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    jobs = [W.notched_square(n=32, n_steps=3, t_max=0.6) for _ in range(3)]
    fp = S.Server.footprint(jobs[0])
    srv = S.Server(int(1.5 * fp), workers=3)  # room for one job at a time
    ids = [srv.submit(w, opts=_opts(S, w), arrival=0.0) for w in jobs]
    res = [srv.wait(i) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["max_active"] == 1 and st["arena_peak"] <= st["arena_bytes"]
    spans = sorted((r["admitted"], r["finished"]) for r in res)
    for (a0, f0), (a1, f1) in zip(spans, spans[1:]):
        assert a1 >= f0
    # later jobs waited for memory: their first-step latency includes the wait
    assert res[2]["latency"][0] >= res[2]["admitted"] - res[2]["arrival"]


def test_arrivals_and_rejection():
    need_gpu()
    from paper_1511_08463_gb300 import binding as B
    from paper_1511_08463_gb300 import sim as S

    w = W.notched_square(n=16, n_steps=2, t_max=0.4)
    fp = S.Server.footprint(w)
    srv = S.Server(4 * fp, workers=2)
    late = srv.submit(w, opts=_opts(S, w), arrival=srv.now() + 0.3)
    early = srv.submit(w, opts=_opts(S, w), arrival=0.0)
    r_late, r_early = srv.wait(late), srv.wait(early)
    assert r_late["admitted"] >= r_late["arrival"] and r_early["admitted"] < r_late["arrival"]
    with pytest.raises(B.PFError):
        srv.submit(W.notched_square(n=64, n_steps=2), opts=_opts(S, w))  # larger than the arena
    srv.close()


def test_solve_batch_concurrent_equals_sequential():
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    ws = [W.notched_square(n=n, n_steps=1, t_max=t) for n, t in
          [(16, 1.5), (32, 1.4), (48, 1.2), (64, 1.0), (32, 1.6), (16, 0.8)]]
    opts = S.make_opts(omega=ws[0].omega, precision="mixed", batch_workers=3)  # as in _direct
    ctx = S.Context(0)
    sims = [S.Sim(w, ctx=ctx) for w in ws]
    st, reps = S.solve_batch(sims, [w.loads[0] for w in ws], opts=opts, ctx=ctx)
    assert st in (0, 3)
    for w, g, r in zip(ws, sims, reps):
        u, a, r1 = _direct(S, w)
        ub, ab, _ = g.get_fields()
        np.testing.assert_array_equal(ub, u)
        np.testing.assert_array_equal(ab, a)
        assert r["energy"] == r1[0]["energy"]


def test_served_jobs_match_oracle():
    """Jobs that ran through the serving loop, next to each other, against the oracle's
    Algorithm 2 on the same schedules: energies at every load step; fields at the end where the
    path is stable (the notched square; where the bar's crack nucleates is a bifurcation decided
    by rounding, so only its energies are compared)."""
    need_gpu()
    from oracle import am
    from oracle.problem import Problem
    from paper_1511_08463_gb300 import sim as S

    from .gpu_util import rel_max, tight_opts

    jobs = [W.notched_square(n=16, n_steps=8, t_max=1.6), W.bar(nx=64, ny=8, n_steps=6)]
    srv = S.Server(4 * sum(S.Server.footprint(w) for w in jobs), workers=2)
    ids = [srv.submit(w, opts=tight_opts(S, omega=w.omega), arrival=0.0) for w in jobs]
    res = [srv.wait(i) for i in ids]
    srv.close()
    for w, r in zip(jobs, res):
        assert r["status"] == 0 and r["steps_done"] == len(w.loads)
        p = Problem(w)
        for (t, dT), rep in zip(w.loads, r["reports"]):
            o = am.load_step(p, t, dT, omega=w.omega, tol=1e-10, maxit=5000)
            assert o["status"] == "converged"
            # absolute floor: at the bar's critical load the damage is zero up to rounding
            np.testing.assert_allclose(rep["energy"], o["energy"], rtol=1e-8,
                                       atol=1e-10 * abs(o["energy"][2]))
        if w.name.startswith("notched"):
            assert rel_max(r["u"], p.u) <= 1e-6
            assert np.abs(r["alpha"] - p.alpha).max() <= 1e-6
    assert res[0]["alpha"].max() > 0.5  # the notched job grew a crack
