"""GPU parity through crack propagation: the 32 x 32 notched square on its 50-step schedule to
t = 2 (AT1, ell = 4h, omega = 1.5), load steps 32-36, in which the crack starts from the notch and
runs through the ligament (energy drop at step 34).  Both sides start from the oracle's state after
step 31 (tests/golden/notched32_step31.npz, written by tests/golden/make_notched32_state.py).

Algorithm 2 (ORAM) and Algorithm 3 (ORAM-N) against the oracle's same algorithms, in FP64 at the
tight tolerances of the parity suite, and the mixed-precision path (FP32 inner solves, FP64
refinement) against the FP64 oracle.  The path is stable here (a mode-I crack on the symmetry
line), so fields are compared at every step."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import am
from oracle.problem import Problem
from tests.gpu_util import need_gpu, rel_max, tight_opts

pytestmark = pytest.mark.gpu

STEPS = range(31, 36)  # schedule indices of load steps 32..36
GOLD = os.path.join(os.path.dirname(__file__), "golden", "notched32_step31.npz")


def _start():
    z = np.load(GOLD)
    w = W.notched_square(n=int(z["n"]))
    p = Problem(w)
    p.u, p.alpha, p.alpha_prev = z["u"].copy(), z["alpha"].copy(), z["alpha_prev"].copy()
    return w, p, (z["u"], z["alpha"], z["alpha_prev"])


@pytest.fixture(scope="module")
def oracle_oram():
    w, p, _ = _start()
    out = []
    for k in STEPS:
        r = am.load_step(p, *w.loads[k], omega=w.omega, tol=1e-10, maxit=5000)
        assert r["status"] == "converged"
        out.append((r, p.u.copy(), p.alpha.copy()))
    return out


def _gpu_sim(state):
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.notched_square(n=32)
    g = S.Sim(w)
    g.set_fields(*state)
    return S, w, g


def test_oram_fp64_through_crack_propagation(oracle_oram):
    w, _, state = _start()
    S, w, g = _gpu_sim(state)
    opts = tight_opts(S, omega=w.omega)
    e_prev = None
    wbar_min = 2.0
    for (k, (r, u_ref, a_ref)) in zip(STEPS, oracle_oram):
        rep = g.load_step(*w.loads[k], opts)
        assert rep["status"] == 0 and rep["u_notconv"] == 0 and rep["alpha_notconv"] == 0
        np.testing.assert_allclose(rep["energy"], r["energy"], rtol=1e-8, atol=1e-14)
        u, a, ap = g.get_fields()
        assert rel_max(u, u_ref) <= 1e-6, (k, rel_max(u, u_ref))
        assert np.abs(a - a_ref).max() <= 1e-6, (k, np.abs(a - a_ref).max())
        assert np.all(a >= ap) and np.all(a <= 1.0)  # bounds and irreversibility
        assert rep["phi_norm"] <= 1e-6 * rep["phi_start"]
        wbar_min = min(wbar_min, rep["omega_bar_min"])
        if e_prev is not None and k == 33:
            assert rep["energy"][2] < e_prev  # the crack runs: the total energy drops
        e_prev = rep["energy"][2]
    # the feasibility rule of Section 2.1 reduced the damage relaxation below omega
    assert wbar_min < w.omega
    # the crack crossed the ligament: damaged band on y = 1/2 up to the right edge (the AT1
    # profile with ell = 4h peaks slightly below 1 at the nodes of this coarse mesh)
    z = np.load(GOLD)
    p = Problem(W.notched_square(n=int(z["n"])))
    on_line = (p.mesh.Y2 == 32) & (p.mesh.X2 >= 56)
    assert a[on_line].min() > 0.95


def test_oramn_fp64_through_crack_propagation():
    w, p, state = _start()
    S, w, g = _gpu_sim(state)
    opts = tight_opts(S, algo="ORAM_N", omega=w.omega, newton_rtol=1e-9)
    newton = 0
    for k in STEPS:
        rep = g.load_step(*w.loads[k], opts)
        ref = am.load_step_oramn(p, *w.loads[k], omega=w.omega, rtol=1e-9)
        assert rep["status"] == 0 and ref["status"] == "converged"
        np.testing.assert_allclose(rep["energy"], ref["energy"], rtol=1e-8, atol=1e-14)
        newton += rep["newton_iters"]
    u, a, _ = g.get_fields()
    assert rel_max(u, p.u) <= 1e-6 and np.abs(a - p.alpha).max() <= 1e-6
    assert newton > 0


def test_mixed_precision_through_crack_propagation(oracle_oram):
    """FP32 inner solves with FP64 residuals: per-step relative energy error <= 1e-6 against the
    FP64 oracle, fields within 1e-5, through the propagation steps."""
    w, _, state = _start()
    S, w, g = _gpu_sim(state)
    opts = tight_opts(S, omega=w.omega, precision="mixed", inner_rtol=1e-4)
    for (k, (r, u_ref, a_ref)) in zip(STEPS, oracle_oram):
        rep = g.load_step(*w.loads[k], opts)
        assert rep["status"] == 0
        assert abs(rep["energy"][2] - r["energy"][2]) <= 1e-6 * abs(r["energy"][2])
        u, a, _ = g.get_fields()
        assert rel_max(u, u_ref) <= 1e-5 and np.abs(a - a_ref).max() <= 1e-5
