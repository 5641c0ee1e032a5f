"""Pins of the oracle's nonlinear solvers (Algorithms 1-3) against closed forms and invariants."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import am, fe
from oracle.problem import Problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")


def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def test_golden_constants():
    g = _golden()
    assert abs(fe.Material(model="AT1").cw - g["c_w"]["AT1"]["value"]) < 1e-15
    assert abs(fe.Material(model="AT2").cw - g["c_w"]["AT2"]["value"]) < 1e-15
    tc = W.bar_critical_displacement(1.0, 1.0, 0.3, 1.0, 0.05)
    assert abs(tc - g["bar_tc_plane_strain"]["value"]) < 5e-5
    dtc = W.thermal_critical_jump(1.0, 0.3, 1.0, 3.0 / 1024.0, 1.0)
    assert abs(dtc - g["thermal_dTc_plane_strain"]["value"]) < 5e-3


def test_bar_config_elastic_phase_and_critical_step():
    """Traction of a bar, 128x16 right mesh, AT1 (Section 4.2, plane-strain reading of t_c):
    alpha == 0 and E = 1/2 E' (t/L)^2 L H for t < t_c; first damage at step 14 of 20."""
    w = W.bar()
    p = Problem(w)
    Ep = w.E / (1 - w.nu ** 2)
    tc = W.bar_critical_displacement(w.lx, w.E, w.nu, w.Gc, w.ell)
    first_damaged = None
    for k, (t, dT) in enumerate(w.loads[:14], start=1):
        r = am.load_step(p, t, dT, omega=1.0, tol=1e-8)
        assert r["status"] == "converged"
        if t < tc:
            assert p.alpha.max() == 0.0
            el = r["energy"][0]
            np.testing.assert_allclose(el, 0.5 * (1 + w.k_ell) * Ep * (t / w.lx) ** 2 * w.lx * w.ly,
                                       rtol=1e-10)
        elif first_damaged is None and p.alpha.max() > 0:
            first_damaged = k
    assert first_damaged == 14


def test_1d_critical_stress():
    """nu = 0 bar without damage Dirichlet data is one-dimensional: homogeneous damage appears
    exactly when E t / L exceeds sigma_c = sqrt(3 Gc E / (8 ell)) (Section 4, first formula)."""
    w = W.bar(nx=16, ny=2, nu=0.0)
    w.fixed = {"left": {"ux": 0.0}, "right": {"ux": 1.0}}
    sc = np.sqrt(3 * w.Gc * w.E / (8 * w.ell))
    for factor, damaged in ((0.999, False), (1.001, True)):
        p = Problem(w)
        t = factor * sc * w.lx / w.E
        am.load_step(p, t, 0.0, omega=1.0, tol=1e-12)
        assert (p.alpha.max() > 0) == damaged
        if damaged:  # homogeneous stationary point: alpha = 1 - 3 Gc / (8 ell E eps^2)
            np.testing.assert_allclose(p.alpha, 1 - 3 * w.Gc / (8 * w.ell * w.E * (t / w.lx) ** 2),
                                       rtol=1e-8)


@pytest.mark.parametrize("ratio", [10, 20])
def test_developed_profile_surface_energy(ratio):
    """A fully developed AT1 crack (alpha = 1 on one column, u = 0) costs Gc per unit length,
    up to an O(h/ell) discretization error; the profile is (1 - |x|/(2 ell))^2."""
    ell = 0.05
    nx = int(round(1.0 / (ell / ratio)))
    nx += nx % 2
    w = W.Workload(name="profile", kind="right", nx=nx, ny=2, x0=-0.5, y0=0, lx=1.0,
                   ly=1.0 / nx * 2, ell=ell, alpha_boxes=[(nx, nx, 0, 4, 1.0)])
    p = Problem(w)
    a, info = am.solve_alpha(p, np.zeros((p.mesh.n_nodes, 2)), p.alpha.copy(), 0.0)
    surf = fe.energy(p.mat, p.geo, np.zeros((p.mesh.n_nodes, 2)), a)[1]
    rel = surf / (w.Gc * w.ly) - 1
    assert 0 < rel < 1.0 / ratio  # converges from above at O(h/ell)
    x = p.mesh.xy[:, 0]
    prof = np.clip(1 - np.abs(x) / (2 * ell), 0, None) ** 2
    assert np.abs(a - prof).max() < 2.0 / ratio


def test_oram_energy_monotone_bounds_irreversibility():
    """For any omega in (0, 2) each ORAM sweep cannot raise the energy (each block step moves
    along the segment towards the exact block minimizer); alpha stays in [alpha_prev, 1]."""
    w = W.notched_square(n=16, n_steps=10, t_max=1.2)
    for omega in (1.0, 1.6):
        p = Problem(w)
        prev = p.alpha.copy()
        for (t, dT) in w.loads[::3]:
            r = am.load_step(p, t, dT, omega=omega, tol=1e-7, record_energy=True)
            e = np.array(r["energies"][1:])
            assert np.all(np.diff(e) <= 1e-12 * np.abs(e).max())
            assert np.all(p.alpha >= prev) and np.all(p.alpha <= 1.0)
            prev = p.alpha.copy()
        assert p.alpha[~(p.alpha_prev == 1)].max() > 0.5  # the crack has grown


def test_oram_and_am_reach_same_stationary_point():
    """On a step with a unique nearby stationary point, AM and ORAM(omega=1.5) agree."""
    w = W.notched_square(n=16, n_steps=10, t_max=1.0)
    res = []
    for omega in (1.0, 1.5):
        p = Problem(w)
        for (t, dT) in w.loads[:6]:
            am.load_step(p, t, dT, omega=omega, tol=1e-11)
        res.append((p.u.copy(), p.alpha.copy()))
    np.testing.assert_allclose(res[0][1], res[1][1], atol=1e-7)
    np.testing.assert_allclose(res[0][0], res[1][0], atol=1e-7 * np.abs(res[0][0]).max())


def test_oramn_matches_oram_and_converges_fast():
    w = W.notched_square(n=16, n_steps=10, t_max=1.0)
    p1, p2 = Problem(w), Problem(w)
    for (t, dT) in w.loads[:6]:
        am.load_step(p1, t, dT, omega=1.5, tol=1e-11)
        r = am.load_step_oramn(p2, t, dT, omega=1.5, switch_tol=1e-2, rtol=1e-10)
        assert r["status"] == "converged"
    np.testing.assert_allclose(p1.alpha, p2.alpha, atol=1e-7)
    np.testing.assert_allclose(p1.u, p2.u, atol=1e-7 * np.abs(p1.u).max())


def test_thermal_no_damage_below_critical_jump():
    """Thermal shock (Section 4.3): purely elastic for dT below dT_c (plane-strain reading);
    above it damage appears first along the exposed face y = 0."""
    w = W.thermal_shock(nx=32, ny=8)
    dtc = W.thermal_critical_jump(w.E, w.nu, w.Gc, w.ell, w.beta)
    p = Problem(w)
    am.load_step(p, 0.0, 0.95 * dtc, omega=1.0, tol=1e-9)
    assert p.alpha.max() == 0.0
    am.load_step(p, 0.0, 1.05 * dtc, omega=1.0, tol=1e-9)
    assert p.alpha.max() > 0
    ybot = p.mesh.Y2 == 0
    # an x-homogeneous band along the exposed face (small end effects of the side conditions)
    assert p.alpha[ybot].min() > 0 and p.alpha[ybot].min() >= p.alpha[~ybot].max() - 1e-12
    assert np.ptp(p.alpha[ybot]) < 0.5 * p.alpha[ybot].max()


def test_omega_bar_midpoint_rule():
    """Reading of Section 2.1 (Algorithm 2's omega_bar): candidates omega, (1 + omega)/2, ...;
    the first for which alpha + omega_bar * dalpha stays in the box; omega itself when <= 1."""
    alpha = np.array([0.2, 0.5, 0.9])
    lo = np.array([0.2, 0.0, 0.9])
    hi = np.ones(3)
    dalpha = np.array([0.0, 0.3, 0.0])  # the largest feasible step is (1 - 0.5)/0.3 = 5/3
    assert am.omega_bar(alpha, dalpha, lo, hi, 1.8) == pytest.approx(1.4)  # 1.8 -> 1.4
    assert am.omega_bar(alpha, dalpha, lo, hi, 1.6) == pytest.approx(1.6)  # feasible as is
    dalpha = np.array([0.0, 0.4, 0.0])  # largest feasible step 1.25: 1.8 -> 1.4 -> 1.2
    assert am.omega_bar(alpha, dalpha, lo, hi, 1.8) == pytest.approx(1.2)
    dalpha = np.array([0.0, -0.45, 0.0])  # towards the lower bound: step <= 0.5/0.45 = 1.11
    assert am.omega_bar(alpha, dalpha, lo, hi, 1.8) == pytest.approx(1.1)  # 1.8 -> 1.4 -> 1.2 -> 1.1
    assert am.omega_bar(alpha, np.array([0.0, 5.0, 0.0]), lo, hi, 0.7) == 0.7  # omega <= 1
    # a step that is infeasible for every candidate above 1 falls back to 1 (the minimizer itself)
    assert am.omega_bar(alpha, np.array([0.0, 0.5, 0.0]), lo, hi, 1.9) == pytest.approx(1.0, abs=1e-8)


def test_dirichlet_lift_sets_prescribed_values_exactly():
    """Reading: the step's data t * g are written into u before the first iteration, and only on
    prescribed dofs."""
    w = W.bar(nx=16, ny=2, n_steps=5)
    p = Problem(w)
    rng = np.random.default_rng(0)
    p.u = rng.normal(size=p.u.shape)
    before = p.u.reshape(-1).copy()
    t = 0.37
    am.begin_step(p, t, 0.0)
    after = p.u.reshape(-1)
    np.testing.assert_array_equal(after[p.u_fixed], t * p.u_load[p.u_fixed])
    np.testing.assert_array_equal(after[~p.u_fixed], before[~p.u_fixed])
    assert np.any(p.u_load[p.u_fixed] != 0)  # the bar's end displacement is a genuine load


def test_surfing_dissipation_rate_is_griffith():
    """Surfing (Section 4.1): with K_I = sqrt(Gc E) the crack runs at the tip speed v, so the
    surface energy grows at Gc v (Griffith).  AT1 with h = ell/5 overestimates the surface
    energy of a developed band by a few percent; the rate must be within 10% of Gc v."""
    w = W.surfing(nx=52, ny=26, ell=0.2, n_steps=8, t_max=1.2)
    p = Problem(w)
    es, ts = [], []
    for (t, dT) in w.loads:
        r = am.load_step(p, t, dT, omega=w.omega, tol=1e-6)
        assert r["status"] == "converged"
        es.append(r["energy"][1])
        ts.append(t)
        assert np.all(p.alpha >= p.alpha_prev) and p.alpha.max() <= 1.0
    rate = (es[-1] - es[3]) / (ts[-1] - ts[3])  # after the start-up transient (t >= 0.6)
    assert abs(rate - w.Gc * w.mode_I["v"]) <= 0.1 * w.Gc * w.mode_I["v"], rate
    # the damage band lies on the crack line y = 0 ahead of the initial crack
    band = (np.abs(p.mesh.xy[:, 1]) < 1e-12) & (p.mesh.xy[:, 0] > 0.3) & (p.mesh.xy[:, 0] < 1.0)
    assert p.alpha[band].min() > 0.9


def test_omega_update_closed_forms():
    """The automated omega rule against the SOR theory it is read from (two-block consistently
    ordered case): at omega = 1 the contraction is mu^2, and the update returns the optimum
    2/(1 + sqrt(1 - mu^2)); at omega above the optimum the SOR eigenvalues have modulus
    omega - 1, and the update leaves omega unchanged; out-of-range input keeps omega."""
    for mu2 in (0.5, 0.9, 0.99):
        opt = 2.0 / (1.0 + np.sqrt(1.0 - mu2))
        assert abs(am.omega_update(mu2, 1.0, 1.99) - opt) < 1e-12
        # at the optimum itself the contraction is omega_opt - 1: fixed point
        assert abs(am.omega_update(opt - 1.0, opt, 1.99) - opt) < 1e-12
    assert am.omega_update(0.9, 1.0, 1.3) == 1.3  # clamped
    assert am.omega_update(1.2, 1.4, 1.9) == 1.4 and am.omega_update(0.0, 1.4, 1.9) == 1.4


def test_omega_update_on_a_linear_two_block_system():
    """Block Gauss-Seidel on a random SPD two-block system: the contraction observed at omega = 1
    fed to the rule gives the omega that minimizes the spectral radius of the block SOR matrix
    (checked against a dense scan of omega)."""
    rng = np.random.default_rng(4)
    n = 6
    B = rng.normal(size=(n, n))
    B *= 0.95 / np.linalg.norm(B, 2)  # [[I, B], [B^T, I]] is SPD, Jacobi radius 0.95
    Z = np.zeros((n, n))
    Dd = np.eye(2 * n)
    Lb = np.block([[Z, Z], [-B.T, Z]])
    Ub = np.block([[Z, -B], [Z, Z]])

    def rho(w):
        M = np.linalg.solve(Dd - w * Lb, w * Ub + (1 - w) * Dd)
        return float(np.abs(np.linalg.eigvals(M)).max())

    w_rule = am.omega_update(rho(1.0), 1.0, 1.99)
    ws = np.linspace(1.0, 1.99, 2000)
    w_best = ws[int(np.argmin([rho(w) for w in ws]))]
    assert abs(w_rule - w_best) < 2e-3
    assert rho(w_rule) < rho(1.0)
