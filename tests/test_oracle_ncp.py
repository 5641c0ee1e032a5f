"""Pins of the oracle's complementarity machinery and damage subproblem (Section 2.4)."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import am, fe
from oracle.ncp import box_qp, box_qp_bruteforce, mcp_residual, phi_fb
from oracle.problem import Problem


def test_fischer_burmeister_zero_set():
    vals = np.array([-2.0, -0.5, 0.0, 0.3, 1.7])
    for a in vals:
        for b in vals:
            z = abs(phi_fb(a, b)) < 1e-15
            assert z == (a >= 0 and b >= 0 and a * b == 0)


def test_mcp_residual_zero_iff_kkt():
    rng = np.random.default_rng(0)
    n = 200
    lo = rng.uniform(-1, 0, n)
    hi = lo + rng.uniform(0.1, 2, n)
    case = rng.integers(0, 3, n)
    x = np.where(case == 0, lo, np.where(case == 1, hi, 0.5 * (lo + hi)))
    F = np.where(case == 0, rng.uniform(0, 1, n), np.where(case == 1, -rng.uniform(0, 1, n), 0.0))
    b = np.ones(n, dtype=bool)
    assert np.abs(mcp_residual(x, F, lo, hi, b)).max() < 1e-15
    # break complementarity at one component of each kind: residual nonzero there only
    for k in range(3):
        i = np.nonzero(case == k)[0][0]
        F2 = F.copy()
        F2[i] = -0.3 if k == 0 else (0.3 if k == 1 else 0.2)
        r = mcp_residual(x, F2, lo, hi, b)
        assert abs(r[i]) > 1e-3 and np.abs(np.delete(r, i)).max() < 1e-15


@pytest.mark.parametrize("seed", range(12))
def test_box_qp_matches_bruteforce(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 8))
    A = rng.normal(size=(n, n))
    H = A @ A.T + 0.3 * np.eye(n)
    g = rng.normal(size=n) * 2
    lo = rng.uniform(-1.0, 0.0, n)
    hi = lo + rng.uniform(0.2, 1.5, n)
    x0 = np.clip(rng.normal(size=n), lo, hi)
    x, info = box_qp(sp.csr_matrix(H), g, x0, lo, hi)
    xb = box_qp_bruteforce(H, g, lo, hi)
    assert info["status"] == "converged"
    np.testing.assert_allclose(x, xb, atol=1e-10)


@pytest.mark.parametrize("model", ["AT1", "AT2"])
@pytest.mark.parametrize("kind", ["right", "crossed"])
def test_homogeneous_damage_closed_form(kind, model):
    """Uniform strain, no damage Dirichlet data, alpha_prev = 0: the exact P1 minimizer is
    uniform, AT1: alpha = clamp(1 - 3Gc/(8 ell q)), AT2: alpha = q/(q + Gc/ell)."""
    w = W.Workload(name="hom", kind=kind, nx=6, ny=4, x0=0, y0=0, lx=1.0, ly=0.8, ell=0.1,
                   model=model)
    p = Problem(w)
    G = np.array([[2.1, 0.4], [0.3, -0.7]])
    u = p.mesh.xy @ G.T
    q = fe.elastic_density(p.mat, p.geo, u)
    assert np.ptp(q) < 1e-12 * q.max()
    q0 = q[0]
    a, info = am.solve_alpha(p, u, np.zeros(p.mesh.n_nodes), 0.0)
    if model == "AT1":
        expect = np.clip(1 - 3 * w.Gc / (8 * w.ell * q0), 0, 1)
    else:
        expect = q0 / (q0 + w.Gc / w.ell)
    assert 0 < expect < 1
    np.testing.assert_allclose(a, expect, atol=1e-12)
    # below threshold (AT1): the bound is active everywhere
    if model == "AT1":
        a2, _ = am.solve_alpha(p, 0.2 * u, np.zeros(p.mesh.n_nodes), 0.0)
        assert np.abs(a2).max() == 0.0


def test_damage_qp_against_bruteforce_on_tiny_mesh():
    """Damage step on a 2x1 crossed mesh (8 nodes): full 3^n enumeration of bound patterns."""
    w = W.Workload(name="tiny", kind="crossed", nx=2, ny=1, x0=0, y0=0, lx=1.0, ly=0.5, ell=0.3)
    p = Problem(w)
    rng = np.random.default_rng(7)
    u = rng.normal(size=(p.mesh.n_nodes, 2)) * 1.5
    q = fe.elastic_density(p.mat, p.geo, u)
    H = fe.damage_hessian(p.mat, p.geo, q)
    g0 = fe.damage_linear_term(p.mat, p.geo, q)
    lo = rng.uniform(0, 0.3, p.mesh.n_nodes)
    p.alpha_prev = lo
    a, info = am.solve_alpha(p, u, lo.copy(), 0.0)
    ab = box_qp_bruteforce(H, g0, lo, np.ones_like(lo))
    np.testing.assert_allclose(a, ab, atol=1e-10)


def _random_mcp(seed, n=24, n_free=5):
    """A strictly convex QP's gradient F = Hx + g with box bounds on all but n_free components."""
    rng = np.random.default_rng(seed)
    A = sp.random(n, n, density=0.25, random_state=seed, format="csr")
    H = (A @ A.T + sp.eye(n) * 0.5).tocsr()
    g = rng.normal(size=n)
    lo = rng.uniform(-1.0, 0.0, n)
    hi = lo + rng.uniform(0.3, 1.5, n)
    bounded = np.ones(n, dtype=bool)
    bounded[rng.choice(n, n_free, replace=False)] = False
    return H, g, lo, hi, bounded, rng


@pytest.mark.parametrize("seed", range(4))
def test_merit_gradient_matches_central_differences(seed):
    """grad(||Phi||^2 / 2) of the steepest-descent fallback of Algorithm 4 against central
    differences, at points where both nested Fischer-Burmeister arguments are nonzero (Phi is
    smooth there).  Points inside the box, on a bound with the gradient pushing outwards, and
    outside the box; unbounded components use Phi = F."""
    from oracle.ncp import _merit_gradient

    H, g, lo, hi, bounded, rng = _random_mcp(seed)
    n = g.size
    merit = lambda x: 0.5 * float(np.sum(mcp_residual(x, H @ x + g, lo, hi, bounded) ** 2))
    for where in ("inside", "on_lower", "outside"):
        if where == "inside":
            x = lo + rng.uniform(0.2, 0.8, n) * (hi - lo)
        elif where == "on_lower":
            x = lo.copy()
        else:
            x = hi + rng.uniform(0.1, 0.3, n)
        x[~bounded] = rng.normal(size=int((~bounded).sum()))
        F = H @ x + g
        # stay away from the kink of phi: both arguments of each nested phi nonzero
        psi = phi_fb(hi - x, -F)
        ok = bounded & ((np.abs(hi - x) + np.abs(F)) > 1e-3) & ((np.abs(x - lo) + np.abs(psi)) > 1e-3)
        assert ok[bounded].all()
        grad = _merit_gradient(x, F, H, lo, hi, bounded)
        h = 1e-6
        fd = np.array([(merit(x + h * e) - merit(x - h * e)) / (2 * h) for e in np.eye(n)])
        np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-7 * max(1.0, np.abs(fd).max()))


def test_steepest_descent_fallback_branch_reaches_the_kkt_point():
    """Algorithm 4's fallback: when the Newton search fails (here a planted bad linear solve
    returning a zero step on the first iteration), the steepest-descent direction of
    the merit function is taken; the iteration still ends at the brute-force KKT point."""
    from oracle.ncp import rs_solve

    rng = np.random.default_rng(3)
    n = 6
    A = rng.normal(size=(n, n))
    H = sp.csr_matrix(A @ A.T + 0.5 * np.eye(n))
    g = rng.normal(size=n) * 2
    lo = rng.uniform(-1.0, 0.0, n)
    hi = lo + rng.uniform(0.2, 1.5, n)
    calls = {"n": 0}

    def bad_first(Ann, b):
        calls["n"] += 1
        d = np.linalg.solve(Ann.toarray(), b)
        return 0.0 * d if calls["n"] == 1 else d

    bounded = np.ones(n, dtype=bool)
    x0 = np.clip(rng.normal(size=n), lo, hi)
    x, info = rs_solve(lambda x: H @ x + g, lambda x: H, x0, lo, hi, bounded, rtol=1e-13,
                       linsolve=bad_first)
    assert info["status"] == "converged" and info["steepest"] >= 1
    np.testing.assert_allclose(x, box_qp_bruteforce(H, g, lo, hi), atol=1e-10)
    # steepest descent alone (no Newton direction): every step accepted, ||Phi|| reduced
    x1, info1 = rs_solve(lambda x: H @ x + g, lambda x: H, x0, lo, hi, bounded, rtol=1e-3,
                         maxit=200, directions=("steepest",))
    assert info1["status"] in ("converged", "maxit") and info1["steepest"] == info1["its"]
    assert info1["phi"] < 0.1 * info1["phi0"]
