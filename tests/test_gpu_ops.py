"""GPU parity of the single operators against the oracle, element by element, on seeded random
fields.  Meshes span several 32 x 8 tiles with ragged tails, plus degenerate 1-cell meshes."""
import numpy as np
import pytest

import workloads as W
from oracle import fe
from oracle.ncp import active_set, mcp_residual
from oracle.problem import Problem

from .gpu_util import need_gpu

pytestmark = pytest.mark.gpu

MESHES = [
    ("right", 70, 19), ("crossed", 45, 37), ("right", 1, 1), ("crossed", 1, 1), ("crossed", 2, 1),
    ("right", 33, 9),
]


def _workload(kind, nx, ny, model="AT1", thermal=False):
    fixed = {"left": {"ux": 0.0, "alpha": 0.0}, "bottom": {"uy": 0.0}, "right": {"ux": 1.0}}
    return W.Workload(name="ops", kind=kind, nx=nx, ny=ny, x0=-0.3, y0=0.2, lx=1.7, ly=0.9,
                      nu=0.27, ell=0.11, model=model, k_ell=1e-5, fixed=fixed,
                      pins=[(2 * nx, 2 * ny, "uy", 0.5)], beta=0.9 if thermal else 0.0,
                      pen=0.3)


def _setup(kind, nx, ny, seed, **kw):
    torch = need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = _workload(kind, nx, ny, **kw)
    p = Problem(w)
    u, alpha = W.random_fields(w, seed, alpha_max=1.0)
    alpha[p.a_fixed] = p.a_value[p.a_fixed]
    g = S.Sim(w)
    g.set_fields(u, alpha, np.minimum(alpha, 0.5 * alpha))
    return torch, S, w, p, g, u, alpha


@pytest.mark.parametrize("kind,nx,ny", MESHES)
def test_elastic_apply_fp64_and_fp32(kind, nx, ny):
    torch, S, w, p, g, u, alpha = _setup(kind, nx, ny, seed=11)
    rng = np.random.default_rng(5)
    x = rng.normal(size=2 * p.mesh.n_nodes)
    K = fe.stiffness(p.mat, p.geo, alpha)
    yref = K @ x
    scale = abs(K) @ np.abs(x) + 1e-300
    xd = torch.tensor(x, device="cuda")
    y = g.elastic_apply(xd).cpu().numpy()
    assert np.all(np.abs(y - yref) <= 1e-12 * scale + 1e-300)
    y32 = g.elastic_apply(xd.float()).double().cpu().numpy()
    assert np.all(np.abs(y32 - yref) <= 2e-5 * scale)
    # operator of the free dofs: rows and columns of prescribed dofs removed
    fr = ~p.u_fixed
    xm = np.where(fr, x, 0.0)
    ym = np.where(fr, K @ xm, 0.0)
    ymg = g.elastic_apply(xd, masked=True).cpu().numpy()
    assert np.all(np.abs(ymg - ym) <= 1e-12 * scale + 1e-300)


@pytest.mark.parametrize("kind,nx,ny", [("right", 70, 19), ("crossed", 45, 37), ("crossed", 1, 1)])
@pytest.mark.parametrize("thermal", [False, True])
def test_elastic_residual(kind, nx, ny, thermal):
    torch, S, w, p, g, u, alpha = _setup(kind, nx, ny, seed=12, thermal=thermal)
    t, dT = 0.37, (2.3 if thermal else 0.0)
    g.set_load(t, dT)
    p.lift(t)
    ug, _, _ = g.get_fields()
    np.testing.assert_array_equal(ug.ravel()[p.u_fixed], p.u.ravel()[p.u_fixed])
    uu = u.copy().ravel()
    uu[p.u_fixed] = p.u.ravel()[p.u_fixed]
    Fu, _ = fe.gradients(p.mat, p.geo, uu.reshape(-1, 2), alpha, dT)
    rref = np.where(~p.u_fixed, -Fu, 0.0)
    K = fe.stiffness(p.mat, p.geo, alpha)
    scale = abs(K) @ np.abs(uu) + np.abs(fe.thermal_load(p.mat, p.geo, alpha, dT)) + 1e-300
    # FP64, and the double-float arithmetic of the mixed path: both within 1e-12 of the terms
    for precision in ("fp64", "mixed"):
        r, n2 = g.elastic_residual(precision=precision)
        r = r.cpu().numpy()
        assert np.all(np.abs(r - rref) <= 1e-12 * scale), precision
        np.testing.assert_allclose(n2, rref @ rref, rtol=1e-10)


@pytest.mark.parametrize("kind,nx,ny", [("right", 70, 19), ("crossed", 45, 37), ("right", 1, 1)])
@pytest.mark.parametrize("model", ["AT1", "AT2"])
def test_damage_operator_gradient_residual_active_set(kind, nx, ny, model):
    torch, S, w, p, g, u, alpha = _setup(kind, nx, ny, seed=13, model=model, thermal=True)
    dT = 1.1
    g.set_load(0.0, dT)
    p.lift(0.0)
    uu = u.copy().ravel()
    uu[p.u_fixed] = p.u.ravel()[p.u_fixed]
    uu = uu.reshape(-1, 2)
    ap = np.minimum(alpha, 0.5 * alpha)
    p.alpha_prev = ap
    q = fe.elastic_density(p.mat, p.geo, uu, dT)
    H = fe.damage_hessian(p.mat, p.geo, q)
    g0 = fe.damage_linear_term(p.mat, p.geo, q)
    rng = np.random.default_rng(8)
    x = rng.normal(size=p.mesh.n_nodes)
    scale = abs(H) @ np.abs(x) + 1e-300
    xd = torch.tensor(x, device="cuda")
    y = g.damage_apply(xd).cpu().numpy()
    assert np.all(np.abs(y - H @ x) <= 1e-12 * scale)
    y32 = g.damage_apply(xd.float()).double().cpu().numpy()
    assert np.all(np.abs(y32 - H @ x) <= 2e-5 * scale)
    Fref = H @ alpha + g0
    fscale = abs(H) @ np.abs(alpha) + np.abs(g0) + 1e-300
    lo, hi = p.lower(), p.upper()
    Pref = mcp_residual(alpha, Fref, lo, hi, np.ones(alpha.size, dtype=bool))
    aref = active_set(alpha, Fref, lo, hi, np.ones(alpha.size, dtype=bool), 1e-10)
    for precision in ("fp64", "mixed"):  # FP64, and the mixed path's double-float
        F, Phi, act, n2 = g.damage_gradient(precision=precision)
        F, Phi, act = F.cpu().numpy(), Phi.cpu().numpy(), act.cpu().numpy()
        assert np.all(np.abs(F - Fref) <= 1e-12 * fscale), precision
        assert np.all(np.abs(Phi - Pref) <= 1e-10 * fscale)
        # decisions agree wherever F is not within rounding of zero
        clear = np.abs(Fref) > 1e-9 * fscale
        np.testing.assert_array_equal(act.astype(bool)[clear], aref[clear])
        np.testing.assert_allclose(n2, Pref @ Pref, rtol=1e-8)


@pytest.mark.parametrize("kind,nx,ny", [("right", 70, 19), ("crossed", 45, 37)])
@pytest.mark.parametrize("model", ["AT1", "AT2"])
def test_energy(kind, nx, ny, model):
    torch, S, w, p, g, u, alpha = _setup(kind, nx, ny, seed=14, model=model, thermal=True)
    g.set_load(0.0, 0.8)
    p.lift(0.0)
    uu = u.copy().ravel()
    uu[p.u_fixed] = p.u.ravel()[p.u_fixed]
    e = g.energy()
    eref = fe.energy(p.mat, p.geo, uu.reshape(-1, 2), alpha, 0.8)
    np.testing.assert_allclose(e, eref, rtol=1e-12)
