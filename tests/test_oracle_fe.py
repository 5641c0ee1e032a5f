"""Pins of the oracle's finite-element model against facts fixed by the mathematics.

Each check here is independent of the oracle's own formulas: textbook special cases, exact
quadrature rules, kernels of the operator, closed-form energies of homogeneous fields and exact
central differences of quadratic functions.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import fe
from oracle.mesh import Mesh, prolongation
from oracle.problem import Problem


def _mesh(kind, nx=5, ny=3, lx=1.3, ly=0.7):
    return Mesh(kind, nx, ny, -0.2, 0.1, lx, ly)


@pytest.mark.parametrize("kind", ["right", "crossed"])
def test_mesh_counts_orientation_area(kind):
    m = _mesh(kind)
    geo = fe.Geometry(m)
    per_cell = 2 if kind == "right" else 4
    assert m.tris.shape == (5 * 3 * per_cell, 3)
    assert m.n_nodes == 6 * 4 + (15 if kind == "crossed" else 0)
    assert np.all(geo.area > 0)  # counter-clockwise
    np.testing.assert_allclose(geo.area.sum(), 1.3 * 0.7, rtol=1e-14)
    np.testing.assert_allclose(geo.area, 1.3 * 0.7 / (15 * per_cell), rtol=1e-13)
    # every interior edge shared by exactly two triangles
    edges = np.sort(np.concatenate([m.tris[:, [0, 1]], m.tris[:, [1, 2]], m.tris[:, [2, 0]]]), axis=1)
    _, counts = np.unique(edges, axis=0, return_counts=True)
    assert set(counts.tolist()) <= {1, 2}


def _cst_textbook(xy, D):
    """Constant-strain triangle stiffness from the classical coordinate-difference form
    (unit thickness): B = 1/(2A) [[y23,0,y31,0,y12,0],[0,x32,0,x13,0,x21],[x32,y23,x13,y31,x21,y12]]."""
    (x1, y1), (x2, y2), (x3, y3) = xy
    A = 0.5 * ((x2 - x1) * (y3 - y1) - (x3 - x1) * (y2 - y1))
    y23, y31, y12 = y2 - y3, y3 - y1, y1 - y2
    x32, x13, x21 = x3 - x2, x1 - x3, x2 - x1
    B = np.array([[y23, 0, y31, 0, y12, 0], [0, x32, 0, x13, 0, x21],
                  [x32, y23, x13, y31, x21, y12]]) / (2 * A)
    return A * B.T @ D @ B


@pytest.mark.parametrize("kind", ["right", "crossed"])
def test_stiffness_alpha0_equals_textbook_cst(kind):
    m = _mesh(kind, nx=2, ny=2)
    geo = fe.Geometry(m)
    mat = fe.Material(E=2.0, nu=0.27, k_ell=0.0)
    # textbook plane-strain D written from E, nu directly
    E, nu = 2.0, 0.27
    D = E / ((1 + nu) * (1 - 2 * nu)) * np.array([[1 - nu, nu, 0], [nu, 1 - nu, 0],
                                                  [0, 0, (1 - 2 * nu) / 2]])
    K = fe.stiffness(mat, geo, np.zeros(m.n_nodes)).toarray()
    Kt = np.zeros_like(K)
    for tri in m.tris:
        ke = _cst_textbook(m.xy[tri], D)
        dofs = np.ravel([[2 * v, 2 * v + 1] for v in tri])
        Kt[np.ix_(dofs, dofs)] += ke
    np.testing.assert_allclose(K, Kt, rtol=1e-12, atol=1e-12 * np.abs(Kt).max())


@pytest.mark.parametrize("kind", ["right", "crossed"])
def test_rigid_body_modes_and_patch(kind):
    m = _mesh(kind)
    geo = fe.Geometry(m)
    mat = fe.Material()
    rng = np.random.default_rng(1)
    alpha = rng.uniform(0, 0.9, m.n_nodes)
    K = fe.stiffness(mat, geo, alpha)
    x, y = m.xy[:, 0], m.xy[:, 1]
    for mode in (np.stack([np.ones_like(x), 0 * x], 1), np.stack([0 * x, np.ones_like(x)], 1),
                 np.stack([-y, x], 1)):
        r = K @ mode.ravel()
        assert np.abs(r).max() < 1e-12 * abs(K).max()
    # symmetric, rank 2n-3
    Kd = K.toarray()
    np.testing.assert_allclose(Kd, Kd.T, atol=1e-14 * np.abs(Kd).max())
    ev = np.linalg.eigvalsh(Kd)
    assert np.sum(ev < 1e-10 * ev.max()) == 3 and ev.min() > -1e-10 * ev.max()
    # patch test with alpha == 0: linear u gives zero force at interior nodes
    K0 = fe.stiffness(mat, geo, np.zeros(m.n_nodes))
    G = np.array([[0.3, -0.2], [0.7, 0.1]])
    u = m.xy @ G.T + np.array([0.05, -0.3])
    r = (K0 @ u.ravel()).reshape(-1, 2)
    interior = (m.X2 > 0) & (m.X2 < 2 * m.nx) & (m.Y2 > 0) & (m.Y2 < 2 * m.ny)
    assert np.abs(r[interior]).max() < 1e-12


def test_energy_of_homogeneous_strain_closed_form():
    m = _mesh("crossed")
    geo = fe.Geometry(m)
    E, nu = 1.7, 0.22
    mat = fe.Material(E=E, nu=nu)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    G = np.array([[0.3, -0.2], [0.5, 0.1]])
    u = m.xy @ G.T
    eps = 0.5 * (G + G.T)
    psi = 0.5 * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps))
    c = 0.37
    alpha = np.full(m.n_nodes, c)
    el, surf, tot = fe.energy(mat, geo, u, alpha)
    area = 1.3 * 0.7
    np.testing.assert_allclose(el, ((1 - c) ** 2 + mat.k_ell) * psi * area, rtol=1e-13)
    np.testing.assert_allclose(surf, mat.Gc / (8 / 3) * (c / mat.ell) * area, rtol=1e-13)
    # AT2 and a linear damage field: gradient part ell |grad a|^2
    mat2 = fe.Material(E=E, nu=nu, model="AT2", ell=0.11)
    a = 0.2 + 0.3 * (m.xy[:, 0] + 0.2) / 1.3
    _, surf2, _ = fe.energy(mat2, geo, 0 * u, a)
    # int a^2 over the rectangle for a linear in x: exact
    x0, x1 = -0.2, 1.1
    ia2 = 0.7 * ((0.2 + 0.3) ** 3 - 0.2 ** 3) / (3 * 0.3 / 1.3)
    expect = mat2.Gc / 2.0 * (ia2 / 0.11 + 0.11 * (0.3 / 1.3) ** 2 * area)
    np.testing.assert_allclose(surf2, expect, rtol=1e-12)


def test_coefficient_mean_matches_exact_quadrature():
    """abar_T against the edge-midpoint rule, exact for quadratic polynomials on a triangle."""
    m = _mesh("right", nx=3, ny=2)
    geo = fe.Geometry(m)
    mat = fe.Material(k_ell=3e-4)
    rng = np.random.default_rng(2)
    alpha = rng.uniform(0, 1, m.n_nodes)
    abar = fe.coefficient_mean(mat, geo, alpha)
    for t, tri in enumerate(m.tris):
        a = alpha[tri]
        mids = [(a[0] + a[1]) / 2, (a[1] + a[2]) / 2, (a[2] + a[0]) / 2]
        quad = np.mean([(1 - v) ** 2 for v in mids]) + 3e-4
        assert abs(abar[t] - quad) < 1e-14


@pytest.mark.parametrize("model", ["AT1", "AT2"])
@pytest.mark.parametrize("kind", ["right", "crossed"])
def test_gradients_and_hessians_by_central_differences(kind, model):
    """The energy is quadratic in u (fixed alpha) and in alpha (fixed u): central differences
    are exact up to rounding."""
    m = _mesh(kind, nx=3, ny=2)
    geo = fe.Geometry(m)
    mat = fe.Material(model=model, beta=0.8, pen=0.3, ell=0.2)
    rng = np.random.default_rng(3)
    n = m.n_nodes
    u = rng.normal(size=(n, 2)) * 0.1
    alpha = rng.uniform(0, 1, n)
    dT = 0.7
    Fu, Fa = fe.gradients(mat, geo, u, alpha, dT)
    h = 1e-3
    E = lambda uu, aa: fe.energy(mat, geo, uu, aa, dT)[2]
    fdu = np.zeros(2 * n)
    for i in range(2 * n):
        up, um = u.copy().ravel(), u.copy().ravel()
        up[i] += h
        um[i] -= h
        fdu[i] = (E(up.reshape(-1, 2), alpha) - E(um.reshape(-1, 2), alpha)) / (2 * h)
    np.testing.assert_allclose(Fu, fdu, rtol=1e-8, atol=1e-9 * np.abs(Fu).max())
    fda = np.zeros(n)
    for i in range(n):
        ap, am_ = alpha.copy(), alpha.copy()
        ap[i] += h
        am_[i] -= h
        fda[i] = (E(u, ap) - E(u, am_)) / (2 * h)
    np.testing.assert_allclose(Fa, fda, rtol=1e-8, atol=1e-9 * np.abs(Fa).max())
    # Hessian blocks against differences of the gradients (gradients are affine in each block)
    p = rng.normal(size=2 * n)
    K = fe.stiffness(mat, geo, alpha)
    Fu_p = fe.gradients(mat, geo, u + p.reshape(-1, 2), alpha, dT)[0]
    np.testing.assert_allclose(K @ p, Fu_p - Fu, rtol=1e-9, atol=1e-10 * np.abs(K @ p).max())
    q = fe.elastic_density(mat, geo, u, dT)
    H = fe.damage_hessian(mat, geo, q)
    s = rng.normal(size=n)
    Fa_s = fe.gradients(mat, geo, u, alpha + s, dT)[1]
    np.testing.assert_allclose(H @ s, Fa_s - Fa, rtol=1e-9, atol=1e-10 * np.abs(H @ s).max())
    # mixed block: E_ua against central differences of E_u in alpha
    B = fe.coupling(mat, geo, u, alpha, dT)
    fdb = np.zeros((2 * n, n))
    for j in range(n):
        ap, am_ = alpha.copy(), alpha.copy()
        ap[j] += h
        am_[j] -= h
        fdb[:, j] = (fe.gradients(mat, geo, u, ap, dT)[0] - fe.gradients(mat, geo, u, am_, dT)[0]) / (2 * h)
    np.testing.assert_allclose(B.toarray(), fdb, rtol=1e-7, atol=1e-9 * np.abs(fdb).max())


def test_plane_strain_uniaxial_bar_solution():
    """Bar with u_x prescribed at both ends and one u_y pin: exact uniaxial stress state,
    sigma_xx = E/(1-nu^2) eps and eps_yy = -nu/(1-nu) eps in plane strain."""
    from oracle import am

    w = W.bar(nx=8, ny=2)
    p = Problem(w)
    p.lift(0.01)
    u = am.solve_u(p, p.alpha, 0.0)
    eps = 0.01 / w.lx
    nu = w.nu
    np.testing.assert_allclose(u[:, 0], eps * p.mesh.xy[:, 0], atol=1e-14)
    np.testing.assert_allclose(u[:, 1], -nu / (1 - nu) * eps * (p.mesh.xy[:, 1] - w.ly / 2),
                               atol=1e-14)
    el = fe.energy(p.mat, p.geo, u, p.alpha)[0]
    np.testing.assert_allclose(el, 0.5 * (1 + 1e-6) * w.E / (1 - nu ** 2) * eps ** 2 * w.lx * w.ly,
                               rtol=1e-12)


def test_thermal_homogeneous_state():
    """Uniform eigenstrain (penetration length >> slab) with top clamped, sides u_x = 0: the
    exact state has eps_xx = 0, sigma_yy = 0 and A0 eps_eff:eps_eff = E/(1-nu^2) (beta dT)^2."""
    from oracle import am

    w = W.thermal_shock(nx=8, ny=4, pen_over_ell=1e15)
    p = Problem(w)
    p.lift(0.0)
    dT = 0.37
    u = am.solve_u(p, p.alpha, dT)
    q = fe.elastic_density(p.mat, p.geo, u, dT)
    np.testing.assert_allclose(q, w.E / (1 - w.nu ** 2) * dT ** 2, rtol=1e-9)


@pytest.mark.parametrize("kind", ["right", "crossed"])
def test_galerkin_coarse_operator_is_mean_of_children(kind):
    """P^T K_h(abar) P == K_2h(mean of the four children's abar): exact because a coarse P1
    function has constant strain on each fine child triangle."""
    mc = Mesh(kind, 3, 2, 0.0, 0.0, 1.2, 0.8)
    mf = Mesh(kind, 6, 4, 0.0, 0.0, 1.2, 0.8)
    gc, gf = fe.Geometry(mc), fe.Geometry(mf)
    mat = fe.Material()
    rng = np.random.default_rng(4)
    af = rng.uniform(1e-3, 1.0, len(gf.area))
    P = prolongation(mc, mf)
    # locate each fine triangle's coarse parent by its centroid
    parent = np.empty(len(gf.area), dtype=int)
    tri = mc.tris
    for t, c in enumerate(gf.centroid):
        p = mc.xy[tri]
        x0, y0 = p[:, 0, 0], p[:, 0, 1]
        det = (p[:, 1, 0] - x0) * (p[:, 2, 1] - y0) - (p[:, 2, 0] - x0) * (p[:, 1, 1] - y0)
        l1 = ((c[0] - x0) * (p[:, 2, 1] - y0) - (p[:, 2, 0] - x0) * (c[1] - y0)) / det
        l2 = ((p[:, 1, 0] - x0) * (c[1] - y0) - (c[0] - x0) * (p[:, 1, 1] - y0)) / det
        inside = np.nonzero((l1 > 0) & (l2 > 0) & (1 - l1 - l2 > 0))[0]
        assert inside.size == 1
        parent[t] = inside[0]
    assert np.all(np.bincount(parent) == 4)
    ac = np.bincount(parent, weights=af) / 4.0
    P2 = np.kron(P.toarray(), np.eye(2))
    Kf = fe.stiffness_from_coefficient(mat, gf, af).toarray()
    Kc = fe.stiffness_from_coefficient(mat, gc, ac).toarray()
    np.testing.assert_allclose(P2.T @ Kf @ P2, Kc, atol=1e-13 * np.abs(Kc).max())
    # the damage Hessian: Laplacian part and constant-weight mass part are exact too
    wc = np.full(len(gc.area), 0.7)
    wf = np.full(len(gf.area), 0.7)
    Hf = fe.damage_hessian_from_weight(mat, gf, wf).toarray()
    Hc = fe.damage_hessian_from_weight(mat, gc, wc).toarray()
    Pd = P.toarray()
    np.testing.assert_allclose(Pd.T @ Hf @ Pd, Hc, atol=1e-13 * np.abs(Hc).max())


def test_thermal_temperature_at_centroids_against_hand_values():
    """eq. (tempfielderfc) at element centroids, against values worked by hand from the printed
    erf table (tests/golden/thermal_centroid_temperature.json): catches a wrong penetration
    scaling (erfc(x2/pen) vs erfc(x2/(2 pen))), a wrong sign, or x2 not measured from y0."""
    import json
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "thermal_centroid_temperature.json")
    with open(path) as fh:
        gold = json.load(fh)
    for case in gold["cases"]:
        m = case["mesh"]
        mesh = Mesh(m["kind"], m["nx"], m["ny"], m["x0"], m["y0"], m["lx"], m["ly"])
        geo = fe.Geometry(mesh)
        mat = fe.Material(beta=1.0, pen=case["pen"])
        T = fe.temperature(mat, geo, case["dT"])
        height = geo.centroid[:, 1] - m["y0"]
        table = case["centroid_height_to_T"]
        seen = set()
        for e in range(T.size):
            k = int(np.argmin([abs(height[e] - h) for h, _ in table]))
            assert abs(height[e] - table[k][0]) < 1e-12, f"unexpected centroid height {height[e]}"
            assert abs(T[e] - table[k][1]) <= 2e-10 * case["dT"], (e, T[e], table[k])
            seen.add(k)
        assert seen == set(range(len(table)))
        # the eigenstrain is beta T on both normal components, no shear (eq. energytshock)
        e0 = fe.eigenstrain(mat, geo, case["dT"])
        np.testing.assert_array_equal(e0[:, 0], T)
        np.testing.assert_array_equal(e0[:, 1], T)
        assert not np.any(e0[:, 2])


def test_mode_I_field_closed_forms_on_special_rays():
    """eq. (surfingloading): ahead of the tip (theta = 0) the opening component vanishes and
    u_x = K/(2 mu) sqrt(r/(2 pi)) (kappa - 1); on the crack faces (theta = pi) u_x = 0 and
    u_y = K/(2 mu) sqrt(r/(2 pi)) (kappa + 1); kappa = (3 - nu)/(1 + nu) in plane stress."""
    mat = fe.Material(nu=0.3, plane="stress")
    K, r = 1.7, 0.09
    kappa = (3 - 0.3) / 1.3
    a = K / (2 * mat.mu) * np.sqrt(r / (2 * np.pi))
    ux, uy = fe.mode_I_displacement(mat, K, r, 0.0)
    assert abs(uy) < 1e-15 and abs(ux - a * (kappa - 1)) < 1e-14
    ux, uy = fe.mode_I_displacement(mat, K, -r, 0.0)
    assert abs(ux) < 1e-15 and abs(uy - a * (kappa + 1)) < 1e-14
    ux, uy = fe.mode_I_displacement(mat, K, 0.0, r)  # theta = pi/2
    assert abs(ux - a * kappa / np.sqrt(2)) < 1e-14 and abs(uy - a * kappa / np.sqrt(2)) < 1e-14
    ux2, uy2 = fe.mode_I_displacement(mat, K, 0.0, -r)  # mirror: u_x even, u_y odd in y
    assert abs(ux2 - ux) < 1e-15 and abs(uy2 + uy) < 1e-15


@pytest.mark.parametrize("kind", ["right", "crossed"])
def test_mode_I_field_is_in_equilibrium(kind):
    """Away from the tip the Mode-I field solves the homogeneous Lame equations: the FE solution
    with that field as Dirichlet data on a square beside the tip converges to it at O(h^2)
    (a wrong kappa, sign or angle convention leaves an O(1) error)."""
    from oracle import am

    errs = []
    for n in (8, 16, 32):
        w = W.Workload(name="eq", kind=kind, nx=n, ny=n, x0=0.5, y0=-0.5, lx=1.0, ly=1.0,
                       plane="stress", fixed={e: {"ux": 1.0, "uy": 1.0} for e in W.EDGES},
                       mode_I=dict(KI=1.0, x_tip0=0.0, v=0.0, y_line=0.0))
        p = Problem(w)
        p.lift(0.0)
        u = am.solve_u(p, p.alpha, 0.0)
        ux, uy = fe.mode_I_displacement(p.mat, 1.0, p.mesh.xy[:, 0], p.mesh.xy[:, 1])
        ex = np.stack([ux, uy], axis=1)
        errs.append(np.abs(u - ex).max() / np.abs(ex).max())
    assert errs[-1] < 1e-3
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0
