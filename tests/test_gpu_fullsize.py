"""GPU parity at the full sizes of the workloads the benchmark and the configurations name
(notched square 1024^2 and 512^2 crossed, thermal slab 1024 x 256 right), in the launch
configuration the benchmark times (mixed precision, CUDA graphs, single-block coarse tail).

The oracle cannot solve these meshes, so parity is checked on outputs it can compute one by
one and on properties that hold at any size:
  * operator outputs (K(alpha) x in FP64 and FP32, the damage gradient F = H alpha + g0, the
    Fischer-Burmeister residual and the active set) at sampled nodes -- corners, edges, tile
    boundaries and the ragged last tile column, random interior vertices and cell centres --
    each evaluated by the oracle's own assembly on the patch of elements around the node;
  * the total energy of the whole mesh (the oracle's vectorized energy handles the full mesh);
  * load steps of the benchmark's schedule: bounds and irreversibility, the optimality residual
    reduced from its value at the lifted start, and mixed precision against FP64 within 1e-6.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fe
from oracle.mesh import Mesh
from oracle.ncp import mcp_residual
from oracle.problem import Problem

from .gpu_util import need_gpu, rel_max

pytestmark = pytest.mark.gpu

TX = 32  # tile width of the stencil kernels (columns of vertices per block)


def _sample_nodes(w, rng, n_random=48):
    nx, ny = w.nx, w.ny
    nv = (nx + 1) * (ny + 1)
    vid = lambda i, j: j * (nx + 1) + i
    picks = {vid(0, 0), vid(nx, 0), vid(0, ny), vid(nx, ny), vid(nx // 2, 0), vid(nx // 2, ny),
             vid(0, ny // 2), vid(nx, ny // 2)}
    for i in (TX - 1, TX, TX + 1, nx - 1, nx):  # tile boundary and the ragged last column
        picks.add(vid(i, ny // 3))
    for _ in range(n_random):
        picks.add(vid(int(rng.integers(1, nx)), int(rng.integers(1, ny))))
    if w.kind == "crossed":
        for _ in range(n_random // 2):
            picks.add(nv + int(rng.integers(0, ny)) * nx + int(rng.integers(0, nx)))
        picks.add(nv + (ny - 1) * nx + nx - 1)
    return sorted(picks)


def _patch(w, node):
    """The oracle mesh of the cells around `node`, the global index of each patch node, and the
    node's index in the patch.  Every element touching the node lies in the patch."""
    nx, ny = w.nx, w.ny
    hx, hy = w.lx / nx, w.ly / ny
    nv = (nx + 1) * (ny + 1)
    if node < nv:
        j, i = divmod(node, nx + 1)
        ci0, ci1 = max(i - 1, 0), min(i, nx - 1)
        cj0, cj1 = max(j - 1, 0), min(j, ny - 1)
    else:
        cj, ci = divmod(node - nv, nx)
        ci0 = ci1 = ci
        cj0 = cj1 = cj
    m = Mesh(w.kind, ci1 - ci0 + 1, cj1 - cj0 + 1, w.x0 + ci0 * hx, w.y0 + cj0 * hy,
             (ci1 - ci0 + 1) * hx, (cj1 - cj0 + 1) * hy)
    gidx = np.empty(m.n_nodes, dtype=np.int64)
    for jp in range(m.ny + 1):
        for ip in range(m.nx + 1):
            gidx[m.vertex(ip, jp)] = (cj0 + jp) * (nx + 1) + ci0 + ip
    if w.kind == "crossed":
        for jp in range(m.ny):
            for ip in range(m.nx):
                gidx[m.centre(ip, jp)] = nv + (cj0 + jp) * nx + ci0 + ip
    pos = int(np.nonzero(gidx == node)[0][0])
    return m, gidx, pos


def _full_size_sim(w, seed):
    torch = need_gpu()
    from paper_1511_08463_gb300 import sim as S

    p = Problem(w)
    u, alpha = W.random_fields(w, seed, alpha_max=1.0, u_scale=0.05)
    alpha[p.a_fixed] = p.a_value[p.a_fixed]
    ap = np.minimum(alpha, 0.5 * alpha)
    ap[p.a_fixed] = p.a_value[p.a_fixed]
    g = S.Sim(w)
    g.set_fields(u, alpha, ap)
    g.set_load(0.7 * w.loads[-1][0], 0.0)
    u, alpha, ap = g.get_fields()  # u after the Dirichlet lift
    return torch, S, g, p, u, alpha, ap


WORKLOADS = {
    "notched_1024": lambda: W.notched_square(n=1024),
    "notched_512": lambda: W.notched_square(n=512),
    "thermal_1024x256": lambda: W.thermal_shock(),
}


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_operators_at_sampled_nodes(name):
    w = WORKLOADS[name]()
    torch, S, g, p, u, alpha, ap = _full_size_sim(w, seed=7)
    rng = np.random.default_rng(3)
    x = rng.normal(size=2 * p.mesh.n_nodes)
    xd = torch.tensor(x, device="cuda")
    y64 = g.elastic_apply(xd).cpu().numpy()
    y32 = g.elastic_apply(xd.float()).double().cpu().numpy()
    F, Phi, act, _ = [v.cpu().numpy() if hasattr(v, "cpu") else v for v in g.damage_gradient()]
    hi = p.upper()
    for node in _sample_nodes(w, rng):
        m, gi, k = _patch(w, node)
        geo = fe.Geometry(m)
        gi2 = np.stack([2 * gi, 2 * gi + 1], axis=1).ravel()
        K = fe.stiffness(p.mat, geo, alpha[gi]).tocsr()
        yref = (K @ x[gi2])[2 * k: 2 * k + 2]
        scale = (abs(K) @ np.abs(x[gi2]))[2 * k: 2 * k + 2] + 1e-300
        got = y64[2 * node: 2 * node + 2]
        assert np.all(np.abs(got - yref) <= 1e-12 * scale), (name, node, got, yref)
        got32 = y32[2 * node: 2 * node + 2]
        assert np.all(np.abs(got32 - yref) <= 2e-5 * scale), (name, node, got32, yref)
        # damage gradient at the lifted displacement (no eigenstrain: load set with dT = 0)
        q = fe.elastic_density(p.mat, geo, u[gi], 0.0)
        H = fe.damage_hessian(p.mat, geo, q).tocsr()
        Fp = H @ alpha[gi] + fe.damage_linear_term(p.mat, geo, q)
        fs = (abs(H) @ np.abs(alpha[gi]))[k] + np.abs(fe.damage_linear_term(p.mat, geo, q))[k]
        assert abs(F[node] - Fp[k]) <= 1e-11 * fs + 1e-300, (name, node, F[node], Fp[k])
        ph = mcp_residual(alpha[node:node + 1], Fp[k:k + 1], ap[node:node + 1], hi[node:node + 1],
                          np.ones(1, dtype=bool))[0]
        assert abs(Phi[node] - ph) <= 1e-11 * (fs + 1.0), (name, node, Phi[node], ph)


@pytest.mark.parametrize("name", ["notched_1024", "thermal_1024x256"])
def test_total_energy_full_mesh(name):
    w = WORKLOADS[name]()
    torch, S, g, p, u, alpha, ap = _full_size_sim(w, seed=9)
    dT = w.loads[len(w.loads) // 2][1]
    g.set_load(0.7 * w.loads[-1][0], dT)
    u, alpha, _ = g.get_fields()
    e_gpu = g.energy()
    e_ref = fe.energy(p.mat, p.geo, u, alpha, dT)
    np.testing.assert_allclose(e_gpu, e_ref, rtol=1e-11, atol=1e-300)


def test_benchmark_load_steps_properties():
    """The benchmark's first load steps at 1024^2 with its options (mixed, graphs, coarse tail):
    bounds, irreversibility, a reduced optimality residual, and FP64 agreement."""
    need_gpu()
    from paper_1511_08463_gb300 import sim as S

    w = W.notched_square(n=1024)
    opts = S.make_opts(algo="ORAM", omega=w.omega, precision="mixed")
    g = S.Sim(w)
    prev_alpha = None
    for (t, dT) in w.loads[:2]:
        u0, a0, _ = g.get_fields()
        g.set_load(t, dT)  # lifted start of the step: its optimality residual
        phi_start = g.full_residual()
        g.set_fields(u0, a0, None)
        rep = g.load_step(t, dT, opts)
        assert rep["status"] == 0
        u, a, ap = g.get_fields()
        assert np.all(a >= ap - 1e-15) and np.all(a <= 1.0 + 1e-15)
        if prev_alpha is not None:
            assert np.all(ap == prev_alpha) and np.all(a >= prev_alpha - 1e-15)
        prev_alpha = a.copy()
        assert g.full_residual() <= 1e-4 * phi_start
    # the same two steps in FP64: energies within 1e-6
    g64 = S.Sim(w)
    o64 = S.make_opts(algo="ORAM", omega=w.omega, precision="fp64")
    for (t, dT) in w.loads[:2]:
        r64 = g64.load_step(t, dT, o64)
    assert abs(rep["energy"][2] - r64["energy"][2]) <= 1e-6 * abs(r64["energy"][2])
    u64, a64, _ = g64.get_fields()
    assert rel_max(u, u64) <= 1e-5 and np.abs(a - a64).max() <= 1e-5
