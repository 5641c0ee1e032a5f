"""P1 finite-element model of the regularized fracture energy (oracle; test infrastructure only).

Follows Section 1.1, eq. (regenergy), with the AT1 model (w(a) = a, Section 1.1 end) and the AT2
model (w(a) = a^2, Section 1.1), a(a) = (1 - a)^2 + k_ell, c_w = 4 int_0^1 sqrt(w):

    E(u, a) = int 1/2 a(a) A0 eps(u):eps(u) + Gc/c_w (w(a)/ell + ell |grad a|^2)

and with the thermal eigenstrain of eq. (energytshock): eps_eff = eps(u) - beta T I, T from
eq. (tempfielderfc) evaluated at element centroids.  Derivatives follow Section 1.2 (E_u, E_alpha,
E_uu, E_ua, E_aa).  Everything is integrated exactly on P1 triangles: the strain is constant per
element, (1/|T|) int_T a(alpha_h) uses the P1 mass matrix, and w is linear or quadratic.

Pins (tests/test_oracle_fe.py): textbook CST stiffness reproduced independently, rigid-body modes
in the kernel, patch test, energy of homogeneous fields against closed forms, exact quadrature
rule check of the element coefficient, central finite differences of the energy (exact for these
quadratics), Galerkin identities on nested meshes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.special import erfc

from .mesh import Mesh


class Material:
    """Isotropic linear elasticity (plane strain by default) plus the damage model constants."""

    def __init__(self, E=1.0, nu=0.3, Gc=1.0, ell=0.05, k_ell=1e-6, model="AT1", plane="strain",
                 beta=0.0, pen=1.0):
        self.E, self.nu, self.Gc, self.ell, self.k_ell = E, nu, Gc, ell, k_ell
        self.model, self.plane, self.beta, self.pen = model, plane, beta, pen
        mu = E / (2.0 * (1.0 + nu))
        if plane == "strain":
            lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
        elif plane == "stress":
            lam = E * nu / (1.0 - nu * nu)
        else:
            raise ValueError(plane)
        self.lam, self.mu = lam, mu
        # Voigt matrix acting on (eps_xx, eps_yy, gamma_xy = 2 eps_xy): A0 eps : eps = e^T D e
        self.D = np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])
        if model == "AT1":
            self.cw = 8.0 / 3.0  # 4 int_0^1 sqrt(a) da
        elif model == "AT2":
            self.cw = 2.0  # 4 int_0^1 a da
        else:
            raise ValueError(model)

    @classmethod
    def from_workload(cls, w):
        return cls(E=w.E, nu=w.nu, Gc=w.Gc, ell=w.ell, k_ell=w.k_ell, model=w.model,
                   plane=w.plane, beta=w.beta, pen=w.pen)


class Geometry:
    """Per-element area and P1 basis-function gradients, computed from node coordinates."""

    def __init__(self, mesh: Mesh):
        self.mesh = mesh
        p = mesh.xy[mesh.tris]  # (M, 3, 2)
        x, y = p[..., 0], p[..., 1]
        det = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
        self.area = 0.5 * det
        g = np.empty((len(det), 3, 2))
        for k in range(3):
            a, b = (k + 1) % 3, (k + 2) % 3
            g[:, k, 0] = (y[:, a] - y[:, b]) / det
            g[:, k, 1] = (x[:, b] - x[:, a]) / det
        self.grad = g
        self.centroid = p.mean(axis=1)
        # strain-displacement matrices B (M, 3, 6), element dofs ordered (u0x,u0y,u1x,u1y,u2x,u2y)
        B = np.zeros((len(det), 3, 6))
        for k in range(3):
            B[:, 0, 2 * k] = g[:, k, 0]
            B[:, 1, 2 * k + 1] = g[:, k, 1]
            B[:, 2, 2 * k] = g[:, k, 1]
            B[:, 2, 2 * k + 1] = g[:, k, 0]
        self.B = B
        t = mesh.tris
        self.edofs = np.stack([2 * t[:, 0], 2 * t[:, 0] + 1, 2 * t[:, 1], 2 * t[:, 1] + 1,
                               2 * t[:, 2], 2 * t[:, 2] + 1], axis=1)


# P1 mass matrix on the reference simplex scaled by 1/|T|: int_T phi_i phi_j = |T| (1+d_ij)/12
MHAT = (np.ones((3, 3)) + np.eye(3)) / 12.0


def coefficient_mean(mat: Material, geo: Geometry, alpha: np.ndarray) -> np.ndarray:
    """abar_T = (1/|T|) int_T a(alpha_h) = 1 - 2 m_T + s_T + k_ell with the P1 mass matrix."""
    a = alpha[geo.mesh.tris]  # (M, 3)
    m = a.mean(axis=1)
    s = np.einsum("ti,ij,tj->t", a, MHAT, a)
    return 1.0 - 2.0 * m + s + mat.k_ell


def mode_I_displacement(mat: Material, KI: float, dx, dy):
    """Asymptotic Mode-I crack-tip displacement of linear elastic fracture mechanics, eq.
    (surfingloading) of Section 4.1: u = KI/(2 mu) sqrt(r/(2 pi)) (kappa - cos theta)
    (cos(theta/2), sin(theta/2)), with (r, theta) the polar coordinates of (dx, dy) around the tip
    (theta in (-pi, pi], theta = pi on the crack line behind the tip).  kappa = (3 - nu)/(1 + nu)
    as printed (plane stress); 3 - 4 nu for plane strain.  Returns (u_x, u_y)."""
    dx = np.asarray(dx, dtype=float)
    dy = np.asarray(dy, dtype=float)
    kappa = (3.0 - mat.nu) / (1.0 + mat.nu) if mat.plane == "stress" else 3.0 - 4.0 * mat.nu
    r = np.hypot(dx, dy)
    th = np.arctan2(dy, dx)
    amp = KI / (2.0 * mat.mu) * np.sqrt(r / (2.0 * np.pi)) * (kappa - np.cos(th))
    return amp * np.cos(0.5 * th), amp * np.sin(0.5 * th)


def temperature(mat: Material, geo: Geometry, dT: float) -> np.ndarray:
    """T at element centroids, eq. (tempfielderfc) with x2 measured from the exposed face y=y0."""
    y = geo.centroid[:, 1] - geo.mesh.y0
    return -dT * erfc(y / mat.pen)


def eigenstrain(mat: Material, geo: Geometry, dT: float) -> np.ndarray:
    """Voigt eigenstrain beta T I per element (gamma_xy = 0), eq. (energytshock)."""
    e0 = np.zeros((len(geo.area), 3))
    if mat.beta != 0.0 and dT != 0.0:
        bt = mat.beta * temperature(mat, geo, dT)
        e0[:, 0] = bt
        e0[:, 1] = bt
    return e0


def strains(geo: Geometry, u: np.ndarray) -> np.ndarray:
    """Voigt strain per element; u has shape (n_nodes, 2)."""
    ue = u.reshape(-1)[geo.edofs]  # (M, 6)
    return np.einsum("tij,tj->ti", geo.B, ue)


def elastic_density(mat: Material, geo: Geometry, u: np.ndarray, dT: float = 0.0) -> np.ndarray:
    """q_T = A0 eps_eff : eps_eff per element."""
    e = strains(geo, u) - eigenstrain(mat, geo, dT)
    return np.einsum("ti,ij,tj->t", e, mat.D, e)


def energy(mat: Material, geo: Geometry, u: np.ndarray, alpha: np.ndarray, dT: float = 0.0):
    """(elastic, surface, total) of eq. (regenergy) / (energytshock), exact on P1."""
    q = elastic_density(mat, geo, u, dT)
    abar = coefficient_mean(mat, geo, alpha)
    el = float(np.sum(0.5 * abar * q * geo.area))
    a = alpha[geo.mesh.tris]
    if mat.model == "AT1":
        wbar = a.mean(axis=1)
    else:
        wbar = np.einsum("ti,ij,tj->t", a, MHAT, a)
    ga = np.einsum("tk,tkd->td", a, geo.grad)
    surf = float(np.sum(mat.Gc / mat.cw * (wbar / mat.ell + mat.ell * np.sum(ga * ga, axis=1))
                        * geo.area))
    return el, surf, el + surf


def stiffness(mat: Material, geo: Geometry, alpha: np.ndarray) -> sp.csr_matrix:
    """Assembled K(alpha) = E_uu (eq. elasticity): sum_T abar_T |T| B^T D B."""
    return stiffness_from_coefficient(mat, geo, coefficient_mean(mat, geo, alpha))


def stiffness_from_coefficient(mat: Material, geo: Geometry, abar: np.ndarray) -> sp.csr_matrix:
    """sum_T abar_T |T| B_T^T D B_T for a given per-element coefficient abar."""
    ke = np.einsum("tki,kl,tlj->tij", geo.B, mat.D, geo.B) * (abar * geo.area)[:, None, None]
    n = 2 * geo.mesh.n_nodes
    rows = np.repeat(geo.edofs, 6, axis=1).ravel()
    cols = np.tile(geo.edofs, (1, 6)).ravel()
    return sp.csr_matrix((ke.ravel(), (rows, cols)), shape=(n, n))


def thermal_load(mat: Material, geo: Geometry, alpha: np.ndarray, dT: float) -> np.ndarray:
    """f with grad_u E = K(alpha) u - f: f = sum_T abar_T |T| B^T D eps0_T."""
    n = 2 * geo.mesh.n_nodes
    f = np.zeros(n)
    e0 = eigenstrain(mat, geo, dT)
    if not np.any(e0):
        return f
    abar = coefficient_mean(mat, geo, alpha)
    fe = np.einsum("tki,kl,tl->ti", geo.B, mat.D, e0) * (abar * geo.area)[:, None]
    np.add.at(f, geo.edofs.ravel(), fe.ravel())
    return f


def damage_constants(mat: Material):
    """(c1, c2, c3): Hessian = sum_T (q_T + c2) M_T + c1 L_T, gradient constant g0 uses c3."""
    c1 = 2.0 * mat.Gc * mat.ell / mat.cw
    if mat.model == "AT1":
        return c1, 0.0, mat.Gc / (mat.cw * mat.ell)
    return c1, 2.0 * mat.Gc / (mat.cw * mat.ell), 0.0


def damage_hessian(mat: Material, geo: Geometry, q: np.ndarray) -> sp.csr_matrix:
    """E_aa (eq. helmholtz) at fixed u: (a''/2 q + Gc w''/(c_w ell)) mass + 2 Gc ell/c_w stiffness."""
    _, c2, _ = damage_constants(mat)
    return damage_hessian_from_weight(mat, geo, q + c2)


def damage_hessian_from_weight(mat: Material, geo: Geometry, wgt: np.ndarray) -> sp.csr_matrix:
    """sum_T wgt_T M_T + c1 L_T for a given per-element mass weight."""
    c1, _, _ = damage_constants(mat)
    me = wgt[:, None, None] * geo.area[:, None, None] * MHAT[None]
    le = c1 * geo.area[:, None, None] * np.einsum("tid,tjd->tij", geo.grad, geo.grad)
    he = me + le
    t = geo.mesh.tris
    n = geo.mesh.n_nodes
    rows = np.repeat(t, 3, axis=1).ravel()
    cols = np.tile(t, (1, 3)).ravel()
    return sp.csr_matrix((he.ravel(), (rows, cols)), shape=(n, n))


def damage_linear_term(mat: Material, geo: Geometry, q: np.ndarray) -> np.ndarray:
    """g0 with E_alpha(alpha) = H alpha + g0 at fixed u (eq. kkt, second derivative form)."""
    _, _, c3 = damage_constants(mat)
    ge = (c3 - q) * geo.area / 3.0
    g0 = np.zeros(geo.mesh.n_nodes)
    np.add.at(g0, geo.mesh.tris.ravel(), np.repeat(ge, 3))
    return g0


def coupling(mat: Material, geo: Geometry, u: np.ndarray, alpha: np.ndarray,
             dT: float = 0.0) -> sp.csr_matrix:
    """E_ua (eq. offdiag) as a (2n x n) matrix: int a'(alpha) A0 eps_eff(u) : eps(v) beta.

    a'(alpha) = -2 (1 - alpha); per element int_T a'(alpha_h) phi_j = -2 |T| (1/3 - (M^ alpha)_j).
    """
    e = strains(geo, u) - eigenstrain(mat, geo, dT)
    sig = e @ mat.D  # (M,3) stress in Voigt (symmetric D)
    a = alpha[geo.mesh.tris]
    wj = -2.0 * geo.area[:, None] * (1.0 / 3.0 - a @ MHAT)  # (M,3): int a'(alpha_h) phi_j
    gi = np.einsum("tki,tk->ti", geo.B, sig)  # (M,6): B^T sigma
    be = gi[:, :, None] * wj[:, None, :]  # (M,6,3)
    t = geo.mesh.tris
    rows = np.repeat(geo.edofs, 3, axis=1).ravel()
    cols = np.tile(t, (1, 6)).ravel()
    n = geo.mesh.n_nodes
    return sp.csr_matrix((be.ravel(), (rows, cols)), shape=(2 * n, n))


def gradients(mat: Material, geo: Geometry, u: np.ndarray, alpha: np.ndarray, dT: float = 0.0):
    """(E_u, E_alpha) as nodal vectors (2n,), (n,)."""
    K = stiffness(mat, geo, alpha)
    Fu = K @ u.reshape(-1) - thermal_load(mat, geo, alpha, dT)
    q = elastic_density(mat, geo, u, dT)
    H = damage_hessian(mat, geo, q)
    Fa = H @ alpha + damage_linear_term(mat, geo, q)
    return Fu, Fa
