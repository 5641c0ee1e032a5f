"""Complementarity residuals and the reduced-space active-set method (oracle; test only).

Section 2.4: an MCP(F, l, u) holds at x iff for every i exactly one of
    F_i = 0 and l_i < x_i < u_i;   F_i >= 0 and x_i = l_i;   F_i <= 0 and x_i = u_i.
The Fischer-Burmeister NCP function phi(a, b) = sqrt(a^2 + b^2) - a - b vanishes iff a >= 0,
b >= 0, ab = 0.  The paper states the NCP case and calls the MCP extension straightforward; the
reading used here nests phi (Billups' construction):

    Phi_i = phi(x_i - l_i, phi(u_i - x_i, -F_i)),

which vanishes iff the MCP holds at i and reduces to phi(x_i - l_i, F_i) as u_i -> infinity.
Components without bounds (displacements) use Phi_i = F_i.

Algorithm 4 (reduced-space active set): active set A = {x_i <= l_i + zeta and F_i > 0} union
{x_i >= u_i - zeta and F_i < 0} (eq. reducedis, both bounds), plus every component whose box is a
single point; zeta being the zero tolerance, active components are taken to lie on their bound
and the step moves them onto it exactly (the paper's d_A = 0 up to that tolerance); solve
J_NN d_N = -F_N (eq. reducednewton); line search on ||Phi||^2 over
projected points pi[x + mu d], mu = 1, 1/2, ..., 2^-20, Armijo constant 1e-4; if it fails, the
steepest-descent direction of ||Phi||^2/2 is tried with the same search.

Pins (tests/test_oracle_ncp.py): phi's zero set, MCP residual zero iff KKT holds (checked
directly), brute-force enumeration of all 3^n bound patterns for small QPs, homogeneous closed
forms of the damage problem.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def phi_fb(a, b):
    return np.sqrt(a * a + b * b) - a - b


def _dphi(a, b):
    """An element of the generalized gradient of phi_fb at (a, b)."""
    r = np.sqrt(a * a + b * b)
    safe = r > 0
    da = np.where(safe, a / np.where(safe, r, 1.0), 1.0 / np.sqrt(2.0)) - 1.0
    db = np.where(safe, b / np.where(safe, r, 1.0), 1.0 / np.sqrt(2.0)) - 1.0
    return da, db


def mcp_residual(x, F, lo, hi, bounded):
    """Phi for the MCP; components with bounded=False use F itself."""
    Phi = np.array(F, dtype=float, copy=True)
    b = bounded
    Phi[b] = phi_fb(x[b] - lo[b], phi_fb(hi[b] - x[b], -F[b]))
    return Phi


def active_sets(x, F, lo, hi, bounded, zeta):
    """(lower-active, upper-active) index masks of eq. reducedis with both bounds; a box that is
    a single point counts as lower-active."""
    low = np.zeros(x.shape, dtype=bool)
    up = np.zeros(x.shape, dtype=bool)
    b = bounded
    low[b] = ((x[b] <= lo[b] + zeta) & (F[b] > 0)) | (hi[b] - lo[b] <= zeta)
    up[b] = ~low[b] & (x[b] >= hi[b] - zeta) & (F[b] < 0)
    return low, up


def active_set(x, F, lo, hi, bounded, zeta):
    low, up = active_sets(x, F, lo, hi, bounded, zeta)
    return low | up


def _merit_gradient(x, F, J, lo, hi, bounded):
    """grad of ||Phi||^2 / 2 = G^T Phi with G a generalized Jacobian of Phi."""
    Phi = mcp_residual(x, F, lo, hi, bounded)
    n = x.size
    # Phi_i = phi(x_i - l_i, psi_i), psi_i = phi(u_i - x_i, -F_i); unbounded: Phi_i = F_i
    diag = np.zeros(n)
    rowscale = np.ones(n)
    b = bounded
    psi = phi_fb(hi[b] - x[b], -F[b])
    pa, pb = _dphi(x[b] - lo[b], psi)
    qa, qb = _dphi(hi[b] - x[b], -F[b])
    # dPhi_i/dx_j = pa d_ij + pb (dpsi_i/dx_j); dpsi_i/dx_j = -qa d_ij - qb J_ij
    diag[b] = pa - pb * qa
    rowscale[b] = -pb * qb
    G = sp.diags(diag) + sp.diags(rowscale) @ J
    return G.T @ Phi


def rs_solve(F, J, x0, lo, hi, bounded, zeta=1e-10, atol=0.0, rtol=1e-12, maxit=200,
             linsolve=None, c_armijo=1e-4, mu_min=2.0 ** -20,
             directions=("newton", "steepest")):
    """Algorithm 4 for MCP(F, lo, hi).  F(x) -> vector, J(x) -> sparse Jacobian.

    directions: the search directions tried in order in every iteration ("newton": the reduced
    Newton step of eq. reducednewton; "steepest": minus the gradient of ||Phi||^2 / 2).

    Returns (x, info) with info = dict(its, phi0, phi, status, steepest) and status in
    {"converged", "maxit", "linesearch"}; steepest counts the iterations whose accepted step
    came from the steepest-descent direction.
    """
    if linsolve is None:
        linsolve = lambda A, b: spla.spsolve(A.tocsc(), b)
    x = np.where(bounded, np.clip(x0, lo, hi), x0).astype(float)
    Fx = F(x)
    Phi = mcp_residual(x, Fx, lo, hi, bounded)
    nphi0 = float(np.linalg.norm(Phi))
    tol = atol + rtol * nphi0
    its = 0
    n_steepest = 0
    status = "converged"
    while float(np.linalg.norm(Phi)) > tol:
        if its >= maxit:
            status = "maxit"
            break
        its += 1
        low, up = active_sets(x, Fx, lo, hi, bounded, zeta)
        N = ~(low | up)
        Jx = J(x).tocsr()
        d = np.zeros_like(x)
        if np.any(N):
            idx = np.nonzero(N)[0]
            d[idx] = linsolve(Jx[idx][:, idx], -Fx[idx])
        # active components lie within the zero tolerance of their bound: the step puts them on it
        d[low] = lo[low] - x[low]
        d[up] = hi[up] - x[up]
        m0 = float(Phi @ Phi)
        accepted = False
        for direction in directions:
            if direction == "steepest":
                d = -_merit_gradient(x, Fx, Jx, lo, hi, bounded)
            mu = 1.0
            while mu >= mu_min:
                xt = x + mu * d
                xt = np.where(bounded, np.clip(xt, lo, hi), xt)
                Ft = F(xt)
                Pt = mcp_residual(xt, Ft, lo, hi, bounded)
                if float(Pt @ Pt) <= (1.0 - 2.0 * c_armijo * mu) * m0:
                    accepted = True
                    break
                mu *= 0.5
            if accepted:
                n_steepest += direction == "steepest"
                break
        if not accepted:
            status = "linesearch"
            break
        x, Fx, Phi = xt, Ft, Pt
    return x, dict(its=its, phi0=nphi0, phi=float(np.linalg.norm(Phi)), status=status,
                   steepest=n_steepest)


def box_qp(H, g, x0, lo, hi, zeta=1e-10, rtol=1e-13, atol=0.0, maxit=200):
    """min 1/2 x^T H x + g^T x on lo <= x <= hi by Algorithm 4 with direct inner solves."""
    H = H.tocsr()
    bounded = np.ones(x0.size, dtype=bool)
    return rs_solve(lambda x: H @ x + g, lambda x: H, x0, lo, hi, bounded, zeta=zeta,
                    atol=atol, rtol=rtol, maxit=maxit)


def box_qp_bruteforce(H, g, lo, hi):
    """Exhaustive solution of a small strictly convex box QP: for every assignment of each
    component to {lower, upper, free}, solve the free block and keep the KKT-consistent point."""
    import itertools

    Hd = H.toarray() if sp.issparse(H) else np.asarray(H)
    n = len(g)
    best = None
    for pattern in itertools.product((0, 1, 2), repeat=n):
        pat = np.array(pattern)
        x = np.where(pat == 0, lo, np.where(pat == 1, hi, 0.0))
        fr = pat == 2
        if np.any(fr):
            rhs = -g[fr] - Hd[np.ix_(fr, ~fr)] @ x[~fr]
            x[fr] = np.linalg.solve(Hd[np.ix_(fr, fr)], rhs)
        if np.any(x < lo - 1e-12) or np.any(x > hi + 1e-12):
            continue
        F = Hd @ x + g
        ok = np.all(np.abs(F[fr]) <= 1e-9 * (1 + np.abs(g).max())) and \
            np.all(F[pat == 0] >= -1e-9) and np.all(F[pat == 1] <= 1e-9)
        if ok:
            val = 0.5 * x @ Hd @ x + g @ x
            if best is None or val < best[0]:
                best = (val, x)
    return None if best is None else best[1]
