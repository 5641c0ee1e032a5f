"""Alternate minimization, its over-relaxation and its composition with Newton (oracle; test only).

* u-subproblem (Algorithm 1/2, first line of the loop): E_u(u, alpha; v) = 0 for all v in C_0,
  i.e. K(alpha)_ff u_f = f_f - K(alpha)_fd ubar_d, solved by sparse LU (the paper's Section 5.1-5.2
  experiments use LU for every linear solve).
* alpha-subproblem: the variational inequality E_alpha(u, alpha; beta) >= 0 on D_alpha_prev is
  the strictly convex box QP 1/2 a^T H a + g0^T a, solved by Algorithm 4 with direct solves.
* ORAM (Algorithm 2): u <- u + omega (u~ - u); alpha <- alpha + omega_bar (alpha~ - alpha) with
  omega_bar chosen by the recursive midpoint rule of Section 2.1 (omega, (1+omega)/2, ...): the
  first candidate keeping alpha in the box; omega_bar = omega when omega <= 1; after 30 halvings
  omega_bar = 1 (alpha~ itself is feasible).  AM (Algorithm 1) is ORAM with omega = 1.
* ORAM-N (Algorithm 3): ORAM until ||Phi|| / ||Phi^0|| <= switch tolerance, then the coupled
  reduced-space Newton method (Algorithm 4 on (u, alpha) with Jacobian [[K, B], [B^T, H]],
  Section 3.3) with backtracking; if Newton does not converge, return to ORAM.

Readings where the paper is silent: the Dirichlet lift is applied before the first iteration
of every load step (over-relaxing u across changed boundary data would overshoot them); the stopping rule is max|alpha^k - alpha^{k-1}| <= tol together with
max|u^k - u^{k-1}| <= tol * max|u^k| (the second part catches an over-relaxed u that has not
settled while alpha no longer moves).

Pins (tests/test_oracle_am.py): energy non-increasing per sweep, bounds and irreversibility, the
bar's elastic phase and critical load, 1D closed forms (critical stress, fully developed profile
energy G_c), ORAM(omega=1) equals AM, ORAM-N and ORAM converge to the same stationary point.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe
from .ncp import box_qp, mcp_residual, rs_solve


def solve_u(prob, alpha, dT):
    """Minimizer of E(., alpha) over C_ubar, keeping the prescribed values already in prob.u."""
    mat, geo = prob.mat, prob.geo
    K = fe.stiffness(mat, geo, alpha).tocsr()
    f = fe.thermal_load(mat, geo, alpha, dT)
    u = prob.u.reshape(-1).copy()
    fr = ~prob.u_fixed
    rhs = f[fr] - K[fr][:, prob.u_fixed] @ u[prob.u_fixed]
    u[fr] = spla.spsolve(K[fr][:, fr].tocsc(), rhs)
    return u.reshape(-1, 2)


def solve_alpha(prob, u, alpha0, dT, zeta=1e-10, rtol=1e-13):
    """Minimizer of E(u, .) over the box lower() <= alpha <= upper() (Algorithm 4, exact solves)."""
    q = fe.elastic_density(prob.mat, prob.geo, u, dT)
    H = fe.damage_hessian(prob.mat, prob.geo, q)
    g0 = fe.damage_linear_term(prob.mat, prob.geo, q)
    a, info = box_qp(H, g0, alpha0, prob.lower(), prob.upper(), zeta=zeta, rtol=rtol)
    return a, info


def omega_bar(alpha, dalpha, lo, hi, omega, max_halvings=30):
    """Section 2.1: try omega, then the midpoint of [1, omega], recursively, until feasible."""
    if omega <= 1.0:
        return omega
    w = omega
    for _ in range(max_halvings + 1):
        trial = alpha + w * dalpha
        if np.all(trial >= lo) and np.all(trial <= hi):
            return w
        w = 0.5 * (1.0 + w)
    return 1.0


def full_residual(prob, u, alpha, dT):
    """Phi of the optimality system (eq. kkt): E_u on free displacement dofs, the MCP residual of
    E_alpha on the damage box."""
    Fu, Fa = fe.gradients(prob.mat, prob.geo, u, alpha, dT)
    Pu = Fu[~prob.u_fixed]
    Pa = mcp_residual(alpha, Fa, prob.lower(), prob.upper(), np.ones(alpha.size, dtype=bool))
    return np.concatenate([Pu, Pa])


def begin_step(prob, t, dT):
    """alpha_prev <- alpha (irreversibility w.r.t. the previous step) and Dirichlet lift."""
    prob.alpha_prev = prob.alpha.copy()
    prob.t, prob.dT = t, dT
    prob.lift(t)


def oram_iteration(prob, omega, dT, zeta=1e-10, qp_rtol=1e-13):
    """One pass of the loop of Algorithm 2; updates prob.u, prob.alpha; returns diagnostics."""
    u_old, a_old = prob.u.copy(), prob.alpha.copy()
    ut = solve_u(prob, a_old, dT)
    u_new = u_old + omega * (ut - u_old)
    at, qinfo = solve_alpha(prob, u_new, a_old, dT, zeta=zeta, rtol=qp_rtol)
    da = at - a_old
    lo, hi = prob.lower(), prob.upper()
    wb = omega_bar(a_old, da, lo, hi, omega)
    a_new = np.clip(a_old + wb * da, lo, hi)
    prob.u, prob.alpha = u_new, a_new
    du = float(np.max(np.abs(u_new - u_old))) if u_new.size else 0.0
    unorm = float(np.max(np.abs(u_new))) if u_new.size else 0.0
    return dict(dalpha=float(np.max(np.abs(a_new - a_old))) if a_new.size else 0.0,
                du_rel=du / unorm if unorm > 0 else du, omega_bar=wb, qp_its=qinfo["its"],
                qp_status=qinfo["status"])


# Automated choice of omega (Section 2.2 conjectures that the best omega minimizes the spectral
# radius of the SOR iteration matrix and leaves its automation open).  Reading: for a two-block
# consistently ordered system, an SOR eigenvalue lam and a Jacobi eigenvalue mu satisfy
# (lam + omega - 1)^2 = lam omega^2 mu^2, and the optimum is omega = 2 / (1 + sqrt(1 - mu^2)).
OMEGA_PERIOD = 5  # iterations between two estimates


def omega_update(rho, omega, omega_max):
    """New omega from the observed contraction rho at the current omega: mu^2 from the SOR
    eigenvalue relation, then the optimum, clamped to [1, omega_max]; omega itself if rho carries
    no estimate (rho outside (0, 1) or mu^2 outside [0, 1))."""
    if not (0.0 < rho < 1.0):
        return omega
    mu2 = (rho + omega - 1.0) ** 2 / (rho * omega * omega)
    if not (0.0 <= mu2 < 1.0):
        return omega
    return min(omega_max, max(1.0, 2.0 / (1.0 + np.sqrt(1.0 - mu2))))


def load_step(prob, t, dT=0.0, omega=1.0, tol=1e-6, maxit=2000, zeta=1e-10, qp_rtol=1e-13,
              record_energy=False, omega_auto=False, omega_max=1.9):
    """Algorithm 2 (Algorithm 1 when omega = 1) for one load step.  omega_auto: every
    OMEGA_PERIOD iterations omega is replaced by omega_update of the contraction of the damage
    change over those iterations, rho = (dalpha_k / dalpha_{k-P})^(1/P)."""
    begin_step(prob, t, dT)
    hist = []
    energies = [fe.energy(prob.mat, prob.geo, prob.u, prob.alpha, dT)[2]] if record_energy else []
    status = "maxit"
    k = 0
    for k in range(1, maxit + 1):
        d = oram_iteration(prob, omega, dT, zeta=zeta, qp_rtol=qp_rtol)
        d["omega"] = omega
        hist.append(d)
        if omega_auto and k % OMEGA_PERIOD == 0 and k > OMEGA_PERIOD:
            prev = hist[k - 1 - OMEGA_PERIOD]["dalpha"]
            if prev > 0.0 and d["dalpha"] > 0.0:
                omega = omega_update((d["dalpha"] / prev) ** (1.0 / OMEGA_PERIOD), omega,
                                     omega_max)
        if record_energy:
            energies.append(fe.energy(prob.mat, prob.geo, prob.u, prob.alpha, dT)[2])
        if d["dalpha"] <= tol and d["du_rel"] <= tol:
            status = "converged"
            break
    return dict(its=k, status=status, hist=hist, energies=energies,
                energy=fe.energy(prob.mat, prob.geo, prob.u, prob.alpha, dT))


# ---------------------------------------------------------------------------------------------
# ORAM-N (Algorithm 3) with the coupled reduced-space Newton method (Algorithm 4, Section 3.3)
# ---------------------------------------------------------------------------------------------
def _coupled_system(prob, dT):
    n = prob.mesh.n_nodes
    fr = np.nonzero(~prob.u_fixed)[0]
    nf = fr.size

    def unpack(z):
        u = prob.u.reshape(-1).copy()
        u[fr] = z[:nf]
        return u.reshape(-1, 2), z[nf:]

    def F(z):
        u, a = unpack(z)
        Fu, Fa = fe.gradients(prob.mat, prob.geo, u, a, dT)
        return np.concatenate([Fu[fr], Fa])

    def J(z):
        u, a = unpack(z)
        K = fe.stiffness(prob.mat, prob.geo, a).tocsr()[fr][:, fr]
        B = fe.coupling(prob.mat, prob.geo, u, a, dT).tocsr()[fr]
        q = fe.elastic_density(prob.mat, prob.geo, u, dT)
        H = fe.damage_hessian(prob.mat, prob.geo, q)
        return sp.bmat([[K, B], [B.T, H]]).tocsr()

    lo = np.concatenate([np.full(nf, -np.inf), prob.lower()])
    hi = np.concatenate([np.full(nf, np.inf), prob.upper()])
    bounded = np.concatenate([np.zeros(nf, dtype=bool), np.ones(n, dtype=bool)])
    z0 = np.concatenate([prob.u.reshape(-1)[fr], prob.alpha])
    return F, J, lo, hi, bounded, z0, unpack


def load_step_oramn(prob, t, dT=0.0, omega=1.0, switch_tol=1e-2, rtol=1e-9, atol=0.0,
                    max_outer=50, max_oram=2000, newton_maxit=20, zeta=1e-10):
    """Algorithm 3 for one load step: returns counts and the final residual norm."""
    begin_step(prob, t, dT)
    phi_start = float(np.linalg.norm(full_residual(prob, prob.u, prob.alpha, dT)))
    tol = atol + rtol * phi_start
    oram_its = newton_its = 0
    status = "maxit"
    for _ in range(max_outer):
        phi0 = float(np.linalg.norm(full_residual(prob, prob.u, prob.alpha, dT)))
        if phi0 <= tol:
            status = "converged"
            break
        phik = phi0
        while phik / phi0 > switch_tol and phik > tol and oram_its < max_oram:
            oram_iteration(prob, omega, dT, zeta=zeta)
            oram_its += 1
            phik = float(np.linalg.norm(full_residual(prob, prob.u, prob.alpha, dT)))
        if phik <= tol:
            status = "converged"
            break
        F, J, lo, hi, bounded, z0, unpack = _coupled_system(prob, dT)
        z, info = rs_solve(F, J, z0, lo, hi, bounded, zeta=zeta, atol=tol, rtol=0.0,
                           maxit=newton_maxit)
        newton_its += info["its"]
        if info["phi"] < phik:  # keep Newton's result only if it reduced the residual
            u, a = unpack(z)
            prob.u, prob.alpha = u, a
        if info["status"] == "converged":
            status = "converged"
            break
        if oram_its >= max_oram:
            break
    phi = float(np.linalg.norm(full_residual(prob, prob.u, prob.alpha, dT)))
    return dict(status=status, oram_its=oram_its, newton_its=newton_its, phi=phi,
                phi_start=phi_start, energy=fe.energy(prob.mat, prob.geo, prob.u, prob.alpha, dT))
