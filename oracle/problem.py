"""Boundary data, bounds and state of one fracture problem (oracle; test infrastructure only).

Turns a ``workloads.Workload`` description into the admissible sets of Section 1.1:
C_ubar (Dirichlet displacement data on parts of the boundary) and D_alpha_prev (the box
alpha_prev <= alpha <= 1, with Dirichlet damage data).  Readings: the Dirichlet lift of each load
step is written into u before the step (so over-relaxation never acts on prescribed values), and
pre-existing cracks are nodes with alpha = alpha_prev = 1.
"""
from __future__ import annotations

import numpy as np

from .fe import Geometry, Material
from .mesh import Mesh

_COMP = {"ux": 0, "uy": 1, "alpha": 2}


class Problem:
    def __init__(self, w):
        self.w = w
        self.mesh = Mesh(w.kind, w.nx, w.ny, w.x0, w.y0, w.lx, w.ly)
        self.geo = Geometry(self.mesh)
        self.mat = Material.from_workload(w)
        n = self.mesh.n_nodes
        self.u_fixed = np.zeros(2 * n, dtype=bool)
        self.u_load = np.zeros(2 * n)  # prescribed value = t * u_load
        self.a_fixed = np.zeros(n, dtype=bool)
        self.a_value = np.zeros(n)
        for edge, comps in w.fixed.items():
            on = self.mesh.on_edge(edge)
            for comp, g in comps.items():
                c = _COMP[comp]
                if c < 2:
                    idx = 2 * np.nonzero(on)[0] + c
                    clash = self.u_fixed[idx] & (self.u_load[idx] != g)
                    if np.any(clash):
                        raise ValueError("conflicting Dirichlet data at a corner")
                    self.u_fixed[idx] = True
                    self.u_load[idx] = g
                else:
                    idx = np.nonzero(on)[0]
                    self.a_fixed[idx] = True
                    self.a_value[idx] = g
        for (x2, y2, comp, g) in w.pins:
            node = np.nonzero((self.mesh.X2 == x2) & (self.mesh.Y2 == y2))[0]
            if node.size != 1:
                raise ValueError("pin is not a node")
            c = _COMP[comp]
            if c < 2:
                self.u_fixed[2 * node[0] + c] = True
                self.u_load[2 * node[0] + c] = g
            else:
                self.a_fixed[node[0]] = True
                self.a_value[node[0]] = g
        # initial state: u = 0, alpha = alpha_prev = 0 except inside the damage boxes
        self.u = np.zeros((n, 2))
        self.alpha = np.zeros(n)
        for (xl, xh, yl, yh, v) in w.alpha_boxes:
            inside = (self.mesh.X2 >= xl) & (self.mesh.X2 <= xh) & (self.mesh.Y2 >= yl) & \
                     (self.mesh.Y2 <= yh)
            self.alpha[inside] = v
        self.alpha[self.a_fixed] = self.a_value[self.a_fixed]
        self.alpha_prev = self.alpha.copy()
        self.t = 0.0
        self.dT = 0.0

    # bounds of the damage box at the current step
    def lower(self):
        lo = self.alpha_prev.copy()
        lo[self.a_fixed] = self.a_value[self.a_fixed]
        return lo

    def upper(self):
        hi = np.ones_like(self.alpha_prev)
        hi[self.a_fixed] = self.a_value[self.a_fixed]
        return hi

    def lift(self, t: float):
        """Write the step's Dirichlet data into u: t*g, or, for a moving Mode-I crack (Section
        4.1, eq. surfingloading), g * u_bar(x - x_tip0 - v t, y - y_line)."""
        uf = self.u.reshape(-1)
        if self.w.mode_I is None:
            uf[self.u_fixed] = t * self.u_load[self.u_fixed]
            return
        from .fe import mode_I_displacement

        m = self.w.mode_I
        dx = self.mesh.xy[:, 0] - (m["x_tip0"] + m["v"] * t)
        dy = self.mesh.xy[:, 1] - m["y_line"]
        ux, uy = mode_I_displacement(self.mat, m["KI"], dx, dy)
        ub = np.stack([ux, uy], axis=1).reshape(-1)
        uf[self.u_fixed] = self.u_load[self.u_fixed] * ub[self.u_fixed]
