"""Structured P1 triangulations of a rectangle (oracle; test infrastructure only).

The paper discretizes with piecewise-linear finite elements on simplicial meshes (Section 1.2,
last paragraphs).  Two structured families are built here:

* ``right``: every grid cell is cut by the diagonal from its lower-left to its upper-right
  corner (two triangles per cell);
* ``crossed``: every grid cell is cut by both diagonals, adding a cell-centre node (four
  triangles per cell).

Node order: the (nx+1) x (ny+1) vertex grid row-major (x fastest), then for ``crossed`` the
nx x ny centre grid row-major.  Every triangle is listed counter-clockwise.

Pins: number of nodes/elements, orientation and total area are checked in the tests.
"""
from __future__ import annotations

import numpy as np


class Mesh:
    def __init__(self, kind: str, nx: int, ny: int, x0: float, y0: float, lx: float, ly: float):
        if kind not in ("right", "crossed"):
            raise ValueError(kind)
        self.kind, self.nx, self.ny = kind, nx, ny
        self.x0, self.y0, self.lx, self.ly = x0, y0, lx, ly
        jj, ii = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        X2 = [2 * ii.ravel()]
        Y2 = [2 * jj.ravel()]
        self.n_vertices = (nx + 1) * (ny + 1)
        if kind == "crossed":
            jc, ic = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
            X2.append(2 * ic.ravel() + 1)
            Y2.append(2 * jc.ravel() + 1)
        self.X2 = np.concatenate(X2).astype(np.int64)
        self.Y2 = np.concatenate(Y2).astype(np.int64)
        self.n_nodes = self.X2.size
        self.xy = np.stack([x0 + lx * self.X2 / (2.0 * nx), y0 + ly * self.Y2 / (2.0 * ny)], axis=1)
        self.tris = self._triangles()

    def vertex(self, i, j):
        return j * (self.nx + 1) + i

    def centre(self, i, j):
        return self.n_vertices + j * self.nx + i

    def _triangles(self):
        nx, ny = self.nx, self.ny
        tri = []
        for j in range(ny):
            for i in range(nx):
                v00, v10 = self.vertex(i, j), self.vertex(i + 1, j)
                v01, v11 = self.vertex(i, j + 1), self.vertex(i + 1, j + 1)
                if self.kind == "right":
                    tri.append((v00, v10, v11))
                    tri.append((v00, v11, v01))
                else:
                    c = self.centre(i, j)
                    tri.append((v00, v10, c))
                    tri.append((v10, v11, c))
                    tri.append((v11, v01, c))
                    tri.append((v01, v00, c))
        return np.asarray(tri, dtype=np.int64)

    # boundary membership of nodes, by edge (only vertices lie on the boundary)
    def on_edge(self, edge: str) -> np.ndarray:
        if edge == "left":
            return self.X2 == 0
        if edge == "right":
            return self.X2 == 2 * self.nx
        if edge == "bottom":
            return self.Y2 == 0
        if edge == "top":
            return self.Y2 == 2 * self.ny
        raise ValueError(edge)


def prolongation(coarse: Mesh, fine: Mesh):
    """Nodal interpolation of coarse P1 functions at the fine nodes (a (n_fine x n_coarse)
    sparse matrix): each fine node is located in a coarse triangle and the coarse barycentric
    coordinates there are the weights."""
    import scipy.sparse as sp

    pts = fine.xy
    tri = coarse.tris
    P = coarse.xy[tri]  # (M,3,2)
    rows, cols, vals = [], [], []
    for a in range(pts.shape[0]):
        x, y = pts[a]
        # barycentric coordinates in every coarse triangle; pick one containing the point
        x0, y0 = P[:, 0, 0], P[:, 0, 1]
        x1, y1 = P[:, 1, 0], P[:, 1, 1]
        x2, y2 = P[:, 2, 0], P[:, 2, 1]
        det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)
        l1 = ((x - x0) * (y2 - y0) - (x2 - x0) * (y - y0)) / det
        l2 = ((x1 - x0) * (y - y0) - (x - x0) * (y1 - y0)) / det
        l0 = 1.0 - l1 - l2
        tol = -1e-12
        inside = np.nonzero((l0 >= tol) & (l1 >= tol) & (l2 >= tol))[0]
        t = inside[0]
        for k, lk in enumerate((l0[t], l1[t], l2[t])):
            if abs(lk) > 1e-14:
                rows.append(a)
                cols.append(tri[t, k])
                vals.append(lk)
    return sp.csr_matrix((vals, (rows, cols)), shape=(fine.n_nodes, coarse.n_nodes))
