"""Equiangular cubed-sphere column mesh for the oracle (test infrastructure only).

The paper runs on a C_n cubed sphere of 6 n^2 columns with a stretched vertical grid
(Sec. 5.1, C192 with 30 quadratically stretched levels); the grid is partitioned only
horizontally and every column holds a contiguous vertical structure (Sec. 4).  This
module builds that mesh from its plain geometric definition:

* panel p maps (xi, eta) in [-pi/4, pi/4]^2 to the sphere by the gnomonic projection of
  the cube face point listed in ``cube_point``;
* cell (p, j, i) spans xi in [-pi/4 + i d, -pi/4 + (i+1) d], eta likewise with j,
  d = pi / (2 n); column index col = p n^2 + j n + i;
* cell centre = image of the centre angles; areas are spherical quadrilateral areas from
  the corner vectors (two spherical triangles, Van Oosterom & Strackee 1983); edge
  lengths and centre distances are great-circle arcs; shallow atmosphere, radius R at
  all heights;
* neighbours are found by matching edge midpoints between cells (a k-d tree query), so
  panel-edge connectivity comes from the geometry, with no orientation table.

Directions are E (+i), W (-i), N (+j), S (-j).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial import cKDTree

DIRS = ("E", "W", "N", "S")


def cube_point(p: int, a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Point on face p of the cube [-1, 1]^3 for a = tan(xi), b = tan(eta)."""
    one = np.ones_like(a)
    if p == 0:
        v = (one, a, b)
    elif p == 1:
        v = (-a, one, b)
    elif p == 2:
        v = (-one, -a, b)
    elif p == 3:
        v = (a, -one, b)
    elif p == 4:
        v = (-b, a, one)
    elif p == 5:
        v = (b, a, -one)
    else:
        raise ValueError(p)
    return np.stack(v, axis=-1)


def _unit(v: np.ndarray) -> np.ndarray:
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def arc(u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Great-circle angle between unit vectors (atan2 of |u x v| and u . v)."""
    return np.arctan2(np.linalg.norm(np.cross(u, v), axis=-1), np.sum(u * v, axis=-1))


def triangle_area(a: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Unit-sphere area of the spherical triangle abc (Van Oosterom & Strackee)."""
    num = np.abs(np.sum(a * np.cross(b, c), axis=-1))
    den = 1.0 + np.sum(a * b, axis=-1) + np.sum(b * c, axis=-1) + np.sum(c * a, axis=-1)
    return 2.0 * np.arctan2(num, den)


class Mesh:
    """Horizontal geometry of C_n plus the vertical grid of its columns."""

    def __init__(self, n: int, z_if: np.ndarray, radius: float):
        self.n = n
        self.ncol = 6 * n * n
        self.R = float(radius)
        self.z_if = np.asarray(z_if, dtype=np.float64)
        self.nlev = len(self.z_if) - 1
        d = 0.5 * math.pi / n
        p, j, i = np.meshgrid(np.arange(6), np.arange(n), np.arange(n), indexing="ij")
        p, j, i = p.ravel(), j.ravel(), i.ravel()
        self.panel, self.j, self.i = p, j, i

        def sphere(xi, eta):
            out = np.empty(xi.shape + (3,))
            for q in range(6):
                m = p == q
                out[m] = cube_point(q, np.tan(xi[m]), np.tan(eta[m]))
            return _unit(out)

        x0 = -0.25 * math.pi + d * i
        y0 = -0.25 * math.pi + d * j
        c00 = sphere(x0, y0)
        c10 = sphere(x0 + d, y0)
        c11 = sphere(x0 + d, y0 + d)
        c01 = sphere(x0, y0 + d)
        self.centre = sphere(x0 + 0.5 * d, y0 + 0.5 * d)
        self.area = self.R ** 2 * (triangle_area(c00, c10, c11) + triangle_area(c00, c11, c01))

        # edge endpoints in the order E, W, N, S
        ends = [(c10, c11), (c00, c01), (c01, c11), (c00, c10)]
        self.edge_len = np.stack([self.R * arc(u, v) for u, v in ends])       # (4, ncol)
        mids = np.concatenate([_unit(u + v) for u, v in ends])              # (4 ncol, 3)
        tree = cKDTree(mids)
        dist, idx = tree.query(mids, k=2)
        own = np.arange(4 * self.ncol)
        other = np.where(idx[:, 0] == own, idx[:, 1], idx[:, 0])
        gap = np.where(idx[:, 0] == own, dist[:, 1], dist[:, 0])
        if np.any(gap > 1e-9) or np.any(other == own):
            raise RuntimeError("cubed-sphere edge matching failed")
        if np.any(other[other] != own):
            raise RuntimeError("cubed-sphere edge matching is not symmetric")
        self.nbr = (other % self.ncol).reshape(4, self.ncol)                 # (4, ncol)
        self.nbr_dir = (other // self.ncol).reshape(4, self.ncol)            # their side
        self.centre_dist = np.stack([self.R * arc(self.centre, self.centre[self.nbr[d_]])
                                     for d_ in range(4)])                    # (4, ncol)

        # vertical grid: layer depths, cell centres and centre-to-centre distances
        self.dz = np.diff(self.z_if)                                          # (nlev,)
        self.zc = 0.5 * (self.z_if[1:] + self.z_if[:-1])
        self.dzc = np.full(self.nlev + 1, np.nan)                             # at faces
        self.dzc[1:-1] = np.diff(self.zc)

    # ---- horizontal face numbering (the library's velocity-vector convention) ----
    def hfaces(self):
        """Horizontal faces of one level: (owner L, other R, owner side) arrays.

        A face joins columns c and c' = nbr[d][c]; it is listed once, under the column
        with the smaller index, ordered by (owner column, side E, W, N, S).
        """
        cols = np.arange(self.ncol)
        keep = (cols[None, :] < self.nbr).T            # (ncol, 4), row-major = (c, side)
        owner, side = np.nonzero(keep)
        return owner, self.nbr[side, owner], side

    def children(self, coarse: "Mesh") -> np.ndarray:
        """(4, ncol_coarse) fine columns making up each coarse column (nested meshes)."""
        assert self.n == 2 * coarse.n
        cn = coarse.n
        P, J, I = coarse.panel, coarse.j, coarse.i
        out = []
        for b in (0, 1):
            for a in (0, 1):
                out.append(P * self.n * self.n + (2 * J + b) * self.n + (2 * I + a))
        return np.stack(out)

    def parent(self) -> np.ndarray:
        """coarse column of every fine column of this mesh under 2x2 coarsening."""
        cn = self.n // 2
        return self.panel * cn * cn + (self.j // 2) * cn + (self.i // 2)
