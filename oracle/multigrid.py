"""Horizontal-only multigrid hierarchy and the V-cycle (oracle).

Test infrastructure only.  Follows Maynard, Melvin & Mueller (arXiv 2002.00756), Sec. 3.6:

* the hierarchy W3 = W3^(1) > W3^(2) > ... > W3^(L) coarsens only horizontally; on the
  equiangular cubed sphere the coarse cell of C_{n/2} is exactly the union of 2x2 fine
  cells of the same panel, and the vertical grid is unchanged;
* prolongation is the natural injection (Eq. prolongation): every fine cell takes the
  value of the coarse cell containing it;
* restriction is its dual on the dual (residual) space: the integrated residual of a
  coarse cell is the sum of the integrated residuals of its children.  In the strong,
  volume-normalised form used here that reads b_c = sum_children V_ch r_ch / V_c;
* coarse operators are rediscretised from the reference profiles represented on the
  coarse level (Sec. 3.6, last paragraph before Algorithm 1): background factors (and,
  for the mixed system, the vertical-face mass factors) are volume-/area-weighted means
  of the children;
* Algorithm 1: recursive V-cycle with n_pre / n_post block-Jacobi smoothing steps,
  residual, restriction, zero coarse initial guess, recursion and prolongation; on the
  coarsest level CoarseSolve = n_coarse block-Jacobi sweeps (Sec. 3.6, text after
  Algorithm 1; n_coarse = 4, Sec. 5.1) starting from zero.
"""
from __future__ import annotations

import numpy as np

from .geometry import Mesh
from .helmholtz import Level, Level9


def restrict_field(fine: Mesh, coarse: Mesh, f: np.ndarray) -> np.ndarray:
    """Volume-weighted mean of the 4 children: sum_ch A_ch f_ch / A_c, level by level."""
    ch = fine.children(coarse)
    f = np.asarray(f, dtype=np.float64)
    acc = np.zeros(f.shape[:-1] + (coarse.ncol,))
    for q in range(4):
        acc += fine.area[ch[q]] * f[..., ch[q]]
    return acc / coarse.area


def restrict_side_field(fine: Mesh, coarse: Mesh, f: np.ndarray) -> np.ndarray:
    """Per-side face field (4, ncol): the edge-length-weighted mean of the two fine faces
    that make up each coarse face (children q = 2b + a lying on that side)."""
    ch = fine.children(coarse)
    f = np.asarray(f, dtype=np.float64).reshape(4, fine.ncol)
    on_side = ((1, 3), (0, 2), (2, 3), (0, 1))      # E: a = 1, W: a = 0, N: b = 1, S: b = 0
    out = np.empty((4, coarse.ncol))
    for d in range(4):
        w = [fine.edge_len[d][ch[q]] for q in on_side[d]]
        v = [f[d][ch[q]] for q in on_side[d]]
        out[d] = (w[0] * v[0] + w[1] * v[1]) / (w[0] + w[1])
    return out


def restrict(fine: Mesh, coarse: Mesh, r: np.ndarray) -> np.ndarray:
    """Restrict(R): dual of injection, b_c = sum_ch V_ch r_ch / V_c (same layer depth)."""
    return restrict_field(fine, coarse, np.asarray(r).reshape(fine.nlev, fine.ncol))


def prolongate(fine: Mesh, xc: np.ndarray) -> np.ndarray:
    """Prolongate(x_c): natural injection, each child takes its parent's value."""
    return np.asarray(xc).reshape(fine.nlev, -1)[:, fine.parent()]


class Hierarchy:
    """Meshes and rediscretised operators on levels 1..L (index 0 = finest)."""

    def __init__(self, n: int, z_if: np.ndarray, radius: float, levels: int, g: np.ndarray,
                 cs_dt: float, mu: np.ndarray | None = None, mu_h: np.ndarray | None = None,
                 gamma2: float = 0.0):
        if n % (1 << (levels - 1)):
            raise ValueError("C_n must be divisible by 2^(L-1)")
        self.meshes = [Mesh(n >> l, z_if, radius) for l in range(levels)]
        nlev = self.meshes[0].nlev
        g = np.asarray(g, dtype=np.float64).reshape(nlev, -1)
        mu = None if mu is None else np.asarray(mu, dtype=np.float64).reshape(nlev + 1, -1)
        self.levels = []
        for l, m in enumerate(self.meshes):
            if l > 0:
                g = restrict_field(self.meshes[l - 1], m, g)
                if mu is not None:
                    mu = restrict_field(self.meshes[l - 1], m, mu)
                if mu_h is not None:
                    mu_h = restrict_side_field(self.meshes[l - 1], m, mu_h)
            # gamma2 > 0: the 9-cell stencil (Sec. 3.5), rediscretised on every level
            self.levels.append(Level9(m, g, cs_dt, gamma2, mu, mu_h) if gamma2 > 0.0 else Level(m, g, cs_dt, mu, mu_h))

    def with_finest(self, level: Level) -> "Hierarchy":
        """The same hierarchy with the finest operator replaced (coarse levels unchanged): the
        hierarchy of a caller-supplied finest operator whose coarse levels are rediscretised
        from background factors."""
        out = Hierarchy.__new__(Hierarchy)
        out.meshes = self.meshes
        out.levels = [level] + self.levels[1:]
        return out

    @property
    def L(self) -> int:
        return len(self.levels)

    def vcycle(self, b: np.ndarray, omega: float = 0.8, n_pre: int = 2, n_post: int = 2,
               n_coarse: int = 4, x0: np.ndarray | None = None, level: int = 0) -> np.ndarray:
        """MGVcycle of Algorithm 1 on ``level`` (0-based), initial guess x0 (default 0)."""
        H = self.levels[level]
        b = np.asarray(b, dtype=np.float64).reshape(H.shape)
        x = np.zeros(H.shape) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(H.shape)
        if level == self.L - 1:
            return H.jacobi(b, x, omega, n_coarse)                      # CoarseSolve
        fine, coarse = self.meshes[level], self.meshes[level + 1]
        x = H.jacobi(b, x, omega, n_pre)                                # pre-smooth
        r = H.residual(b, x)                                            # R = B - H x
        bc = restrict(fine, coarse, r)                                  # B^(l+1)
        xc = self.vcycle(bc, omega, n_pre, n_post, n_coarse, None, level + 1)
        x = x + prolongate(fine, xc)                                    # correction
        return H.jacobi(b, x, omega, n_post)                            # post-smooth

    def as_preconditioner(self, omega=0.8, n_pre=2, n_post=2, n_coarse=4):
        return lambda r: self.vcycle(r, omega, n_pre, n_post, n_coarse).ravel()
