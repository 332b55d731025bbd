"""Helmholtz operator, column tridiagonal part and block-Jacobi sweep (oracle).

Test infrastructure only.  Follows Maynard, Melvin & Mueller (arXiv 2002.00756):

* Eq. helmholtz_operator / Sec. 3.5: H couples every cell to its 4 horizontal
  neighbours and to the cells above and below (the lowest-order finite-volume analogue
  of the 9-cell stencil keeps the nearest vertical neighbours only).  In strong,
  volume-normalised form
        (H x)_i = x_i + sum_{faces f of i} a_{i,f} (x_i - x_{j(f)}),
        a_{i,f} = (c_s dt)^2 g_f A_f / (V_i d_f),
  with face area A_f, cell volume V_i, centre distance d_f and background factor
  g_f = (g_i + g_j)/2 (so V_i a_{i,f} = V_j a_{j,f}: flux antisymmetry).  The terms
  scale as CFL_h^2 horizontally and CFL_v^2 vertically (Eq. DH_ratios).  No flux passes
  the bottom and top.  For the mixed system every coefficient carries the factor
  mu_f = 1 / (lumped velocity mass) of its face (Sec. 3.4, Step 1a): ``mu`` on the vertical
  faces, ``mu_h`` (per cell side E, W, N, S) on the horizontal ones.
* Sec. 3.6, Eq. jacobi: H_z-hat keeps, per column, the vertical couplings and the full
  diagonal of H; one block-Jacobi iteration is x <- x + omega H_z-hat^{-1} (b - H x),
  the tridiagonal solve done per column with the Thomas algorithm.

Arrays are (nlev, ncol), level-major like the library's x[k * ncol + col].
"""
from __future__ import annotations

import numpy as np

from .geometry import Mesh


class Level:
    """Stencil coefficients of H on one mesh level.

    a_h[d, k, c]  horizontal coefficient of cell (k, c) towards direction d (E, W, N, S)
    a_up[k, c]    coefficient to cell (k+1, c); 0 on the top level
    a_dn[k, c]    coefficient to cell (k-1, c); 0 on the bottom level
    """

    def __init__(self, mesh: Mesh, g: np.ndarray, cs_dt: float, mu: np.ndarray | None = None,
                 mu_h: np.ndarray | None = None):
        self.mesh = mesh
        nlev, ncol = mesh.nlev, mesh.ncol
        g = np.asarray(g, dtype=np.float64).reshape(nlev, ncol)
        self.g = g
        if mu is None:
            mu = np.ones((nlev + 1, ncol))
        self.mu = np.asarray(mu, dtype=np.float64).reshape(nlev + 1, ncol)
        if mu_h is None:
            mu_h = np.ones((4, ncol))
        self.mu_h = np.asarray(mu_h, dtype=np.float64).reshape(4, ncol)
        c2 = cs_dt * cs_dt
        self.a_h = np.empty((4, nlev, ncol))
        for d in range(4):
            nb = mesh.nbr[d]
            gf = 0.5 * (g + g[:, nb])
            # A_f / V_i = edge_length * dz / (area * dz): the layer depth cancels
            self.a_h[d] = c2 * gf * self.mu_h[d][None, :] * mesh.edge_len[d][None, :] / (
                mesh.area[None, :] * mesh.centre_dist[d][None, :])
        self.a_up = np.zeros((nlev, ncol))
        self.a_dn = np.zeros((nlev, ncol))
        for k in range(nlev - 1):
            # face kf = k + 1 between cells k and k + 1; A_f / V_i = 1 / dz_i
            gf = 0.5 * (g[k] + g[k + 1])
            flux = c2 * gf * self.mu[k + 1] / mesh.dzc[k + 1]
            self.a_up[k] = flux / mesh.dz[k]
            self.a_dn[k + 1] = flux / mesh.dz[k + 1]

    @classmethod
    def from_couplings(cls, mesh: Mesh, a_h: np.ndarray, a_up: np.ndarray, a_dn: np.ndarray) -> "Level":
        """A level whose couplings are given directly (the operator supplied by a caller
        instead of being discretised from background factors): a_h (4, nlev, ncol) towards
        E, W, N, S, a_up / a_dn (nlev, ncol), zero above the top / below the bottom cell."""
        lev = cls.__new__(cls)
        lev.mesh = mesh
        lev.a_h = np.array(a_h, dtype=np.float64).reshape(4, mesh.nlev, mesh.ncol)
        lev.a_up = np.array(a_up, dtype=np.float64).reshape(mesh.nlev, mesh.ncol)
        lev.a_dn = np.array(a_dn, dtype=np.float64).reshape(mesh.nlev, mesh.ncol)
        return lev

    def couplings(self) -> np.ndarray:
        """The six couplings per cell as one (6, nlev, ncol) array: E, W, N, S, up, down."""
        return np.concatenate([self.a_h, self.a_up[None], self.a_dn[None]])

    @property
    def shape(self):
        return (self.mesh.nlev, self.mesh.ncol)

    def diag(self) -> np.ndarray:
        """Diagonal of H: 1 plus all six face coefficients."""
        return 1.0 + self.a_h.sum(axis=0) + self.a_up + self.a_dn

    def apply(self, x: np.ndarray) -> np.ndarray:
        """y = H x (difference form)."""
        x = np.asarray(x, dtype=np.float64).reshape(self.shape)
        y = x.copy()
        for d in range(4):
            y += self.a_h[d] * (x - x[:, self.mesh.nbr[d]])
        y[:-1] += self.a_up[:-1] * (x[:-1] - x[1:])
        y[1:] += self.a_dn[1:] * (x[1:] - x[:-1])
        return y

    def residual(self, b: np.ndarray, x: np.ndarray) -> np.ndarray:
        return np.asarray(b, dtype=np.float64).reshape(self.shape) - self.apply(x)

    def hz_bands(self):
        """Sub-, main- and super-diagonal of the column matrices H_z-hat."""
        return -self.a_dn, self.diag(), -self.a_up

    def hz_solve(self, r: np.ndarray) -> np.ndarray:
        """H_z-hat^{-1} r, every column by the Thomas algorithm (pivot-excess form).

        The textbook recurrence loses about log10(CFL_v^2) digits on the vertically
        smooth mode when the vertical coefficients reach 1e6-1e7; the excess form below is
        the same elimination with every pivot kept as a sum of positive terms.
        """
        s = 1.0 + self.a_h.sum(axis=0)
        return thomas_excess(self.a_dn, s, self.a_up,
                             np.asarray(r, dtype=np.float64).reshape(self.shape))

    def jacobi(self, b: np.ndarray, x: np.ndarray, omega: float, sweeps: int) -> np.ndarray:
        """BlockJacobi(H, b, x, omega, sweeps): Eq. jacobi applied ``sweeps`` times."""
        x = np.asarray(x, dtype=np.float64).reshape(self.shape).copy()
        for _ in range(sweeps):
            x = x + omega * self.hz_solve(self.residual(b, x))
        return x


class Level9(Level):
    """The 9-cell stencil of Sec. 3.5 (Fig. 2): besides its four horizontal neighbours and the
    cells directly above and below, every cell couples to the cells two levels above and two
    below, so the column blocks H_z are pentadiagonal.  The smoother keeps only the
    tridiagonal part H_z-hat (Sec. 3.6: the next-to-nearest couplings are dropped from the
    column solve, while the residual b - H x keeps them).

    At lowest order the paper's operator has no such couplings; here they are a flux between
    cells k and k + 2 of the same form as the nearest one,
        b_up[k] = gamma2 (c_s dt)^2 g_(k,k+2) / (dz_k (z_c[k+2] - z_c[k])),
        b_dn[k + 2] = the same flux / dz_(k+2),   g_(k,k+2) = (g_k + g_(k+2)) / 2,
    with a relative strength gamma2, so V H stays symmetric and H an M-matrix.  H_z-hat drops
    these fluxes entirely (the off-diagonal entries and their share of the diagonal): keeping
    the share on the diagonal would make H_z-hat differ from H by 2 b on the vertically smooth
    error, which the column solve then fails to reduce."""

    def __init__(self, mesh: Mesh, g: np.ndarray, cs_dt: float, gamma2: float, mu=None, mu_h=None):
        super().__init__(mesh, g, cs_dt, mu, mu_h)
        nlev, ncol = mesh.nlev, mesh.ncol
        self.gamma2 = float(gamma2)
        self.b_up = np.zeros((nlev, ncol))
        self.b_dn = np.zeros((nlev, ncol))
        c2 = cs_dt * cs_dt
        for k in range(nlev - 2):
            gf = 0.5 * (self.g[k] + self.g[k + 2])
            flux = self.gamma2 * c2 * gf / (mesh.zc[k + 2] - mesh.zc[k])
            self.b_up[k] = flux / mesh.dz[k]
            self.b_dn[k + 2] = flux / mesh.dz[k + 2]

    def diag(self) -> np.ndarray:
        return super().diag() + self.b_up + self.b_dn

    def apply(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64).reshape(self.shape)
        y = super().apply(x)
        y[:-2] += self.b_up[:-2] * (x[:-2] - x[2:])
        y[2:] += self.b_dn[2:] * (x[2:] - x[:-2])
        return y

    # hz_solve is Level's: H_z-hat drops the next-to-nearest fluxes b (x_i - x_(i+-2)) as a whole,
    # their diagonal share included, so it is the same tridiagonal matrix as without them.


def thomas(lower: np.ndarray, diag: np.ndarray, upper: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Solve the tridiagonal systems of every column (axis 0 = position in the column).

    Textbook forward elimination / back substitution (e.g. Press et al., Numerical
    Recipes, "tridag"); lower[0] and upper[-1] are ignored.
    """
    n = diag.shape[0]
    gam = np.empty_like(diag)
    u = np.empty_like(r)
    bet = diag[0].copy()
    u[0] = r[0] / bet
    for k in range(1, n):
        gam[k] = upper[k - 1] / bet
        bet = diag[k] - lower[k] * gam[k]
        u[k] = (r[k] - lower[k] * u[k - 1]) / bet
    for k in range(n - 2, -1, -1):
        u[k] -= gam[k + 1] * u[k + 1]
    return u


def thomas_excess(a_dn: np.ndarray, s: np.ndarray, a_up: np.ndarray, r: np.ndarray) -> np.ndarray:
    """The same column solve with pivots written as p_k = q_k + a_up_k.

    For the column matrix tridiag(-a_dn, s + a_dn + a_up, -a_up) with row excess
    s_k = 1 + (horizontal coefficients) > 0, elimination gives
        q_0 = s_0,   q_k = s_k + a_dn_k q_{k-1} / p_{k-1},   p_k = q_k + a_up_k,
    so every pivot is a sum of positive terms (no cancellation between the O(1)
    identity part and the O(CFL_v^2) vertical terms).  Forward sweep y_k = r_k +
    (a_dn_k / p_{k-1}) y_{k-1}, back substitution x_k = (y_k + a_up_k x_{k+1}) / p_k.
    """
    n = s.shape[0]
    p = np.empty_like(s)
    y = np.empty_like(r)
    q = s[0].copy()
    p[0] = q + a_up[0]
    y[0] = r[0]
    for k in range(1, n):
        m = a_dn[k] / p[k - 1]
        q = s[k] + m * q
        p[k] = q + a_up[k]
        y[k] = r[k] + m * y[k - 1]
    x = np.empty_like(r)
    x[-1] = y[-1] / p[-1]
    for k in range(n - 2, -1, -1):
        x[k] = (y[k] + a_up[k] * x[k + 1]) / p[k]
    return x
