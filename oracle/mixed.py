"""Reduced mixed (velocity, pressure) system and its Schur-complement preconditioner (oracle).

Test infrastructure only.  Follows Maynard, Melvin & Mueller (arXiv 2002.00756):

* Sec. 3.3, Eq. linear_matrix: the quasi-Newton linear system couples velocity u (faces,
  RT0 at lowest order), density, potential temperature and pressure.  After the
  elimination of theta (Step 1a, Eq. eliminate_theta) the velocity block becomes
  M2-bar = M2 + P M_theta^{-1} P^z, whose extra term acts on vertical velocity only;
  after the elimination of rho (Step 1b) a 2x2 (u, p) system remains.  The reduced
  lowest-order system used here is, in strong volume-normalised form,

      velocity row f:  (M-bar u)_f + (kappa_f / d_f) (p_R(f) - p_L(f))   = r_u,f
      pressure row i:  p_i + (c_s dt / V_i) sum_f sigma_if A_f u_f        = r_p,i

  with kappa_f = c_s dt g_f, sigma_if = +1 when the face normal points out of cell i.
  Each coupling carries one factor of the time step (the linearised momentum and
  pressure equations of Sec. 3.3, Eq. linear_continuum, each hold one tau dt), scaled by
  the sound speed so that gradient and divergence are both O(CFL); their product gives
  the Helmholtz coefficients (c_s dt)^2 g_f A_f / (V_i d_f).  M-bar = I + eps B_w, where
  B_w couples each interior vertical face to the interior vertical faces directly above
  (weight beta_up) and below (beta_dn) in its column
  (non-symmetric, the folded buoyancy term of Step 1a).  The top and bottom faces carry
  no flux: their rows are identity rows and they do not enter D or G.
* Sec. 3.4: lumping M-bar to its row sums (diagonal M-ring) gives the Schur-complement
  preconditioner, Steps 1-3:
      B   = r_p - D M-ring^{-1} r_u                         (Eq. helmholtz right side)
      Pi' ~ H^{-1} B,  H = I - D M-ring^{-1} G             (Eq. helmholtz_operator)
      u'  = M-ring^{-1} (r_u - G Pi')                      (Eq. eliminate_u)
  H is the Helmholtz operator of ``helmholtz.Level`` with the coefficients of every face
  scaled by mu_f = 1 / M-ring_f.
* Sec. 3.3, Eq. M2muCdef, optional terms of M2^{mu,C} = M2 + tau_u dt (M_mu + M_C):
  - ``consistent``: the consistent (non-lumped) lowest-order Raviart-Thomas mass M2 in
    place of its lumped form, on the reference cell (the lumped mass stays 1 per face, the
    normalisation of this strong form).  Per cell, with every face basis function taken
    along the cell's own axis (xi for E/W, eta for N/S, up for bottom/top) and unit flux:
    integral of a basis function with itself 1/3, with the opposite face's 1/6, with a
    perpendicular one 0; in the vertical the same pattern couples faces kf and kf +- 1.
  - ``f0`` = tau_u dt 2 Omega: the implicit Coriolis term (M_C)_ij = 2 int v_i . (Omega x
    v_j) dV in the traditional approximation (only the local vertical component Omega
    sin(lat) of the rotation, lat at the cell centre, rotation axis = z): per cell
    F_c = f0 sin(lat_c) times int psi_a . (z x psi_b) = -1/4 for an xi-face a and an
    eta-face b, +1/4 for an eta-face a and a xi-face b (skew-symmetric, no work done).
  Both are assembled with the global orientation: a face's basis is the cell-axis basis
  times tau = +-1, the sign of the face normal (from the lower- to the higher-numbered
  column) along that axis.  The lumped diagonal M-ring is the row sum of M-bar taken in
  each cell's own axes (all tau = +1) over the retained unknowns; it equals the literal
  row sum wherever the global orientation agrees with the cells' axes (everywhere inside
  a panel) and does not depend on the orientation at panel edges.

Velocity vector layout (the library's convention): [u_h, u_v]; u_h is (nlev, 2 ncol)
level-major over the horizontal faces of ``Mesh.hfaces`` order; u_v is (nlev+1, ncol),
face kf lying between cells kf-1 (below) and kf (above), kf = 0 and nlev the boundary.
"""
from __future__ import annotations

import numpy as np

import scipy.sparse as sp

from .geometry import Mesh

OUTWARD = (1.0, -1.0, 1.0, -1.0)     # sides E, W, N, S: outward normal along +xi, -xi, +eta, -eta


def element_matrices():
    """Per-cell matrices of the horizontal faces E, W, N, S, basis along the cell axes:
    (consistent mass, Coriolis for unit F).  Reference cell [0,1]^2 (x xi, y eta), basis
    E: x e_x, W: (1 - x) e_x, N: y e_y, S: (1 - y) e_y."""
    M = np.array([[1 / 3, 1 / 6, 0, 0], [1 / 6, 1 / 3, 0, 0],
                  [0, 0, 1 / 3, 1 / 6], [0, 0, 1 / 6, 1 / 3]])
    C = np.array([[0, 0, -0.25, -0.25], [0, 0, -0.25, -0.25],
                  [0.25, 0.25, 0, 0], [0.25, 0.25, 0, 0]])
    return M, C


class MixedSystem:
    def __init__(self, mesh: Mesh, g: np.ndarray, cs_dt: float, beta_up: np.ndarray,
                 beta_dn: np.ndarray, eps: float, consistent: bool = False, f0: float = 0.0):
        self.mesh = mesh
        nlev, ncol = mesh.nlev, mesh.ncol
        self.nlev, self.ncol = nlev, ncol
        g = np.asarray(g, dtype=np.float64).reshape(nlev, ncol)
        self.cs_dt = cs_dt
        self.L, self.R, side = mesh.hfaces()
        self._side = side
        self.nhf = len(self.L)
        self.nh = nlev * self.nhf
        self.nv = (nlev + 1) * ncol
        self.nu = self.nh + self.nv
        self.np = nlev * ncol
        ell = mesh.edge_len[side, self.L]
        dist = mesh.centre_dist[side, self.L]
        # gradient weights kappa_f / d_f and divergence weights A_f / V_i
        self.kd_h = cs_dt * 0.5 * (g[:, self.L] + g[:, self.R]) / dist[None, :]   # (nlev, nhf)
        self.div_hL = cs_dt * ell / mesh.area[self.L]                            # (nhf,)
        self.div_hR = cs_dt * ell / mesh.area[self.R]
        self.div_v = cs_dt / mesh.dz                                              # (nlev,)
        self.kd_v = np.zeros((nlev + 1, ncol))
        for kf in range(1, nlev):
            self.kd_v[kf] = cs_dt * 0.5 * (g[kf - 1] + g[kf]) / mesh.dzc[kf]
        # velocity mass M-bar = I + eps B_w on vertical faces; couplings only between
        # interior faces of the same column
        interior = np.zeros(nlev + 1, dtype=bool)
        interior[1:nlev] = True
        up_ok = interior.copy()
        up_ok[nlev - 1:] = False        # face kf couples to kf+1 only if kf+1 is interior
        dn_ok = interior.copy()
        dn_ok[:2] = False               # face kf couples to kf-1 only if kf-1 is interior
        off = 1.0 / 6.0 if consistent else 0.0
        self.mv = 2.0 / 3.0 if consistent else 1.0                            # self weight
        self.w_up = (eps * np.asarray(beta_up, dtype=np.float64).reshape(nlev + 1, ncol) + off) * up_ok[:, None]
        self.w_dn = (eps * np.asarray(beta_dn, dtype=np.float64).reshape(nlev + 1, ncol) + off) * dn_ok[:, None]
        self.m_lump = self.mv + self.w_up + self.w_dn                         # row sums (Sec. 3.4)
        self.m_lump[0] = self.m_lump[nlev] = 1.0                              # identity rows
        self.mu = 1.0 / self.m_lump                                           # (nlev+1, ncol)
        self._horizontal_mass(consistent, f0)

    def _horizontal_mass(self, consistent: bool, f0: float):
        """M_h = M2 + tau_u dt M_C on the horizontal faces of one level (level-independent),
        assembled cell by cell from ``element_matrices``, and its lumped diagonal."""
        mesh, ncol = self.mesh, self.ncol
        face_of = np.empty((4, ncol), dtype=np.int64)
        for f in range(self.nhf):
            L, R, s = self.L[f], self.R[f], self._side[f]
            face_of[s, L] = f
            face_of[mesh.nbr_dir[s, L], R] = f
        self.face_of = face_of
        Me, Ce = element_matrices()
        if not consistent:
            Me = 0.5 * np.eye(4)            # lumped mass, 1 per face over its two cells
        self.F = f0 * mesh.centre[:, 2]     # tau_u dt 2 Omega sin(lat) per cell
        rows, cols, vals = [], [], []
        m_h = np.zeros(self.nhf)
        for c in range(ncol):
            E = Me + self.F[c] * Ce
            tau = [OUTWARD[s] * (1.0 if self.L[face_of[s, c]] == c else -1.0) for s in range(4)]
            for a in range(4):
                m_h[face_of[a, c]] += E[a].sum()            # row sum in the cell's own axes
                for b in range(4):
                    if E[a, b] != 0.0:
                        rows.append(face_of[a, c])
                        cols.append(face_of[b, c])
                        vals.append(tau[a] * tau[b] * E[a, b])
        self.Mh = sp.csr_matrix((vals, (rows, cols)), shape=(self.nhf, self.nhf))
        self.m_h = m_h
        self.mu_h = 1.0 / m_h[face_of]                      # (4, ncol) per cell side

    # ---- blocks ----
    def split(self, v: np.ndarray):
        v = np.asarray(v, dtype=np.float64).ravel()
        u, p = v[: self.nu], v[self.nu:]
        return (u[: self.nh].reshape(self.nlev, self.nhf), u[self.nh:].reshape(self.nlev + 1, self.ncol),
                p.reshape(self.nlev, self.ncol))

    def join(self, uh, uv, p) -> np.ndarray:
        return np.concatenate([uh.ravel(), uv.ravel(), p.ravel()])

    def grad(self, p: np.ndarray):
        """G p on faces: (kappa_f / d_f)(p_R - p_L); zero on the boundary faces."""
        p = p.reshape(self.nlev, self.ncol)
        gh = self.kd_h * (p[:, self.R] - p[:, self.L])
        gv = np.zeros((self.nlev + 1, self.ncol))
        gv[1:self.nlev] = self.kd_v[1:self.nlev] * (p[1:] - p[:-1])
        return gh, gv

    def div(self, uh: np.ndarray, uv: np.ndarray) -> np.ndarray:
        """D u in cells: (c_s dt / V_i) sum_f sigma_if A_f u_f over the interior faces."""
        out = np.zeros((self.nlev, self.ncol))
        np.add.at(out, (slice(None), self.L), self.div_hL[None, :] * uh)
        np.add.at(out, (slice(None), self.R), -self.div_hR[None, :] * uh)
        dv = self.div_v
        out[:-1] += dv[:-1, None] * uv[1:self.nlev]       # top face of cell k (faces 1..nlev-1)
        out[1:] -= dv[1:, None] * uv[1:self.nlev]         # bottom face of cell k (faces 1..nlev-1)
        return out

    def mass(self, uv: np.ndarray) -> np.ndarray:
        """M-bar on vertical faces (boundary rows: identity)."""
        y = uv.copy()
        y[1:-1] *= self.mv
        y[:-1] += self.w_up[:-1] * uv[1:]
        y[1:] += self.w_dn[1:] * uv[:-1]
        return y

    def mass_h(self, uh: np.ndarray) -> np.ndarray:
        """M_h on the horizontal faces, level by level."""
        return np.asarray(self.Mh @ uh.T).T

    # ---- operator and preconditioner ----
    def apply(self, v: np.ndarray) -> np.ndarray:
        """A_mixed [u; p] (Eq. linear_matrix, reduced lowest-order form)."""
        uh, uv, p = self.split(v)
        gh, gv = self.grad(p)
        return self.join(self.mass_h(uh) + gh, self.mass(uv) + gv, p + self.div(uh, uv))

    def precond(self, v: np.ndarray, helmholtz_solve) -> np.ndarray:
        """Approximate Schur complement (Sec. 3.4, Steps 1-3) with a given H^{-1}."""
        ruh, ruv, rp = self.split(v)
        B = rp - self.div(ruh / self.m_h, ruv / self.m_lump)    # Step 1
        pi = np.asarray(helmholtz_solve(B), dtype=np.float64).reshape(self.nlev, self.ncol)  # Step 2
        gh, gv = self.grad(pi)
        uh = (ruh - gh) / self.m_h                               # Step 3
        uv = (ruv - gv) / self.m_lump
        return self.join(uh, uv, pi)
