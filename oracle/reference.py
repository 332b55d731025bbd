"""Assembled matrices and direct solves: the plain definition of the solutions (oracle).

Test infrastructure only.  ``pressure_solve`` and ``mixed_solve`` approximate the
solution of a linear system (Eq. helmholtz and Eq. linear_matrix of Maynard, Melvin &
Mueller, arXiv 2002.00756).  The reference solution x* is that of the assembled sparse
matrix: by sparse LU (scipy.sparse.linalg.spsolve) or dense LU on small problems, and
otherwise by the oracle's GCR to a relative residual of 1e-12 measured with the
assembled matrix itself, so that x* does not depend on the matrix-free code it checks.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .helmholtz import Level
from .krylov import gcr
from .mixed import MixedSystem


def assemble_helmholtz(H: Level) -> sp.csr_matrix:
    """H as a sparse matrix, row i = k * ncol + c, entry by entry from the coefficients."""
    nlev, ncol = H.shape
    N = nlev * ncol
    idx = np.arange(N).reshape(nlev, ncol)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [H.diag().ravel()]
    for d in range(4):
        rows.append(idx.ravel())
        cols.append(idx[:, H.mesh.nbr[d]].ravel())
        vals.append(-H.a_h[d].ravel())
    rows.append(idx[:-1].ravel())
    cols.append(idx[1:].ravel())
    vals.append(-H.a_up[:-1].ravel())
    rows.append(idx[1:].ravel())
    cols.append(idx[:-1].ravel())
    vals.append(-H.a_dn[1:].ravel())
    if hasattr(H, "b_up"):          # the 9-cell stencil: couplings two levels up and down
        rows.append(idx[:-2].ravel())
        cols.append(idx[2:].ravel())
        vals.append(-H.b_up[:-2].ravel())
        rows.append(idx[2:].ravel())
        cols.append(idx[:-2].ravel())
        vals.append(-H.b_dn[2:].ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


def assemble_mixed(S: MixedSystem) -> sp.csr_matrix:
    """[[M-bar, G], [D, I]] as one sparse matrix over [u_h, u_v, p] (M-bar: M_h on the
    horizontal faces of every level, the vertical couplings of ``MixedSystem.mass``)."""
    nlev, ncol, nhf = S.nlev, S.ncol, S.nhf
    rows, cols, vals = [], [], []

    def put(r, c, v):
        r, c, v = np.broadcast_arrays(r, c, v)
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(v.ravel())

    uh = np.arange(S.nh).reshape(nlev, nhf)
    uv = S.nh + np.arange(S.nv).reshape(nlev + 1, ncol)
    pp = S.nu + np.arange(S.np).reshape(nlev, ncol)
    # velocity rows: horizontal faces, M_h on every level
    Mh = S.Mh.tocoo()
    for k in range(nlev):
        put(uh[k][Mh.row], uh[k][Mh.col], Mh.data)
    put(uh, pp[:, S.R], S.kd_h)
    put(uh, pp[:, S.L], -S.kd_h)
    # velocity rows: vertical faces
    self_w = np.full((nlev + 1, ncol), S.mv)
    self_w[0] = self_w[-1] = 1.0                        # boundary faces: identity rows
    put(uv, uv, self_w)
    put(uv[:-1], uv[1:], S.w_up[:-1])
    put(uv[1:], uv[:-1], S.w_dn[1:])
    put(uv[1:nlev], pp[1:], S.kd_v[1:nlev])
    put(uv[1:nlev], pp[:-1], -S.kd_v[1:nlev])
    # pressure rows
    put(pp, pp, 1.0)
    put(pp[:, S.L], uh, S.div_hL[None, :])
    put(pp[:, S.R], uh, -S.div_hR[None, :])
    put(pp[:-1], uv[1:nlev], S.div_v[:-1, None])
    put(pp[1:], uv[1:nlev], -S.div_v[1:, None])
    n = S.nu + S.np
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    A = A.tocsr()
    A.eliminate_zeros()
    return A


def direct_solve(A: sp.spmatrix, b: np.ndarray) -> np.ndarray:
    """Sparse LU solve (dense LU below 3000 unknowns)."""
    b = np.asarray(b, dtype=np.float64).ravel()
    if A.shape[0] <= 3000:
        return np.linalg.solve(A.toarray(), b)
    return spla.spsolve(A.tocsc(), b)


def adjoint_solve(A: sp.spmatrix, g: np.ndarray) -> np.ndarray:
    """lambda = A^{-T} g: the gradient dL/db of L(x(b)), x = A^{-1} b, given g = dL/dx (the
    plain definition, a direct solve with the transposed matrix)."""
    return direct_solve(sp.csr_matrix(A.T), g)


def coefficient_gradient(H: Level, x: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """dL/da for L(x), x = H^{-1} b, given lam = H^{-T} dL/dx: differentiating H x = b gives
    dL = -<lam, dH x>, and (dH x)_i = sum_f da_{i,f} (x_i - x_j), so
        dL/da_{i,f} = -lam_i (x_i - x_{j(f)}).
    Returned as (6, nlev, ncol): E, W, N, S, up, down (zero where a face has no neighbour)."""
    x = np.asarray(x, dtype=np.float64).reshape(H.shape)
    lam = np.asarray(lam, dtype=np.float64).reshape(H.shape)
    out = np.zeros((6,) + H.shape)
    for d in range(4):
        out[d] = -lam * (x - x[:, H.mesh.nbr[d]])
    out[4, :-1] = -lam[:-1] * (x[:-1] - x[1:])
    out[5, 1:] = -lam[1:] * (x[1:] - x[:-1])
    return out


def iterative_reference(A: sp.spmatrix, b: np.ndarray, P, tol: float = 1e-12,
                        maxiter: int = 400) -> np.ndarray:
    """GCR on the assembled matrix to a relative residual ``tol`` (checked again at the end)."""
    b = np.asarray(b, dtype=np.float64).ravel()
    x, _, _ = gcr(lambda v: A @ v, b, P, tol=tol, restart=20, maxiter=maxiter)
    res = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    if res > 10 * tol:
        raise RuntimeError(f"reference solve reached only {res:.3e}")
    return x


def mixed_coefficient_gradient(S, x: np.ndarray, lam: np.ndarray, eps: float):
    """dL/dg, dL/dbeta_up, dL/dbeta_dn for L(x), A(g, beta) x = rhs, given lam = A^-T dL/dx.

    Differentiating A x = rhs gives dL = -<lam, dA x>.  In the mixed operator (Sec. 3.3-3.4)
    the background factors g enter only the gradient weights kappa_f / d_f = c_s dt g_f / d_f
    with g_f = (g_i + g_j) / 2 (velocity rows: kd_f (p_R - p_L)), and beta enters the vertical
    velocity mass as eps beta (row kf, column kf + 1 for beta_up, kf - 1 for beta_dn, between
    interior faces only).  Returns arrays shaped like g (nlev, ncol) and beta (nlev+1, ncol)."""
    uh, uv, p = S.split(x)
    lh, lv, _ = S.split(lam)
    m = S.mesh
    nlev, ncol = S.nlev, S.ncol
    dist = m.centre_dist[S._side, S.L]
    dg = np.zeros((nlev, ncol))
    # horizontal faces: d kd / d g_L = d kd / d g_R = c_s dt / (2 dist)
    gk = -lh * (p[:, S.R] - p[:, S.L]) * (S.cs_dt / (2.0 * dist))[None, :]
    np.add.at(dg, (slice(None), S.L), gk)
    np.add.at(dg, (slice(None), S.R), gk)
    # vertical faces kf = 1 .. nlev-1 between cells kf-1 and kf
    for kf in range(1, nlev):
        gv = -lv[kf] * (p[kf] - p[kf - 1]) * S.cs_dt / (2.0 * m.dzc[kf])
        dg[kf - 1] += gv
        dg[kf] += gv
    db_up = np.zeros((nlev + 1, ncol))
    db_dn = np.zeros((nlev + 1, ncol))
    for kf in range(1, nlev - 1):        # face kf couples to kf + 1 (both interior)
        db_up[kf] = -eps * lv[kf] * uv[kf + 1]
    for kf in range(2, nlev):            # face kf couples to kf - 1 (both interior)
        db_dn[kf] = -eps * lv[kf] * uv[kf - 1]
    return dg, db_up, db_dn
