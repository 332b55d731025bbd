"""Pins of the oracle's mixed (u, p) operator and Schur-complement preconditioner."""
import numpy as np
import pytest

import synthetic as syn
from oracle.geometry import Mesh
from oracle.helmholtz import Level
from oracle.krylov import gcr
from oracle.mixed import MixedSystem
from oracle.multigrid import Hierarchy
from oracle.reference import assemble_helmholtz, assemble_mixed, direct_solve

R = 6371.0e3
CSDT = 340.0 * 600.0


def _system(n=3, nlev=5, eps=0.05, seed=21):
    cfg = syn.small_config(n, nlev, seed=seed, mixed=True, eps=eps)
    inp = syn.make_inputs(cfg)
    m = Mesh(n, inp["z_if"], R)
    S = MixedSystem(m, inp["g"], CSDT, inp["beta_up"], inp["beta_dn"], eps)
    return S, inp, cfg


def test_sizes_follow_the_rt0_count():
    S, _, cfg = _system()
    assert S.nu == cfg.n_uface and S.np == cfg.ncell
    assert S.nhf == 2 * cfg.ncol


def test_apply_matches_assembled_matrix():
    S, inp, _ = _system()
    A = assemble_mixed(S)
    v = np.random.default_rng(0).standard_normal(S.nu + S.np)
    ref = A @ v
    assert np.allclose(S.apply(v), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_boundary_faces_are_identity_rows():
    S, _, _ = _system()
    A = assemble_mixed(S).tocsr()
    uv = S.nh + np.arange(S.nv).reshape(S.nlev + 1, S.ncol)
    for r in np.concatenate([uv[0], uv[-1]]):
        row = A.getrow(r)
        assert row.nnz == 1 and row[0, r] == 1.0
    # no flux through lid and surface: those faces do not appear in any pressure row
    pcols = A[S.nu:, :].tocsc()
    for c in np.concatenate([uv[0], uv[-1]]):
        assert pcols.getcol(c).nnz == 0


def test_discrete_integration_by_parts():
    # c_s dt sum_f (A_f d_f / kappa_f) (G p)_f u_f = - sum_i V_i p_i (D u)_i  (G = -D^T up to weights)
    S, inp, _ = _system()
    m = S.mesh
    rng = np.random.default_rng(1)
    p = rng.standard_normal((S.nlev, S.ncol))
    uh = rng.standard_normal((S.nlev, S.nhf))
    uv = rng.standard_normal((S.nlev + 1, S.ncol))
    uv[0] = uv[-1] = 0.0
    gh, gv = S.grad(p)
    L, Rr, side = m.hfaces()
    A_h = m.edge_len[side, L][None, :] * m.dz[:, None]
    w_h = A_h / S.kd_h                               # A_f d_f / kappa_f
    w_v = np.zeros_like(gv)
    w_v[1:-1] = m.area[None, :] / S.kd_v[1:-1]
    lhs = S.cs_dt * (np.sum(w_h * gh * uh) + np.sum(w_v * gv * uv))
    V = m.dz[:, None] * m.area[None, :]
    rhs = -np.sum(V * p * S.div(uh, uv))
    assert lhs == pytest.approx(rhs, rel=1e-11)


def test_schur_complement_of_lumped_system_is_the_helmholtz_operator():
    # H = I - D M-ring^{-1} G from the assembled blocks equals the stencil operator with
    # vertical coefficients scaled by 1 / M-ring (Sec. 3.4, Eq. helmholtz_operator)
    S, inp, _ = _system(n=2, nlev=4)
    A = assemble_mixed(S).toarray()
    nu = S.nu
    M, G, D = A[:nu, :nu], A[:nu, nu:], A[nu:, :nu]
    lump = M.sum(axis=1)
    H_schur = np.eye(S.np) - D @ (G / lump[:, None])
    H = assemble_helmholtz(Level(S.mesh, inp["g"], CSDT, S.mu)).toarray()
    assert np.allclose(H_schur, H, rtol=1e-12, atol=1e-9)


def test_exact_schur_preconditioner_without_coupling():
    # eps = 0: M-bar is diagonal, lumping is exact, so with an exact Helmholtz solve the
    # preconditioner is A^{-1} and GCR converges in one iteration
    S, inp, _ = _system(n=2, nlev=4, eps=0.0)
    H = assemble_helmholtz(Level(S.mesh, inp["g"], CSDT, S.mu))
    solve = lambda B: direct_solve(H, B)
    rhs = np.concatenate([inp["rhs_u"], inp["rhs_p"]])
    z = S.precond(rhs, solve)
    assert np.allclose(S.apply(z), rhs, rtol=1e-9, atol=1e-9)
    _, it, _ = gcr(S.apply, rhs, lambda r: S.precond(r, solve), tol=1e-10)
    assert it == 1


def test_mixed_gcr_with_mg_schur_matches_dense_lu():
    S, inp, cfg = _system(n=2, nlev=6)
    h = Hierarchy(2, inp["z_if"], R, 2, inp["g"], CSDT, mu=S.mu)
    rhs = np.concatenate([inp["rhs_u"], inp["rhs_p"]])
    x, it, hist = gcr(S.apply, rhs, lambda r: S.precond(r, h.as_preconditioner()), tol=1e-12)
    xs = direct_solve(assemble_mixed(S), rhs)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    assert np.all(np.diff(hist) <= 0)
