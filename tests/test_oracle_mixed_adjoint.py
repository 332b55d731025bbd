"""Pins of the adjoint of the mixed (u, p) system: the oracle's A^{-T} g (a direct solve with
the transposed matrix) and the similarity the GPU adjoint solve relies on.

With face weights W_f = A_f d_f / g_f, cell volumes V_i, S = diag(W, V) and J = diag(I, -I),
the discrete integration by parts of Sec. 3.3's gradient and divergence (W G = -D^T V) gives
    A^T = S J A-hat J S^{-1},   A-hat = [[W^{-1} M-bar^T W, G], [D, I]],
the mixed operator with its velocity mass replaced by W^{-1} M-bar^T W."""
import numpy as np
import pytest
import scipy.sparse as sp

import synthetic as syn
from oracle.problem import mixed_problem
from oracle.reference import adjoint_solve, assemble_mixed, direct_solve


def _case(consistent, rotation, n=2, nlev=4, seed=71):
    cfg = syn.small_config(n, nlev, levels=1, seed=syn.BASE_SEED + seed, mixed=True,
                           consistent_mass=consistent, rotation=rotation)
    inp = syn.make_inputs(cfg)
    S, _ = mixed_problem(cfg, inp)
    return S, inp


def face_weights(S):
    """W_f = A_f d_f / g_f on [u_h, u_v] (1 on the boundary faces) and V_i on the cells,
    from the geometry: A_f = edge length x layer depth or cell area, d_f = centre distance."""
    m = S.mesh
    side = S._side
    cs_dt = S.cs_dt
    Wh = (m.edge_len[side, S.L][None, :] * m.dz[:, None]) * cs_dt / S.kd_h
    Wv = np.ones((S.nlev + 1, S.ncol))
    Wv[1:-1] = m.area[None, :] * cs_dt / S.kd_v[1:-1]
    V = m.dz[:, None] * m.area[None, :]
    return np.concatenate([Wh.ravel(), Wv.ravel()]), V.ravel()


@pytest.mark.parametrize("consistent,rotation", [(False, 0.0), (True, 5e-4)])
def test_mixed_adjoint_identity(consistent, rotation):
    """<A^{-T} g, b> = <g, A^{-1} b> for random b, g; the untransposed solve fails it."""
    S, _ = _case(consistent, rotation)
    A = assemble_mixed(S)
    rng = np.random.default_rng(4)
    n = S.nu + S.np
    g, b = rng.standard_normal(n), rng.standard_normal(n)
    lam, x = adjoint_solve(A, g), direct_solve(A, b)
    assert abs(lam @ b - g @ x) <= 1e-11 * np.linalg.norm(lam) * np.linalg.norm(b)
    wrong = direct_solve(A, g)
    assert abs(wrong @ b - g @ x) > 1e-6 * np.linalg.norm(wrong) * np.linalg.norm(b)


@pytest.mark.parametrize("consistent,rotation", [(False, 0.0), (True, 5e-4)])
def test_transposed_mixed_operator_is_similar_to_the_transposed_mass_system(consistent, rotation):
    S, _ = _case(consistent, rotation)
    A = assemble_mixed(S).toarray()
    W, V = face_weights(S)
    nu = S.nu
    s = np.concatenate([W, V])
    j = np.concatenate([np.ones(nu), -np.ones(S.np)])
    Ahat = (j / s)[:, None] * A.T * (s * j)[None, :]        # J S^-1 A^T S J
    scale = np.abs(A).max()
    # off-diagonal blocks: G and D of A itself
    assert np.allclose(Ahat[:nu, nu:], A[:nu, nu:], rtol=1e-12, atol=1e-13 * scale)
    assert np.allclose(Ahat[nu:, :nu], A[nu:, :nu], rtol=1e-12, atol=1e-13 * scale)
    assert np.allclose(Ahat[nu:, nu:], np.eye(S.np))
    # velocity block: W^-1 M-bar^T W
    M = A[:nu, :nu]
    assert np.allclose(Ahat[:nu, :nu], (M.T * W[None, :]) / W[:, None], rtol=1e-12, atol=1e-15)
    if consistent or rotation:
        assert not np.allclose(Ahat[:nu, :nu], M)              # the mass is not W-symmetric


def test_mixed_coefficient_gradient_matches_central_differences():
    """dL/dg and dL/dbeta of L = <w, A(g, beta)^-1 rhs> from
    oracle.reference.mixed_coefficient_gradient against central differences of single
    background factors (interior and top cells) and single mass couplings."""
    from oracle.reference import mixed_coefficient_gradient
    cfg = syn.small_config(2, 5, levels=1, seed=syn.BASE_SEED + 81, mixed=True,
                           consistent_mass=True, rotation=5e-4)
    inp = syn.make_inputs(cfg)
    rhs = np.concatenate([inp["rhs_u"], inp["rhs_p"]])
    S, _ = mixed_problem(cfg, inp)
    w = syn.normal(82, 0, S.nu + S.np)
    A = assemble_mixed(S)
    x = direct_solve(A, rhs)
    dg, dbu, dbd = mixed_coefficient_gradient(S, x, adjoint_solve(A, w), cfg.eps)

    def loss(**kw):
        i2 = dict(inp, **kw)
        S2, _ = mixed_problem(cfg, i2)
        return w @ direct_solve(assemble_mixed(S2), rhs)

    ncol = S.ncol
    g = inp["g"].reshape(cfg.nlev, ncol)
    for (k, c) in [(0, 3), (2, 10), (cfg.nlev - 1, 17)]:
        h = 1e-5 * g[k, c]
        gp, gm = g.copy(), g.copy()
        gp[k, c] += h
        gm[k, c] -= h
        fd = (loss(g=gp.ravel()) - loss(g=gm.ravel())) / (2 * h)
        assert abs(fd - dg[k, c]) <= 1e-6 * abs(dg[k, c]) + 1e-12, (k, c, fd, dg[k, c])
    for name, arr, grad, kf in [("beta_up", inp["beta_up"], dbu, 2), ("beta_dn", inp["beta_dn"], dbd, 3)]:
        b = arr.reshape(cfg.nlev + 1, ncol)
        c = 5
        h = 1e-4
        bp, bm = b.copy(), b.copy()
        bp[kf, c] += h
        bm[kf, c] -= h
        fd = (loss(**{name: bp.ravel()}) - loss(**{name: bm.ravel()})) / (2 * h)
        assert abs(fd - grad[kf, c]) <= 1e-6 * abs(grad[kf, c]) + 1e-12, (name, fd, grad[kf, c])
    # couplings that do not exist carry no gradient
    assert np.all(dbu[0] == 0) and np.all(dbu[cfg.nlev - 1:] == 0) and np.all(dbd[:2] == 0)
