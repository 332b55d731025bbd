"""Pins of the oracle's consistent velocity mass and implicit Coriolis term (Sec. 3.3,
Eq. M2muCdef) and of their lumped form in the Schur-complement preconditioner (Sec. 3.4)."""
import numpy as np
import pytest

import synthetic as syn
from oracle.geometry import Mesh
from oracle.helmholtz import Level
from oracle.krylov import gcr
from oracle.mixed import MixedSystem, element_matrices
from oracle.multigrid import Hierarchy
from oracle.reference import assemble_helmholtz, assemble_mixed, direct_solve

R = 6371.0e3
CSDT = 340.0 * 600.0


def _system(n=6, nlev=4, eps=0.05, consistent=True, f0=0.2, seed=61):
    cfg = syn.small_config(n, nlev, seed=seed, mixed=True, eps=eps)
    inp = syn.make_inputs(cfg)
    S = MixedSystem(Mesh(n, inp["z_if"], R), inp["g"], CSDT, inp["beta_up"], inp["beta_dn"], eps,
                    consistent=consistent, f0=f0)
    return S, inp


def test_element_matrices_are_the_integrals_of_the_rt0_basis():
    """Gauss-Legendre quadrature (exact for these polynomials) of int psi_a . psi_b and
    int psi_a . (z x psi_b) over the reference cell, basis along the cell axes."""
    xg, wg = np.polynomial.legendre.leggauss(3)
    xg, wg = 0.5 * (xg + 1.0), 0.5 * wg
    X, Y = np.meshgrid(xg, xg, indexing="ij")
    W = np.outer(wg, wg)
    zero = np.zeros_like(X)
    basis = [(X, zero), (1.0 - X, zero), (zero, Y), (zero, 1.0 - Y)]     # E, W, N, S
    mass = np.array([[np.sum(W * (a[0] * b[0] + a[1] * b[1])) for b in basis] for a in basis])
    # z x (v_x, v_y) = (-v_y, v_x)
    cor = np.array([[np.sum(W * (a[0] * -b[1] + a[1] * b[0])) for b in basis] for a in basis])
    M, C = element_matrices()
    assert np.allclose(M, mass, atol=1e-15)
    assert np.allclose(C, cor, atol=1e-15)


def _panel_interior_faces(S, panel):
    """(xi-faces, eta-faces) whose two cells lie one cell or more inside ``panel``."""
    m = S.mesh
    inner = (m.panel == panel) & (m.i >= 1) & (m.i <= m.n - 2) & (m.j >= 1) & (m.j <= m.n - 2)
    both = inner[S.L] & inner[S.R]
    xi = both & (S._side <= 1)
    return np.nonzero(xi)[0], np.nonzero(both & (S._side >= 2))[0]


@pytest.mark.parametrize("panel", [0, 4])
def test_uniform_flow_inside_a_panel(panel):
    """A uniform flow U e_xi has flux U through every xi-face of the panel (normals point
    along +xi inside a panel).  The consistent mass returns it unchanged (2/3 + 1/6 + 1/6);
    the Coriolis term F z x (U e_xi) = F U e_eta puts (F_L + F_R) U / 2 on the eta-faces.
    Likewise U e_eta gives -(F_L + F_R) U / 2 on the xi-faces."""
    S, _ = _system(consistent=True, f0=0.2)
    m = S.mesh
    on = m.panel[S.L] == panel
    on &= m.panel[S.R] == panel
    xi_f, eta_f = _panel_interior_faces(S, panel)
    assert len(xi_f) > 0 and len(eta_f) > 0
    U = 1.7
    Fm = 0.5 * (S.F[S.L] + S.F[S.R])
    u = np.where(on & (S._side <= 1), U, 0.0)
    y = S.Mh @ u
    assert np.allclose(y[xi_f], U, rtol=1e-14)
    assert np.allclose(y[eta_f], Fm[eta_f] * U, rtol=1e-13)
    u = np.where(on & (S._side >= 2), U, 0.0)
    y = S.Mh @ u
    assert np.allclose(y[eta_f], U, rtol=1e-14)
    assert np.allclose(y[xi_f], -Fm[xi_f] * U, rtol=1e-13)


def test_consistent_mass_is_spd_and_coriolis_is_skew():
    S0, _ = _system(n=3, consistent=True, f0=0.0)
    S1, _ = _system(n=3, consistent=True, f0=0.3)
    M = S0.Mh.toarray()
    C = S1.Mh.toarray() - M
    assert np.allclose(M, M.T, atol=1e-15)
    ev = np.linalg.eigvalsh(M)
    # each cell's 2x2 blocks [[1/3, 1/6], [1/6, 1/3]] have eigenvalues 1/6 and 1/2; a face
    # sums two cells: 1/3 <= spectrum <= 1 (1 for a uniform flow along a panel)
    assert ev.min() >= 1 / 3 - 1e-12 and ev.max() <= 1.0 + 1e-12
    assert np.abs(C + C.T).max() <= 1e-15
    u = np.random.default_rng(5).standard_normal(S1.nhf)
    assert abs(u @ C @ u) <= 1e-14 * (u @ u)          # the Coriolis term does no work
    assert np.abs(C).max() > 0.01


def test_lumped_mass_rows():
    """Horizontal: inside a panel M-ring is the literal row sum of M_h; everywhere it is
    the sum over the face's two cells of the element row sums, 1/3 + 1/6 -+ F_c / 2 (- for
    a xi-face of the cell, + for an eta-face).  Vertical: 2/3 + 1/6 + 1/6 inside the column,
    5/6 next to the surface and the lid (the boundary faces are not unknowns)."""
    S, _ = _system(consistent=True, f0=0.2, eps=0.0)
    rows = np.asarray(S.Mh.sum(axis=1)).ravel()
    for panel in range(6):
        xi_f, eta_f = _panel_interior_faces(S, panel)
        f = np.concatenate([xi_f, eta_f])
        assert np.allclose(S.m_h[f], rows[f], rtol=1e-14)
    m = S.mesh
    sideR = m.nbr_dir[S._side, S.L]
    sgn = lambda side: np.where(side <= 1, -1.0, 1.0)
    closed = (0.5 + sgn(S._side) * S.F[S.L] / 2) + (0.5 + sgn(sideR) * S.F[S.R] / 2)
    assert np.allclose(S.m_h, closed, rtol=1e-14)
    assert S.m_h.min() > 0.5
    nlev = S.nlev
    assert np.allclose(S.m_lump[1], 5 / 6) and np.allclose(S.m_lump[nlev - 1], 5 / 6)
    assert np.allclose(S.m_lump[2:nlev - 1], 1.0)
    # without the consistent mass and the rotation the lumped mass is the identity
    S0, _ = _system(consistent=False, f0=0.0, eps=0.0)
    assert np.all(S0.m_h == 1.0) and np.all(S0.m_lump == 1.0)
    assert (S0.Mh != S0.Mh.T).nnz == 0 and np.allclose(S0.Mh.diagonal(), 1.0)


def test_schur_complement_of_the_lumped_system_scales_every_face():
    """I - D M-ring^{-1} G from the assembled blocks, with M-ring the lumped diagonal,
    is the stencil operator with every coefficient scaled by 1 / M-ring of its face."""
    S, inp = _system(n=2, nlev=4, consistent=True, f0=0.3)
    A = assemble_mixed(S).toarray()
    nu = S.nu
    G, D = A[:nu, nu:], A[nu:, :nu]
    lump = np.concatenate([np.tile(S.m_h, S.nlev), S.m_lump.ravel()])
    H_schur = np.eye(S.np) - D @ (G / lump[:, None])
    H = assemble_helmholtz(Level(S.mesh, inp["g"], CSDT, S.mu, S.mu_h)).toarray()
    assert np.allclose(H_schur, H, rtol=1e-12, atol=1e-9)
    # mu_h is one value per face, seen identically from both of its cells
    m = S.mesh
    for d in range(4):
        assert np.allclose(S.mu_h[d], S.mu_h[m.nbr_dir[d], m.nbr[d]])


def test_coarse_face_factor_is_the_edge_weighted_mean_of_its_fine_faces():
    S, inp = _system(n=4, nlev=3, consistent=True, f0=0.3)
    h = Hierarchy(4, inp["z_if"], R, 2, inp["g"], CSDT, mu=S.mu, mu_h=S.mu_h)
    fine, coarse = h.meshes
    ch = fine.children(coarse)
    C = 5
    # E side of coarse column C: the E faces of its children q = 1 and q = 3
    a, b = ch[1][C], ch[3][C]
    w = fine.edge_len[0][[a, b]]
    assert h.levels[1].mu_h[0][C] == pytest.approx((w[0] * S.mu_h[0][a] + w[1] * S.mu_h[0][b]) / w.sum(),
                                                   rel=1e-14)
    # and consistent from both sides of every coarse face
    for d in range(4):
        assert np.allclose(h.levels[1].mu_h[d], h.levels[1].mu_h[coarse.nbr_dir[d], coarse.nbr[d]], rtol=1e-14)


def test_coarse_face_field_conserves_edge_integrals():
    """restrict_side_field against geometry alone.  For every coarse cell and side, the children
    whose neighbour on that side lies outside the cell (found from the fine mesh's connectivity,
    not from the child numbering) are the two fine faces that make up the coarse face: their
    great-circle lengths add up to the coarse mesh's own edge length, and the restricted value
    conserves the edge integral, L_C f_C = sum_f l_f f_f.  A constant restricts to itself."""
    from oracle.multigrid import restrict_side_field
    z = np.linspace(0.0, 1000.0, 3)
    fine, coarse = Mesh(8, z, R), Mesh(4, z, R)
    parent = fine.parent()
    f = syn.normal(77, 0, 4 * fine.ncol).reshape(4, fine.ncol)
    out = restrict_side_field(fine, coarse, f)
    for d in range(4):
        for C in range(coarse.ncol):
            kids = np.nonzero(parent == C)[0]
            side = [k for k in kids if parent[fine.nbr[d][k]] != C]
            assert len(side) == 2
            lf = fine.edge_len[d][side]
            assert lf.sum() == pytest.approx(coarse.edge_len[d][C], rel=1e-12)
            assert coarse.edge_len[d][C] * out[d][C] == pytest.approx(float(np.dot(lf, f[d][side])), rel=1e-12)
    assert np.allclose(restrict_side_field(fine, coarse, np.full((4, fine.ncol), 2.5)), 2.5, rtol=1e-15)


def test_mixed_gcr_with_consistent_mass_and_rotation_matches_direct_solve():
    """GCR(5) with the lumped Schur-complement MG preconditioner on the full M2^{mu,C}
    system (Earth's rotation, tau_u dt 2 Omega = 0.0437) converges to the direct solution."""
    cfg = syn.small_config(4, 6, levels=2, seed=syn.BASE_SEED + 62, mixed=True,
                           consistent_mass=True, rotation=7.292e-5)
    inp = syn.make_inputs(cfg)
    from oracle.problem import mixed_problem
    S, h = mixed_problem(cfg, inp)
    assert np.abs(S.F).max() == pytest.approx(0.5 * 600 * 2 * 7.292e-5, rel=0.2)
    rhs = np.concatenate([inp["rhs_u"], inp["rhs_p"]])
    x, it, hist = gcr(S.apply, rhs, lambda r: S.precond(r, h.as_preconditioner()), tol=1e-12)
    xs = direct_solve(assemble_mixed(S), rhs)
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    assert np.all(np.diff(hist) <= 0)
