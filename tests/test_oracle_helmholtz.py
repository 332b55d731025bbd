"""Pins of the oracle's Helmholtz operator, Thomas solve and block-Jacobi sweep."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import synthetic as syn
from oracle.geometry import Mesh
from oracle.helmholtz import Level, thomas, thomas_excess
from oracle.reference import assemble_helmholtz

R = 6371.0e3
CSDT = 340.0 * 600.0


def _level(n=4, nlev=6, seed=7, g=None, mu=None):
    m = Mesh(n, syn.z_interfaces(nlev), R)
    if g is None:
        g = np.exp(0.1 * syn.normal(seed, 1, nlev * m.ncol)).reshape(nlev, m.ncol)
    return Level(m, g, CSDT, mu)


def _vol(L):
    return L.mesh.dz[:, None] * L.mesh.area[None, :]


def test_constant_field_maps_to_itself():
    L = _level()
    x = np.full(L.shape, 3.25)
    assert np.array_equal(L.apply(x), x)


def test_volume_weighted_symmetry_and_conservation():
    L = _level(n=5, nlev=7)
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(L.shape), rng.standard_normal(L.shape)
    V = _vol(L)
    lhs, rhs = np.sum(y * V * L.apply(x)), np.sum(x * V * L.apply(y))
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(y * V * L.apply(x)))
    # flux form: the volume-integrated exchange terms cancel pairwise
    ex = V * (L.apply(x) - x)
    assert abs(ex.sum()) <= 1e-12 * np.abs(ex).sum()


def test_linear_profile_has_no_interior_vertical_divergence():
    # g = 1 and x = z (horizontally uniform): every vertical flux equals c^2 exactly, so the
    # interior divergence vanishes and only the no-flux lid and surface rows change
    nlev = 9
    m = Mesh(3, syn.z_interfaces(nlev), R)
    L = Level(m, np.ones((nlev, m.ncol)), CSDT)
    x = np.repeat(m.zc[:, None], m.ncol, axis=1)
    y = L.apply(x)
    assert np.allclose(y[1:-1], x[1:-1], rtol=1e-12, atol=1e-9 * CSDT ** 2 / m.dz.min())
    assert np.allclose(y[0] - x[0], -CSDT ** 2 / m.dz[0], rtol=1e-12)
    assert np.allclose(y[-1] - x[-1], CSDT ** 2 / m.dz[-1], rtol=1e-12)


def test_horizontal_coefficients_c1_closed_form():
    # C1: six cells (the cube faces); every edge is a cube edge of angle acos(1/3), every
    # cell has area 4 pi R^2 / 6 and adjacent face centres are pi/2 apart
    m = Mesh(1, syn.z_interfaces(2), R)
    L = Level(m, np.ones((2, 6)), CSDT)
    ref = CSDT ** 2 * (R * math.acos(1 / 3)) / ((4 * math.pi * R * R / 6) * (R * math.pi / 2))
    assert np.allclose(L.a_h, ref, rtol=1e-13)


def test_horizontal_coefficients_c2_closed_form():
    # C2: 24 congruent cells.  Cell (i=1, j=1) of panel 0 has its E and N edges on cube
    # edges (half of an acos(1/3) arc each) and its W and S edges from the face centre to
    # an edge midpoint (angle pi/4).  Its centre is (1, t, t)/|.|, t = tan(pi/8).
    m = Mesh(2, syn.z_interfaces(2), R)
    L = Level(m, np.ones((2, 24)), CSDT)
    t = math.tan(math.pi / 8)
    unit = lambda v: np.array(v) / np.linalg.norm(v)
    ang = lambda a, b: math.acos(np.clip(np.dot(unit(a), unit(b)), -1, 1))
    c = (1, t, t)
    area = 4 * math.pi * R * R / 24
    e_cube, e_in = R * math.acos(1 / 3) / 2, R * math.pi / 4
    d_E = R * ang(c, (t, 1, t))        # across the cube edge onto the +Y face
    d_N = R * ang(c, (t, t, 1))        # across the cube edge onto the +Z face
    d_W = R * ang(c, (1, -t, t))
    d_S = R * ang(c, (1, t, -t))
    col = 0 * 4 + 1 * 2 + 1
    ref = CSDT ** 2 / area * np.array([e_cube / d_E, e_in / d_W, e_cube / d_N, e_in / d_S])
    assert np.allclose(L.a_h[:, 0, col], ref, rtol=1e-12)


def test_assembled_matrix_matches_apply():
    L = _level(n=3, nlev=5)
    A = assemble_helmholtz(L)
    x = np.random.default_rng(1).standard_normal(L.shape)
    assert np.allclose(A @ x.ravel(), L.apply(x).ravel(), rtol=1e-13, atol=1e-9)
    # an M-matrix with unit row excess: row sums are exactly 1
    assert np.allclose(A.sum(axis=1).A.ravel(), 1.0, rtol=0, atol=1e-7)
    assert np.all(A.diagonal() > 0)


def _random_columns(nlev, ncol, seed, vmax=1e7):
    rng = np.random.default_rng(seed)
    a_up = np.exp(rng.uniform(0, math.log(vmax), (nlev, ncol)))
    a_dn = np.exp(rng.uniform(0, math.log(vmax), (nlev, ncol)))
    a_up[-1] = 0.0
    a_dn[0] = 0.0
    s = 1.0 + rng.uniform(0, 20, (nlev, ncol))
    r = rng.standard_normal((nlev, ncol))
    return a_dn, s, a_up, r


def test_thomas_matches_lapack_banded_solver():
    a_dn, s, a_up, r = _random_columns(30, 8, 3, vmax=1e3)
    x = thomas(-a_dn, s + a_dn + a_up, -a_up, r)
    for c in range(8):
        ab = np.zeros((3, 30))
        ab[0, 1:] = -a_up[:-1, c]
        ab[1] = s[:, c] + a_dn[:, c] + a_up[:, c]
        ab[2, :-1] = -a_dn[1:, c]
        assert np.allclose(x[:, c], sla.solve_banded((1, 1), ab, r[:, c]), rtol=1e-12, atol=1e-14)


def test_excess_form_agrees_with_textbook_thomas():
    a_dn, s, a_up, r = _random_columns(70, 16, 4, vmax=1e7)
    x1 = thomas(-a_dn, s + a_dn + a_up, -a_up, r)
    x2 = thomas_excess(a_dn, s, a_up, r)
    res = lambda x: r - (s + a_dn + a_up) * x + np.vstack([a_up[:-1] * x[1:], 0 * x[:1]]) \
        + np.vstack([0 * x[:1], a_dn[1:] * x[:-1]])
    scale = np.abs(r).max()
    assert np.abs(res(x2)).max() <= 1e-9 * scale
    assert np.allclose(x1, x2, rtol=1e-7, atol=1e-12 * np.abs(x2).max())


def test_excess_form_is_accurate_at_extreme_aspect_ratio():
    # against a 50-digit LU solve: the vertically smooth mode at CFL_v^2 ~ 7e6
    mpmath = pytest.importorskip("mpmath")
    a_dn, s, a_up, _ = _random_columns(70, 2, 6, vmax=7e6)
    r = np.ones_like(s)
    x = thomas_excess(a_dn, s, a_up, r)
    mpmath.mp.dps = 50
    for c in range(2):
        A = mpmath.zeros(70, 70)
        for k in range(70):
            A[k, k] = mpmath.mpf(s[k, c]) + mpmath.mpf(a_dn[k, c]) + mpmath.mpf(a_up[k, c])
            if k > 0:
                A[k, k - 1] = -mpmath.mpf(a_dn[k, c])
            if k < 69:
                A[k, k + 1] = -mpmath.mpf(a_up[k, c])
        ref = np.array([float(v) for v in mpmath.lu_solve(A, mpmath.matrix([1] * 70))])
        assert np.abs(x[:, c] - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("omega", [1.0, 0.5])
def test_vertical_only_problem_one_sweep_is_exact(omega):
    L = _level(n=3, nlev=12)
    L.a_h[:] = 0.0                       # H == H_z-hat: block Jacobi is a direct solve
    b = np.random.default_rng(2).standard_normal(L.shape)
    x = L.jacobi(b, np.zeros(L.shape), omega, 1)
    exact = sla.solve(assemble_helmholtz(L).toarray(), b.ravel()).reshape(L.shape)
    assert np.allclose(x, omega * exact, rtol=1e-10, atol=1e-13)


def test_jacobi_sweep_is_the_damped_block_iteration():
    # x1 = x0 + omega Hz^{-1}(b - H x0) with Hz = block-diagonal part of the assembled H
    L = _level(n=2, nlev=5)
    A = assemble_helmholtz(L).toarray()
    nlev, ncol = L.shape
    k_of = np.arange(nlev * ncol) // ncol
    c_of = np.arange(nlev * ncol) % ncol
    same_col = c_of[:, None] == c_of[None, :]
    near = np.abs(k_of[:, None] - k_of[None, :]) <= 1
    Hz = np.where(same_col & near, A, 0.0)
    rng = np.random.default_rng(5)
    b, x0 = rng.standard_normal(nlev * ncol), rng.standard_normal(nlev * ncol)
    ref = x0 + 0.8 * np.linalg.solve(Hz, b - A @ x0)
    got = L.jacobi(b, x0, 0.8, 1).ravel()
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-12)


def test_mu_scales_only_vertical_coefficients():
    L1 = _level(n=2, nlev=4)
    mu = np.full((5, 24), 0.5)
    L2 = Level(L1.mesh, L1.g, CSDT, mu)
    assert np.array_equal(L1.a_h, L2.a_h)
    assert np.allclose(L2.a_up, 0.5 * L1.a_up) and np.allclose(L2.a_dn, 0.5 * L1.a_dn)


def test_level_from_couplings_brute_force_dense_matrix():
    """A level given by arbitrary couplings (a caller's operator): its assembled matrix equals
    the dense matrix built entry by entry from the definition (H x)_i = x_i + sum_f a_if (x_i - x_j),
    and it maps constants to themselves whatever the couplings."""
    from oracle.geometry import Mesh
    from oracle.helmholtz import Level
    from oracle.reference import assemble_helmholtz
    import synthetic as syn
    mesh = Mesh(2, syn.z_interfaces(3), 6.371e6)
    nlev, ncol = mesh.nlev, mesh.ncol
    rng = np.random.default_rng(5)
    a_h = rng.uniform(0.0, 2.0, (4, nlev, ncol))
    a_up = rng.uniform(0.0, 3.0, (nlev, ncol))
    a_dn = rng.uniform(0.0, 3.0, (nlev, ncol))
    a_up[-1] = 0.0
    a_dn[0] = 0.0
    lev = Level.from_couplings(mesh, a_h, a_up, a_dn)
    N = nlev * ncol
    A = np.eye(N)
    for k in range(nlev):
        for c in range(ncol):
            i = k * ncol + c
            for d in range(4):
                j = k * ncol + mesh.nbr[d][c]
                A[i, i] += a_h[d, k, c]
                A[i, j] -= a_h[d, k, c]
            if k + 1 < nlev:
                A[i, i] += a_up[k, c]
                A[i, i + ncol] -= a_up[k, c]
            if k > 0:
                A[i, i] += a_dn[k, c]
                A[i, i - ncol] -= a_dn[k, c]
    assert np.allclose(assemble_helmholtz(lev).toarray(), A, rtol=0, atol=1e-14)
    assert np.allclose(lev.apply(np.full(N, 2.5)), 2.5, rtol=1e-14, atol=0)
    assert np.array_equal(lev.couplings(), np.concatenate([a_h, a_up[None], a_dn[None]]))


def test_nine_point_level_against_its_definition():
    """Level9 (the 9-cell stencil of Sec. 3.5): the assembled matrix equals the dense matrix
    built entry by entry (7-cell stencil plus fluxes to the cells two levels up and down),
    V H is symmetric, constants map to themselves, gamma2 = 0 gives the 7-cell level, and one
    block-Jacobi sweep is x0 + omega Hz^-1 (b - H x0) with Hz the tridiagonal column matrix
    without the next-to-nearest fluxes."""
    from oracle.geometry import Mesh
    from oracle.helmholtz import Level, Level9
    from oracle.reference import assemble_helmholtz
    import synthetic as syn
    mesh = Mesh(2, syn.z_interfaces(6), 6.371e6)
    nlev, ncol = mesh.nlev, mesh.ncol
    g = np.exp(0.1 * syn.normal(4, 1, nlev * ncol)).reshape(nlev, ncol)
    L7 = Level(mesh, g, CSDT)
    L9 = Level9(mesh, g, CSDT, 0.3)
    A7 = assemble_helmholtz(L7).toarray()
    A = A7.copy()
    c2 = CSDT * CSDT
    for k in range(nlev - 2):
        for c in range(ncol):
            flux = 0.3 * c2 * 0.5 * (g[k, c] + g[k + 2, c]) / (mesh.zc[k + 2] - mesh.zc[k])
            i, j = k * ncol + c, (k + 2) * ncol + c
            A[i, i] += flux / mesh.dz[k]
            A[i, j] -= flux / mesh.dz[k]
            A[j, j] += flux / mesh.dz[k + 2]
            A[j, i] -= flux / mesh.dz[k + 2]
    A9 = assemble_helmholtz(L9).toarray()
    assert np.allclose(A9, A, rtol=1e-13, atol=0)
    V = (mesh.area[None, :] * mesh.dz[:, None]).ravel()
    VA = V[:, None] * A9
    assert np.allclose(VA, VA.T, rtol=1e-12, atol=1e-12 * np.abs(VA).max())
    assert np.allclose(L9.apply(np.full(nlev * ncol, -1.5)), -1.5, rtol=1e-13, atol=0)
    x = syn.normal(4, 2, nlev * ncol)
    assert np.array_equal(Level9(mesh, g, CSDT, 0.0).apply(x), L7.apply(x))
    assert np.allclose(L9.apply(x).ravel(), A9 @ x, rtol=1e-12, atol=1e-9)
    k_of = np.arange(nlev * ncol) // ncol
    c_of = np.arange(nlev * ncol) % ncol
    Hz = np.where((c_of[:, None] == c_of[None, :]) & (np.abs(k_of[:, None] - k_of[None, :]) <= 1), A7, 0.0)
    b, x0 = syn.normal(4, 3, nlev * ncol), syn.normal(4, 5, nlev * ncol)
    ref = x0 + 0.8 * np.linalg.solve(Hz, b - A9 @ x0)
    assert np.allclose(L9.jacobi(b, x0, 0.8, 1).ravel(), ref, rtol=1e-10, atol=1e-12)
