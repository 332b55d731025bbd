"""Pins of the oracle's GCR against the minimal-residual definition and direct solves."""
import numpy as np
import pytest

import synthetic as syn
from oracle.krylov import gcr
from oracle.multigrid import Hierarchy
from oracle.reference import assemble_helmholtz, direct_solve

R = 6371.0e3
CSDT = 340.0 * 600.0


def _nonsym(n=40, seed=0):
    rng = np.random.default_rng(seed)
    return np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.4, rng.standard_normal(n)


def _min_residual(A, b, P, k):
    """min ||b - A x|| over x in P K_k(A P, b), from an orthonormal Krylov basis."""
    AP = A @ P
    K = np.empty((len(b), k))
    v = b.copy()
    for j in range(k):
        K[:, j] = v
        v = AP @ v
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(AP @ Q, b, rcond=None)
    return np.linalg.norm(b - AP @ Q @ y) / np.linalg.norm(b)


@pytest.mark.parametrize("precond", [False, True])
def test_unrestarted_gcr_is_minimal_residual(precond):
    A, b = _nonsym()
    P = np.diag(1.0 / np.diag(A)) if precond else np.eye(len(b))
    _, _, hist = gcr(lambda v: A @ v, b, lambda r: P @ r, tol=1e-30, restart=1000, maxiter=8)
    for k in range(1, 9):
        assert hist[k] == pytest.approx(_min_residual(A, b, P, k), rel=1e-8)


def test_restarted_gcr_residual_is_monotone_and_converges():
    A, b = _nonsym(60, 1)
    x, it, hist = gcr(lambda v: A @ v, b, None, tol=1e-10, restart=5, maxiter=400)
    assert np.all(np.diff(hist) <= 1e-15)
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-10
    # a restart discards the directions: iteration 6 can no longer be the global minimum
    _, _, h5 = gcr(lambda v: A @ v, b, None, tol=1e-30, restart=5, maxiter=6)
    assert h5[6] >= _min_residual(A, b, np.eye(60), 6) * (1 - 1e-10)


def test_exact_preconditioner_converges_in_one_iteration():
    A, b = _nonsym(30, 2)
    Ainv = np.linalg.inv(A)
    _, it, hist = gcr(lambda v: A @ v, b, lambda r: Ainv @ r, tol=1e-12)
    assert it == 1 and hist[-1] < 1e-12


def test_mg_preconditioned_gcr_matches_direct_solve():
    n, nlev = 4, 6
    g = np.exp(0.1 * syn.normal(5, 1, nlev * 6 * n * n))
    h = Hierarchy(n, syn.z_interfaces(nlev), R, 2, g, CSDT)
    H = h.levels[0]
    b = syn.normal(5, 2, nlev * 6 * n * n)
    x, it, hist = gcr(H.apply, b, h.as_preconditioner(), tol=1e-12, restart=5)
    xs = direct_solve(assemble_helmholtz(H), b)
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    assert np.all(np.diff(hist) <= 0)


def test_breakdown_is_reported():
    with pytest.raises(FloatingPointError):
        gcr(lambda v: 0 * v, np.ones(4), None, tol=1e-8)


def test_adjoint_solve_satisfies_the_adjoint_identity_and_the_volume_similarity():
    """adjoint_solve: <A^-T g, b> = <g, A^-1 b> for every b, g; and for the Helmholtz
    operator A^T = V A V^-1 with V the cell volumes (area x layer depth, closed forms of the
    geometry), the relation the GPU adjoint solve relies on."""
    from oracle.problem import pressure_hierarchy
    from oracle.reference import adjoint_solve
    cfg = syn.small_config(4, 5, levels=1, seed=syn.BASE_SEED + 41)
    inp = syn.make_inputs(cfg)
    H = pressure_hierarchy(cfg, inp).levels[0]
    A = assemble_helmholtz(H)
    rng = np.random.default_rng(3)
    g, b = rng.standard_normal(cfg.ncell), rng.standard_normal(cfg.ncell)
    lam, x = adjoint_solve(A, g), direct_solve(A, b)
    assert abs(lam @ b - g @ x) <= 1e-12 * np.linalg.norm(lam) * np.linalg.norm(b)
    V = (H.mesh.area[None, :] * H.mesh.dz[:, None]).ravel()
    D = A.toarray()
    assert np.allclose(D.T, V[:, None] * D / V[None, :], rtol=1e-12, atol=1e-12 * np.abs(D).max())
    # and a plain mistake (the untransposed solve) is caught by the identity
    x2 = direct_solve(A, g)
    assert abs(x2 @ b - g @ x) > 1e-6 * np.linalg.norm(x2) * np.linalg.norm(b)


def test_coefficient_gradient_matches_central_differences():
    """dL/da_{i,f} = -lam_i (x_i - x_j) (oracle.reference.coefficient_gradient) against central
    differences of L = <w, H(a)^-1 b> in single coefficients, horizontal and vertical."""
    from oracle.problem import pressure_hierarchy
    from oracle.reference import adjoint_solve, coefficient_gradient
    cfg = syn.small_config(4, 5, levels=1, seed=syn.BASE_SEED + 51)
    inp = syn.make_inputs(cfg)
    H = pressure_hierarchy(cfg, inp).levels[0]
    b = inp["rhs"]
    w = syn.normal(52, 0, cfg.ncell)
    A = assemble_helmholtz(H)
    x = direct_solve(A, b)
    G = coefficient_gradient(H, x, adjoint_solve(A, w))

    def loss():
        return w @ direct_solve(assemble_helmholtz(H), b)

    for (arr, idx, gi) in [(H.a_h[0], (2, 5), (0, 2, 5)), (H.a_h[3], (1, 17), (3, 1, 17)),
                           (H.a_up, (1, 9), (4, 1, 9)), (H.a_dn, (3, 30), (5, 3, 30))]:
        a0 = arr[idx]
        h = 1e-4 * a0
        arr[idx] = a0 + h
        lp = loss()
        arr[idx] = a0 - h
        lm = loss()
        arr[idx] = a0
        fd = (lp - lm) / (2 * h)
        assert abs(fd - G[gi]) <= 1e-6 * abs(G[gi]) + 1e-12, (gi, fd, G[gi])


def test_bicgstab_iterates_match_the_library_routine():
    """BiCGStab with a right preconditioner is the algorithm scipy implements (Templates form):
    after the same number of steps, with the same preconditioner, the iterates agree."""
    import scipy.sparse.linalg as spla
    from oracle.krylov import bicgstab
    A, b = _nonsym(50, 3)
    Dinv = 1.0 / np.diag(A)
    for k in (1, 2, 5):
        x, it, _ = bicgstab(lambda v: A @ v, b, lambda r: Dinv * r, tol=0.0, maxiter=k)
        M = spla.LinearOperator(A.shape, matvec=lambda r: Dinv * r)
        xs, info = spla.bicgstab(A, b, rtol=0.0, atol=0.0, maxiter=k, M=M)
        assert it == k and info == k
        assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def test_bicgstab_exact_preconditioner_stops_at_the_half_step():
    from oracle.krylov import bicgstab
    A, b = _nonsym(30, 4)
    Ainv = np.linalg.inv(A)
    x, it, hist = bicgstab(lambda v: A @ v, b, lambda r: Ainv @ r, tol=1e-12)
    assert it == 0.5 and hist[-1] <= 1e-12
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=0)


@pytest.mark.parametrize("precond", ["jacobi", "mg"])
def test_bicgstab_on_the_helmholtz_problem_matches_direct_solve(precond):
    """Krylov(eps_H) and Krylov-MG(eps_H, L) of Table 1 on a small Helmholtz problem: the true
    residual is below eps_H and the error below the conditioning bound."""
    from oracle.krylov import bicgstab
    n, nlev = 4, 6
    g = np.exp(0.1 * syn.normal(6, 1, nlev * 6 * n * n))
    hier = Hierarchy(n, syn.z_interfaces(nlev), R, 2, g, CSDT)
    H = hier.levels[0]
    b = syn.normal(6, 2, nlev * 6 * n * n)
    P = (lambda r: H.jacobi(r, np.zeros_like(r), 1.0, 1).ravel()) if precond == "jacobi" else \
        hier.as_preconditioner()
    xs = direct_solve(assemble_helmholtz(H), b)
    for eps in (1e-2, 1e-6, 1e-10):
        x, it, hist = bicgstab(lambda v: H.apply(v).ravel(), b, P, tol=eps)
        res = np.linalg.norm(b - H.apply(x).ravel()) / np.linalg.norm(b)
        assert res <= eps * (1 + 1e-6) and hist[-1] <= eps
        assert it >= 0.5
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
