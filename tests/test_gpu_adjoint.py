"""The differentiable pressure solve: pressure_solve_adjoint and the torch autograd wrapper.

* lambda = H^-T g from the library against the oracle's transposed direct solve, to the
  solution accuracy the forward solves are held to (1e-8 relative).  The solver's tolerance
  applies to the volume-scaled system H y = V^-1 g (lambda = V y), and the layer volumes of
  this column vary about tenfold, so the solves run to 1e-12;
* gradients through `solve` (backward = adjoint solve) against the oracle's adjoint and
  against central differences of the loss (exact for the linear map up to the solver
  tolerance), for an FP64 and an FP32 V-cycle."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00756_gb300.build import build
    build()
    import paper_2002_00756_gb300 as mg
    from oracle.problem import pressure_hierarchy
    from oracle.reference import assemble_helmholtz
    cfg = syn.small_config(12, 9, levels=2, seed=syn.BASE_SEED + 42)
    inp = syn.make_inputs(cfg)
    A = assemble_helmholtz(pressure_hierarchy(cfg, inp).levels[0])
    return mg, cfg, inp, A


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_matches_transposed_direct_solve(setup, precision):
    from oracle.reference import adjoint_solve
    mg, cfg, inp, A = setup
    h = mg.mg_setup_config(cfg, inp, precision=precision)
    g = syn.normal(43, 0, cfg.ncell)
    lam = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
    info = mg.pressure_solve_adjoint(h, torch.from_numpy(g).cuda(), lam, tol=1e-12)
    assert info.converged
    ref = adjoint_solve(A, g)
    assert np.linalg.norm(lam.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    h.destroy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autograd_gradient(setup, precision):
    from oracle.reference import adjoint_solve
    mg, cfg, inp, A = setup
    h = mg.mg_setup_config(cfg, inp, precision=precision)
    w = torch.from_numpy(syn.normal(44, 0, cfg.ncell)).cuda()
    b = torch.from_numpy(inp["rhs"]).cuda().requires_grad_(True)
    x = mg.solve(h, b, tol=1e-12)
    loss = (w * x).sum()
    loss.backward()
    grad = b.grad.detach()
    ref = adjoint_solve(A, w.cpu().numpy())
    assert np.linalg.norm(grad.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    # central differences along random directions (the map is linear: exact up to the tolerance)
    with torch.no_grad():
        for seed in (45, 46, 47):
            d = torch.from_numpy(syn.normal(seed, 0, cfg.ncell)).cuda()
            lp = (w * mg.solve(h, b + d, tol=1e-12)).sum()
            lm = (w * mg.solve(h, b - d, tol=1e-12)).sum()
            fd = float(lp - lm) / 2.0
            an = float((grad * d).sum())
            assert abs(fd - an) <= 1e-8 * (abs(an) + float(w.norm() * d.norm()) * 1e-3)
    h.destroy()


def test_coefficient_gradient(setup):
    """helmholtz_coefficient_gradient against the oracle's dL/da = -lam_i (x_i - x_j) (itself
    pinned by central differences), evaluated at the oracle's own x and lambda."""
    from oracle.problem import pressure_hierarchy
    from oracle.reference import adjoint_solve, coefficient_gradient, direct_solve
    mg, cfg, inp, A = setup
    H = pressure_hierarchy(cfg, inp).levels[0]
    x = direct_solve(A, inp["rhs"])
    lam = adjoint_solve(A, syn.normal(48, 0, cfg.ncell))
    ref = coefficient_gradient(H, x, lam).reshape(6, -1)
    h = mg.mg_setup_config(cfg, inp)
    grad = torch.full((6 * cfg.ncell,), float("nan"), dtype=torch.float64, device="cuda")
    mg.helmholtz_coefficient_gradient(h, torch.from_numpy(lam).cuda(), torch.from_numpy(x).cuda(), grad)
    got = grad.cpu().numpy().reshape(6, -1)
    # one product of a difference per entry: rounding of the last bits only
    assert np.allclose(got, ref, rtol=1e-14, atol=1e-14 * np.abs(ref).max())
    h.destroy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_differentiable_solve_at_c96l70(setup, precision):
    """The differentiable-solve workload, C96L70 (3,870,720 unknowns, 4 levels): L = 1/2 ||W x||^2
    with seeded diagonal weights W, x = H^-1 b.  dL/db from the autograd backward pass against
    (1) central differences with h = 1e-6 along 32 seeded directions, to 1e-6 relative, and
    (2) the oracle's gradient lam = H^-T (W^2 x*): x* and lam by the oracle's GCR to 1e-11 on its
    own operator and on the transposed assembled matrix (the residual of lam is measured with
    A^T itself, so the preconditioner used there only speeds it up)."""
    import scipy.sparse as sp
    from oracle.krylov import gcr
    from oracle.problem import pressure_hierarchy
    from oracle.reference import assemble_helmholtz
    mg = setup[0]
    cfg = syn.config("c96")
    inp = syn.make_inputs(cfg)
    wt = np.exp(0.5 * syn.normal(cfg.seed, 90, cfg.ncell))
    W = torch.from_numpy(wt).cuda()
    h = mg.mg_setup_config(cfg, inp, precision=precision)
    b = torch.from_numpy(inp["rhs"]).cuda().requires_grad_(True)
    tol = 1e-13
    x = mg.solve(h, b, tol=tol)
    (0.5 * ((W * x) ** 2).sum()).backward()
    grad = b.grad.detach()
    # Central differences of L along 32 seeded N(0, 1) directions d, L(+) - L(-) formed as
    # 1/2 <W (x+ - x-), W (x+ + x-)> (no two large sums subtracted), x(b +- h d) solved with the
    # FP64 V-cycle.  The loss is quadratic in b, so the difference quotient is exact for every h
    # but for the solves' errors:
    #  * h = 1: those errors (~1e-13 relative) stay far below the change, so the quotient is
    #    the directional derivative itself: checked to 1e-6 of its value;
    #  * h = 1e-6: the solves' errors are divided by h, and <dL/db, d> of a random d is about
    #    1/sqrt(N) of ||dL/db|| ||d|| at N = 3.9e6: checked to 1e-6 of ||dL/db|| ||d||.
    key = ("c96", "fd")
    if key not in _oracle_cache:
        hf = mg.mg_setup_config(cfg, inp, precision="fp64")
        fds = []
        with torch.no_grad():
            for i in range(32):
                d = torch.from_numpy(syn.normal(cfg.seed, 100 + i, cfg.ncell)).cuda()
                row = []
                for hs in (1.0, 1e-6):
                    xp = mg.solve(hf, b + hs * d, tol=tol)
                    xm = mg.solve(hf, b - hs * d, tol=tol)
                    row.append(0.5 * float(((W * (xp - xm)) * (W * (xp + xm))).sum()) / (2.0 * hs))
                fds.append(row)
        hf.destroy()
        _oracle_cache[key] = fds
    worst1, worst6 = 0.0, 0.0
    gnorm = float(grad.norm())
    for i, (fd1, fd6) in enumerate(_oracle_cache[key]):
        d = torch.from_numpy(syn.normal(cfg.seed, 100 + i, cfg.ncell)).cuda()
        an = float((grad * d).sum())
        worst1 = max(worst1, abs(fd1 - an) / abs(an))
        worst6 = max(worst6, abs(fd6 - an) / (gnorm * float(d.norm())))
    print(f"C96L70 {precision}: central differences over 32 directions: h = 1 worst {worst1:.3e} of "
          f"<dL/db, d>; h = 1e-6 worst {worst6:.3e} of ||dL/db|| ||d||")
    assert worst1 <= 1e-6 and worst6 <= 1e-6
    key = ("c96", "oracle")
    if key not in _oracle_cache:
        hier = pressure_hierarchy(cfg, inp)
        H = hier.levels[0]
        P = hier.as_preconditioner(cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse)
        xs, _, hist = gcr(H.apply, inp["rhs"], P, tol=1e-11, restart=cfg.gcr_restart, maxiter=80)
        assert hist[-1] <= 1e-11
        AT = sp.csr_matrix(assemble_helmholtz(H).T)
        vol = (H.mesh.area[None, :] * H.mesh.dz[:, None]).ravel()
        PT = lambda r: vol * P(r / vol)          # a preconditioner for A^T = V A V^-1
        gx = wt * wt * xs
        lam, _, hist = gcr(lambda v: AT @ v, gx, PT, tol=1e-11, restart=cfg.gcr_restart, maxiter=80)
        res = np.linalg.norm(gx - AT @ lam) / np.linalg.norm(gx)
        assert res <= 1e-10
        _oracle_cache[key] = lam
    lam = _oracle_cache[key]
    err = np.linalg.norm(grad.cpu().numpy() - lam) / np.linalg.norm(lam)
    print(f"C96L70 {precision}: dL/db against the oracle gradient {err:.3e}")
    assert err <= 1e-8
    h.destroy()


_oracle_cache = {}
