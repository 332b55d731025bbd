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
