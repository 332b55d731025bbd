"""Caller-supplied stencil coefficients: mg_setup_coeffs, mg_set_coefficients and dL/dcoeff
through the torch autograd wrapper.

* The oracle's own couplings handed to mg_setup_coeffs reproduce the oracle's operator
  (elementwise rounding bound) and V-cycle (1e-12), and the solve its direct solution.
* A flux-symmetric operator that no set of background factors describes (every face and
  vertical coupling scaled by its own factor): helmholtz_apply and the V-cycle against the
  oracle level built from the same couplings, with coarse levels rediscretised from g.
* Couplings that break flux symmetry, are negative or cross the lid are refused and leave
  the handle's operator unchanged.
* solve(h, b, coeffs=a): dL/da from the backward pass against the oracle's -lam_i (x_i - x_j)
  at the oracle's x and lam, and against central differences along flux-symmetric directions.
"""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00756_gb300.build import build
    build()
    import paper_2002_00756_gb300 as m
    m.load()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def symmetric_scaling(H, amp=0.5):
    """Couplings of H with every horizontal face and every vertical face scaled by its own
    factor (the same from both cells, so V_i a_if = V_j a_jf still holds)."""
    nlev, ncol = H.shape
    k = np.arange(nlev)[:, None]
    c = np.arange(ncol)[None, :]
    a_h = np.empty_like(H.a_h)
    for d in range(4):
        nb = H.mesh.nbr[d][None, :]
        a_h[d] = H.a_h[d] * (1.0 + amp * np.sin(0.37 * (c + nb) + 0.11 * k))
    psi = 1.0 + amp * np.cos(0.23 * c + 0.7 * k)          # factor of the face above cell k
    a_up = H.a_up * psi
    a_dn = np.zeros_like(H.a_dn)
    a_dn[1:] = H.a_dn[1:] * psi[:-1]
    return a_h, a_up, a_dn


def setup_case(name="c12"):
    from oracle.problem import pressure_hierarchy
    cfg = syn.config(name) if name in syn.CONFIGS else syn.small_config(20, 9, levels=3, seed=syn.BASE_SEED + 71)
    inp = syn.make_inputs(cfg)
    return cfg, inp, pressure_hierarchy(cfg, inp)


@pytest.mark.parametrize("name", ["c12", "c20l9"])
def test_oracle_couplings_reproduce_the_oracle(mg, name):
    from oracle.reference import assemble_helmholtz, direct_solve
    from test_gpu_parity import abs_apply_scale
    cfg, inp, hier = setup_case(name)
    H = hier.levels[0]
    h = mg.mg_setup_config(cfg, inp, coeffs=H.couplings())
    x = syn.normal(72, 0, cfg.ncell)
    y = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
    mg.helmholtz_apply(h, dev(x), y)
    assert np.all(np.abs(host(y) - H.apply(x).ravel()) <= 1e-12 * abs_apply_scale(H, x))
    v = torch.empty_like(y)
    mg.vcycle(h, dev(inp["rhs"]), v)
    ref = hier.vcycle(inp["rhs"], cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse).ravel()
    assert np.linalg.norm(host(v) - ref) <= 1e-12 * np.linalg.norm(ref)
    xs = direct_solve(assemble_helmholtz(H), inp["rhs"])
    xg = torch.zeros_like(y)
    assert mg.pressure_solve(h, dev(inp["rhs"]), xg, tol=1e-11).converged
    assert np.linalg.norm(host(xg) - xs) <= 1e-8 * np.linalg.norm(xs)
    h.destroy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_operator_no_background_factor_describes(mg, precision):
    from oracle.helmholtz import Level
    from oracle.reference import assemble_helmholtz, direct_solve
    from test_gpu_parity import abs_apply_scale
    cfg, inp, hier = setup_case("c20l9")
    H0 = hier.levels[0]
    H = Level.from_couplings(H0.mesh, *symmetric_scaling(H0))
    hh = hier.with_finest(H)
    h = mg.mg_setup_config(cfg, inp, precision=precision, coeffs=H.couplings())
    x = syn.normal(73, 0, cfg.ncell)
    y = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
    mg.helmholtz_apply(h, dev(x), y)
    assert np.all(np.abs(host(y) - H.apply(x).ravel()) <= 1e-12 * abs_apply_scale(H, x))
    v = torch.empty_like(y)
    mg.vcycle(h, dev(inp["rhs"]), v)
    ref = hh.vcycle(inp["rhs"], cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse).ravel()
    tol = 1e-12 if precision == "fp64" else 1e-4
    assert np.linalg.norm(host(v) - ref) <= tol * np.linalg.norm(ref)
    xs = direct_solve(assemble_helmholtz(H), inp["rhs"])
    xg = torch.zeros_like(y)
    info = mg.pressure_solve(h, dev(inp["rhs"]), xg, tol=1e-11)
    assert info.converged
    assert np.linalg.norm(host(xg) - xs) <= 1e-8 * np.linalg.norm(xs)
    h.destroy()


def test_set_coefficients_on_the_device(mg):
    from oracle.helmholtz import Level
    from test_gpu_parity import abs_apply_scale
    cfg, inp, hier = setup_case("c12")
    H0 = hier.levels[0]
    H = Level.from_couplings(H0.mesh, *symmetric_scaling(H0, 0.3))
    h = mg.mg_setup_config(cfg, inp, precision="fp32")
    mg.mg_set_coefficients(h, dev(H.couplings()))
    x = syn.normal(74, 0, cfg.ncell)
    y = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
    mg.helmholtz_apply(h, dev(x), y)
    assert np.all(np.abs(host(y) - H.apply(x).ravel()) <= 1e-12 * abs_apply_scale(H, x))
    # the GCR operator is the new one too: the solve's true residual under the oracle's H
    xg = torch.zeros_like(y)
    assert mg.pressure_solve(h, dev(inp["rhs"]), xg, tol=1e-10).converged
    res = np.linalg.norm(inp["rhs"] - H.apply(host(xg)).ravel()) / np.linalg.norm(inp["rhs"])
    assert res <= 1.05e-10
    h.destroy()


def test_refused_couplings_leave_the_operator_unchanged(mg):
    cfg, inp, hier = setup_case("c12")
    H = hier.levels[0]
    a = H.couplings()
    h = mg.mg_setup_config(cfg, inp)
    x = dev(syn.normal(75, 0, cfg.ncell))
    y0 = torch.empty_like(x)
    mg.helmholtz_apply(h, x, y0)
    bad = []
    b = a.copy()
    b[0, 3, 5] *= 1.001                  # one side of one face: not flux-symmetric
    bad.append(b)
    b = a.copy()
    b[1, 0, 0] = -b[1, 0, 0]             # negative (and asymmetric)
    bad.append(b)
    b = a.copy()
    b[4, -1, 7] = 1.0                    # flux through the lid
    bad.append(b)
    b = a.copy()
    b[5, 0, 2] = 1.0                     # flux through the surface
    bad.append(b)
    b = a.copy()
    b[2, 4, 9] = np.nan
    bad.append(b)
    for b in bad:
        with pytest.raises(mg.MGError) as e:
            mg.mg_set_coefficients(h, dev(b))
        assert e.value.status == mg.MG_ERR_ARG
        with pytest.raises(mg.MGError):
            mg.mg_setup_config(cfg, inp, coeffs=b)
    y1 = torch.empty_like(x)
    mg.helmholtz_apply(h, x, y1)
    assert torch.equal(y0, y1)
    h.destroy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_autograd_coefficient_gradient(mg, precision):
    """L = 1/2 ||W x||^2 with x = H(a)^-1 b: dL/db and dL/da from one backward pass."""
    from oracle.reference import adjoint_solve, assemble_helmholtz, coefficient_gradient, direct_solve
    cfg = syn.small_config(8, 6, levels=2, seed=syn.BASE_SEED + 76)
    inp = syn.make_inputs(cfg)
    from oracle.problem import pressure_hierarchy
    H = pressure_hierarchy(cfg, inp).levels[0]
    a = H.couplings()
    wt = np.exp(0.5 * syn.normal(77, 0, cfg.ncell))
    h = mg.mg_setup_config(cfg, inp, precision=precision)
    W = dev(wt)
    b = dev(inp["rhs"]).requires_grad_(True)
    coef = dev(a).requires_grad_(True)
    x = mg.solve(h, b, tol=1e-13, coeffs=coef)
    loss = 0.5 * ((W * x) ** 2).sum()
    loss.backward()
    A = assemble_helmholtz(H)
    xs = direct_solve(A, inp["rhs"])
    lam = adjoint_solve(A, wt * wt * xs)
    assert np.linalg.norm(host(b.grad) - lam) <= 1e-8 * np.linalg.norm(lam)
    ref = coefficient_gradient(H, xs, lam).ravel()
    got = host(coef.grad)
    assert np.linalg.norm(got - ref) <= 1e-8 * np.linalg.norm(ref)
    # central differences along flux-symmetric directions: every coupling scaled together, the
    # horizontal couplings alone, and each face scaled by its own factor.  L(+) - L(-) is
    # formed as 1/2 <W (x+ - x-), W (x+ + x-)> (the same number without subtracting two large
    # sums); the step is large enough that the solves' residual (1e-13) stays far below the
    # change it causes, small enough that the O(h^2) term stays below 1e-8
    from oracle.helmholtz import Level
    horiz = a.copy()
    horiz[4:] = 0.0
    dirs = [(a, 1e-6), (horiz, 1e-6),
            (Level.from_couplings(H.mesh, *symmetric_scaling(H, 0.3)).couplings() - a, 1e-4)]
    with torch.no_grad():
        for i, (dd, hstep) in enumerate(dirs):
            d = dev(dd)
            xp = mg.solve(h, b, tol=1e-13, coeffs=coef + hstep * d)
            xm = mg.solve(h, b, tol=1e-13, coeffs=coef - hstep * d)
            fd = 0.5 * float(((W * (xp - xm)) * (W * (xp + xm))).sum()) / (2.0 * hstep)
            an = float((coef.grad * d).sum())
            print(f"{precision} direction {i}: central difference {fd:.12e}, backward pass {an:.12e}")
            assert abs(fd - an) <= 1e-6 * abs(an), (i, fd, an)
    h.destroy()
