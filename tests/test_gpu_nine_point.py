"""The 9-cell stencil (Sec. 3.5, Fig. 2) with the tridiagonal smoother H_z-hat (Sec. 3.6) on the
GPU against the oracle's Level9 hierarchy.

* apply, residual + restriction: elementwise, rounding bound of the terms involved;
* block-Jacobi sweeps (residual with the full stencil, column solve without the next-to-nearest
  fluxes) and the V-cycle: FP64 to 1e-11 / 1e-12 relative, the FP32 V-cycle per element;
* pressure solve and BiCGStab pressure solve against the direct solution / the oracle's BiCGStab;
* the adjoint solve (V H symmetric here too) against the transposed direct solve.
"""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GAMMA2 = 0.25
CASES = {
    "c12": syn.Config("c12g", n=12, nlev=30, levels=3, seed=syn.BASE_SEED + 0, gamma2=GAMMA2),
    "c20l9": syn.small_config(20, 9, levels=3, seed=syn.BASE_SEED + 14, gamma2=GAMMA2),
    "c6l7": syn.small_config(6, 7, levels=2, seed=syn.BASE_SEED + 11, gamma2=GAMMA2),
    "c5l3": syn.small_config(5, 3, levels=1, seed=syn.BASE_SEED + 12, gamma2=GAMMA2),
    "c2l2": syn.small_config(2, 2, levels=2, seed=syn.BASE_SEED + 62, gamma2=GAMMA2),
}


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00756_gb300.build import build
    build()
    import paper_2002_00756_gb300 as m
    m.load()
    return m


_cache = {}


def problem(name):
    if name not in _cache:
        from oracle.problem import pressure_hierarchy
        cfg = CASES[name]
        inp = syn.make_inputs(cfg)
        _cache[name] = (cfg, inp, pressure_hierarchy(cfg, inp))
    return _cache[name]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def abs_scale9(H, x):
    """sum of |terms| of (H x)_i for the 9-cell stencil."""
    ax = np.abs(np.asarray(x).reshape(H.shape))
    s = ax.copy()
    for d in range(4):
        s += np.abs(H.a_h[d]) * (ax + ax[:, H.mesh.nbr[d]])
    s[:-1] += np.abs(H.a_up[:-1]) * (ax[:-1] + ax[1:])
    s[1:] += np.abs(H.a_dn[1:]) * (ax[1:] + ax[:-1])
    s[:-2] += np.abs(H.b_up[:-2]) * (ax[:-2] + ax[2:])
    s[2:] += np.abs(H.b_dn[2:]) * (ax[2:] + ax[:-2])
    return s.ravel()


@pytest.mark.parametrize("name", list(CASES))
def test_apply_every_level(mg, name):
    cfg, inp, hier = problem(name)
    h = mg.mg_setup_config(cfg, inp)
    for l, H in enumerate(hier.levels):
        x = syn.normal(3, l, H.mesh.nlev * H.mesh.ncol)
        y = torch.empty_like(dev(x))
        if l == 0:
            mg.helmholtz_apply(h, dev(x), y)
        else:
            mg.mg_level_apply(h, l, dev(x), y)
        assert np.all(np.abs(host(y) - H.apply(x).ravel()) <= 1e-12 * abs_scale9(H, x)), l
    h.destroy()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("sweeps,start", [(1, "zero"), (3, "random")])
def test_sweeps_every_level(mg, name, sweeps, start):
    cfg, inp, hier = problem(name)
    h = mg.mg_setup_config(cfg, inp)
    for l, H in enumerate(hier.levels):
        n = H.mesh.nlev * H.mesh.ncol
        b = syn.normal(4, l, n)
        x0 = np.zeros(n) if start == "zero" else syn.normal(5, l, n)
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        mg.mg_smooth(h, l, dev(b), None if start == "zero" else dev(x0), out, sweeps)
        ref = H.jacobi(b, x0, cfg.omega, sweeps).ravel()
        err = np.linalg.norm(host(out) - ref) / np.linalg.norm(ref)
        assert err <= 1e-11, (l, err)
    h.destroy()


@pytest.mark.parametrize("name", ["c12", "c20l9", "c6l7", "c2l2"])
def test_residual_restriction(mg, name):
    from oracle.multigrid import restrict
    cfg, inp, hier = problem(name)
    h = mg.mg_setup_config(cfg, inp)
    for l in range(hier.L - 1):
        H, fine, coarse = hier.levels[l], hier.meshes[l], hier.meshes[l + 1]
        n = H.mesh.nlev * H.mesh.ncol
        b, x = syn.normal(6, l, n), syn.normal(7, l, n)
        bc = torch.empty(H.mesh.nlev * coarse.ncol, dtype=torch.float64, device="cuda")
        mg.mg_residual_restrict(h, l, dev(b), dev(x), bc)
        ref = restrict(fine, coarse, H.residual(b, x)).ravel()
        scale = restrict(fine, coarse, (np.abs(b) + abs_scale9(H, x)).reshape(H.shape)).ravel()
        assert np.all(np.abs(host(bc) - ref) <= 1e-12 * scale), l
    h.destroy()


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle(mg, name):
    cfg, inp, hier = problem(name)
    ref = hier.vcycle(inp["rhs"], cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse).ravel()
    for prec in ("fp64", "fp32"):
        h = mg.mg_setup_config(cfg, inp, precision=prec)
        x = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
        mg.vcycle(h, dev(inp["rhs"]), x)
        got = host(x)
        if prec == "fp64":
            assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        else:
            assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))
        h.destroy()


@pytest.mark.parametrize("name", ["c12", "c20l9", "c6l7"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_pressure_solve(mg, name, precision):
    from oracle.reference import assemble_helmholtz, direct_solve
    cfg, inp, hier = problem(name)
    xs = direct_solve(assemble_helmholtz(hier.levels[0]), inp["rhs"])
    h = mg.mg_setup_config(cfg, inp, precision=precision)
    x = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
    info = mg.pressure_solve(h, dev(inp["rhs"]), x, tol=1e-11)
    assert info.converged
    err = np.linalg.norm(host(x) - xs) / np.linalg.norm(xs)
    print(f"9-cell {name} {precision}: {info.iters} iterations, error {err:.2e}")
    assert err <= 1e-8
    h.destroy()


def test_bicgstab_and_adjoint(mg):
    from oracle.krylov import bicgstab
    from oracle.reference import adjoint_solve, assemble_helmholtz
    cfg, inp, hier = problem("c12")
    H = hier.levels[0]
    h = mg.mg_setup_config(cfg, inp)
    mg.mg_set_pressure_solver(h, "bicgstab_jacobi", eps=1e-6, omega=1.0, sweeps=1)
    x = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
    info = mg.helmholtz_solve(h, dev(inp["rhs"]), x)
    ref, it, _ = bicgstab(lambda v: H.apply(v).ravel(), inp["rhs"],
                          lambda r: H.jacobi(r, np.zeros(H.shape), 1.0, 1).ravel(), tol=1e-6)
    assert info.converged and info.iterations == it
    assert np.linalg.norm(host(x) - ref) <= 1e-8 * np.linalg.norm(ref)
    g = syn.normal(8, 0, cfg.ncell)
    lam = torch.zeros_like(x)
    assert mg.pressure_solve_adjoint(h, dev(g), lam, tol=1e-12).converged
    lref = adjoint_solve(assemble_helmholtz(H), g)
    assert np.linalg.norm(host(lam) - lref) <= 1e-8 * np.linalg.norm(lref)
    h.destroy()


def test_unsupported_calls(mg):
    cfg, inp, hier = problem("c6l7")
    lib = mg.load()
    h = mg.mg_setup_config(cfg, inp)
    v = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
    g6 = torch.zeros(6 * cfg.ncell, dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MGError) as e:
        mg.helmholtz_coefficient_gradient(h, v, v, g6)
    assert e.value.status == mg.MG_ERR_UNSUPPORTED
    with pytest.raises(mg.MGError):
        mg.mg_set_coefficients(h, g6)
    with pytest.raises(mg.MGError):
        mg.mg_autotune(h)
    with pytest.raises(mg.MGError):
        mg.mg_smooth_noalloc(h, 0, v, None, v.clone(), 1)
    for prec in ("fp32_bf16", "fp32_p64"):
        with pytest.raises(mg.MGError) as e:
            mg.mg_setup_config(cfg, inp, precision=prec)
        assert e.value.status == mg.MG_ERR_UNSUPPORTED
    import ctypes
    out = ctypes.c_void_p()
    prm = mg._Params(2, 0.8, 2, 2, 4, 0, 5, 10)
    assert lib.mg_setup_9pt(None, ctypes.byref(prm), None, 0.25, ctypes.byref(out)) == mg.MG_ERR_ARG
    h.destroy()
