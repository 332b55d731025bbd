"""The differentiable mixed solve: mixed_apply_transpose, mixed_solve_adjoint and the torch
autograd wrapper solve_mixed, against the oracle's transposed matrix and transposed direct
solve, with the lumped system and with the consistent velocity mass and Coriolis term.

The library evaluates A^T as S J A-hat J S^-1 (S = diag(W, V) face weights and cell volumes)
and solves the A-hat system, so its tolerance applies to the scaled residual; the solves run
to 1e-12 and are held to 1e-8 against the oracle, the accuracy the forward solves are held to.
At C48L30, where the oracle has no direct solve, the adjoint identity <lambda, b> = <g, x>
with the forward GPU solve x = A^-1 b checks the pair."""
import dataclasses

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = {
    "m4l6": syn.small_config(4, 6, levels=2, seed=syn.BASE_SEED + 72, mixed=True),
    "m2l4": syn.small_config(2, 4, levels=2, seed=syn.BASE_SEED + 73, mixed=True),
    "m4l6f4": syn.small_config(4, 6, levels=2, seed=syn.BASE_SEED + 74, mixed=True,
                               consistent_mass=True, rotation=5.0e-4),
    "m2l4f4": syn.small_config(2, 4, levels=2, seed=syn.BASE_SEED + 75, mixed=True,
                               consistent_mass=True, rotation=5.0e-4),
}
LARGE = {
    "c48": syn.config("c48"),
    "c48f4": dataclasses.replace(syn.config("c48"), name="c48f4", consistent_mass=True, rotation=7.292e-5),
}
_cache = {}


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00756_gb300.build import build
    build()
    import paper_2002_00756_gb300 as m
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def problem(name):
    if name not in _cache:
        from oracle.problem import mixed_problem
        from oracle.reference import assemble_mixed
        cfg = CASES.get(name) or LARGE[name]
        inp = syn.make_inputs(cfg)
        S, _ = mixed_problem(cfg, inp)
        A = assemble_mixed(S) if name in CASES else None
        _cache[name] = (cfg, inp, S, A)
    return _cache[name]


def _zeros(n):
    return torch.zeros(n, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("name", list(CASES))
def test_transposed_operator_matches_the_oracle_matrix(mg, name):
    cfg, inp, S, A = problem(name)
    h = mg.mg_setup_config(cfg, inp)
    v = syn.normal(76, 0, S.nu + S.np)
    yu, yp = _zeros(S.nu), _zeros(S.np)
    mg.mixed_apply_transpose(h, dev(v[:S.nu]), dev(v[S.nu:]), yu, yp)
    ref = A.T @ v
    scale = abs(A).T @ np.abs(v)
    got = np.concatenate([host(yu), host(yp)])
    assert np.all(np.abs(got - ref) <= 1e-12 * scale + 1e-300)
    h.destroy()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_solve_matches_transposed_direct_solve(mg, name, precision):
    from oracle.reference import adjoint_solve
    cfg, inp, S, A = problem(name)
    h = mg.mg_setup_config(cfg, inp, precision=precision)
    g = syn.normal(77, 0, S.nu + S.np)          # surface and lid faces included
    lu, lp = _zeros(S.nu), _zeros(S.np)
    info = mg.mixed_solve_adjoint(h, dev(g[:S.nu]), dev(g[S.nu:]), lu, lp, tol=1e-12)
    assert info.converged, info
    ref = adjoint_solve(A, g)
    got = np.concatenate([host(lu), host(lp)])
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"{name} {precision}: iters {info.iters}, error {err:.2e}")
    assert err <= 1e-8
    h.destroy()


@pytest.mark.parametrize("name", list(LARGE))
def test_adjoint_identity_at_c48(mg, name):
    cfg, inp, S, _ = problem(name)
    h = mg.mg_setup_config(cfg, inp, precision="fp32")
    b_u, b_p = dev(inp["rhs_u"]), dev(inp["rhs_p"])
    g = syn.normal(78, 0, S.nu + S.np)
    u, p = _zeros(S.nu), _zeros(S.np)
    assert mg.mixed_solve(h, b_u, b_p, u, p, tol=1e-11).converged
    lu, lp = _zeros(S.nu), _zeros(S.np)
    info = mg.mixed_solve_adjoint(h, dev(g[:S.nu]), dev(g[S.nu:]), lu, lp, tol=1e-11)
    assert info.converged, info
    lam = np.concatenate([host(lu), host(lp)])
    x = np.concatenate([host(u), host(p)])
    b = np.concatenate([inp["rhs_u"], inp["rhs_p"]])
    lhs, rhs = lam @ b, g @ x
    print(f"{name}: adjoint iters {info.iters}, <lam, b> {lhs:.12e}, <g, x> {rhs:.12e}")
    assert abs(lhs - rhs) <= 1e-8 * np.linalg.norm(lam) * np.linalg.norm(b)
    h.destroy()


@pytest.mark.parametrize("name", ["m4l6", "m4l6f4"])
def test_autograd_gradient_and_central_differences(mg, name):
    """L = <w_u, u> + <w_p, p> for (u, p) = solve_mixed(rhs): rhs.grad against the oracle's
    A^-T w and against central differences of L along random directions."""
    from oracle.reference import adjoint_solve
    cfg, inp, S, A = problem(name)
    h = mg.mg_setup_config(cfg, inp, precision="fp32")
    w = syn.normal(79, 0, S.nu + S.np)
    wu, wp = dev(w[:S.nu]), dev(w[S.nu:])
    ru = dev(inp["rhs_u"]).requires_grad_(True)
    rp = dev(inp["rhs_p"]).requires_grad_(True)
    u, p = mg.solve_mixed(h, ru, rp, tol=1e-12)
    loss = (wu * u).sum() + (wp * p).sum()
    loss.backward()
    grad = np.concatenate([host(ru.grad), host(rp.grad)])
    ref = adjoint_solve(A, w)
    assert np.linalg.norm(grad - ref) <= 1e-8 * np.linalg.norm(ref)

    def L(du, dp):
        with torch.no_grad():
            uu, pp = mg.solve_mixed(h, dev(inp["rhs_u"]) + du, dev(inp["rhs_p"]) + dp, tol=1e-12)
            return float((wu * uu).sum() + (wp * pp).sum())

    rng = np.random.default_rng(80)
    for _ in range(3):
        d = rng.standard_normal(S.nu + S.np)
        du, dp = dev(d[:S.nu]), dev(d[S.nu:])
        eps = 1e-3
        fd = (L(eps * du, eps * dp) - L(-eps * du, -eps * dp)) / (2 * eps)
        assert abs(fd - grad @ d) <= 1e-6 * abs(grad @ d) + 1e-9 * np.linalg.norm(grad) * np.linalg.norm(d)
    h.destroy()


@pytest.mark.parametrize("name", ["m4l6", "m2l4f4", "m4l6f4"])
def test_coefficient_gradient(mg, name):
    """mixed_coefficient_gradient against oracle.reference.mixed_coefficient_gradient: on the
    oracle's own solution and adjoint (the kernel's arithmetic, to rounding), and end to end
    from the GPU's forward and adjoint solves (to the solves' accuracy)."""
    from oracle.reference import adjoint_solve, direct_solve, mixed_coefficient_gradient
    cfg, inp, S, A = problem(name)
    h = mg.mg_setup_config(cfg, inp, precision="fp32")
    rhs = np.concatenate([inp["rhs_u"], inp["rhs_p"]])
    w = syn.normal(83, 0, S.nu + S.np)
    x = direct_solve(A, rhs)
    lam = adjoint_solve(A, w)
    ref = mixed_coefficient_gradient(S, x, lam, cfg.eps)
    nv = (S.nlev + 1) * S.ncol
    gg, gu, gd = _zeros(S.np), _zeros(nv), _zeros(nv)
    mg.mixed_coefficient_gradient(h, dev(lam[:S.nu]), dev(x[:S.nu]), dev(x[S.nu:]), gg, gu, gd)
    for got, r in zip((gg, gu, gd), ref):
        r = r.ravel()
        assert np.allclose(host(got), r, rtol=1e-12, atol=1e-13 * np.abs(r).max())
    # end to end: GPU solution and adjoint
    u, p = _zeros(S.nu), _zeros(S.np)
    assert mg.mixed_solve(h, dev(inp["rhs_u"]), dev(inp["rhs_p"]), u, p, tol=1e-12).converged
    lu, lp = _zeros(S.nu), _zeros(S.np)
    assert mg.mixed_solve_adjoint(h, dev(w[:S.nu]), dev(w[S.nu:]), lu, lp, tol=1e-12).converged
    mg.mixed_coefficient_gradient(h, lu, u, p, gg, gu, gd)
    for got, r in zip((gg, gu, gd), ref):
        r = r.ravel()
        assert np.linalg.norm(host(got) - r) <= 1e-8 * np.linalg.norm(r)
    h.destroy()
