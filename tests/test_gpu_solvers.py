"""The pressure solvers of Table 1 (Sec. 4.1, Eq. solver_notation; Sec. 5.1) against the oracle.

K_H(A_H, P_H, eps_H) is one of: MG(L), PreOnly with one V-cycle; line relaxation, PreOnly with
P_H^(Jac)(0.8, 10); Krylov(eps_H), BiCGStab with P_H^(Jac)(1.0, 1); Krylov-MG(eps_H, L), BiCGStab
with one V-cycle.  Checked on their own (helmholtz_solve) against the oracle's block-Jacobi
iteration and BiCGStab (the same iteration count, the iterate to 1e-8, the true residual below
eps_H), and inside the mixed solve (Step 2 of the Schur-complement preconditioner): the solution
against a direct solve and the outer iteration count against the oracle's GCR with the same
pressure solver.
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


# (kind, eps_H, omega, sweeps) of Table 1
TABLE1 = {
    "line_relaxation": ("jacobi", 0.0, 0.8, 10),
    "krylov_1e-2": ("bicgstab_jacobi", 1e-2, 1.0, 1),
    "krylov_1e-3": ("bicgstab_jacobi", 1e-3, 1.0, 1),
    "krylov_1e-6": ("bicgstab_jacobi", 1e-6, 1.0, 1),
    "mg": ("mg", 0.0, 0.8, 0),
    "krylov_mg_1e-2": ("bicgstab_mg", 1e-2, 0.8, 0),
    "krylov_mg_1e-6": ("bicgstab_mg", 1e-6, 0.8, 0),
}


def oracle_pressure_solver(hier, cfg, kind, eps, omega, sweeps):
    """The oracle's K_H: returns (solve(b) -> x, iterations of the last solve)."""
    from oracle.krylov import bicgstab
    H = hier.levels[0]
    mgP = hier.as_preconditioner(cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse)
    jac = lambda r: H.jacobi(r, np.zeros(H.shape), omega, sweeps).ravel()
    last = {"it": 0.0}
    if kind == "mg":
        return mgP, last
    if kind == "jacobi":
        return jac, last
    P = jac if kind == "bicgstab_jacobi" else mgP

    def solve(b):
        x, it, _ = bicgstab(lambda v: H.apply(v).ravel(), b, P, tol=eps, maxiter=200)
        last["it"] = it
        return x
    return solve, last


@pytest.mark.parametrize("name", list(TABLE1))
@pytest.mark.parametrize("case", ["c12", "c20l9"])
def test_pressure_solver_alone(mg, case, name):
    from oracle.problem import pressure_hierarchy
    cfg = syn.config("c12") if case == "c12" else syn.small_config(20, 9, levels=3, seed=syn.BASE_SEED + 91)
    inp = syn.make_inputs(cfg)
    hier = pressure_hierarchy(cfg, inp)
    kind, eps, omega, sweeps = TABLE1[name]
    h = mg.mg_setup_config(cfg, inp, precision="fp64")
    mg.mg_set_pressure_solver(h, kind, eps=eps, omega=omega, sweeps=sweeps)
    b = dev(inp["rhs"])
    x = torch.full_like(b, float("nan"))
    info = mg.helmholtz_solve(h, b, x)
    assert info.converged, info
    solve, last = oracle_pressure_solver(hier, cfg, kind, eps, omega, sweeps)
    ref = solve(inp["rhs"])
    got = host(x)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print(f"{case} {name}: iterations gpu {info.iterations} oracle {last['it']}, difference {err:.2e}")
    if kind == "mg":
        v = torch.empty_like(b)
        mg.vcycle(h, b, v)
        assert torch.equal(v, x)
    assert info.iterations == last["it"]
    assert err <= (1e-10 if kind in ("mg", "jacobi") else 1e-8)
    if kind.startswith("bicgstab"):
        H = hier.levels[0]
        res = np.linalg.norm(inp["rhs"] - H.apply(got).ravel()) / np.linalg.norm(inp["rhs"])
        assert res <= eps * (1 + 1e-6)
        n, it = mg.mg_inner_stats(h)
        assert n == 1 and it == info.iterations
    h.destroy()


MIXED_CASE = syn.small_config(8, 10, levels=3, seed=syn.BASE_SEED + 92, mixed=True)


@pytest.mark.parametrize("name", list(TABLE1))
def test_mixed_solve_with_each_pressure_solver(mg, name):
    from oracle.krylov import gcr
    from oracle.problem import mixed_problem
    from oracle.reference import assemble_mixed, direct_solve
    cfg = MIXED_CASE
    inp = syn.make_inputs(cfg)
    S, hier = mixed_problem(cfg, inp)
    kind, eps, omega, sweeps = TABLE1[name]
    rhs = np.concatenate([inp["rhs_u"], inp["rhs_p"]])
    xs = direct_solve(assemble_mixed(S), rhs)
    solve, _ = oracle_pressure_solver(hier, cfg, kind, eps, omega, sweeps)
    _, oit, _ = gcr(S.apply, rhs, lambda r: S.precond(r, solve), tol=1e-10, restart=cfg.gcr_restart, maxiter=200)
    for precision in ("fp64", "fp32"):
        h = mg.mg_setup_config(cfg, inp, precision=precision)
        mg.mg_set_pressure_solver(h, kind, eps=eps, omega=omega, sweeps=sweeps)
        u = torch.zeros(S.nu, dtype=torch.float64, device="cuda")
        p = torch.zeros(S.np, dtype=torch.float64, device="cuda")
        mg.mg_inner_stats(h)
        info = mg.mixed_solve(h, dev(inp["rhs_u"]), dev(inp["rhs_p"]), u, p, tol=1e-10)
        assert info.converged, info
        got = np.concatenate([host(u), host(p)])
        err = np.linalg.norm(got - xs) / np.linalg.norm(xs)
        n, it = mg.mg_inner_stats(h)
        print(f"{name} {precision}: outer iterations gpu {info.iters} oracle {oit}, error {err:.2e}, "
              f"inner solves {n} iterations {it}")
        assert err <= 1e-8
        if precision == "fp64":
            assert abs(info.iters - oit) <= 1
        if kind.startswith("bicgstab"):
            assert n == info.iters and it >= 0.5 * n
        h.destroy()


def test_pressure_solver_arguments(mg):
    cfg = syn.config("c12")
    inp = syn.make_inputs(cfg)
    h = mg.mg_setup_config(cfg, inp)
    for kw in (dict(kind="jacobi", sweeps=0), dict(kind="bicgstab_mg", eps=-1.0),
               dict(kind="bicgstab_jacobi", max_iter=0)):
        with pytest.raises(mg.MGError):
            mg.mg_set_pressure_solver(h, **kw)
    ps = mg._PSolver(9, 1e-2, 0.8, 1, 10)
    assert mg.load().mg_set_pressure_solver(h.ptr, ps) == mg.MG_ERR_ARG
    # a BiCGStab solve that stops at its iteration limit reports it
    mg.mg_set_pressure_solver(h, "bicgstab_jacobi", eps=1e-14, omega=1.0, sweeps=1, max_iter=2)
    b = dev(inp["rhs"])
    x = torch.zeros_like(b)
    info = mg.helmholtz_solve(h, b, x)
    assert info.status == mg.MG_ERR_NOT_CONVERGED and info.iterations == 2.0
    h.destroy()
