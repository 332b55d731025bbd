"""GPU parity at the benchmarked size, C192L70 (15,482,880 unknowns), in the launch
configuration bench.py times (FP32 V-cycle, FP64 GCR(5), 4 levels).

* Helmholtz apply (FP64): every output against the oracle, elementwise rounding bound.
* V-cycle: FP64 to 1e-12 and FP32 to 1e-4 relative against the oracle's V-cycle.
* pressure_solve at tol 1e-8: the true residual of the GPU solution recomputed by the oracle.
* The FP32-preconditioned solve against the oracle's solution x* (GCR on the oracle's own
  operator to a relative residual of 1e-11): relative error <= 1e-8.
"""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

_cache = {}


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_00756_gb300.build import build
    build()
    import paper_2002_00756_gb300 as mg
    from oracle.problem import pressure_hierarchy
    cfg = syn.config("c192")
    inp = syn.make_inputs(cfg)
    hier = pressure_hierarchy(cfg, inp)
    return mg, cfg, inp, hier


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_apply_full_size(setup):
    mg, cfg, inp, hier = setup
    from test_gpu_parity import abs_apply_scale
    h = mg.mg_setup_config(cfg, inp, precision="fp32")
    x = syn.normal(31, 1, cfg.ncell)
    y = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
    mg.helmholtz_apply(h, dev(x), y)
    H = hier.levels[0]
    assert np.all(np.abs(host(y) - H.apply(x).ravel()) <= 1e-12 * abs_apply_scale(H, x))


def test_vcycle_full_size(setup):
    mg, cfg, inp, hier = setup
    ref = hier.vcycle(inp["rhs"], cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse).ravel()
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-4)):
        h = mg.mg_setup_config(cfg, inp, precision=prec)
        x = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
        mg.vcycle(h, dev(inp["rhs"]), x)
        err = np.linalg.norm(host(x) - ref) / np.linalg.norm(ref)
        print(f"C192L70 {prec} V-cycle relative error vs oracle: {err:.3e}")
        assert err <= tol
        h.destroy()


def test_benchmarked_solve_residual(setup):
    mg, cfg, inp, hier = setup
    h = mg.mg_setup_config(cfg, inp, precision="fp32")
    x = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
    info = mg.pressure_solve(h, dev(inp["rhs"]), x, tol=1e-8)
    assert info.converged and info.rel_res <= 1e-8
    b = inp["rhs"]
    true_res = np.linalg.norm(b - hier.levels[0].apply(host(x)).ravel()) / np.linalg.norm(b)
    print(f"C192L70 fp32 solve: {info.iters} iterations, reported {info.rel_res:.3e}, true {true_res:.3e}")
    assert true_res <= 1.05e-8


def test_fp32_preconditioned_solve_matches_oracle_solution(setup):
    from oracle.krylov import gcr
    mg, cfg, inp, hier = setup
    H = hier.levels[0]
    xs, it, hist = gcr(H.apply, inp["rhs"], hier.as_preconditioner(cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse),
                       tol=1e-11, restart=cfg.gcr_restart, maxiter=60)
    assert hist[-1] <= 1e-11
    h = mg.mg_setup_config(cfg, inp, precision="fp32")
    x = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
    info = mg.pressure_solve(h, dev(inp["rhs"]), x, tol=1e-10)
    assert info.converged
    err = np.linalg.norm(host(x) - xs) / np.linalg.norm(xs)
    print(f"C192L70 fp32-preconditioned solve (tol 1e-10, {info.iters} its) vs oracle x*: {err:.3e}")
    assert err <= 1e-8
