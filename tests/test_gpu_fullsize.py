"""GPU parity at the benchmarked size, C192L70 (15,482,880 unknowns), in the launch
configuration bench.py times (FP32 V-cycle, FP64 GCR(5), 4 levels), and at two sizes that
reach the launch shapes only large levels use.

* Helmholtz apply (FP64): every output against the oracle, elementwise rounding bound.
* V-cycle, per element: |x_gpu - x_oracle| <= c max|x_oracle| with c = 1e-11 (FP64; measured
  1.1e-12) and c = FP32_VCYCLE_ELEMENT (FP32; measured 2.4e-7 to 2.8e-7 on the large-level
  shapes), so a wrong neighbour, face or child anywhere (e.g. along one panel edge) fails.
* FP32 V-cycles at C96L20 (55,296 columns: the copy-ring residual + restriction) and C144L12
  (124,416 columns: 24 levels per thread, one ragged chunk), per element.
* The FP32 V-cycle (FP32 Thomas pivots on every level) against the FP64 one (FP64 pivots) and
  against MG_FP32_P64 (FP32 data, FP64 elimination on the finest level), per element, and the
  preconditioned solves' iteration counts and errors against the oracle; the same V-cycle
  comparison at the largest time step of the CFL study (dt = 1200 s, CFL_h about 7.9).
* The exact solve bench.py times (FP32 V-cycle, tol SOLVE_TOL, x0 = 0): true residual and
  relative error against the oracle's solution x* (oracle GCR on its own operator to a
  relative residual of 1e-11) <= 1e-8.
"""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

_cache = {}

# worst element of the FP32 V-cycle against the oracle's, relative to its largest element
FP32_VCYCLE_ELEMENT = 1e-6


def element_err(x, ref):
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


def oracle_solution(cfg, inp, hier):
    """x* of the headline workload: the oracle's GCR on its own operator to 1e-11 (cached)."""
    if "xs" not in _cache:
        from oracle.krylov import gcr
        xs, it, hist = gcr(hier.levels[0].apply, inp["rhs"],
                           hier.as_preconditioner(cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse),
                           tol=1e-11, restart=cfg.gcr_restart, maxiter=60)
        assert hist[-1] <= 1e-11
        _cache["xs"] = xs
    return _cache["xs"]


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
    out = {}
    for prec, tol in (("fp64", 1e-11), ("fp32", FP32_VCYCLE_ELEMENT), ("fp32_p64", FP32_VCYCLE_ELEMENT)):
        h = mg.mg_setup_config(cfg, inp, precision=prec)
        x = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
        mg.vcycle(h, dev(inp["rhs"]), x)
        out[prec] = host(x)
        err = np.linalg.norm(out[prec] - ref) / np.linalg.norm(ref)
        el = element_err(out[prec], ref)
        print(f"C192L70 {prec} V-cycle vs oracle: relative 2-norm {err:.3e}, worst element {el:.3e} of max")
        assert el <= tol
        h.destroy()
    # FP32 pivots (FP32 V-cycle) against FP64 pivots (FP64 V-cycle; FP32 V-cycle with the finest
    # level eliminated in FP64), element by element
    for a, b in (("fp32", "fp64"), ("fp32_p64", "fp64"), ("fp32", "fp32_p64")):
        el = element_err(out[a], out[b])
        print(f"C192L70 {a} V-cycle vs {b} V-cycle: worst element {el:.3e} of max")
        assert el <= FP32_VCYCLE_ELEMENT
    assert not np.array_equal(out["fp32"], out["fp32_p64"])   # the FP64 elimination ran


def test_pivot_precision_at_largest_time_step(setup):
    """dt = 1200 s (CFL_h about 7.9, the paper's C192 time step): the V-cycle with FP32 pivots,
    with the finest level's elimination in FP64, and in FP64 throughout, element by element."""
    import dataclasses
    mg, cfg, inp, _ = setup
    cfg = dataclasses.replace(cfg, dt=1200.0)
    inp = syn.make_inputs(cfg)
    out = {}
    for prec in ("fp64", "fp32", "fp32_p64"):
        h = mg.mg_setup_config(cfg, inp, precision=prec)
        x = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
        mg.vcycle(h, dev(inp["rhs"]), x)
        out[prec] = host(x)
        h.destroy()
    for a in ("fp32", "fp32_p64"):
        el = element_err(out[a], out["fp64"])
        print(f"C192L70 dt 1200 s: {a} V-cycle vs fp64 V-cycle: worst element {el:.3e} of max")
        assert el <= FP32_VCYCLE_ELEMENT


@pytest.mark.parametrize("n,nlev", [(96, 20), (144, 12)])
def test_fp32_vcycle_large_level_shapes(setup, n, nlev):
    """Levels of 40k columns or more use the copy-ring residual + restriction, levels of 100k
    or more 24 levels per thread: both against the oracle, element by element."""
    mg = setup[0]
    from oracle.problem import pressure_hierarchy
    cfg = syn.small_config(n, nlev, levels=2, seed=syn.BASE_SEED + 81)
    inp = syn.make_inputs(cfg)
    hier = pressure_hierarchy(cfg, inp)
    ref = hier.vcycle(inp["rhs"], cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse).ravel()
    h = mg.mg_setup_config(cfg, inp, precision="fp32")
    x = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
    mg.vcycle(h, dev(inp["rhs"]), x)
    el = element_err(host(x), ref)
    print(f"C{n}L{nlev} fp32 V-cycle: worst element {el:.3e} of max")
    assert el <= FP32_VCYCLE_ELEMENT
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


def test_benchmarked_solve_error(setup):
    """The solve bench.py times, from x = 0 at its tolerance: relative error against x*."""
    from bench import SOLVE_TOL
    mg, cfg, inp, hier = setup
    xs = oracle_solution(cfg, inp, hier)
    for prec in ("fp32", "fp32_p64", "fp64"):
        h = mg.mg_setup_config(cfg, inp, precision=prec)
        x = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
        info = mg.pressure_solve(h, dev(inp["rhs"]), x, tol=SOLVE_TOL)
        assert info.converged
        err = np.linalg.norm(host(x) - xs) / np.linalg.norm(xs)
        print(f"C192L70 {prec}-preconditioned solve at tol {SOLVE_TOL:g}: {info.iters} iterations, "
              f"relative error vs oracle x* {err:.3e}, worst element {element_err(host(x), xs):.3e} of max")
        assert err <= 1e-8
        h.destroy()


def test_fp32_preconditioned_solve_matches_oracle_solution(setup):
    mg, cfg, inp, hier = setup
    xs = oracle_solution(cfg, inp, hier)
    h = mg.mg_setup_config(cfg, inp, precision="fp32")
    x = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
    info = mg.pressure_solve(h, dev(inp["rhs"]), x, tol=1e-10)
    assert info.converged
    err = np.linalg.norm(host(x) - xs) / np.linalg.norm(xs)
    print(f"C192L70 fp32-preconditioned solve (tol 1e-10, {info.iters} its) vs oracle x*: {err:.3e}")
    assert err <= 1e-8
