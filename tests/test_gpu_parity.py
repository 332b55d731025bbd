"""GPU parity: every kernel path of libmgsolve.so against the FP64 CPU oracle.

All calls go through the C ABI (ctypes binding).  Tolerances:
  * FP64 kernels: elementwise |gpu - oracle| <= 1e-12 * s_i, where s_i is the sum of the
    absolute values of the terms that make up output i (a rounding-order bound);
  * FP64 V-cycle: 1e-12 relative in the 2-norm (same arithmetic, different summation order);
  * FP32 V-cycle: 1e-4 relative, BF16 coefficients: 5e-2 relative (stated per result:
    BF16 keeps 8 significant bits of every coefficient);
  * solves: relative error <= 1e-8 against the oracle's reference solution x* (sparse LU
    or GCR to a relative residual of 1e-12 on the assembled matrix).
"""
import dataclasses

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "c12": (syn.config("c12"), None),
    "c6l7": (syn.small_config(6, 7, levels=2, seed=syn.BASE_SEED + 11), None),
    "c5l3": (syn.small_config(5, 3, levels=1, seed=syn.BASE_SEED + 12), None),
    "c4l1": (syn.small_config(4, 1, levels=3, seed=syn.BASE_SEED + 13), None),
    "c20l9": (syn.small_config(20, 9, levels=3, seed=syn.BASE_SEED + 14), None),
    # degenerate meshes: one cell per panel (every neighbour on another panel), and a
    # hierarchy whose coarsest level is that mesh, with a single-level column
    "c1l4": (syn.small_config(1, 4, levels=1, seed=syn.BASE_SEED + 61), None),
    "c2l3": (syn.small_config(2, 3, levels=2, seed=syn.BASE_SEED + 62), None),
    "c2l1": (syn.small_config(2, 1, levels=2, seed=syn.BASE_SEED + 63), None),
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


def problem(name, levels=None):
    key = (name, levels)
    if key not in _cache:
        from oracle.problem import pressure_hierarchy
        cfg, _ = CASES[name]
        inp = syn.make_inputs(cfg)
        _cache[key] = (cfg, inp, pressure_hierarchy(cfg, inp, levels))
    return _cache[key]


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def abs_apply_scale(H, x):
    """sum of |terms| of (H x)_i: |x_i| + sum_f |a_if| (|x_i| + |x_j|)."""
    ax = np.abs(np.asarray(x).reshape(H.shape))
    s = ax.copy()
    for d in range(4):
        s += np.abs(H.a_h[d]) * (ax + ax[:, H.mesh.nbr[d]])
    s[:-1] += np.abs(H.a_up[:-1]) * (ax[:-1] + ax[1:])
    s[1:] += np.abs(H.a_dn[1:]) * (ax[1:] + ax[:-1])
    return s.ravel()


@pytest.mark.parametrize("name", list(CASES))
def test_helmholtz_apply(mg, name):
    cfg, inp, hier = problem(name)
    h = mg.mg_setup_config(cfg, inp)
    x = syn.normal(5, 9, cfg.ncell)
    y = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
    mg.helmholtz_apply(h, dev(x), y)
    ref = hier.levels[0].apply(x).ravel()
    bound = 1e-12 * abs_apply_scale(hier.levels[0], x)
    assert np.all(np.abs(host(y) - ref) <= bound)


@pytest.mark.parametrize("name", ["c12", "c20l9", "c4l1"])
def test_level_apply_every_level(mg, name):
    cfg, inp, hier = problem(name)
    h = mg.mg_setup_config(cfg, inp)
    for l, H in enumerate(hier.levels):
        x = syn.normal(6, l, H.mesh.nlev * H.mesh.ncol)
        y = torch.empty_like(dev(x))
        mg.mg_level_apply(h, l, dev(x), y)
        assert np.all(np.abs(host(y) - H.apply(x).ravel()) <= 1e-12 * abs_apply_scale(H, x)), l


@pytest.mark.parametrize("name", ["c12", "c6l7", "c4l1", "c20l9", "c2l3", "c1l4"])
@pytest.mark.parametrize("sweeps,start", [(1, "zero"), (2, "zero"), (1, "random"), (3, "random")])
def test_block_jacobi_sweeps(mg, name, sweeps, start):
    cfg, inp, hier = problem(name)
    h = mg.mg_setup_config(cfg, inp)
    for l, H in enumerate(hier.levels):
        n = H.mesh.nlev * H.mesh.ncol
        b = syn.normal(7, l, n)
        x0 = np.zeros(n) if start == "zero" else syn.normal(8, l, n)
        out = torch.empty(n, dtype=torch.float64, device="cuda")
        mg.mg_smooth(h, l, dev(b), None if start == "zero" else dev(x0), out, sweeps)
        ref = H.jacobi(b, x0, cfg.omega, sweeps).ravel()
        # rounding of b - H x (terms up to CFL_v^2 |x|) reaches the result through
        # Hz^{-1}, whose gain on the vertically smooth mode is O(1): propagate the
        # summation-order bound of every sweep's residual through Hz^{-1} (an M-matrix,
        # so |Hz^{-1} e| <= Hz^{-1} |e|)
        bound, xi = 1e-12 * np.linalg.norm(ref), x0
        for _ in range(sweeps):
            s = abs_apply_scale(H, xi) + np.abs(b)
            bound += 32 * np.finfo(float).eps * cfg.omega * np.linalg.norm(H.hz_solve(s))
            xi = H.jacobi(b, xi, cfg.omega, 1)
        assert np.linalg.norm(host(out) - ref) <= bound, (l, np.linalg.norm(host(out) - ref), bound)


@pytest.mark.parametrize("name", ["c12", "c20l9", "c4l1"])
def test_residual_restrict_and_prolong(mg, name):
    from oracle.multigrid import prolongate, restrict
    cfg, inp, hier = problem(name)
    h = mg.mg_setup_config(cfg, inp)
    for l in range(hier.L - 1):
        H, fine, coarse = hier.levels[l], hier.meshes[l], hier.meshes[l + 1]
        n, nc = fine.nlev * fine.ncol, coarse.nlev * coarse.ncol
        b, x = syn.normal(9, l, n), syn.normal(10, l, n)
        bc = torch.empty(nc, dtype=torch.float64, device="cuda")
        mg.mg_residual_restrict(h, l, dev(b), dev(x), bc)
        ref = restrict(fine, coarse, H.residual(b, x)).ravel()
        scale = restrict(fine, coarse, abs_apply_scale(H, x).reshape(H.shape) + np.abs(b).reshape(H.shape)).ravel()
        assert np.all(np.abs(host(bc) - ref) <= 1e-12 * scale)
        xc = syn.normal(11, l, nc)
        xf = dev(x)
        mg.mg_prolong_add(h, l, dev(xc), xf)
        assert np.array_equal(host(xf), (x.reshape(H.shape) + prolongate(fine, xc)).ravel())


@pytest.mark.parametrize("name", list(CASES))
def test_vcycle_fp64(mg, name):
    cfg, inp, hier = problem(name)
    h = mg.mg_setup_config(cfg, inp)
    b = inp["rhs"]
    x = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
    mg.vcycle(h, dev(b), x)
    ref = hier.vcycle(b, cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse).ravel()
    assert np.linalg.norm(host(x) - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("n_pre,n_post,n_coarse", [(0, 2, 4), (2, 0, 4), (1, 3, 1), (0, 0, 2), (3, 1, 6)])
def test_vcycle_smoothing_counts(mg, n_pre, n_post, n_coarse):
    cfg, inp, hier = problem("c20l9")
    h = mg.mg_setup(cfg.n, cfg.nlev, inp["z_if"], inp["g"], radius=cfg.radius, cs_dt=cfg.cs * cfg.dt,
                    levels=cfg.levels, omega=cfg.omega, n_pre=n_pre, n_post=n_post, n_coarse=n_coarse)
    b = inp["rhs"]
    x = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
    mg.vcycle(h, dev(b), x)
    ref = hier.vcycle(b, cfg.omega, n_pre, n_post, n_coarse).ravel()
    assert np.linalg.norm(host(x) - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("fp32_p64", 1e-4), ("fp32_bf16", 5e-2)])
@pytest.mark.parametrize("name", ["c12", "c20l9", "c5l3", "c2l3", "c4l1", "c2l1"])
def test_vcycle_reduced_precision(mg, name, precision, tol):
    cfg, inp, hier = problem(name)
    h = mg.mg_setup_config(cfg, inp, precision=precision)
    b = inp["rhs"]
    x = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
    mg.vcycle(h, dev(b), x)
    ref = hier.vcycle(b, cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse).ravel()
    err = np.linalg.norm(host(x) - ref) / np.linalg.norm(ref)
    print(f"{name} {precision} V-cycle relative error vs FP64 oracle: {err:.3e}")
    assert err <= tol


# 6 * 66^2 = 26136 columns: FP32 sweeps with the full 128-thread blocks of the large
# levels and a ragged last block (26136 = 408 * 64 + 24 columns), an odd column height
# (9: the upper half of each column is one level shorter) and an odd coarse n (33).  FP32
# rounding reaches the V-cycle result at about 1e-7 relative; a wrong neighbour or
# coefficient in any part of the mesh is far above the 2e-6 allowed here.
CASES["c66l9"] = (syn.small_config(66, 9, levels=2, seed=syn.BASE_SEED + 15), None)


@pytest.mark.parametrize("precision", ["fp32", "fp32_p64"])
@pytest.mark.parametrize("n_pre,n_post,n_coarse", [(2, 2, 4), (0, 2, 4), (1, 3, 1), (2, 0, 2)])
def test_vcycle_fp32_large_ragged_level(mg, n_pre, n_post, n_coarse, precision):
    cfg, inp, hier = problem("c66l9")
    assert cfg.ncol >= 128 * 150 and cfg.ncol % 64 != 0 and cfg.nlev % 2 == 1
    h = mg.mg_setup(cfg.n, cfg.nlev, inp["z_if"], inp["g"], radius=cfg.radius, cs_dt=cfg.cs * cfg.dt,
                    levels=cfg.levels, omega=cfg.omega, n_pre=n_pre, n_post=n_post, n_coarse=n_coarse,
                    precision=precision)
    b = inp["rhs"]
    x = torch.empty(cfg.ncell, dtype=torch.float64, device="cuda")
    mg.vcycle(h, dev(b), x)
    ref = hier.vcycle(b, cfg.omega, n_pre, n_post, n_coarse).ravel()
    err = np.linalg.norm(host(x) - ref) / np.linalg.norm(ref)
    print(f"c66l9 {precision} V-cycle ({n_pre},{n_post},{n_coarse}) relative error vs FP64 oracle: {err:.3e}")
    assert err <= 2e-6


def _xstar(name):
    from oracle.reference import assemble_helmholtz, direct_solve
    cfg, inp, hier = problem(name)
    key = ("xstar", name)
    if key not in _cache:
        _cache[key] = direct_solve(assemble_helmholtz(hier.levels[0]), inp["rhs"])
    return _cache[key]


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_p64", "fp32_bf16"])
@pytest.mark.parametrize("name", ["c12", "c20l9", "c5l3", "c2l3", "c1l4"])
def test_pressure_solve(mg, name, precision):
    from oracle.krylov import gcr
    cfg, inp, hier = problem(name)
    h = mg.mg_setup_config(cfg, inp, precision=precision)
    x = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
    info = mg.pressure_solve(h, dev(inp["rhs"]), x, tol=1e-10)
    assert info.converged and info.rel_res <= 1e-10
    xs = _xstar(name)
    err = np.linalg.norm(host(x) - xs) / np.linalg.norm(xs)
    assert err <= 1e-8, err
    # the recursive residual the solver reports is the true one
    true_res = np.linalg.norm(inp["rhs"] - hier.levels[0].apply(host(x)).ravel()) / np.linalg.norm(inp["rhs"])
    assert true_res <= 2e-10
    if precision == "fp64":
        _, it, _ = gcr(hier.levels[0].apply, inp["rhs"], hier.as_preconditioner(cfg.omega, cfg.n_pre, cfg.n_post,
                                                                                 cfg.n_coarse), tol=1e-10)
        assert abs(info.iters - it) <= 1


def test_solver_status_paths(mg):
    cfg, inp, hier = problem("c6l7")
    h = mg.mg_setup_config(cfg, inp, max_iter=1)
    x = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
    info = mg.pressure_solve(h, dev(inp["rhs"]), x, tol=1e-14)
    assert info.status == mg.MG_ERR_NOT_CONVERGED and info.iters == 1
    h2 = mg.mg_setup_config(cfg, inp)
    zero = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
    x.fill_(3.0)
    info = mg.pressure_solve(h2, zero, x, tol=1e-8)
    assert info.converged and info.iters == 0 and float(x.abs().max()) == 0.0
    bad = dev(inp["rhs"])
    bad[17] = float("nan")
    info = mg.pressure_solve(h2, bad, x, tol=1e-8)
    assert info.status == mg.MG_ERR_BREAKDOWN
    with pytest.raises(mg.MGError):
        mg.vcycle(h2, bad, bad)
    u = torch.zeros(10, dtype=torch.float64, device="cuda")
    assert mg.load().mixed_solve(h2.ptr, mg._raw_ptr(u), mg._raw_ptr(u), mg._raw_ptr(u), mg._raw_ptr(u), 1e-8, None,
                                 mg._stream(None)) == mg.MG_ERR_UNSUPPORTED


def test_repeat_calls_are_bitwise_deterministic(mg):
    cfg, inp, hier = problem("c12")
    h = mg.mg_setup_config(cfg, inp, precision="fp32")
    b = dev(inp["rhs"])
    outs = []
    for _ in range(3):
        x = torch.zeros_like(b)
        mg.pressure_solve(h, b, x, tol=1e-9)
        outs.append(host(x))
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


def test_graph_replay_matches_direct_launches(mg):
    """GCR iterations run from captured CUDA graphs after the first solve on a handle, and
    as direct launches while per-launch profiling is on: both give bitwise the same x."""
    cfg, inp, hier = problem("c20l9")
    h = mg.mg_setup_config(cfg, inp, precision="fp32")
    b = dev(inp["rhs"])
    x1 = torch.zeros_like(b)
    mg.pressure_solve(h, b, x1, tol=1e-9)          # captures the graphs
    x2 = torch.zeros_like(b)
    i2 = mg.pressure_solve(h, b, x2, tol=1e-9)     # replays them
    mg.mg_profile_start(h, 1 << 14)
    x3 = torch.zeros_like(b)
    i3 = mg.pressure_solve(h, b, x3, tol=1e-9)     # direct launches
    recs = mg.mg_profile_stop(h)
    assert len(recs) > 0 and i2.iters == i3.iters
    assert torch.equal(x1, x2) and torch.equal(x2, x3)


# ---------------------------------------------------------------------------------------
# mixed (u, p) system

MIXED = {
    "m4l6": syn.small_config(4, 6, levels=2, seed=syn.BASE_SEED + 21, mixed=True),
    "m2l4": syn.small_config(2, 4, levels=2, seed=syn.BASE_SEED + 64, mixed=True),   # coarsest C1
    "c48": syn.config("c48"),
    # consistent velocity mass and implicit Coriolis term (Eq. M2muCdef): a strong rotation
    # (tau_u dt 2 Omega ~ 0.3) on small meshes, the Earth's on C48L30
    "m4l6f4": syn.small_config(4, 6, levels=2, seed=syn.BASE_SEED + 65, mixed=True,
                               consistent_mass=True, rotation=5.0e-4),
    "m2l4f4": syn.small_config(2, 4, levels=2, seed=syn.BASE_SEED + 66, mixed=True,
                               consistent_mass=True, rotation=5.0e-4),
    "c48f4": dataclasses.replace(syn.config("c48"), name="c48f4", consistent_mass=True, rotation=7.292e-5),
}


def mixed_problem(name):
    key = ("mixed", name)
    if key not in _cache:
        from oracle.problem import mixed_problem as mp
        cfg = MIXED[name]
        inp = syn.make_inputs(cfg)
        S, hier = mp(cfg, inp)
        _cache[key] = (cfg, inp, S, hier)
    return _cache[key]


@pytest.mark.parametrize("name", list(MIXED))
def test_mixed_apply_and_schur(mg, name):
    cfg, inp, S, hier = mixed_problem(name)
    h = mg.mg_setup_config(cfg, inp)
    v = syn.normal(12, 0, S.nu + S.np)
    yu = torch.empty(S.nu, dtype=torch.float64, device="cuda")
    yp = torch.empty(S.np, dtype=torch.float64, device="cuda")
    mg.mixed_apply(h, dev(v[:S.nu]), dev(v[S.nu:]), yu, yp)
    ref = S.apply(v)
    absS = abs(S.apply(np.abs(v)))   # sums of |terms| up to the sign of the differences
    got = np.concatenate([host(yu), host(yp)])
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * absS.max())
    mg.schur_precond(h, dev(v[:S.nu]), dev(v[S.nu:]), yu, yp)
    pref = S.precond(v, hier.as_preconditioner(cfg.omega, cfg.n_pre, cfg.n_post, cfg.n_coarse))
    got = np.concatenate([host(yu), host(yp)])
    assert np.linalg.norm(got - pref) <= 1e-11 * np.linalg.norm(pref)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_p64"])
@pytest.mark.parametrize("name", list(MIXED))
def test_mixed_solve(mg, name, precision):
    from oracle.reference import assemble_mixed, direct_solve, iterative_reference
    cfg, inp, S, hier = mixed_problem(name)
    key = ("mxstar", name)
    rhs = np.concatenate([inp["rhs_u"], inp["rhs_p"]])
    if key not in _cache:
        A = assemble_mixed(S)
        if S.nu + S.np <= 20000:
            _cache[key] = direct_solve(A, rhs)
        else:
            _cache[key] = iterative_reference(A, rhs, lambda r: S.precond(r, hier.as_preconditioner()))
    xs = _cache[key]
    h = mg.mg_setup_config(cfg, inp, precision=precision)
    u = torch.zeros(S.nu, dtype=torch.float64, device="cuda")
    p = torch.zeros(S.np, dtype=torch.float64, device="cuda")
    info = mg.mixed_solve(h, dev(inp["rhs_u"]), dev(inp["rhs_p"]), u, p, tol=1e-11)
    assert info.converged, info
    got = np.concatenate([host(u), host(p)])
    err = np.linalg.norm(got - xs) / np.linalg.norm(xs)
    perr = np.linalg.norm(got[S.nu:] - xs[S.nu:]) / np.linalg.norm(xs[S.nu:])
    print(f"{name} {precision}: iters {info.iters}, error {err:.2e}, pressure error {perr:.2e}")
    assert err <= 1e-8 and perr <= 1e-8


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_p64"])
def test_solve_is_scale_invariant(mg, precision):
    """H x = 2^-70 b gives 2^-70 x, bit for bit, in the same iterations: every scalar of GCR and
    every value of the V-cycle scales by a power of two (residual norms down to 1e-30 and
    their squares included), so no step may flush, saturate or stop early on small data."""
    cfg, inp, hier = problem("c12")
    h = mg.mg_setup_config(cfg, inp, precision=precision)
    b = dev(inp["rhs"])
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    i1 = mg.pressure_solve(h, b, x1, tol=1e-10)
    i2 = mg.pressure_solve(h, b * 2.0 ** -70, x2, tol=1e-10)
    assert i1.converged and i2.converged and i1.iters == i2.iters, (i1, i2)
    assert torch.equal(x2, x1 * 2.0 ** -70)
