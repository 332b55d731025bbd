"""Failure detection by host-side injection (no GPU fault is made): every device and pinned-host
allocation of a set-up is made to fail in turn (mg_inject_alloc_failure).  Each attempt must
return MG_ERR_NOMEM, release everything it had allocated (mg_live_allocations back to its value
before), leave the CUDA context usable, and a set-up afterwards must solve as before.  Covered:
the pressure handle in FP64, FP32 and FP32 with FP64 finest pivots, the mixed handle with the
consistent mass and Coriolis term, the 9-cell handle, the caller-coefficient handle, and the
one-launch ensemble.
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


def _makers(mg):
    """name -> (make() -> handle, solve(handle) -> converged)."""
    from oracle.problem import pressure_hierarchy
    pc = syn.small_config(6, 7, levels=2, seed=syn.BASE_SEED + 11)
    pin = syn.make_inputs(pc)
    mc = syn.small_config(4, 6, levels=2, seed=syn.BASE_SEED + 65, mixed=True, consistent_mass=True,
                          rotation=5.0e-4)
    mi = syn.make_inputs(mc)
    nc = syn.small_config(6, 7, levels=2, seed=syn.BASE_SEED + 11, gamma2=0.25)
    ni = syn.make_inputs(nc)
    coeffs = pressure_hierarchy(pc, pin).levels[0].couplings()

    def pressure(cfg, inp):
        def solve(h):
            x = torch.zeros(cfg.ncell, dtype=torch.float64, device="cuda")
            return mg.pressure_solve(h, dev(inp["rhs"]), x, tol=1e-10).converged
        return solve

    def mixed_solve(h):
        u = torch.zeros(h.nu, dtype=torch.float64, device="cuda")
        p = torch.zeros(h.ncell, dtype=torch.float64, device="cuda")
        return mg.mixed_solve(h, dev(mi["rhs_u"]), dev(mi["rhs_p"]), u, p, tol=1e-10).converged

    return {
        "fp64": (lambda: mg.mg_setup_config(pc, pin, precision="fp64"), pressure(pc, pin)),
        "fp32": (lambda: mg.mg_setup_config(pc, pin, precision="fp32"), pressure(pc, pin)),
        "fp32_p64": (lambda: mg.mg_setup_config(pc, pin, precision="fp32_p64"), pressure(pc, pin)),
        "mixed": (lambda: mg.mg_setup_config(mc, mi, precision="fp32"), mixed_solve),
        "nine": (lambda: mg.mg_setup_config(nc, ni), pressure(nc, ni)),
        "coeffs": (lambda: mg.mg_setup_config(pc, pin, coeffs=coeffs), pressure(pc, pin)),
    }


@pytest.mark.parametrize("kind", ["fp64", "fp32", "fp32_p64", "mixed", "nine", "coeffs"])
def test_every_setup_allocation_failure_is_released(mg, kind):
    lib = mg.load()
    make, solve = _makers(mg)[kind]
    live0 = lib.mg_live_allocations()
    lib.mg_inject_alloc_failure(0)
    h = make()
    n = lib.mg_inject_alloc_failure(0)   # allocations one set-up attempts
    assert lib.mg_live_allocations() > live0
    h.destroy()
    assert lib.mg_live_allocations() == live0
    assert n >= 10, n
    for k in range(1, n + 1):
        lib.mg_inject_alloc_failure(k)
        with pytest.raises(mg.MGError) as e:
            make()
        assert e.value.status == mg.MG_ERR_NOMEM, (k, e.value.status)
        assert lib.mg_live_allocations() == live0, k
    # one past the last allocation: the set-up completes
    lib.mg_inject_alloc_failure(n + 1)
    h = make()
    lib.mg_inject_alloc_failure(0)
    assert solve(h)
    h.destroy()
    assert lib.mg_live_allocations() == live0
    torch.cuda.synchronize()


def test_ensemble_allocation_failures_are_released(mg):
    lib = mg.load()
    cfgs = [syn.small_config(n, 7, levels=2, seed=syn.BASE_SEED + 40 + n) for n in (4, 6)]
    inps = [syn.make_inputs(c) for c in cfgs]
    hs = [mg.mg_setup_config(c, i, precision="fp32") for c, i in zip(cfgs, inps)]
    bs = [dev(i["rhs"]) for i in inps]
    xs = [torch.zeros_like(b) for b in bs]
    live0 = lib.mg_live_allocations()
    lib.mg_inject_alloc_failure(0)
    e = mg.Ensemble(hs, bs, xs, tol=1e-10)
    n = lib.mg_inject_alloc_failure(0)
    e.destroy()
    assert lib.mg_live_allocations() == live0 and n >= 1
    for k in range(1, n + 1):
        lib.mg_inject_alloc_failure(k)
        with pytest.raises(mg.MGError) as err:
            mg.Ensemble(hs, bs, xs, tol=1e-10)
        assert err.value.status == mg.MG_ERR_NOMEM
        assert lib.mg_live_allocations() == live0, k
    lib.mg_inject_alloc_failure(0)
    e = mg.Ensemble(hs, bs, xs, tol=1e-10)
    assert all(i.converged for i in e.solve())
    e.destroy()
    for h in hs:
        h.destroy()
