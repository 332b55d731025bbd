"""ensemble_pressure_solve: independent pressure solves with interleaved iterations.

Each member must get exactly what pressure_solve gives it alone (the same kernels in the same
order: bit for bit, same iteration count and status), whatever the other members are: here a
mix of meshes, level counts, V-cycle precisions, a zero right-hand side (no iteration) and a
member that stops at its iteration limit.  One member's solution is also checked against the
oracle's operator (true residual)."""
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


MEMBERS = [  # (config, precision, max_iter, rhs scale)
    (syn.config("c12"), "fp32", 200, 1.0),
    (syn.small_config(16, 9, levels=2, seed=syn.BASE_SEED + 31), "fp64", 200, 1.0),
    (syn.small_config(20, 9, levels=3, seed=syn.BASE_SEED + 32), "fp32_bf16", 200, 1.0),
    (syn.small_config(8, 30, levels=3, seed=syn.BASE_SEED + 33), "fp32", 200, 0.0),
    (syn.small_config(24, 12, levels=4, seed=syn.BASE_SEED + 34), "fp32", 2, 1.0),
    (syn.small_config(16, 10, levels=3, seed=syn.BASE_SEED + 36), "fp32_p64", 200, 1.0),
]


def test_members_match_their_single_solves(mg):
    hs, bs, refs = [], [], []
    for cfg, prec, max_iter, scale in MEMBERS:
        inp = syn.make_inputs(cfg, mixed=False)
        h = mg.mg_setup_config(cfg, inp, precision=prec, mixed=False, max_iter=max_iter)
        b = torch.from_numpy(scale * inp["rhs"]).cuda()
        x = torch.full_like(b, float("nan"))
        refs.append((x, mg.pressure_solve(h, b, x, tol=1e-9)))
        hs.append(h)
        bs.append(b)
    for call in range(2):   # the second call meets every handle's cached graphs
        xs = [torch.full_like(b, float("nan")) for b in bs]
        infos = mg.ensemble_pressure_solve(hs, bs, xs, tol=1e-9)
        torch.cuda.synchronize()
        for i, ((xr, ir), x, info) in enumerate(zip(refs, xs, infos)):
            assert info.status == ir.status and info.iters == ir.iters, (call, i, info, ir)
            assert torch.equal(x, xr), (call, i)
    assert infos[3].iters == 0 and float(xs[3].abs().max()) == 0.0
    assert infos[4].status == mg.MG_ERR_NOT_CONVERGED and infos[4].iters == 2
    assert all(infos[i].converged for i in range(4))
    # the first member against the oracle's operator
    from oracle.problem import pressure_hierarchy
    cfg = MEMBERS[0][0]
    inp = syn.make_inputs(cfg, mixed=False)
    H = pressure_hierarchy(cfg, inp).levels[0]
    x0 = xs[0].cpu().numpy()
    true = np.linalg.norm(inp["rhs"] - H.apply(x0).ravel()) / np.linalg.norm(inp["rhs"])
    assert true <= 1.05e-9
    with pytest.raises(mg.MGError):
        mg.ensemble_pressure_solve([hs[0], hs[0]], [bs[0], bs[0]], [xs[0], xs[0].clone()])   # a handle twice
    for h in hs:
        h.destroy()


def test_one_graph_launch_matches_single_solves(mg):
    """mg_ensemble: every member's whole solve in one CUDA graph (device-side convergence
    decisions).  Each member gets what pressure_solve gives it alone, bit for bit, with the same
    iteration count and status, including a zero right-hand side, a member stopped by its
    iteration limit and a member whose right-hand side holds a NaN (breakdown)."""
    hs, bs, xs = [], [], []
    members = MEMBERS + [(syn.small_config(8, 12, levels=2, seed=syn.BASE_SEED + 35), "fp32", 200, 1.0)]
    for cfg, prec, max_iter, scale in members:
        inp = syn.make_inputs(cfg, mixed=False)
        h = mg.mg_setup_config(cfg, inp, precision=prec, mixed=False, max_iter=max_iter)
        b = torch.from_numpy(scale * inp["rhs"]).cuda()
        hs.append(h)
        bs.append(b)
        xs.append(torch.full_like(b, float("nan")))
    bs[-1][5] = float("nan")
    ens = mg.Ensemble(hs, bs, xs, tol=1e-9)
    for call in range(2):
        if call == 1:   # new right-hand sides in the bound buffers (member 3 keeps b = 0)
            for i, b in enumerate(bs[:-1]):
                if i != 3:
                    b.mul_(-0.5).add_(0.25 * torch.from_numpy(syn.normal(60 + i, 0, b.numel())).cuda())
        refs = []
        for h, b in zip(hs, bs):
            x = torch.full_like(b, float("nan"))
            refs.append((x, mg.pressure_solve(h, b, x, tol=1e-9)))
        infos = ens.solve()
        torch.cuda.synchronize()
        for i, ((xr, ir), x, info) in enumerate(zip(refs, xs, infos)):
            assert info.status == ir.status and info.iters == ir.iters, (call, i, info, ir)
            assert info.rel_res == ir.rel_res or (np.isnan(info.rel_res) and np.isnan(ir.rel_res)) or \
                ir.status == mg.MG_ERR_BREAKDOWN
            if ir.status != mg.MG_ERR_BREAKDOWN:
                assert torch.equal(x, xr), (call, i)
            assert info.ms > 0.0
        assert infos[3].iters == 0 and infos[3].converged
        assert infos[4].status == mg.MG_ERR_NOT_CONVERGED and infos[4].iters == 2
        assert infos[-1].status == mg.MG_ERR_BREAKDOWN
    ens.destroy()
    for h in hs:
        h.destroy()


@pytest.mark.parametrize("one_launch", [False, True])
def test_every_member_against_the_oracle_operator(mg, one_launch):
    """Members of the benchmarked kind (C32 and larger, 30 / 50 / 70 levels, 4-level FP32
    V-cycle) and small ones: every member's true residual under the oracle's operator."""
    from oracle.problem import pressure_hierarchy
    shapes = [(32, 30), (40, 50), (48, 70), (8, 30), (16, 50), (24, 70)]
    hs, bs, xs, ops = [], [], [], []
    for i, (n, nlev) in enumerate(shapes):
        cfg = syn.small_config(n, nlev, levels=4 if n % 8 == 0 else 3, seed=syn.BASE_SEED + 300 + i)
        inp = syn.make_inputs(cfg, mixed=False)
        hs.append(mg.mg_setup_config(cfg, inp, precision="fp32", mixed=False))
        bs.append(torch.from_numpy(inp["rhs"]).cuda())
        xs.append(torch.zeros_like(bs[-1]))
        ops.append((pressure_hierarchy(cfg, inp).levels[0], inp["rhs"]))
    if one_launch:
        ens = mg.Ensemble(hs, bs, xs, tol=1e-9)
        infos = ens.solve()
        ens.destroy()
    else:
        infos = mg.ensemble_pressure_solve(hs, bs, xs, tol=1e-9)
    for (H, rhs), x, info, shp in zip(ops, xs, infos, shapes):
        assert info.converged, (shp, info)
        true = np.linalg.norm(rhs - H.apply(x.cpu().numpy()).ravel()) / np.linalg.norm(rhs)
        print(f"member C{shp[0]}L{shp[1]}: {info.iters} iterations, true residual {true:.3e}")
        assert true <= 1.05e-9, shp
    for h in hs:
        h.destroy()
