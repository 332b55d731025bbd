"""mg_autotune: the launch shapes it picks per level change times only.  The V-cycle and the
solve give the same result, bit for bit, before and after tuning, on a level set that uses the
generic restriction (n = 12) and on one whose FP32 levels take both restriction kernels (n = 32)."""
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
    return m


@pytest.mark.parametrize("n,nlev,levels,precision", [(12, 30, 3, "fp64"), (32, 30, 3, "fp32"),
                                                     (32, 20, 3, "fp32_bf16")])
def test_autotune_keeps_results_bit_identical(mg, n, nlev, levels, precision):
    cfg = syn.small_config(n, nlev, levels=levels, seed=syn.BASE_SEED + 90 + n)
    inp = syn.make_inputs(cfg)
    h = mg.mg_setup_config(cfg, inp, precision=precision)
    b = torch.from_numpy(inp["rhs"]).cuda()
    x0 = torch.zeros_like(b)
    mg.vcycle(h, b, x0)
    s0 = torch.zeros_like(b)
    i0 = mg.pressure_solve(h, b, s0, tol=1e-10)
    choices = mg.mg_autotune(h)
    assert len(choices) == levels
    for l, (bd, kc, ring) in enumerate(choices):
        assert bd in (64, 128)
        if l + 1 < levels:
            assert kc in (4, 8, 16, 24, 35, 70) and ring in (0, 1)
        else:
            assert (kc, ring) == (0, -1)
    x1 = torch.zeros_like(b)
    mg.vcycle(h, b, x1)
    assert torch.equal(x0, x1)
    s1 = torch.zeros_like(b)
    i1 = mg.pressure_solve(h, b, s1, tol=1e-10)
    assert i0.converged and i1.converged and i0.iters == i1.iters
    assert torch.equal(s0, s1)
    h.destroy()
