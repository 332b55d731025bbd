"""mg_smooth_noalloc: block-Jacobi smoothing for callers that cannot allocate device memory.

Callers running a real-time loop, living inside a framework whose memory pool owns the
device or held to a fixed device-memory budget cannot call cudaMalloc when they smooth; this entry
point keeps its intermediate iterate in a fixed device array inside the library instead.
The test calls it through the C ABI and compares it with mg_smooth (same kernels, so the
results agree to the parity tolerance of the other tests, 1e-12 relative), twice in a
row so that the second call meets the array as the first one left it.  It passes run on
its own in a fresh process and after the rest of the suite.
"""
import ctypes

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


def _rel(a, b):
    return float((a - b).norm() / b.norm())


@pytest.mark.parametrize("sweeps,start", [(1, "zero"), (2, "random"), (3, "random"), (3, "alias")])
def test_matches_mg_smooth_on_two_calls_in_a_row(mg, sweeps, start):
    cfg = syn.config("c12")
    inp = syn.make_inputs(cfg)
    h = mg.mg_setup_config(cfg, inp)
    for level in range(cfg.levels):
        n = h.level_cells(level)
        for call in range(2):
            b = torch.from_numpy(syn.normal(40 + call, level, n)).cuda()
            x0 = torch.from_numpy(syn.normal(50 + call, level, n)).cuda()
            ref = torch.empty_like(b)
            mg.mg_smooth(h, level, b, None if start == "zero" else x0, ref, sweeps)
            out = x0.clone() if start == "alias" else torch.full_like(b, float("nan"))
            x_in = None if start == "zero" else (out if start == "alias" else x0)
            mg.mg_smooth_noalloc(h, level, b, x_in, out, sweeps)
            torch.cuda.synchronize()
            assert _rel(out, ref) <= 1e-12, (level, call, _rel(out, ref))
    h.destroy()


def test_status_codes_through_the_c_abi(mg):
    lib = mg.load()
    cfg = syn.config("c12")
    inp = syn.make_inputs(cfg)
    h = mg.mg_setup_config(cfg, inp)
    n = h.level_cells(0)
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    vp = lambda t: ctypes.c_void_p(t.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.mg_smooth_noalloc(h.ptr, 0, vp(b), None, vp(x), 1, s) == mg.MG_OK
    assert lib.mg_smooth_noalloc(h.ptr, 0, vp(b), None, vp(b), 1, s) == mg.MG_ERR_ARG      # b aliases x_out
    assert lib.mg_smooth_noalloc(h.ptr, 9, vp(b), None, vp(x), 1, s) == mg.MG_ERR_ARG      # no such level
    assert lib.mg_smooth_noalloc(h.ptr, 0, vp(b), None, vp(x), -1, s) == mg.MG_ERR_ARG
    h.destroy()
    # a level above the fixed array's size is refused before anything runs
    big = syn.small_config(128, 30, levels=1)
    assert 6 * 128 * 128 * 30 > mg.MG_NOALLOC_MAX_CELLS
    hb = mg.mg_setup_config(big, syn.make_inputs(big))
    nb = hb.level_cells(0)
    bb = torch.zeros(nb, dtype=torch.float64, device="cuda")
    xb = torch.zeros_like(bb)
    assert lib.mg_smooth_noalloc(hb.ptr, 0, vp(bb), None, vp(xb), 1, s) == mg.MG_ERR_ARG
    hb.destroy()
