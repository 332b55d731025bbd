"""The seeded input generator: published splitmix64 outputs, determinism, distributions."""
import numpy as np

import synthetic as syn


def test_splitmix64_known_answers():
    # splitmix64 seeded with 0 (Steele, Lea & Flood 2014) starts with these three outputs
    g = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        got = [int(syn._mix64(np.array([g * np.uint64(i)], dtype=np.uint64))[0]) for i in (1, 2, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_streams_are_deterministic_and_distinct():
    a = syn.normal(1, 2, 1000)
    assert np.array_equal(a, syn.normal(1, 2, 1000))
    assert not np.array_equal(a, syn.normal(1, 3, 1000))
    assert np.array_equal(syn.normal(1, 2, 10), a[:10])


def test_distributions():
    u = syn.uniform(7, 1, 200000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.005
    z = syn.normal(7, 2, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_workload_shapes():
    cfg = syn.config("c48")
    inp = syn.make_inputs(cfg)
    assert inp["g"].shape == (30, 13824) and inp["rhs"].shape == (414720,)
    assert inp["rhs_u"].shape == (cfg.n_uface,) and cfg.n_uface == 1257984
    rv = inp["rhs_u"][cfg.n_hface:].reshape(31, 13824)
    assert np.all(rv[0] == 0) and np.all(rv[-1] == 0)
    lg = np.log(inp["g"])
    assert abs(lg.std() - 0.1) < 0.002
    assert syn.config("c192").ncell == 15482880
