"""Pins of the oracle's intergrid transfers and V-cycle (Algorithm 1)."""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle.geometry import Mesh
from oracle.multigrid import Hierarchy, prolongate, restrict
from oracle.reference import assemble_helmholtz

R = 6371.0e3
CSDT = 340.0 * 600.0


def _hier(n=4, nlev=4, levels=2, seed=11, cs_dt=CSDT, gamma2=0.0):
    z = syn.z_interfaces(nlev)
    ncol = 6 * n * n
    g = np.exp(0.1 * syn.normal(seed, 1, nlev * ncol)).reshape(nlev, ncol)
    return Hierarchy(n, z, R, levels, g, cs_dt, gamma2=gamma2)


def test_restriction_is_the_volume_adjoint_of_injection():
    h = _hier(n=8, nlev=3, levels=2)
    fine, coarse = h.meshes
    rng = np.random.default_rng(0)
    r = rng.standard_normal((3, fine.ncol))
    y = rng.standard_normal((3, coarse.ncol))
    Vf = fine.dz[:, None] * fine.area[None, :]
    Vc = coarse.dz[:, None] * coarse.area[None, :]
    lhs = np.sum(Vc * restrict(fine, coarse, r) * y)
    rhs = np.sum(Vf * r * prolongate(fine, y))
    assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(Vf * r))


def test_transfer_special_cases():
    h = _hier(n=8, nlev=3, levels=2)
    fine, coarse = h.meshes
    assert np.array_equal(prolongate(fine, np.full((3, coarse.ncol), 2.5)), np.full((3, fine.ncol), 2.5))
    assert np.allclose(restrict(fine, coarse, np.full((3, fine.ncol), -1.5)), -1.5, rtol=1e-14)
    r = np.random.default_rng(1).standard_normal((3, fine.ncol))
    Vf = fine.dz[:, None] * fine.area[None, :]
    Vc = coarse.dz[:, None] * coarse.area[None, :]
    assert abs(np.sum(Vc * restrict(fine, coarse, r)) - np.sum(Vf * r)) < 1e-12 * np.sum(np.abs(Vf * r))
    # a single child's residual lands in its parent only, weighted by the area ratio
    e = np.zeros((3, fine.ncol))
    e[1, 17] = 1.0
    b = restrict(fine, coarse, e)
    p = fine.parent()[17]
    assert np.count_nonzero(b) == 1 and b[1, p] == pytest.approx(fine.area[17] / coarse.area[p], rel=1e-14)


def test_coarse_levels_rediscretise_restricted_factors():
    h = _hier(n=8, nlev=3, levels=3)
    # constant factors stay constant, so the coarse operator is the C_{n/2} operator with g = 1
    g1 = Hierarchy(8, syn.z_interfaces(3), R, 3, np.ones((3, 384)), CSDT)
    for l in range(3):
        assert np.allclose(g1.levels[l].g, 1.0, rtol=1e-14)
    for l in (1, 2):
        f, c = h.meshes[l - 1], h.meshes[l]
        Vf, Vc = f.area, c.area
        assert np.allclose((h.levels[l].g * Vc).sum(axis=1), (h.levels[l - 1].g * Vf).sum(axis=1), rtol=1e-13)


def _dense_vcycle_matrix(h, level, omega, n_pre, n_post, n_coarse):
    """Algorithm 1 written as matrix algebra on dense assembled operators."""
    H = assemble_helmholtz(h.levels[level]).toarray()
    nlev, ncol = h.levels[level].shape
    k_of = np.arange(nlev * ncol) // ncol
    c_of = np.arange(nlev * ncol) % ncol
    Hz = np.where((c_of[:, None] == c_of[None, :]) & (np.abs(k_of[:, None] - k_of[None, :]) <= 1), H, 0.0)
    lev = h.levels[level]
    if hasattr(lev, "b_up"):
        # 9-cell stencil: H_z-hat drops the next-to-nearest fluxes, their diagonal share too
        Hz -= np.diag((lev.b_up + lev.b_dn).ravel())
    B = omega * np.linalg.inv(Hz)
    I = np.eye(len(H))
    S = I - B @ H

    def sweeps(m):  # x = sum_{i<m} S^i B b from a zero start
        acc, Si = np.zeros_like(H), I
        for _ in range(m):
            acc += Si @ B
            Si = S @ Si
        return acc, Si

    if level == h.L - 1:
        return sweeps(n_coarse)[0]
    fine, coarse = h.meshes[level], h.meshes[level + 1]
    nc = nlev * coarse.ncol
    P = np.zeros((nlev * ncol, nc))
    par = fine.parent()
    for k in range(nlev):
        P[k * ncol + np.arange(ncol), k * coarse.ncol + par] = 1.0
    Vf = np.tile(fine.area, nlev) * np.repeat(fine.dz, ncol)
    Vc = np.tile(coarse.area, nlev) * np.repeat(coarse.dz, coarse.ncol)
    Rm = (P * Vf[:, None]).T / Vc[:, None]
    Mc = _dense_vcycle_matrix(h, level + 1, omega, n_pre, n_post, n_coarse)
    Mpre, _ = sweeps(n_pre)
    Mpost, Spost = sweeps(n_post)
    M = Mpre + P @ Mc @ Rm @ (I - H @ Mpre)
    return Spost @ M + Mpost


@pytest.mark.parametrize("gamma2", [0.0, 0.25])
@pytest.mark.parametrize("levels,n_pre,n_post", [(2, 2, 2), (3, 1, 2), (2, 0, 3)])
def test_vcycle_equals_dense_matrix_form(levels, n_pre, n_post, gamma2):
    h = _hier(n=4, nlev=5, levels=levels, gamma2=gamma2)
    M = _dense_vcycle_matrix(h, 0, 0.8, n_pre, n_post, 3)
    b = np.random.default_rng(3).standard_normal(h.levels[0].shape)
    got = h.vcycle(b, 0.8, n_pre, n_post, 3).ravel()
    assert np.allclose(got, M @ b.ravel(), rtol=1e-10, atol=1e-13)


def test_one_level_vcycle_is_n_coarse_sweeps():
    h = _hier(n=4, nlev=5, levels=1)
    b = np.random.default_rng(4).standard_normal(h.levels[0].shape)
    ref = h.levels[0].jacobi(b, np.zeros_like(b), 0.8, 4)
    assert np.array_equal(h.vcycle(b, 0.8, 2, 2, 4), ref)


def _contraction(n, cfl_h, nlev=10, levels=3, iters=8):
    """Asymptotic error reduction of x <- x + V(b - H x) at a fixed horizontal CFL."""
    dx = 0.5 * math.pi * R / n
    h = _hier(n=n, nlev=nlev, levels=levels, cs_dt=cfl_h * dx)
    H = h.levels[0]
    e = np.random.default_rng(9).standard_normal(H.shape)
    rho = []
    for _ in range(iters):
        e2 = e - h.vcycle(H.apply(e))
        rho.append(np.linalg.norm(e2) / np.linalg.norm(e))
        e = e2
    return rho[-1]


def test_vcycle_contraction_is_mesh_independent():
    # Sec. 3.6: with the vertical treated exactly, the hierarchy removes the horizontal
    # error at all scales, so the contraction factor at fixed CFL_h does not grow with n.
    # The paper prints no factor for this operator: the absolute value is parity unpinned.
    rhos = [_contraction(n, 4.0) for n in (8, 16, 32)]
    assert max(rhos) < 0.5
    assert max(rhos) / min(rhos) < 1.5


def test_level_count_rule_at_large_cfl():
    # Sec. 3.6: the coarse-level problem is well conditioned once 4^-(l-1) CFL_h^2 = O(1),
    # so L = log2(CFL_h) + 1 levels suffice; fewer levels converge ever more slowly
    # (Table 2: MG(1) needs far more outer iterations than MG(L >= 2)).
    rho = [_contraction(16, 8.0, levels=L) for L in (1, 2, 3, 4)]
    assert rho[0] > rho[1] > rho[2] > rho[3]
    assert rho[3] < 0.5


def test_nine_point_vcycle_contraction_is_mesh_independent():
    # the 9-cell stencil (Sec. 3.5) smoothed with the tridiagonal H_z-hat: the V-cycle still
    # contracts independently of the mesh, and about as fast as on the 7-cell stencil
    def rho(n, gamma2):
        dx = 0.5 * math.pi * R / n
        h = _hier(n=n, nlev=10, levels=3, cs_dt=4.0 * dx, gamma2=gamma2)
        H = h.levels[0]
        e = np.random.default_rng(9).standard_normal(H.shape)
        for _ in range(8):
            e2 = e - h.vcycle(H.apply(e))
            r = np.linalg.norm(e2) / np.linalg.norm(e)
            e = e2
        return r
    r9 = [rho(n, 0.25) for n in (8, 16, 32)]
    assert max(r9) < 0.5 and max(r9) / min(r9) < 1.5
    assert abs(rho(16, 0.25) - rho(16, 0.0)) < 0.05
