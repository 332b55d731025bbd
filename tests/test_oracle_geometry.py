"""Pins of the oracle's cubed-sphere geometry against closed forms and the paper's figures."""
import json
import math
import os

import numpy as np
import pytest

import synthetic as syn
from oracle.geometry import Mesh, arc, cube_point

R = 6371.0e3
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_mesh_figures.json")))


def _mesh(n, nlev=4):
    return Mesh(n, syn.z_interfaces(nlev), R)


def _gnomonic_cell_area(x1, x2, y1, y2):
    """Closed-form area of an equiangular gnomonic cell, x = tan(xi), y = tan(eta)
    (Rancic, Purser & Mesinger 1996): F(x, y) = atan(x y / sqrt(1 + x^2 + y^2))."""
    F = lambda x, y: np.arctan(x * y / np.sqrt(1.0 + x * x + y * y))
    return R * R * (F(x2, y2) - F(x1, y2) - F(x2, y1) + F(x1, y1))


@pytest.mark.parametrize("n", [1, 2, 3, 6, 12])
def test_total_area_is_sphere(n):
    m = _mesh(n)
    assert abs(m.area.sum() / (4 * math.pi * R * R) - 1.0) < 1e-13


@pytest.mark.parametrize("n", [3, 8])
def test_cell_area_closed_form(n):
    m = _mesh(n)
    d = 0.5 * math.pi / n
    x1 = np.tan(-0.25 * math.pi + d * m.i)
    x2 = np.tan(-0.25 * math.pi + d * (m.i + 1))
    y1 = np.tan(-0.25 * math.pi + d * m.j)
    y2 = np.tan(-0.25 * math.pi + d * (m.j + 1))
    ref = _gnomonic_cell_area(x1, x2, y1, y2)
    assert np.allclose(m.area, ref, rtol=1e-12, atol=0)


@pytest.mark.parametrize("n", [1, 2, 5, 8])
def test_neighbours_are_a_consistent_pairing(n):
    m = _mesh(n)
    cols = np.arange(m.ncol)
    # the neighbour across side d sees us across side nbr_dir
    assert np.all(m.nbr[m.nbr_dir, m.nbr] == cols[None, :])
    # 4 distinct neighbours, never itself
    s = np.sort(m.nbr, axis=0)
    assert np.all(s[1:] != s[:-1]) and np.all(m.nbr != cols[None, :])
    # shared edges have one length and one centre distance seen from both sides
    assert np.allclose(m.edge_len[m.nbr_dir, m.nbr], m.edge_len, rtol=1e-13)
    assert np.allclose(m.centre_dist[m.nbr_dir, m.nbr], m.centre_dist, rtol=1e-13)


def test_interior_neighbours_follow_panel_indexing():
    n = 6
    m = _mesh(n)
    inner = (m.i > 0) & (m.i < n - 1) & (m.j > 0) & (m.j < n - 1)
    c = np.nonzero(inner)[0]
    assert np.all(m.nbr[0, c] == c + 1) and np.all(m.nbr[1, c] == c - 1)
    assert np.all(m.nbr[2, c] == c + n) and np.all(m.nbr[3, c] == c - n)


def test_each_panel_touches_four_others():
    n = 4
    m = _mesh(n)
    for p in range(6):
        cols = np.nonzero(m.panel == p)[0]
        touched = set(m.panel[m.nbr[:, cols]].ravel()) - {p}
        opposite = {0: 2, 2: 0, 1: 3, 3: 1, 4: 5, 5: 4}[p]
        assert touched == set(range(6)) - {p, opposite}


@pytest.mark.parametrize("n", [3, 7])
def test_panel_side_is_a_cube_edge_arc(n):
    m = _mesh(n)
    # cells of panel 0 on its +i side: their E edges make up one cube edge, which spans
    # the angle acos(1/3) between cube vertices (1,1,-1) and (1,1,1)
    side = (m.panel == 0) & (m.i == n - 1)
    assert abs(m.edge_len[0, side].sum() - R * math.acos(1.0 / 3.0)) < 1e-6


@pytest.mark.parametrize("n", [4, 9])
def test_centre_row_lies_on_a_great_circle(n):
    m = _mesh(n)
    for j in range(n):
        row = np.nonzero((m.panel == 0) & (m.j == j))[0]
        total = m.centre_dist[0, row[:-1]].sum()
        direct = R * arc(m.centre[row[0]], m.centre[row[-1]])
        assert abs(total - direct) < 1e-6 * R / n


def test_face_numbering_lists_every_edge_once():
    m = _mesh(5)
    L, Rr, side = m.hfaces()
    assert len(L) == 2 * m.ncol
    assert np.all(L < Rr)
    pairs = set(zip(L.tolist(), Rr.tolist()))
    assert len(pairs) == len(L)
    # ordered by owner column
    assert np.all(np.diff(L) >= 0)


def test_coarse_mesh_is_nested():
    fine, coarse = _mesh(8), _mesh(4)
    ch = fine.children(coarse)
    assert np.allclose(fine.area[ch].sum(axis=0), coarse.area, rtol=1e-13)
    assert np.all(fine.parent()[ch] == np.arange(coarse.ncol)[None, :])


def test_cube_point_faces_are_outward():
    for p in range(6):
        v = cube_point(p, np.array([0.0]), np.array([0.0]))[0]
        assert np.count_nonzero(v) == 1 and abs(v).sum() == 1.0


def test_paper_mesh_figures():
    g = GOLDEN["c192l30"]
    z = syn.z_interfaces(g["nlev"])
    assert abs(z[1] - z[0] - g["dz_min_m"]) < 1.0
    assert 6 * g["n"] ** 2 * g["nlev"] == pytest.approx(g["pressure_unknowns"], rel=0.01)
    m = Mesh(g["n"], z, R)
    dx = m.centre_dist.mean()
    assert dx / 1e3 == pytest.approx(g["dx_km"], rel=0.05)
    assert g["cs"] * g["dt"] / (0.5 * math.pi * R / g["n"]) == pytest.approx(g["cfl_h"], rel=0.02)
    assert g["cs"] * g["dt"] / (z[1] - z[0]) == pytest.approx(g["cfl_v"], rel=0.15)
    g2 = GOLDEN["c1152l30"]
    assert 6 * g2["n"] ** 2 * g2["nlev"] == pytest.approx(g2["pressure_unknowns"], rel=0.01)
    assert g2["cs"] * g2["dt"] / (0.5 * math.pi * R / g2["n"]) == pytest.approx(g2["cfl_h"], rel=0.02)
    assert 0.5 * math.pi * R / g2["n"] / 1e3 == pytest.approx(g2["dx_km"], rel=0.05)
