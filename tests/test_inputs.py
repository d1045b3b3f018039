"""Checks of the seeded input generators (geometry closure, colouring, DVS
quadrature) -- no method arithmetic involved."""
import math

import numpy as np
import pytest

from paper_2303_10846_gb300 import inputs as I


def _closure(m):
    acc = np.zeros((m.n_cell, 3))
    np.add.at(acc, m.face_cell[:, 0], m.face_normal * m.face_area[:, None])
    it = m.face_cell[:, 1] >= 0
    np.add.at(acc, m.face_cell[it, 1], -m.face_normal[it] * m.face_area[it, None])
    return np.abs(acc).max()


def test_hex_cavity_geometry():
    m = I.hex_cavity(8)
    assert m.n_cell == 512 and m.n_face == 1344 + 384
    assert (m.face_cell[:, 1] >= 0).sum() == 1344
    assert (m.face_cell[:, 1] == -2).sum() == 64            # lid
    assert _closure(m) < 1e-14
    assert m.n_colour == 2
    assert abs(m.cell_volume.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("kw", [dict(h_wall=0.7, growth=1.6, h_max=1.0, box_half=1.2),
                                dict(h_wall=0.25, growth=1.3, h_max=0.6)])
def test_tet_sphere_geometry(kw):
    m = I.tet_sphere(**kw)
    assert _closure(m) < 1e-12
    assert np.all(m.cell_volume > 0)
    bh = kw.get("box_half", 2.5)
    # the wall is a polyhedron inscribed in the sphere: volume error ~ area * sag
    assert 0 <= m.cell_volume.sum() - (8 * bh ** 3 - math.pi / 6) < 1.5 * kw["h_wall"] ** 2
    fc = m.face_cell
    it = fc[:, 1] >= 0
    assert np.all(m.cell_colour[fc[it, 0]] != m.cell_colour[fc[it, 1]])
    # normals point from left to right / outward
    d = m.face_center - m.cell_center[fc[:, 0]]
    assert np.all(np.einsum("ij,ij->i", d, m.face_normal) > 0)
    wall = fc[:, 1] == -1
    assert np.all(np.abs(np.linalg.norm(m.face_center[wall], axis=1) - 0.5) < 0.5 * kw["h_wall"])


def test_gauss_hermite_dvs_integrates_maxwellian_moments():
    d = I.gauss_hermite_dvs(8, RT=0.5, centre=(0.2, 0.0, -0.1))
    U = np.array([0.2, 0.0, -0.1])
    c = d.u - U
    M = np.exp(-(c * c).sum(1)) / math.pi ** 1.5
    assert abs(d.w @ M - 1.0) < 1e-13
    assert np.abs((d.w * M) @ d.u - U).max() < 1e-13
    assert abs(d.w @ (0.5 * (c * c).sum(1) * M) - 0.75) < 1e-13


def test_unstructured_dvs_criterion():
    U = (5 * math.sqrt(0.7), 0.0, 0.0)
    d = I.unstructured_dvs(U, 1.0, 1.0, 5.0, True, target=3000)
    assert abs(d.K - 3000) < 150 and np.all(d.w > 0)
    T0 = 1.0 + 0.2 * 25
    r = 3 * math.sqrt(0.5 * T0)
    assert abs(d.w.sum() - 4 / 3 * math.pi * r ** 3) / (4 / 3 * math.pi * r ** 3) < 0.05
    assert np.all(np.linalg.norm(d.u - 0.4 * np.array(U), axis=1) < r)
    n_ball = (np.linalg.norm(d.u - np.array(U), axis=1) < 3 * math.sqrt(0.5)).sum()
    assert abs(n_ball - I.refined_ball_cells(1.0)) < 60         # Eq. solve_weight: 730
