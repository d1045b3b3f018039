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


def _axisym_volume(prof):
    """Volume of revolution of a closed (x, r) profile (Pappus: 2 pi * area * centroid r)."""
    P = np.asarray(prof)
    P = np.concatenate([P, P[:1]])
    x, r = P[:, 0], P[:, 1]
    cross = x[:-1] * r[1:] - x[1:] * r[:-1]
    area = 0.5 * cross.sum()
    rc = ((r[:-1] + r[1:]) * cross).sum() / (6.0 * area)
    return abs(2.0 * math.pi * area * rc)


@pytest.mark.parametrize("which", ["capsule", "cone"])
def test_axisymmetric_body_meshes(which):
    """Closed, positive, properly coloured; the meshed volume is the box minus the body
    (inscribed faceting: small deficit); wall faces lie on the body."""
    if which == "capsule":
        prof = I.capsule_profile()
        lo, hi, aoa = np.array([-3.2, -4, -4]), np.array([4.8, 4, 4]), 25.0
    else:
        prof = I.sphere_cone_profile()
        lo, hi, aoa = np.array([-4, -5, -5]), np.array([10, 5, 5]), 0.0
    m, dist = I.tet_axisym_body(prof, aoa, lo, hi, 0.15, 1.3, 0.8, 7, which)
    assert _closure(m) < 1e-12
    assert np.all(m.cell_volume > 0) and np.all(dist > 0)
    box = np.prod(hi - lo)
    body = _axisym_volume(prof)
    # the body is replaced by a faceted hole; the volume error is about surface area x
    # a fraction of the wall spacing
    area = 2 * math.pi * np.sum(0.5 * (prof[1:, 1] + prof[:-1, 1]) * np.hypot(*np.diff(prof, axis=0).T))
    assert abs(m.cell_volume.sum() - (box - body)) < 0.2 * area * 0.15
    fc = m.face_cell
    it = fc[:, 1] >= 0
    assert np.all(m.cell_colour[fc[it, 0]] != m.cell_colour[fc[it, 1]])
    wall = fc[:, 1] == -1
    assert wall.sum() > 100 and (fc[:, 1] == -2).sum() > 100
    # wall face centres are on the body surface (within the faceting sag)
    xc = 0.5 * (prof[:, 0].min() + prof[:, 0].max())
    a = math.radians(aoa)
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    b = (m.face_center[wall] - [xc, 0, 0]) @ Rz + [xc, 0, 0]
    sd = I._axisym_sdf(prof, b[:, 0], np.hypot(b[:, 1], b[:, 2]))
    assert np.max(np.abs(sd)) < 0.05


def test_capsule_and_scale_workload_sizes():
    """The capsule configuration: ~200k tetrahedra x ~6,000 velocities (Mach 10, 25
    degrees); the scale DVS: ~8,000 velocities (the mesh is built on the GPU runs)."""
    wl = I.capsule_workload()
    assert 190_000 < wl.mesh.n_cell < 220_000 and 5_500 < wl.dvs.K < 6_500
    assert wl.bcs[0].T == pytest.approx(300.0 / 142.0)
    U = np.asarray(wl.bcs[1].U)
    assert np.linalg.norm(U) == pytest.approx(10.0 * math.sqrt(1.4 * I.R_GAS))
    a = math.sqrt(1.4 * I.R_GAS)
    d = I.unstructured_dvs((8 * a, 0, 0), 1.0, 1.0, 8.0, transitional=False, target=8000, seed=20266)
    assert 7_500 < d.K < 8_500


def test_unstructured_dvs_criterion_variants():
    """The constants of the Sec. 4.4 criterion as parameters: the defaults are the
    criterion's (3 sqrt(R T0) transitional, centre 0.4 U), the outer radius and centre
    follow their factors, and without refined balls the size is the target and the
    weights fill the outer ball."""
    U, Ma = (3.0, 0.0, 0.0), 3.0
    T0 = 1.0 * (1.0 + 0.2 * Ma * Ma)
    a = I.unstructured_dvs(U, 1.0, 1.0, Ma, True, target=600)
    b = I.unstructured_dvs(U, 1.0, 1.0, Ma, True, target=600, radius_factor=3.0, centre_factor=0.4,
                           ball_radius_factor=3.0, refine=True)
    assert np.array_equal(a.u, b.u) and np.array_equal(a.w, b.w)
    for rf, cf in ((3.0, 0.4), (4.0, 0.2)):
        d = I.unstructured_dvs(U, 1.0, 1.0, Ma, True, target=600, radius_factor=rf, centre_factor=cf,
                               refine=False)
        r = rf * math.sqrt(I.R_GAS * T0)
        c = cf * np.asarray(U)
        dist = np.linalg.norm(d.u - c, axis=1)
        assert dist.max() <= r and dist.max() > 0.85 * r
        assert abs(d.K - 600) < 0.25 * 600
        vol = 4.0 / 3.0 * math.pi * r ** 3
        assert 0.85 * vol < d.w.sum() <= vol
        centroid = (d.w[:, None] * d.u).sum(0) / d.w.sum()
        assert np.linalg.norm(centroid - c) < 0.05 * r


def test_freestream_turned_by_the_angle_of_attack():
    from paper_2303_10846_gb300 import studies as S
    U = (2.0, 0.0, 0.0)
    for plane in ("xz", "xy"):
        for a in (0.0, 10.0, -25.0):
            Ua, el = S.freestream_at(U, a, plane)
            Ua, el = np.asarray(Ua), np.asarray(el)
            assert abs(np.linalg.norm(Ua) - 2.0) < 1e-14 and abs(np.linalg.norm(el) - 1.0) < 1e-14
            assert abs(Ua @ el) < 1e-14
            assert abs(math.degrees(math.atan2(Ua[2] if plane == "xz" else Ua[1], Ua[0])) - a) < 1e-12


def test_turned_workload_turns_freestream_initial_field_and_velocity_space():
    """Turning the workload by an angle turns the farfield velocity, the initial
    velocities and every discrete velocity about the same axis, leaving the weights,
    the body and the mesh as they are (so a velocity space built around the freestream
    still surrounds it)."""
    from paper_2303_10846_gb300 import studies as S
    from tests import workloads as TW
    wl = TW.tiny_tet()
    wa = S.turned_workload(wl, 20.0, "xz")
    U, _ = S.freestream_at(wl.ref["U"], 20.0, "xz")
    far = [b for b in wa.bcs if b.kind == I.BC_FARFIELD][0]
    assert np.allclose(far.U, U, atol=1e-14) and np.allclose(wa.ref["U"], U, atol=1e-14)
    assert np.array_equal(wa.dvs.w, wl.dvs.w) and wa.mesh is wl.mesh
    assert np.allclose(np.linalg.norm(wa.dvs.u, axis=1), np.linalg.norm(wl.dvs.u, axis=1))
    # the first moment of the DVS (weighted mean velocity) turns with the freestream
    m0 = (wl.dvs.w[:, None] * wl.dvs.u).sum(0)
    m1 = (wa.dvs.w[:, None] * wa.dvs.u).sum(0)
    assert np.allclose(m1, S._turn(m0[None], 20.0, "xz")[0], atol=1e-12 * np.abs(m0).max())
    assert np.allclose(wa.prim0[:, 1:4], S._turn(wl.prim0[:, 1:4], 20.0, "xz"))
    assert np.array_equal(wa.prim0[:, [0, 4, 5]], wl.prim0[:, [0, 4, 5]])
