"""Pins of the oracle's aerodynamic loads (lift, drag, lift-to-drag ratio and pitching
moment, the quantities of the paper's blunted-cone and capsule results in Sec. 4)
against an independent recombination of the per-face wall quantities, the transfer
theorem of moments and the invariances of the coefficient definitions (no GPU)."""
import numpy as np
import pytest

import oracle as O
from tests import workloads as TW


@pytest.fixture(scope="module")
def flow():
    wl = TW.tiny_tet(n_gh=4, lim=1)
    o = O.Oracle(wl)
    o.iterate(6)
    return wl, o


def _walls(wl):
    m = wl.mesh
    bcs = wl.bcs
    fc = m.face_cell
    return np.array([f for f in range(m.n_face)
                     if fc[f, 1] < 0 and bcs[-1 - fc[f, 1]].kind == 0])


def test_loads_equal_the_recombined_wall_pressure_and_shear(flow):
    """F = sum A (p_w n + tau) and M = sum A (x_f - x_ref) x (p_w n + tau) from the
    per-face pressure and shear of the surface routine (Eqs. cp, cf)."""
    wl, o = flow
    per, force, _ = o.surface()
    wf = _walls(wl)
    m = wl.mesh
    assert len(wf) == len(per)
    traction = per[:, :1] * m.face_normal[wf] + per[:, 1:4]
    A = m.face_area[wf][:, None]
    x_ref = np.array([0.1, -0.2, 0.05])
    out = o.aero(x_ref=x_ref)
    F = (A * traction).sum(0)
    M = (A * np.cross(m.face_center[wf] - x_ref, traction)).sum(0)
    sc = np.max(np.abs(A * traction)) * len(wf)
    assert np.max(np.abs(out[:3] - F)) < 1e-13 * sc
    assert np.max(np.abs(out[:3] - force)) < 1e-13 * sc
    assert np.max(np.abs(out[3:6] - M)) < 1e-13 * sc
    assert np.max(np.abs(out[3:6])) > 1e-6 * sc           # a non-trivial moment


def test_moment_transfer_theorem_and_pitch_sign(flow):
    """M(x1) = M(x0) + (x0 - x1) x F; moving the reference point upstream by d along
    the flow changes C_m by -d C_L / L (lift aft of the reference point pitches the
    nose down)."""
    wl, o = flow
    x0 = np.array([0.0, 0.0, 0.0])
    x1 = np.array([0.3, 0.2, -0.4])
    a0, a1 = o.aero(x_ref=x0, L_ref=2.0), o.aero(x_ref=x1, L_ref=2.0)
    F = a0[:3]
    sc = np.max(np.abs(a0[3:6])) + np.max(np.abs(F))
    assert np.max(np.abs(a1[3:6] - (a0[3:6] + np.cross(x0 - x1, F)))) < 1e-13 * sc
    U = np.asarray(wl.ref["U"], float)
    eD = U / np.linalg.norm(U)
    d = 0.7
    a2 = o.aero(x_ref=x0 - d * eD, L_ref=2.0)
    assert abs(a0[7]) > 1e-8
    assert abs((a2[8] - a0[8]) - (-d * a0[7] / 2.0)) < 1e-12 * (abs(a0[8]) + abs(a0[7]))


def test_coefficient_invariances(flow):
    """The lift direction is used only through its unit part normal to the flow:
    adding a multiple of the flow direction or scaling it changes nothing, reversing
    it reverses C_L and C_m; C_D > 0 for the sphere; L/D = C_L/C_D; the coefficients
    scale as 1/(q S) and 1/(q S L)."""
    wl, o = flow
    U = np.asarray(wl.ref["U"], float)
    e = np.array([0.0, 0.3, 1.0])
    a = o.aero(lift_dir=e, S_ref=0.8, L_ref=1.5)
    b = o.aero(lift_dir=3.0 * e + 2.0 * U, S_ref=0.8, L_ref=1.5)
    c = o.aero(lift_dir=-e, S_ref=0.8, L_ref=1.5)
    sc = np.max(np.abs(a[6:9]))
    assert np.max(np.abs(a[6:9] - b[6:9])) < 1e-13 * sc
    assert abs(c[6] - a[6]) < 1e-13 * sc and abs(c[7] + a[7]) < 1e-13 * sc and abs(c[8] + a[8]) < 1e-13 * sc
    assert a[6] > 0
    assert abs(a[9] - a[7] / a[6]) < 1e-14 * abs(a[9])
    d = o.aero(lift_dir=e, S_ref=1.6, L_ref=3.0, rho_inf=2.0)
    assert np.max(np.abs(d[6:8] - a[6:8] / 4.0)) < 1e-13 * sc
    assert abs(d[8] - a[8] / 8.0) < 1e-13 * sc
    with pytest.raises(ValueError):
        o.aero(lift_dir=U)
