"""Patches (tests/patch.py) reproduce the whole-mesh oracle for their inner cells: the
ground the full-size sampled GPU checks stand on.  A patch oracle fed the whole-mesh
oracle's state gives the same reconstructed face values (Eq. flux_solve_phi_phi, two
rings around the face's cells), the same last point update of the micro PR-SGS (Eq.
implicit_mic_final_equ, one ring) and the same Step-6 update (Eqs. solve_rho -
solve_qrot), bit for bit: the per-cell face lists keep their order."""
import numpy as np

import oracle as O
from tests import patch as PT
from tests import workloads as TW


def _full(n_iter=3):
    wl = TW.tiny_tet(n_gh=5, lim=1, first_order_iters=0, cfl_imp=20.0)
    o = O.Oracle(wl)
    o.iterate(n_iter)
    return wl, o


def _rows(buf, rows, N, K, nfield=2):
    return buf.reshape(nfield, N, K)[:, rows, :]


def test_patch_reconstruction_matches_whole_mesh():
    wl, o = _full()
    N, K = wl.mesh.n_cell, wl.dvs.K
    phi = o.get(O.BUF_PHI)
    W, q = o.get(O.BUF_W), o.get(O.BUF_Q)
    o.step("gradient")
    o.step("faces")
    face0 = o.get(O.BUF_FACE0).reshape(2, wl.mesh.n_face, K)
    interior = np.nonzero(wl.mesh.face_cell[:, 1] >= 0)[0]
    rng = np.random.default_rng(3)
    for f in rng.choice(interior, 6, replace=False):
        a, b = wl.mesh.face_cell[f]
        pw, g2l, fidx = PT.patch_workload(wl, [a, b], 2)
        P = np.array(sorted(g2l, key=g2l.get))
        op = O.Oracle(pw)
        op.set_state(W[P], q[P], _rows(phi, P, N, K).reshape(-1))
        op.step("gradient")
        op.step("faces")
        got = op.get(O.BUF_FACE0).reshape(2, pw.mesh.n_face, K)[:, PT.local_face(fidx, f)]
        assert np.array_equal(got, face0[:, f]), f"face {f}"


def test_patch_micro_point_and_update_match_whole_mesh():
    wl, o = _full()
    N, K = wl.mesh.n_cell, wl.dvs.K
    for st in ("gradient", "faces", "fluxes", "macro"):
        o.step(st)
    phi_n = o.get(O.BUF_PHI)
    q_n = o.get(O.BUF_Q)
    Wt, taut = o.get(O.BUF_WT), o.get(O.BUF_TAUT)
    o.step("micro")
    res, dphi = o.get(O.BUF_RES), o.get(O.BUF_DPHI)
    o.step("update")
    phi1, W1, q1 = o.get(O.BUF_PHI), o.get(O.BUF_W), o.get(O.BUF_Q)
    # colour 0 is the last colour of the last (backward) sweep: its neighbours' final
    # increments are the ones its last point update read
    cells = np.nonzero(wl.mesh.cell_colour == 0)[0][:6]
    for i in cells:
        pw, g2l, _ = PT.patch_workload(wl, [i], 1, cfl_imp=wl.params.cfl_imp)
        P = np.array(sorted(g2l, key=g2l.get))
        li = g2l[int(i)]
        op = O.Oracle(pw)
        op.set_state(W1[P], q_n[P], _rows(phi_n, P, N, K).reshape(-1))
        op.put(O.BUF_RES, _rows(res, P, N, K).reshape(-1))
        op.put(O.BUF_DPHI, _rows(dphi, P, N, K).reshape(-1))
        op.put(O.BUF_WT, Wt[P].reshape(-1))
        op.put(O.BUF_TAUT, taut[P])
        op.micro_point(li, False, 0)
        n = len(P)
        assert np.array_equal(op.get(O.BUF_DPHI).reshape(2, n, K)[:, li], dphi.reshape(2, N, K)[:, i])
        op.update_cell(li)
        assert np.array_equal(op.get(O.BUF_PHI).reshape(2, n, K)[:, li], phi1.reshape(2, N, K)[:, i])
        assert np.array_equal(op.get(O.BUF_W).reshape(n, 6)[li], W1.reshape(N, 6)[i])
        assert np.array_equal(op.get(O.BUF_Q).reshape(n, 6)[li], q1.reshape(N, 6)[i])
