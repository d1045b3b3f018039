"""Sub-mesh ("patch") workloads for sampled oracle checks at sizes the oracle cannot run
whole.

A patch is a set of cells of a workload's mesh grown by face-neighbour rings.  Every
face that touches the patch is kept, in the mesh's own face order (so each cell's face
list, and with it every per-cell sum of the oracle, keeps its order): faces between two
patch cells stay interior faces, real boundary faces keep their condition, and faces
that lead out of the patch become boundary faces of one extra farfield condition.  The
cells of the inner rings then have exactly their neighbourhood in the full mesh: the
oracle evaluates on the patch, for those cells, what it would evaluate on the whole
mesh.  Only mesh bookkeeping lives here; the arithmetic of the method is the oracle's.
"""
from __future__ import annotations

import copy
import dataclasses

import numpy as np

from paper_2303_10846_gb300 import inputs as I


def cell_faces(mesh):
    """CSR of cell -> faces in increasing face order: (offsets[N+1], faces)."""
    fc = mesh.face_cell
    F = mesh.n_face
    cells = np.concatenate([fc[:, 0], fc[:, 1]])
    faces = np.concatenate([np.arange(F), np.arange(F)])
    keep = cells >= 0
    cells, faces = cells[keep], faces[keep]
    order = np.lexsort((faces, cells))
    cells, faces = cells[order], faces[order]
    off = np.zeros(mesh.n_cell + 1, np.int64)
    np.add.at(off, cells + 1, 1)
    return np.cumsum(off), faces


def neighbours(mesh, csr, i):
    off, faces = csr
    out = []
    for f in faces[off[i]:off[i + 1]]:
        a, b = mesh.face_cell[f]
        j = b if a == i else a
        if j >= 0:
            out.append(int(j))
    return out


def grow(mesh, csr, cells, rings):
    sel = set(int(c) for c in cells)
    front = set(sel)
    for _ in range(rings):
        new = set()
        for i in front:
            new.update(neighbours(mesh, csr, i))
        new -= sel
        sel |= new
        front = new
    return np.array(sorted(sel), np.int64)


def patch_workload(wl, cells, rings, cfl_imp=None):
    """The patch of `cells` grown by `rings` face-neighbour rings, as a workload.

    Returns (workload, local index of every patch cell's global index as a dict,
    global indices of the patch faces in patch order).  The parameters keep the
    workload's, with the start-up switches off (first_order_iters = 0, no implicit-CFL
    ramp; cfl_imp if given), so that a fresh oracle on the patch evaluates the limited
    second-order iteration at the given implicit step."""
    m = wl.mesh
    csr = cell_faces(m)
    P = grow(m, csr, cells, rings)
    g2l = {int(g): l for l, g in enumerate(P)}
    inP = np.zeros(m.n_cell, bool)
    inP[P] = True
    fc = m.face_cell
    a, b = fc[:, 0], fc[:, 1]
    touch = inP[a] | ((b >= 0) & inP[np.maximum(b, 0)])
    fidx = np.nonzero(touch)[0]
    nbc = len(wl.bcs)
    new_fc = np.empty((len(fidx), 2), np.int64)
    nrm = m.face_normal[fidx].copy()
    for t, f in enumerate(fidx):
        fa, fb = int(a[f]), int(b[f])
        if inP[fa] and fb >= 0 and inP[fb]:
            new_fc[t] = (g2l[fa], g2l[fb])
        elif inP[fa] and fb < 0:
            new_fc[t] = (g2l[fa], fb)                       # a real boundary face
        elif inP[fa]:
            new_fc[t] = (g2l[fa], -1 - nbc)                 # leads out of the patch
        else:
            new_fc[t] = (g2l[fb], -1 - nbc)                 # seen from the right cell
            nrm[t] = -nrm[t]
    mesh = I.Mesh(face_cell=new_fc, face_normal=nrm, face_area=m.face_area[fidx].copy(),
                  face_center=m.face_center[fidx].copy(), cell_center=m.cell_center[P].copy(),
                  cell_volume=m.cell_volume[P].copy(), cell_colour=m.cell_colour[P].copy(),
                  name=f"patch_of_{m.name}")
    params = dataclasses.replace(wl.params, first_order_iters=0, cfl_imp0=0.0, cfl_ramp=1.0,
                                 limiter_freeze=0)
    if cfl_imp is not None:
        params = dataclasses.replace(params, cfl_imp=float(cfl_imp))
    ref = wl.ref
    bcs = list(wl.bcs) + [I.BC(I.BC_FARFIELD, float(ref.get("rho", 1.0)),
                               tuple(ref.get("U", (0.0, 0.0, 0.0))), float(ref.get("T", 1.0)))]
    w2 = copy.copy(wl)
    w2.mesh, w2.params, w2.bcs = mesh, params, bcs
    w2.prim0 = wl.prim0[P].copy()
    w2.name = f"patch_{len(P)}_of_{wl.name}"
    return w2, g2l, fidx


def local_face(fidx, f):
    """Patch index of global face f."""
    t = np.searchsorted(fidx, f)
    assert fidx[t] == f
    return int(t)
