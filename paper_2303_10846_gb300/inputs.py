"""Seeded synthetic inputs: unstructured physical meshes, discrete velocity spaces
(DVS) and flow conditions.

This module only *builds inputs*.  It holds none of the scheme's arithmetic: no
equilibrium, flux, moment or solver formula lives here.  Both the CUDA library and
the CPU oracle receive exactly what it produces (geometry, velocity points and
weights, colouring, boundary/initial conditions as primitive variables).

Workload shapes follow the paper's test cases (Sec. 4): diatomic nitrogen with a
VHS viscosity law (omega = 0.74), everything dimensionless with
U_ref = sqrt(2 R T_ref) (Eqs. ref_quantities / reference), i.e. R = 1/2, T_inf = 1,
rho_inf = 1.  The paper's meshes and DVS are not available, so they are replaced by
seeded generators of the same kind:

* ``hex_cavity``: the lid-driven cubic cavity of Sec. 4.1 as an n^3 hexahedral
  lattice handed over as unstructured cell/face lists.
* ``tet_sphere``: a sphere in a cubic box (Sec. 4.2) as a seeded Delaunay
  tetrahedral mesh graded towards the wall.
* ``gauss_hermite_dvs``: tensor Gauss-Hermite velocity points.
* ``unstructured_dvs``: the unstructured-DVS generation criterion of Sec. 4.4
  (outer ball centred at 0.4 U_inf with radius 3 or 5 sqrt(R T0), Eq. solve_t0;
  refined balls of radius 3 sqrt(R T) at U_inf and 0 whose cell count follows the
  average-weight fit Eq. solve_weight).  Points are the centroids of seeded
  Delaunay tetrahedra in velocity space, weights their volumes (Sec. 3.2, text
  after Eq. implicit_mac_equ_mac_flux).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

# Boundary-condition kinds understood by both the library and the oracle.
BC_WALL = 0        # diffuse reflection with full accommodation (U_w, T_w)
BC_FARFIELD = 1    # incoming freestream Maxwellian (rho, U, T)

R_GAS = 0.5        # dimensionless specific gas constant: U_ref = sqrt(2 R T_ref)


# ----------------------------------------------------------------------------------
# data containers
# ----------------------------------------------------------------------------------
@dataclass
class Mesh:
    """Unstructured finite-volume mesh as flat arrays.

    face_cell[f] = (left, right); right < 0 marks a boundary face whose boundary
    condition id is -1-right.  face_normal is the unit normal pointing from left to
    right (outward for boundary faces).  cell_colour is a proper colouring of the
    cell adjacency graph (no two face neighbours share a colour).
    """
    face_cell: np.ndarray      # int64 [F,2]
    face_normal: np.ndarray    # float64 [F,3]
    face_area: np.ndarray      # float64 [F]
    face_center: np.ndarray    # float64 [F,3]
    cell_center: np.ndarray    # float64 [N,3]
    cell_volume: np.ndarray    # float64 [N]
    cell_colour: np.ndarray    # int32 [N]
    name: str = "mesh"

    @property
    def n_cell(self) -> int:
        return int(self.cell_volume.shape[0])

    @property
    def n_face(self) -> int:
        return int(self.face_area.shape[0])

    @property
    def n_colour(self) -> int:
        return int(self.cell_colour.max()) + 1 if self.n_cell else 0


@dataclass
class DVS:
    """Discrete velocity space: points u[K,3] and quadrature weights w[K]."""
    u: np.ndarray
    w: np.ndarray
    name: str = "dvs"

    @property
    def K(self) -> int:
        return int(self.w.shape[0])


@dataclass
class Params:
    """Scheme parameters (identical field order to the C ``rk_params`` struct).

    omega0, omega1, delta: Rykov-model constants for nitrogen.  The paper uses them
    (Eqs. frot, halftime_solve_qtra/qrot, solve_qtr/qrot) without giving values;
    the defaults are the nitrogen values used in the Rykov-model literature.
    """
    R: float = R_GAS
    Z_rot: float = 3.5
    omega_vis: float = 0.74
    mu_ref: float = 0.05
    T_ref: float = 1.0
    omega0: float = 0.2354
    omega1: float = 0.3049
    delta: float = 1.0 / 1.55
    cfl_s: float = 0.8
    cfl_imp: float = 1.0e3
    cfl_imp0: float = 0.0     # <= 0: no ramp
    cfl_ramp: float = 1.0
    lim_k: float = 0.3
    n_micro_sgs: int = 2
    n_macro_sgs: int = 40
    limiter: int = 1          # 0 unlimited, 1 Venkatakrishnan, 2 first order
    first_order_iters: int = 0
    limiter_freeze: int = 0   # > 0: limiter values of iteration limiter_freeze - 1 reused
    viscosity_law: int = 0    # 0 power law (omega_vis), 1 Sutherland (sutherland_c)
    sutherland_c: float = 111.0 / 273.0   # C_s of nitrogen (111 K) over a 273 K unit

    def as_dict(self):
        return asdict(self)


@dataclass
class BC:
    """Boundary condition for one bc id.  WALL: U = wall velocity, T = wall
    temperature (rho unused).  FARFIELD: freestream rho, U, T."""
    kind: int
    rho: float
    U: tuple
    T: float


@dataclass
class Workload:
    """One complete synthetic problem: mesh, DVS, parameters, boundary conditions
    and the uniform initial state (primitive variables per cell)."""
    name: str
    mesh: Mesh
    dvs: DVS
    params: Params
    bcs: list
    prim0: np.ndarray           # [N,6]: rho, Ux, Uy, Uz, T_tr, T_rot
    ref: dict = field(default_factory=dict)   # freestream reference for coefficients
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------------
def greedy_colour(n_cell: int, face_cell: np.ndarray, max_colours: int = 0) -> np.ndarray:
    """Deterministic greedy colouring in cell-index order: each cell takes the
    smallest colour not used by an already coloured face neighbour.  With
    max_colours > 0, cells left with a larger colour are then moved into the first
    max_colours colours where possible, directly or by swapping the two colours of a
    Kempe chain around them (a mesh whose cells have at most 4 neighbours is
    4-colourable unless it contains 5 mutually adjacent cells); cells that cannot be
    moved keep their colour, so the result is always a proper colouring."""
    nbrs = [[] for _ in range(n_cell)]
    for a, b in face_cell:
        if b >= 0:
            nbrs[a].append(int(b))
            nbrs[b].append(int(a))
    colour = np.full(n_cell, -1, dtype=np.int32)
    for i in range(n_cell):
        used = {int(colour[j]) for j in nbrs[i] if colour[j] >= 0}
        c = 0
        while c in used:
            c += 1
        colour[i] = c
    if max_colours <= 0:
        return colour
    for v in np.nonzero(colour >= max_colours)[0].tolist():
        used = {int(colour[j]) for j in nbrs[v]}
        free = [c for c in range(max_colours) if c not in used]
        if free:
            colour[v] = free[0]
            continue
        moved = False
        for a in range(max_colours):
            for b in range(a + 1, max_colours):
                # Kempe chain of colours (a, b) from v's neighbours of colour a
                starts = [j for j in nbrs[v] if colour[j] == a]
                seen, stack = set(starts), list(starts)
                while stack:
                    x = stack.pop()
                    for y in nbrs[x]:
                        if y not in seen and colour[y] in (a, b):
                            seen.add(y)
                            stack.append(y)
                if any(colour[j] == b for j in nbrs[v] if j in seen):
                    continue                      # the chain reaches a neighbour of colour b
                for x in seen:
                    colour[x] = b if colour[x] == a else a
                colour[v] = a
                moved = True
                break
            if moved:
                break
    # balance the classes: in cell order, move a cell from a class above the mean
    # size into the smallest class its neighbours leave free (sweeps of the colour
    # order are then launches of similar size)
    C = int(colour.max()) + 1
    size = np.bincount(colour, minlength=C).astype(np.int64)
    mean = n_cell / C
    for v in range(n_cell):
        cv = int(colour[v])
        if size[cv] <= mean:
            continue
        used = {int(colour[j]) for j in nbrs[v]}
        cand = [c for c in range(C) if c not in used and c != cv and size[c] < mean]
        if cand:
            c = min(cand, key=lambda x: (size[x], x))
            colour[v] = c
            size[cv] -= 1
            size[c] += 1
    # renumber so that the colours in use are 0..C-1 (largest classes first)
    vals, counts = np.unique(colour, return_counts=True)
    order = vals[np.argsort(-counts, kind="stable")]
    remap = np.empty(order.max() + 1, dtype=np.int32)
    remap[order] = np.arange(len(order), dtype=np.int32)
    return remap[colour]


def _morton_key(p: np.ndarray, bits: int = 10) -> np.ndarray:
    lo, hi = p.min(axis=0), p.max(axis=0)
    q = ((p - lo) / np.maximum(hi - lo, 1e-300) * ((1 << bits) - 1)).astype(np.int64)
    key = np.zeros(len(p), dtype=np.int64)
    for b in range(bits):
        for d in range(3):
            key |= ((q[:, d] >> b) & 1) << (3 * b + d)
    return key


def _hilbert2(x: np.ndarray, y: np.ndarray, order: int) -> np.ndarray:
    """Index along the 2-D Hilbert curve of order `order` of integer points (x, y)."""
    x = x.astype(np.int64).copy()
    y = y.astype(np.int64).copy()
    d = np.zeros(x.shape, np.int64)
    s = 1 << (order - 1)
    while s > 0:
        rx = ((x & s) > 0).astype(np.int64)
        ry = ((y & s) > 0).astype(np.int64)
        d += s * s * ((3 * rx) ^ ry)
        rot = ry == 0
        flip = rot & (rx == 1)
        x[flip] = s - 1 - x[flip]
        y[flip] = s - 1 - y[flip]
        x[rot], y[rot] = y[rot].copy(), x[rot].copy()
        s >>= 1
    return d


def direction_order(u: np.ndarray, bits: int = 6) -> np.ndarray:
    """Order of velocity points by direction (a Hilbert curve over an equal-area grid of
    cos(polar angle) x azimuth), then by speed.  The upwind split of every face,
    the sign of u . n, depends only on the direction of u, so neighbours in this order
    mostly fall on the same side of every face: a chunk of consecutive velocities then
    needs a neighbour's row less often.  Any order of the points is the same velocity
    space; this one only changes memory traffic."""
    r = np.linalg.norm(u, axis=1)
    d = u / np.maximum(r, 1e-300)[:, None]
    nb = 1 << bits
    zi = np.clip(((d[:, 2] + 1.0) * 0.5 * nb).astype(np.int64), 0, nb - 1)
    ph = np.arctan2(d[:, 1], d[:, 0])
    pi_ = np.clip(((ph + math.pi) / (2.0 * math.pi) * nb).astype(np.int64), 0, nb - 1)
    return np.lexsort((r, _hilbert2(zi, pi_, bits)))


def _fibonacci_sphere(n: int, rng: np.random.Generator) -> np.ndarray:
    """n quasi-uniform unit vectors, randomly rotated."""
    if n <= 0:
        return np.zeros((0, 3))
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    v = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    # random rotation (QR of a Gaussian matrix)
    qm, rm = np.linalg.qr(rng.standard_normal((3, 3)))
    qm = qm * np.sign(np.diag(rm))
    return v @ qm.T


def _tets_to_mesh(pts, tets, keep, wall_test, name):
    """Turn kept Delaunay tetrahedra into a face-based unstructured mesh.
    wall_test(face_centroid) -> True for body-wall boundary faces (bc 0), other
    boundary faces are farfield (bc 1)."""
    from scipy.spatial import Delaunay  # noqa: F401  (caller already used it)

    tets = tets[keep]
    nt = len(tets)
    P = pts[tets]                                     # [nt,4,3]
    cen = P.mean(axis=1)
    vol = np.abs(np.einsum("ij,ij->i", P[:, 1] - P[:, 0],
                           np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))) / 6.0
    order = np.argsort(_morton_key(cen), kind="stable")
    tets, cen, vol = tets[order], cen[order], vol[order]
    # faces: sorted vertex triple -> list of (tet, local face)
    fv = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]],
                         tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]], axis=0)
    owner = np.concatenate([np.arange(nt)] * 4)
    fs = np.sort(fv, axis=1)
    key = (fs[:, 0].astype(np.int64) * len(pts) + fs[:, 1]) * len(pts) + fs[:, 2]
    o = np.lexsort((owner, key))
    key_s, own_s, fv_s = key[o], owner[o], fv[o]
    same_next = np.zeros(len(key_s), dtype=bool)
    same_next[:-1] = key_s[:-1] == key_s[1:]
    first = np.ones(len(key_s), dtype=bool)
    first[1:] = key_s[1:] != key_s[:-1]
    left, right, verts = [], [], []
    idx = np.nonzero(first)[0]
    for t in idx:
        if same_next[t]:
            left.append(own_s[t]); right.append(own_s[t + 1])
        else:
            left.append(own_s[t]); right.append(-1)
        verts.append(fv_s[t])
    left = np.array(left, dtype=np.int64)
    right = np.array(right, dtype=np.int64)
    verts = np.array(verts, dtype=np.int64)
    V = pts[verts]
    fc = V.mean(axis=1)
    nrm = np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0])
    area = 0.5 * np.linalg.norm(nrm, axis=1)
    nrm = nrm / np.linalg.norm(nrm, axis=1)[:, None]
    # orient from left cell outward
    flip = np.einsum("ij,ij->i", fc - cen[left], nrm) < 0
    nrm[flip] *= -1.0
    bnd = right < 0
    is_wall = np.array([wall_test(c) for c in fc[bnd]], dtype=bool)
    bc_id = np.where(is_wall, 0, 1)
    right[bnd] = -1 - bc_id
    # face order: interior faces by (left,right), boundary faces after them
    fo = np.lexsort((right, left, bnd))
    face_cell = np.stack([left, right], axis=1)[fo]
    mesh = Mesh(face_cell=face_cell, face_normal=nrm[fo], face_area=area[fo],
                face_center=fc[fo], cell_center=cen, cell_volume=vol,
                cell_colour=np.zeros(nt, dtype=np.int32), name=name)
    mesh.cell_colour = greedy_colour(nt, face_cell, max_colours=4)
    return mesh


# ----------------------------------------------------------------------------------
# physical meshes
# ----------------------------------------------------------------------------------
def hex_cavity(n: int = 8, L: float = 1.0) -> Mesh:
    """n^3 uniform hexahedral lattice on [0,L]^3 as unstructured lists.
    bc 0 = stationary walls, bc 1 = lid (the z = L face)."""
    h = L / n
    idx = lambda x, y, z: x + n * (y + n * z)
    cc = np.array([[(x + 0.5) * h, (y + 0.5) * h, (z + 0.5) * h]
                   for z in range(n) for y in range(n) for x in range(n)])
    fcell, fn, fc = [], [], []
    e = np.eye(3)
    for z in range(n):
        for y in range(n):
            for x in range(n):
                c = idx(x, y, z)
                p = np.array([x, y, z])
                for d in range(3):
                    q = p.copy(); q[d] += 1
                    ctr = (p + 0.5) * h; ctr[d] = (p[d] + 1) * h
                    if q[d] < n:
                        fcell.append((c, idx(*q))); fn.append(e[d]); fc.append(ctr)
    # boundary faces
    for z in range(n):
        for y in range(n):
            for x in range(n):
                c = idx(x, y, z)
                p = np.array([x, y, z])
                for d in range(3):
                    for side in (0, 1):
                        if (side == 0 and p[d] == 0) or (side == 1 and p[d] == n - 1):
                            ctr = (p + 0.5) * h
                            ctr[d] = 0.0 if side == 0 else L
                            nrm = e[d] * (1.0 if side == 1 else -1.0)
                            bc = 1 if (d == 2 and side == 1) else 0
                            fcell.append((c, -1 - bc)); fn.append(nrm); fc.append(ctr)
    face_cell = np.array(fcell, dtype=np.int64)
    mesh = Mesh(face_cell=face_cell,
                face_normal=np.array(fn, dtype=np.float64),
                face_area=np.full(len(fcell), h * h),
                face_center=np.array(fc, dtype=np.float64),
                cell_center=cc, cell_volume=np.full(n ** 3, h ** 3),
                cell_colour=np.zeros(n ** 3, dtype=np.int32), name=f"hex_cavity_{n}")
    mesh.cell_colour = greedy_colour(mesh.n_cell, face_cell)
    return mesh


def tet_sphere(radius: float = 0.5, box_half: float = 2.5, h_wall: float = 0.05,
               growth: float = 1.12, h_max: float = 0.4, seed: int = 20261) -> Mesh:
    """Seeded Delaunay tetrahedral mesh around a sphere (centred at the origin) in
    the box [-box_half, box_half]^3.  Points lie on concentric quasi-uniform shells
    whose spacing grows geometrically from h_wall at the wall to h_max, plus a
    jittered lattice on the box surface.  Tetrahedra with centroid inside the
    sphere are removed.  bc 0 = sphere wall, bc 1 = box farfield."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    pts = []
    r, h = radius, h_wall
    corner = box_half * math.sqrt(3.0)
    first = True
    while r < corner + h_max:
        n = max(8, int(round(4.0 * math.pi * r * r / (0.866 * h * h))))
        v = _fibonacci_sphere(n, rng)
        if first:
            p = radius * v
            first = False
        else:
            rr = r + 0.15 * h * (rng.random(n) - 0.5)
            p = v * rr[:, None]
        inside = np.all(np.abs(p) < box_half - 0.35 * h, axis=1)
        pts.append(p[inside])
        r += 0.82 * h
        h = min(h * growth, h_max)
    # box surface: lattice with spacing ~h_max, jittered in-plane, exact on planes
    m = int(math.ceil(2 * box_half / h_max))
    g = np.linspace(-box_half, box_half, m + 1)
    for d in range(3):
        for s in (-box_half, box_half):
            a, b = np.meshgrid(g, g, indexing="ij")
            a, b = a.ravel(), b.ravel()
            interior = (np.abs(a) < box_half - 1e-12) & (np.abs(b) < box_half - 1e-12)
            ja = a + interior * 0.2 * h_max * (rng.random(a.size) - 0.5)
            jb = b + interior * 0.2 * h_max * (rng.random(b.size) - 0.5)
            p = np.zeros((a.size, 3))
            od = [x for x in range(3) if x != d]
            p[:, d] = s; p[:, od[0]] = ja; p[:, od[1]] = jb
            pts.append(p)
    pts = np.unique(np.round(np.concatenate(pts, axis=0), 12), axis=0)
    tri = Delaunay(pts)
    tets = tri.simplices.astype(np.int64)
    cen = pts[tets].mean(axis=1)
    P = pts[tets]
    vol = np.abs(np.einsum("ij,ij->i", P[:, 1] - P[:, 0],
                           np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))) / 6.0
    keep = (np.linalg.norm(cen, axis=1) > radius) & (vol > 1e-14)
    wall_r = radius + 0.5 * h_wall
    return _tets_to_mesh(pts, tets, keep,
                         lambda c: np.linalg.norm(c) < wall_r,
                         f"tet_sphere_{int(keep.sum())}")


# axisymmetric bodies (profile in the (x, r) half plane, nose on the axis at x = 0
# facing -x), used for the capsule and the sphere-cone
def _profile_segments(prof):
    P = np.asarray(prof, dtype=np.float64)
    return P[:-1], P[1:]


def _axisym_sdf(prof, x, r):
    """Signed distance (negative inside) from points (x, r) to the closed region
    bounded by the profile polyline and the axis."""
    A, B = _profile_segments(prof)
    out = np.empty(len(x))
    for s0 in range(0, len(x), 65536):
        px, pr = x[s0:s0 + 65536, None], r[s0:s0 + 65536, None]
        ab = B - A
        t = ((px - A[:, 0]) * ab[:, 0] + (pr - A[:, 1]) * ab[:, 1]) / np.maximum((ab ** 2).sum(1), 1e-300)
        t = np.clip(t, 0.0, 1.0)
        dx = px - (A[:, 0] + t * ab[:, 0])
        dr = pr - (A[:, 1] + t * ab[:, 1])
        d = np.sqrt(dx * dx + dr * dr).min(axis=1)
        # inside: crossings of a ray towards +r with the closed polygon (profile + axis)
        Q = np.concatenate([np.asarray(prof), np.asarray(prof)[:1]], axis=0)
        qa, qb = Q[:-1], Q[1:]
        cross = ((qa[:, 0] <= px) & (qb[:, 0] > px)) | ((qb[:, 0] <= px) & (qa[:, 0] > px))
        tt = (px - qa[:, 0]) / np.where(qb[:, 0] != qa[:, 0], qb[:, 0] - qa[:, 0], 1.0)
        rc = qa[:, 1] + tt * (qb[:, 1] - qa[:, 1])
        inside = (np.sum(cross & (rc > pr), axis=1) % 2) == 1
        out[s0:s0 + 65536] = np.where(inside, -d, d)
    return out


def _resample(poly, h):
    """Points along a polyline at arc-length spacing about h (ends included)."""
    P = np.asarray(poly)
    seg = np.linalg.norm(np.diff(P, axis=0), axis=1)
    s = np.concatenate([[0.0], np.cumsum(seg)])
    n = max(2, int(round(s[-1] / h)) + 1)
    t = np.linspace(0.0, s[-1], n)
    return np.stack([np.interp(t, s, P[:, 0]), np.interp(t, s, P[:, 1])], axis=1)


def _offset_profile(prof, d):
    """The profile moved outward by d along its vertex normals (in the (x, r) plane)."""
    P = np.asarray(prof, dtype=np.float64)
    t = np.gradient(P, axis=0)
    t /= np.maximum(np.linalg.norm(t, axis=1), 1e-300)[:, None]
    nrm = np.stack([-t[:, 1], t[:, 0]], axis=1)      # left of the direction of travel
    Q = P + d * nrm
    Q[:, 1] = np.maximum(Q[:, 1], 0.0)
    return Q


def tet_axisym_body(prof, aoa_deg: float, box_lo, box_hi, h_wall: float, growth: float,
                    h_max: float, seed: int, name: str):
    """Seeded Delaunay tetrahedral mesh around an axisymmetric body given by its (x, r)
    profile (from the nose on the axis to the back on the axis, body on the left of the
    direction of travel), turned by aoa_deg about z (flow along +x), in the box
    [box_lo, box_hi].  Points lie on offset surfaces of the body whose spacing grows
    geometrically from h_wall to h_max, each revolved in rings of spacing h, plus a
    jittered lattice on the box faces.  bc 0 = body wall, bc 1 = farfield.
    Returns (mesh, distance of every cell centre to the body)."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    prof = np.asarray(prof, dtype=np.float64)
    box_lo, box_hi = np.asarray(box_lo, float), np.asarray(box_hi, float)
    a = math.radians(aoa_deg)
    Rz = np.array([[math.cos(a), -math.sin(a), 0.0], [math.sin(a), math.cos(a), 0.0], [0.0, 0.0, 1.0]])
    xc = 0.5 * (prof[:, 0].min() + prof[:, 0].max())
    span = np.linalg.norm(box_hi - box_lo)
    fine = _resample(prof, 0.25 * h_wall)
    pts, d, h = [], 0.0, h_wall
    while d < span:
        layer = _resample(_offset_profile(fine, d) if d > 0 else fine, h)
        for x, r in layer:
            n = 1 if r < 0.3 * h else max(3, int(round(2.0 * math.pi * r / h)))
            th = 2.0 * math.pi * (np.arange(n) + rng.random()) / n
            ring = np.stack([np.full(n, x), r * np.cos(th), r * np.sin(th)], axis=1)
            if d > 0:
                ring += 0.1 * h * (rng.random((n, 3)) - 0.5)
            pts.append(ring)
        d += 0.82 * h
        h = min(h * growth, h_max)
    P = np.concatenate(pts, axis=0)
    body = P.copy()
    P = (P - [xc, 0.0, 0.0]) @ Rz.T + [xc, 0.0, 0.0]
    sd = _axisym_sdf(prof, body[:, 0], np.hypot(body[:, 1], body[:, 2]))
    ok = np.all((P > box_lo + 0.3 * h_max) & (P < box_hi - 0.3 * h_max), axis=1)
    ok &= (sd > -1e-9) & ((sd > 0.3 * h_wall) | (np.abs(sd) < 1e-9))
    pts = [P[ok]]
    for dd in range(3):
        m = int(math.ceil((box_hi[dd] - box_lo[dd]) / h_max))
        od = [x for x in range(3) if x != dd]
        ga = np.linspace(box_lo[od[0]], box_hi[od[0]], int(math.ceil((box_hi[od[0]] - box_lo[od[0]]) / h_max)) + 1)
        gb = np.linspace(box_lo[od[1]], box_hi[od[1]], int(math.ceil((box_hi[od[1]] - box_lo[od[1]]) / h_max)) + 1)
        A_, B_ = np.meshgrid(ga, gb, indexing="ij")
        A_, B_ = A_.ravel(), B_.ravel()
        inner = ((A_ > box_lo[od[0]] + 1e-12) & (A_ < box_hi[od[0]] - 1e-12) &
                 (B_ > box_lo[od[1]] + 1e-12) & (B_ < box_hi[od[1]] - 1e-12))
        for sv in (box_lo[dd], box_hi[dd]):
            q = np.zeros((A_.size, 3))
            q[:, dd] = sv
            q[:, od[0]] = A_ + inner * 0.2 * h_max * (rng.random(A_.size) - 0.5)
            q[:, od[1]] = B_ + inner * 0.2 * h_max * (rng.random(B_.size) - 0.5)
            pts.append(q)
    pts = np.unique(np.round(np.concatenate(pts, axis=0), 12), axis=0)
    tri = Delaunay(pts)
    tets = tri.simplices.astype(np.int64)
    Pt = pts[tets]
    cen = Pt.mean(axis=1)
    vol = np.abs(np.einsum("ij,ij->i", Pt[:, 1] - Pt[:, 0],
                           np.cross(Pt[:, 2] - Pt[:, 0], Pt[:, 3] - Pt[:, 0]))) / 6.0
    back = (cen - [xc, 0.0, 0.0]) @ Rz + [xc, 0.0, 0.0]        # into the body frame
    sdc = _axisym_sdf(prof, back[:, 0], np.hypot(back[:, 1], back[:, 2]))
    keep = (sdc > 0.0) & (vol > 1e-14)

    def wall_test(c):
        b = (c - [xc, 0.0, 0.0]) @ Rz + [xc, 0.0, 0.0]
        return _axisym_sdf(prof, np.array([b[0]]), np.array([math.hypot(b[1], b[2])]))[0] < 0.25 * h_wall

    mesh = _tets_to_mesh(pts, tets, keep, wall_test, f"{name}_{int(keep.sum())}")
    bc = (mesh.cell_center - [xc, 0.0, 0.0]) @ Rz + [xc, 0.0, 0.0]
    dist = _axisym_sdf(prof, bc[:, 0], np.hypot(bc[:, 1], bc[:, 2]))
    return mesh, dist


def capsule_profile(R_n: float = 1.0, r_max: float = 0.8, cone_deg: float = 33.0, r_back: float = 0.3,
                    n_arc: int = 64):
    """Blunt capsule: spherical-cap heat shield of radius R_n up to the shoulder radius
    r_max, conical afterbody closing at cone_deg to r_back, flat back."""
    th_c = math.asin(r_max / R_n)
    th = np.linspace(0.0, th_c, n_arc)
    cap = np.stack([R_n * (1.0 - np.cos(th)), R_n * np.sin(th)], axis=1)
    xs = cap[-1, 0]
    xb = xs + (r_max - r_back) / math.tan(math.radians(cone_deg))
    return np.concatenate([cap, [[xb, r_back], [xb, 0.0]]], axis=0)


def sphere_cone_profile(R_n: float = 1.0, half_deg: float = 15.0, length: float = 4.0, n_arc: int = 64):
    """Sphere-cone: nose of radius R_n, tangent cone of half angle half_deg up to x =
    length, flat base."""
    tc = math.radians(90.0 - half_deg)
    th = np.linspace(0.0, tc, n_arc)
    nose = np.stack([R_n * (1.0 - np.cos(th)), R_n * np.sin(th)], axis=1)
    xt, rt = nose[-1]
    rb = rt + (length - xt) * math.tan(math.radians(half_deg))
    return np.concatenate([nose, [[length, rb], [length, 0.0]]], axis=0)


# ----------------------------------------------------------------------------------
# discrete velocity spaces
# ----------------------------------------------------------------------------------
def gauss_hermite_dvs(n: int = 8, RT: float = R_GAS, centre=(0.0, 0.0, 0.0)) -> DVS:
    """Tensor Gauss-Hermite points for a Maxwellian of temperature RT centred at
    `centre`: u = centre + sqrt(2 RT) x, w = sqrt(2 RT)^3 w_x w_y w_z e^{|x|^2}, so
    that sum_k w_k f(u_k) approximates the integral of f over velocity space."""
    x, wx = np.polynomial.hermite.hermgauss(n)
    s = math.sqrt(2.0 * RT)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    WX, WY, WZ = np.meshgrid(wx, wx, wx, indexing="ij")
    u = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1) * s + np.asarray(centre)
    w = (WX * WY * WZ).ravel() * np.exp(X.ravel() ** 2 + Y.ravel() ** 2 + Z.ravel() ** 2) * s ** 3
    return DVS(u=u, w=w, name=f"gh{n}")


def _ball_points(centre, radius, spacing, rng, surface=True):
    """Jittered lattice points inside a ball plus (optionally) Fibonacci points on
    its surface."""
    m = int(math.ceil(radius / spacing))
    g = (np.arange(-m, m + 1)) * spacing
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    p = p + 0.3 * spacing * (rng.random(p.shape) - 0.5)
    p = p[np.linalg.norm(p, axis=1) < radius - 0.3 * spacing]
    out = [p + np.asarray(centre)]
    if surface:
        ns = max(12, int(round(4 * math.pi * radius ** 2 / (0.866 * spacing ** 2))))
        out.append(np.asarray(centre) + radius * _fibonacci_sphere(ns, rng))
    return np.concatenate(out, axis=0)


def refined_ball_cells(T: float) -> float:
    """Cell count in a refined ball from the average-weight fit of Sec. 4.4
    (Eq. solve_weight): count = 730 [arctan((T - 1)/40) + 1]."""
    return 730.0 * (math.atan((T - 1.0) / 40.0) + 1.0)


def unstructured_dvs(U_inf, T_inf: float, T_w: float, Ma: float, transitional: bool,
                     target: int = 3000, seed: int = 20262, gamma: float = 1.4,
                     radius_factor: float | None = None, centre_factor: float = 0.4,
                     ball_radius_factor: float = 3.0, refine: bool = True) -> DVS:
    """Unstructured DVS following the generation criterion of Sec. 4.4.

    Outer ball: centre 0.4 U_inf, radius 3 sqrt(R T0) (transitional) or
    5 sqrt(R T0) (near-continuum), T0 = T_inf (1 + (gamma-1)/2 Ma^2) (Eq. solve_t0).
    Refined balls: centre U_inf radius 3 sqrt(R T_inf) and centre 0 radius
    3 sqrt(R T_w), each with about refined_ball_cells(T) cells.  The remaining
    cells (target minus the refined ones) fill the outer ball.  Velocity points are
    tetrahedron centroids of a seeded Delaunay triangulation, weights their volumes.

    For studies of the criterion: radius_factor replaces the 3 / 5 of the outer
    radius, centre_factor the 0.4 of its centre, ball_radius_factor the 3 of the
    refined balls; refine=False leaves the refined balls out.
    """
    from scipy.spatial import Delaunay
    U_inf = np.asarray(U_inf, dtype=np.float64)
    T0 = T_inf * (1.0 + 0.5 * (gamma - 1.0) * Ma * Ma)
    c_out = centre_factor * U_inf
    rf = radius_factor if radius_factor is not None else (3.0 if transitional else 5.0)
    r_out = rf * math.sqrt(R_GAS * T0)
    balls = [(U_inf, ball_radius_factor * math.sqrt(R_GAS * T_inf), refined_ball_cells(T_inf)),
             (np.zeros(3), ball_radius_factor * math.sqrt(R_GAS * T_w), refined_ball_cells(T_w))]
    if not refine:
        balls = []
    n_ref = sum(b[2] for b in balls)
    n_out = max(200.0, target - n_ref)
    v_ref = sum(4.0 / 3.0 * math.pi * b[1] ** 3 for b in balls)
    v_out = 4.0 / 3.0 * math.pi * r_out ** 3 - v_ref
    # initial spacings from ~6 tetrahedra per point, then a few multiplicative
    # corrections so that each region holds its prescribed number of cells
    h_out = (v_out / (n_out / 6.0)) ** (1.0 / 3.0)
    h_b = [(4.0 / 3.0 * math.pi * r ** 3 / (nc / 6.0)) ** (1.0 / 3.0) for _, r, nc in balls]

    def build(h_out, h_b):
        rng = np.random.default_rng(seed)
        p0 = _ball_points(c_out, r_out, h_out, rng, surface=True)
        for c, r, _ in balls:
            p0 = p0[np.linalg.norm(p0 - c, axis=1) > r + 0.3 * h_out]
        pts = [p0]
        for (c, r, _), hb in zip(balls, h_b):
            pb = _ball_points(c, r, hb, rng, surface=True)
            pb = pb[np.linalg.norm(pb - c_out, axis=1) < r_out - 0.2 * hb]
            pts.append(pb)
        pts = np.concatenate(pts, axis=0)
        tri = Delaunay(pts)
        P = pts[tri.simplices]
        vol = np.abs(np.einsum("ij,ij->i", P[:, 1] - P[:, 0],
                               np.cross(P[:, 2] - P[:, 0], P[:, 3] - P[:, 0]))) / 6.0
        keep = vol > 1e-12 * vol.max()
        return P[keep].mean(axis=1), vol[keep]

    for _ in range(4):
        u, w = build(h_out, h_b)
        in_ball = [np.linalg.norm(u - c, axis=1) < r for c, r, _ in balls]
        n_b = [int(m.sum()) for m in in_ball]
        n_o = len(w) - sum(n_b)
        h_out *= (n_o / n_out) ** (1.0 / 3.0)
        h_b = [hb * (nb / nc) ** (1.0 / 3.0) for hb, nb, (_, _, nc) in zip(h_b, n_b, balls)]
    u, w = build(h_out, h_b)
    order = direction_order(u)
    return DVS(u=u[order], w=w[order], name=f"udvs{len(w)}")


# ----------------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------------
def mu_ref_from_kn(kn: float, omega: float, length: float = 1.0, alpha: float = 1.0) -> float:
    """Reference viscosity for a given Knudsen number (VHS mean free path, Bird):
    lambda = 4 alpha (5-2w)(7-2w) / (5 (alpha+1)(alpha+2)) * mu / (rho sqrt(2 pi R T)),
    with rho = 1, R T = 1/2 (so sqrt(2 pi R T) = sqrt(pi)).  The paper states Kn
    but not this conversion."""
    return (kn * length * 5.0 * (alpha + 1.0) * (alpha + 2.0) * math.sqrt(math.pi)
            / (4.0 * alpha * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega)))


def uniform_prim(n_cell: int, rho: float, U, T: float) -> np.ndarray:
    prim = np.zeros((n_cell, 6))
    prim[:, 0] = rho
    prim[:, 1:4] = np.asarray(U, dtype=np.float64)
    prim[:, 4] = T
    prim[:, 5] = T
    return prim


def cavity_workload(n: int = 8, n_gh: int = 8, kn: float = 0.075, ma_lid: float = 0.16,
                    Z_rot: float = 3.5, cfl_imp: float = 1.0e3) -> Workload:
    """Lid-driven cubic cavity (Sec. 4.1 shape): n^3 hex cells, n_gh^3 Gauss-Hermite
    DVS, lid along +x at Mach ma_lid (a = sqrt(gamma R T) with gamma = 7/5), all
    walls diffuse at T_w = 1, gas initially at rest with rho = 1, T = 1."""
    mesh = hex_cavity(n)
    dvs = gauss_hermite_dvs(n_gh)
    a = math.sqrt(1.4 * R_GAS * 1.0)
    U_lid = ma_lid * a
    params = Params(Z_rot=Z_rot, mu_ref=mu_ref_from_kn(kn, 0.74), cfl_imp=cfl_imp)
    bcs = [BC(BC_WALL, 1.0, (0.0, 0.0, 0.0), 1.0), BC(BC_WALL, 1.0, (U_lid, 0.0, 0.0), 1.0)]
    return Workload(name=f"cavity_{n}^3_gh{n_gh}", mesh=mesh, dvs=dvs, params=params,
                    bcs=bcs, prim0=uniform_prim(mesh.n_cell, 1.0, (0, 0, 0), 1.0),
                    ref=dict(rho=1.0, U=(U_lid, 0.0, 0.0), T=1.0),
                    meta=dict(kn=kn, ma_lid=ma_lid, U_lid=U_lid))


def sphere_workload(h_wall: float = 0.065, growth: float = 1.15, h_max: float = 0.4,
                    dvs_target: int = 3000, ma: float = 5.0, kn: float = 0.1,
                    Z_rot: float = 3.5, T_w: float = 1.0, cfl_imp: float = 50.0,
                    mesh_seed: int = 20261, dvs_seed: int = 20262,
                    box_half: float = 2.5, dvs_options: dict | None = None) -> Workload:
    """Sphere of diameter 1 at Mach `ma` along +x, Kn on the diameter (Sec. 4.2
    shape): seeded Delaunay tetrahedra in a 10R box, unstructured DVS from the
    Sec. 4.4 criterion, farfield on the box, diffuse wall at T_w."""
    mesh = tet_sphere(0.5, box_half, h_wall, growth, h_max, seed=mesh_seed)
    a = math.sqrt(1.4 * R_GAS)
    U = (ma * a, 0.0, 0.0)
    dvs = unstructured_dvs(U, 1.0, T_w, ma, transitional=(kn >= 0.1), target=dvs_target,
                           seed=dvs_seed, **(dvs_options or {}))
    params = Params(Z_rot=Z_rot, mu_ref=mu_ref_from_kn(kn, 0.74), cfl_imp=cfl_imp,
                    cfl_imp0=2.0, cfl_ramp=1.3, first_order_iters=10)
    bcs = [BC(BC_WALL, 1.0, (0.0, 0.0, 0.0), T_w), BC(BC_FARFIELD, 1.0, U, 1.0)]
    # Initial field: rho = 1, T = 1 everywhere; the velocity grows linearly from 0 at
    # the wall to U_inf one diameter away (an impulsive uniform start empties the
    # near wake to vacuum in the first iterations).
    prim = uniform_prim(mesh.n_cell, 1.0, U, 1.0)
    r = np.linalg.norm(mesh.cell_center, axis=1)
    prim[:, 1:4] *= np.clip((r - 0.5) / 1.0, 0.0, 1.0)[:, None]
    return Workload(name=f"sphere_ma{ma:g}_kn{kn:g}_N{mesh.n_cell}_K{dvs.K}", mesh=mesh,
                    dvs=dvs, params=params, bcs=bcs, prim0=prim,
                    ref=dict(rho=1.0, U=U, T=1.0),
                    meta=dict(ma=ma, kn=kn, T_w=T_w))


def capsule_workload(h_wall: float = 0.047, growth: float = 1.12, h_max: float = 0.39,
                     dvs_target: int = 6000, ma: float = 10.0, kn: float = 0.01,
                     aoa: float = 25.0, T_w: float = 300.0 / 142.0, Z_rot: float = 3.5,
                     cfl_imp: float = 100.0, mesh_seed: int = 20263,
                     dvs_seed: int = 20264, dvs_options: dict | None = None) -> Workload:
    """Blunt capsule (spherical-cap heat shield R = 1 up to the shoulder radius 0.8,
    33-degree conical afterbody to radius 0.3, flat back) at 25 degrees angle of
    attack, Mach 10 along +x, Kn on the maximum diameter (1.6), T_w = 300/142 T_inf,
    in the box [-3.2, 4.8] x [-4, 4]^2; near-continuum DVS (outer radius 5 sqrt(R T0))."""
    prof = capsule_profile()
    D = 1.6
    mesh, dist = tet_axisym_body(prof, aoa, [-3.2, -4.0, -4.0], [4.8, 4.0, 4.0], h_wall, growth,
                                 h_max, mesh_seed, "tet_capsule")
    a = math.sqrt(1.4 * R_GAS)
    U = (ma * a, 0.0, 0.0)
    dvs = unstructured_dvs(U, 1.0, T_w, ma, transitional=(kn >= 0.1), target=dvs_target,
                           seed=dvs_seed, **(dvs_options or {}))
    params = Params(Z_rot=Z_rot, mu_ref=mu_ref_from_kn(kn, 0.74, length=D), cfl_imp=cfl_imp,
                    cfl_imp0=2.0, cfl_ramp=1.3, first_order_iters=10)
    bcs = [BC(BC_WALL, 1.0, (0.0, 0.0, 0.0), T_w), BC(BC_FARFIELD, 1.0, U, 1.0)]
    prim = uniform_prim(mesh.n_cell, 1.0, U, 1.0)
    prim[:, 1:4] *= np.clip(dist / D, 0.0, 1.0)[:, None]
    return Workload(name=f"capsule_ma{ma:g}_kn{kn:g}_aoa{aoa:g}_N{mesh.n_cell}_K{dvs.K}", mesh=mesh,
                    dvs=dvs, params=params, bcs=bcs, prim0=prim, ref=dict(rho=1.0, U=U, T=1.0),
                    meta=dict(ma=ma, kn=kn, aoa=aoa, T_w=T_w, length=D, profile=prof.tolist()))


def cone_scale_workload(h_wall: float = 0.065, growth: float = 1.12, h_max: float = 0.45,
                        dvs_target: int = 8000, ma: float = 8.0, kn: float = 0.005,
                        T_w: float = 1.0, Z_rot: float = 3.5, cfl_imp: float = 20.0,
                        first_order_iters: int = 20, cfl_ramp: float = 1.2,
                        mesh_seed: int = 20265, dvs_seed: int = 20266) -> Workload:
    """Scale case: sphere-cone (nose radius 1, 15-degree half angle, length 4, flat
    base) at zero incidence, Mach 8, Kn on the nose radius, T_w = T_inf (the case gives
    none), in the box [-4, 10] x [-5, 5]^2: ~500k tetrahedra x ~8,000 velocities.
    Start-up: 20 first-order iterations and an implicit CFL ramped by 1.2 per iteration
    up to 20 (with the limited second-order scheme switched on at an implicit CFL of
    30 or more, this case turned non-finite within 10 iterations)."""
    prof = sphere_cone_profile()
    mesh, dist = tet_axisym_body(prof, 0.0, [-4.0, -5.0, -5.0], [10.0, 5.0, 5.0], h_wall, growth,
                                 h_max, mesh_seed, "tet_cone")
    a = math.sqrt(1.4 * R_GAS)
    U = (ma * a, 0.0, 0.0)
    dvs = unstructured_dvs(U, 1.0, T_w, ma, transitional=(kn >= 0.1), target=dvs_target,
                           seed=dvs_seed)
    params = Params(Z_rot=Z_rot, mu_ref=mu_ref_from_kn(kn, 0.74, length=1.0), cfl_imp=cfl_imp,
                    cfl_imp0=2.0, cfl_ramp=cfl_ramp, first_order_iters=first_order_iters)
    bcs = [BC(BC_WALL, 1.0, (0.0, 0.0, 0.0), T_w), BC(BC_FARFIELD, 1.0, U, 1.0)]
    prim = uniform_prim(mesh.n_cell, 1.0, U, 1.0)
    prim[:, 1:4] *= np.clip(dist / 1.0, 0.0, 1.0)[:, None]
    return Workload(name=f"cone_ma{ma:g}_kn{kn:g}_N{mesh.n_cell}_K{dvs.K}", mesh=mesh, dvs=dvs,
                    params=params, bcs=bcs, prim0=prim, ref=dict(rho=1.0, U=U, T=1.0),
                    meta=dict(ma=ma, kn=kn, T_w=T_w, length=1.0, profile=prof.tolist()))
