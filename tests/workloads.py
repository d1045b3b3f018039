"""Tiny workloads for the oracle pins and the parity tests, built only from the
seeded generators in paper_2303_10846_gb300.inputs."""
from __future__ import annotations

import math

import numpy as np

from paper_2303_10846_gb300 import inputs as I


def tiny_cavity(n=2, n_gh=4, **kw) -> I.Workload:
    return I.cavity_workload(n=n, n_gh=n_gh, **kw)


def tiny_tet(ma=1.0, n_gh=6, seed=7, lim=1, first_order_iters=0, cfl_imp=50.0,
             box_half=1.2, h_wall=0.7, growth=1.6, h_max=1.0) -> I.Workload:
    """~190 tetrahedra around a sphere of radius 0.5, farfield box, a shifted
    Gauss-Hermite DVS covering the freestream and the wall Maxwellians."""
    mesh = I.tet_sphere(0.5, box_half, h_wall, growth, h_max, seed=seed)
    a = math.sqrt(1.4 * I.R_GAS)
    U = (ma * a, 0.0, 0.0)
    dvs = I.gauss_hermite_dvs(n_gh, RT=I.R_GAS * 1.6, centre=(0.5 * U[0], 0.0, 0.0))
    params = I.Params(Z_rot=3.5, mu_ref=I.mu_ref_from_kn(0.2, 0.74), cfl_imp=cfl_imp,
                      limiter=lim, first_order_iters=first_order_iters)
    bcs = [I.BC(I.BC_WALL, 1.0, (0.0, 0.0, 0.0), 1.2), I.BC(I.BC_FARFIELD, 1.0, U, 1.0)]
    prim = I.uniform_prim(mesh.n_cell, 1.0, U, 1.0)
    r = np.linalg.norm(mesh.cell_center, axis=1)
    prim[:, 1:4] *= np.clip((r - 0.5) / 0.5, 0.2, 1.0)[:, None]
    return I.Workload(name="tiny_tet", mesh=mesh, dvs=dvs, params=params, bcs=bcs,
                      prim0=prim, ref=dict(rho=1.0, U=U, T=1.0))
