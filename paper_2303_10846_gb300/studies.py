"""Parameter studies on top of the solver (host-side loops over library calls; every
iteration and every load integral runs in the CUDA kernels of librykov).

* Angle-of-attack sweeps: the lift, drag, lift-to-drag and pitching-moment curves that
  Sec. 4 reports for the blunted cone and the capsule.  The freestream is turned in a
  plane together with the velocity space built around it; each angle is converged
  from the initial field.
* DVS-criterion studies: the unstructured velocity-space criterion of Sec. 4.4 with
  its constants varied (outer radius factor, centre factor, refined-ball radius, with
  or without refined balls, size K), each variant iterated to convergence, so that the
  surface coefficients can be compared across velocity spaces.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import inputs as I
from .rykov import RK_FARFIELD, RK_OK, Solver


def freestream_at(U, aoa_deg: float, plane: str = "xz"):
    """The freestream of speed |U| along +x turned by aoa_deg towards +z (plane "xz")
    or +y ("xy"), and the lift direction normal to it in that plane."""
    s = float(np.linalg.norm(U))
    a = math.radians(aoa_deg)
    if plane == "xz":
        return (s * math.cos(a), 0.0, s * math.sin(a)), (-math.sin(a), 0.0, math.cos(a))
    if plane == "xy":
        return (s * math.cos(a), s * math.sin(a), 0.0), (-math.sin(a), math.cos(a), 0.0)
    raise ValueError("plane must be 'xz' or 'xy'")


def _turn(v, aoa_deg: float, plane: str):
    """Velocity vectors v [n, 3] turned by aoa_deg in the plane of freestream_at."""
    a = math.radians(aoa_deg)
    ca, sa = math.cos(a), math.sin(a)
    j = 2 if plane == "xz" else 1
    out = np.array(v, dtype=np.float64, copy=True)
    out[:, 0] = ca * v[:, 0] - sa * v[:, j]
    out[:, j] = sa * v[:, 0] + ca * v[:, j]
    return out


def turned_workload(wl: I.Workload, aoa_deg: float, plane: str = "xz") -> I.Workload:
    """The workload with its freestream turned by aoa_deg: farfield velocities, the
    initial velocities and the discrete velocities all turned about the same axis, so
    that a velocity space built around the freestream by the Sec. 4.4 criterion (outer
    ball centred at 0.4 U_inf, refined ball at U_inf) still surrounds it.  The body and
    the mesh stay where they are."""
    import dataclasses
    U0 = np.asarray(wl.ref["U"], dtype=np.float64)
    U, _ = freestream_at(U0, aoa_deg, plane)
    bcs = [dataclasses.replace(b, U=tuple(_turn(np.asarray([b.U], float), aoa_deg, plane)[0]))
           if b.kind == RK_FARFIELD else b for b in wl.bcs]
    prim = np.array(wl.prim0, dtype=np.float64, copy=True)
    prim[:, 1:4] = _turn(prim[:, 1:4], aoa_deg, plane)
    dvs = I.DVS(u=_turn(wl.dvs.u, aoa_deg, plane), w=wl.dvs.w, name=f"{wl.dvs.name}@{aoa_deg:g}")
    ref = dict(wl.ref)
    ref["U"] = tuple(U)
    return dataclasses.replace(wl, bcs=bcs, prim0=prim, dvs=dvs, ref=ref,
                               name=f"{wl.name}_aoa{aoa_deg:g}")


def aoa_sweep(wl: I.Workload, angles_deg, precision: str = "mixed", n_iter: int = 600,
              tol: float = 1e-6, plane: str = "xz", x_ref=(0.0, 0.0, 0.0), S_ref: float = 1.0,
              L_ref: float = 1.0):
    """Converge the workload at each angle of attack (turned_workload, from its initial
    field) and return one record per angle: iterations, final residual, wall time,
    force, moment, C_D, C_L, C_m and L/D (rk_aero with the turned freestream and its
    lift direction)."""
    U0 = np.asarray(wl.ref["U"], dtype=np.float64)
    out = []
    for a in angles_deg:
        wa = turned_workload(wl, a, plane)
        U, e_l = freestream_at(U0, a, plane)
        s = Solver(wa, precision)
        t0 = time.perf_counter()
        rc, n, res = s.iterate(n_iter, tol)
        wall = time.perf_counter() - t0
        if rc != RK_OK:
            raise RuntimeError(f"aoa_sweep: iteration failed at {a} degrees ({rc})")
        ld = s.aero(x_ref=x_ref, S_ref=S_ref, L_ref=L_ref, lift_dir=e_l, rho_inf=wl.ref["rho"], U_inf=U)
        out.append(dict(aoa=float(a), iterations=n, residual=float(np.max(res)), wall_s=wall,
                        force=ld[0:3].tolist(), moment=ld[3:6].tolist(), C_D=float(ld[6]),
                        C_L=float(ld[7]), C_m=float(ld[8]), L_over_D=float(ld[9])))
        s.close()
    return out


def dvs_study(make_workload, variants, precision: str = "mixed", n_iter: int = 600,
              tol: float = 1e-6, S_ref: float = 1.0):
    """Run one workload per DVS variant to convergence.  make_workload(**variant)
    returns the workload (e.g. lambda **v: inputs.sphere_workload(dvs_target=...,
    dvs_options=v)); each record holds the variant, K, the iterations, the residual,
    C_D (along the freestream) and the wall heat."""
    out = []
    for v in variants:
        wl = make_workload(**v)
        s = Solver(wl, precision)
        t0 = time.perf_counter()
        rc, n, res = s.iterate(n_iter, tol)
        wall = time.perf_counter() - t0
        if rc != RK_OK:
            raise RuntimeError(f"dvs_study: iteration failed for {v} ({rc})")
        ld = s.aero(S_ref=S_ref)
        _, _, heat = s.surface()
        out.append(dict(variant=dict(v), K=int(wl.dvs.K), iterations=n, residual=float(np.max(res)),
                        wall_s=wall, C_D=float(ld[6]), heat=float(heat)))
        s.close()
    return out
