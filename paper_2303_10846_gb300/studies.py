"""Parameter studies on top of the solver (host-side loops over library calls; every
iteration and every load integral runs in the CUDA kernels of librykov).

* Angle-of-attack sweeps: the lift, drag, lift-to-drag and pitching-moment curves that
  Sec. 4 reports for the blunted cone and the capsule.  The freestream of the farfield
  boundaries is turned in a plane; each angle continues from the previous converged
  state.
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
from .rykov import RK_FARFIELD, RK_OK, Solver, _c, _ptr


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


def set_farfield_velocity(solver: Solver, U) -> None:
    """Give every farfield boundary of the solver's workload the velocity U (density
    and temperature unchanged)."""
    Uc = _c(U, np.float64)
    for b, bc in enumerate(solver.wl.bcs):
        if bc.kind == RK_FARFIELD:
            solver._check(solver.L.rk_set_bc(solver.h, b, RK_FARFIELD, float(bc.rho), _ptr(Uc), float(bc.T)))


def _turn(v, aoa_deg: float, plane: str):
    """Velocity vectors v [n, 3] turned by aoa_deg in the plane of freestream_at."""
    a = math.radians(aoa_deg)
    ca, sa = math.cos(a), math.sin(a)
    j = 2 if plane == "xz" else 1
    out = np.array(v, dtype=np.float64, copy=True)
    out[:, 0] = ca * v[:, 0] - sa * v[:, j]
    out[:, j] = sa * v[:, 0] + ca * v[:, j]
    return out


def aoa_sweep(wl: I.Workload, angles_deg, precision: str = "mixed", n_iter: int = 600,
              tol: float = 1e-6, plane: str = "xz", x_ref=(0.0, 0.0, 0.0), S_ref: float = 1.0,
              L_ref: float = 1.0, solver: Solver | None = None, restart: bool = True):
    """Converge the workload at each angle of attack in turn and return one record per
    angle: iterations, final residual, force, moment, C_D, C_L, C_m and L/D (rk_aero
    with the turned freestream and its lift direction).

    The first angle starts from the workload's initial field with its velocities turned
    by that angle.  Each later angle continues from the previous converged state; with
    restart=True that state is set again (rk_set_state), so that the start-up of the
    iteration (first-order iterations, implicit-CFL ramp) damps the jump of the
    boundary condition."""
    import torch
    s = solver if solver is not None else Solver(wl, precision)
    U0 = np.asarray(wl.ref["U"], dtype=np.float64)
    rho = wl.ref["rho"]
    out = []
    for n_a, a in enumerate(angles_deg):
        U, e_l = freestream_at(U0, a, plane)
        set_farfield_velocity(s, U)
        if n_a == 0:
            prim = np.array(wl.prim0, dtype=np.float64, copy=True)
            prim[:, 1:4] = _turn(prim[:, 1:4], a, plane)
            s.set_state_prim(prim)
        elif restart:
            W, q, _ = s.moments()
            dist = s.get_distribution()
            Wd = torch.from_numpy(W).to(dist.device)
            qd = torch.from_numpy(q).to(dist.device)
            s._check(s.L.rk_set_state(s.h, _ptr(Wd), _ptr(qd), _ptr(dist), 1))
        t0 = time.perf_counter()
        rc, n, res = s.iterate(n_iter, tol)
        wall = time.perf_counter() - t0
        if rc != RK_OK:
            raise RuntimeError(f"aoa_sweep: iteration failed at {a} degrees ({rc})")
        ld = s.aero(x_ref=x_ref, S_ref=S_ref, L_ref=L_ref, lift_dir=e_l, rho_inf=rho, U_inf=U)
        out.append(dict(aoa=float(a), iterations=n, residual=float(np.max(res)), wall_s=wall,
                        force=ld[0:3].tolist(), moment=ld[3:6].tolist(), C_D=float(ld[6]),
                        C_L=float(ld[7]), C_m=float(ld[8]), L_over_D=float(ld[9])))
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
