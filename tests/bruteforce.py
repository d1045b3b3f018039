"""Independent NumPy restatement of one implicit iteration (Steps 2-6 of Sec. 3.5),
for tiny meshes only.

It is written separately from the C oracle and in a different style: velocities are
vectorised, cells are visited one at a time, the least-squares gradient uses
``numpy.linalg.lstsq``, the Gauss-Seidel sweeps are plain sequential sweeps over
the cells sorted by (colour, index) with the coefficients written with sign() exactly
as in Eq. implicit_mic_final_equ, and Venkatakrishnan's limiter is written in its
original (1/Delta_2)[...] form.  Agreement with the oracle to round-off pins the
oracle's transcription (tests/test_oracle_solver.py).  Readings of the paper where it
is silent are the same as the oracle's (they are part of the method definition).
"""
from __future__ import annotations

import numpy as np


def _prim(W, R):
    rho = W[0]
    U = W[1:4] / rho
    ke = 0.5 * rho * U @ U
    return rho, U, (W[4] - ke) / (2.5 * rho * R), (W[4] - ke - W[5]) / (1.5 * rho * R), W[5] / (rho * R)


class BruteForce:
    def __init__(self, wl, params=None):
        self.wl = wl
        self.p = params if params is not None else wl.params
        m, d = wl.mesh, wl.dvs
        self.N, self.F, self.K = m.n_cell, m.n_face, d.K
        self.u, self.w = d.u.copy(), d.w.copy()
        self.m = m
        self.faces_of = [[] for _ in range(self.N)]
        for f, (a, b) in enumerate(m.face_cell):
            self.faces_of[a].append(f)
            if b >= 0:
                self.faces_of[b].append(f)
        self.order = sorted(range(self.N), key=lambda i: (int(m.cell_colour[i]), i))
        self.bcs = wl.bcs
        R = self.p.R
        # CFL step, local physical step, implicit step
        self.dt = np.zeros(self.N)
        for i in range(self.N):
            tot = np.zeros(self.K)
            for f in self.faces_of[i]:
                sgn = 1.0 if m.face_cell[f, 0] == i else -1.0
                un = self.u @ (sgn * m.face_normal[f])
                tot += m.face_area[f] * np.where(un > 0, un, 0.0)
            self.dt[i] = self.p.cfl_s * m.cell_volume[i] / tot.max()
        self.s = np.array([min(self.dt[a], self.dt[b]) if b >= 0 else self.dt[a]
                           for a, b in m.face_cell])
        self.iter = 0
        # Step 1: equilibrium initial state
        self.W = np.zeros((self.N, 6))
        self.q = np.zeros((self.N, 6))
        self.phi = np.zeros((2, self.N, self.K))
        for i, pr in enumerate(wl.prim0):
            rho, U, Ttr, Trot = pr[0], pr[1:4], pr[4], pr[5]
            self.W[i] = [rho, *(rho * U), 0.5 * rho * U @ U + 1.5 * rho * R * Ttr + rho * R * Trot,
                         rho * R * Trot]
            self.phi[:, i] = self.equilibrium(self.W[i], self.q[i])

    # -- model -----------------------------------------------------------------------
    def maxwell(self, rho, U, T):
        RT = self.p.R * T
        c = self.u - U
        return rho / (2 * np.pi * RT) ** 1.5 * np.exp(-(c * c).sum(1) / (2 * RT))

    def equilibrium(self, W, q, state=None):
        """Rykov reduced equilibria G*, R* (Eqs. eqdf_G* - eqdf_Rrot)."""
        P = self.p
        R = P.R
        if state is None:
            rho, U, T, Ttr, Trot = _prim(W, R)
        else:
            rho, U, T, Ttr, Trot = state
        qtr, qrot = q[:3], q[3:]
        c = self.u - U
        c2 = (c * c).sum(1)
        m_tr = self.maxwell(rho, U, Ttr)
        m_eq = self.maxwell(rho, U, T)
        Gtr = m_tr * (1 + (c @ qtr) / (15 * R * Ttr * rho * R * Ttr) * (c2 / (R * Ttr) - 5))
        Grot = m_eq * (1 + P.omega0 * (c @ qtr) / (15 * R * T * rho * R * T) * (c2 / (R * T) - 5))
        Htr = R * Trot * (Gtr + (1 - P.delta) * (c @ qrot) / (R * Ttr * rho * R * Trot) * m_tr)
        Hrot = R * T * (Grot + P.omega1 * (1 - P.delta) * (c @ qrot) / (R * T * rho * R * T) * m_eq)
        Z = P.Z_rot
        return np.stack([(Z - 1) / Z * Gtr + Grot / Z, (Z - 1) / Z * Htr + Hrot / Z])

    def tau(self, rho, Ttr):
        P = self.p
        return P.mu_ref * (Ttr / P.T_ref) ** P.omega_vis / (rho * P.R * Ttr)

    def cfl_imp(self):
        P = self.p
        if P.cfl_imp0 <= 0 or P.cfl_ramp <= 1:
            return P.cfl_imp
        return min(P.cfl_imp, P.cfl_imp0 * P.cfl_ramp ** self.iter)

    # -- Step 2 (a): gradient and limiter --------------------------------------------
    def gradient(self):
        m, P = self.m, self.p
        lim = 2 if self.iter < P.first_order_iters else P.limiter
        self.grad = np.zeros((2, self.N, self.K, 3))
        for i in range(self.N):
            rows, nbrs = [], []
            for f in self.faces_of[i]:
                a, b = m.face_cell[f]
                j = b if a == i else a
                if j >= 0:
                    rows.append(m.cell_center[j] - m.cell_center[i]); nbrs.append(j)
                else:
                    rows.append(m.face_center[f] - m.cell_center[i]); nbrs.append(-1)
            A = np.array(rows)
            for fd in range(2):
                dphi = np.array([self.phi[fd, j] - self.phi[fd, i] if j >= 0 else np.zeros(self.K)
                                 for j in nbrs])                     # [m, K]
                g = np.linalg.lstsq(A, dphi, rcond=None)[0].T       # [K, 3]
                if lim == 2:
                    L = np.zeros(self.K)
                elif lim == 0:
                    L = np.ones(self.K)
                else:
                    interior = [r for r, j in zip(dphi, nbrs) if j >= 0]
                    dmax = np.maximum(0.0, np.max(interior, axis=0)) if interior else np.zeros(self.K)
                    dmin = np.minimum(0.0, np.min(interior, axis=0)) if interior else np.zeros(self.K)
                    # threshold relative to the cell value (per velocity)
                    eps2 = (P.lim_k * m.cell_volume[i] ** (1.0 / 3.0)) ** 3 * self.phi[fd, i] ** 2
                    L = np.ones(self.K)
                    for f in self.faces_of[i]:
                        d2 = g @ (m.face_center[f] - m.cell_center[i])
                        d1 = np.where(d2 > 0, dmax, dmin)
                        with np.errstate(divide="ignore", invalid="ignore"):
                            psi = (1.0 / d2) * (((d1 ** 2 + eps2) * d2 + 2 * d2 ** 2 * d1)
                                                / (d1 ** 2 + 2 * d2 ** 2 + d1 * d2 + eps2))
                        psi = np.where(d2 == 0, 1.0, psi)
                        L = np.minimum(L, psi)
                self.grad[fd, i] = g * L[:, None]

    # -- Step 2 (b)-(d) -----------------------------------------------------------------
    def faces(self):
        m, P, R = self.m, self.p, self.p.R
        Z = P.Z_rot
        self.face = np.zeros((2, self.F, self.K))
        self.face0 = np.zeros((2, self.F, self.K))
        self.fstate = np.zeros((self.F, 16))
        for f, (a, b) in enumerate(m.face_cell):
            n, xf, s = m.face_normal[f], m.face_center[f], self.s[f]
            un = self.u @ n

            def recon(c):
                r = xf - self.u * s - m.cell_center[c]             # [K,3]
                return np.stack([self.phi[fd, c] + (r * self.grad[fd, c]).sum(1) for fd in range(2)])

            if b >= 0:
                ph0 = np.where(un > 0, recon(a), recon(b))
                g0, h0 = ph0
                rho = self.w @ g0
                U = (self.w * g0) @ self.u / rho
                E = self.w @ (0.5 * (self.u ** 2).sum(1) * g0 + h0)
                Er0 = self.w @ h0
                ke = 0.5 * rho * U @ U
                T = (E - ke) / (2.5 * rho * R)
                tau = self.tau(rho, (E - ke - Er0) / (1.5 * rho * R))
                Erot = (Z * tau * Er0 + s * rho * R * T) / (Z * tau + s)
                Ttr = (E - ke - Erot) / (1.5 * rho * R)
                Trot = Erot / (rho * R)
                c = self.u - U
                c2 = (c * c).sum(1)
                qtr = tau * 0.5 * ((self.w * c2 * g0) @ c) / (tau + s - s / 3 * (1 - 1 / Z + P.omega0 / Z))
                qrot = tau * ((self.w * h0) @ c) / (tau + s - s * (1 - P.delta) * (1 - 1 / Z + P.omega1 / Z))
                eq = self.equilibrium(None, np.concatenate([qtr, qrot]), (rho, U, T, Ttr, Trot))
                self.face[:, f] = (tau * ph0 + s * eq) / (tau + s)
                self.face0[:, f] = ph0
                self.fstate[f] = [rho, *U, T, Ttr, Trot, tau, *qtr, *qrot, s, 0.0]
            else:
                bc = self.bcs[-1 - b]
                inner = recon(a)
                Tb = bc.T
                if bc.kind == 0:
                    M = self.maxwell(1.0, np.asarray(bc.U), Tb)
                else:
                    M = self.maxwell(bc.rho, np.asarray(bc.U), Tb)
                outside = np.stack([M, R * Tb * M])
                ph0 = np.where(un > 0, inner, outside)
                rho_w = 0.0
                if bc.kind == 0:
                    rho_w = (self.w * np.where(un > 0, un, 0)) @ ph0[0] / \
                        ((self.w * np.where(un < 0, -un, 0)) @ M)
                    face = np.where(un > 0, ph0, rho_w * ph0)
                else:
                    face = ph0
                self.face0[:, f] = ph0
                self.face[:, f] = face
                self.fstate[f, 14] = s
                self.fstate[f, 15] = rho_w

    # -- Step 2 (e), Step 3 -------------------------------------------------------------
    def fluxes(self):
        m = self.m
        self.microF = np.zeros((2, self.N, self.K))
        self.macroF = np.zeros((self.N, 6))
        Phi = np.stack([np.ones(self.K), self.u[:, 0], self.u[:, 1], self.u[:, 2],
                        0.5 * (self.u ** 2).sum(1)])
        for i in range(self.N):
            for f in self.faces_of[i]:
                n = m.face_normal[f] * (1.0 if m.face_cell[f, 0] == i else -1.0)
                un = self.u @ n
                A_V = m.face_area[f] / m.cell_volume[i]
                self.microF[:, i] += A_V * un * self.face[:, f]
                g, h = self.face[:, f]
                wun = self.w * un
                mac = np.concatenate([Phi @ (wun * g), [wun @ h]])
                mac[4] += wun @ h
                self.macroF[i] += A_V * mac

    # -- Step 4 -------------------------------------------------------------------------
    def euler(self, W, n):
        rho = W[0]
        U = W[1:4] / rho
        p = 0.4 * (W[4] - 0.5 * rho * U @ U)
        Un = U @ n
        return np.array([rho * Un, *(W[1:4] * Un + p * n), (W[4] + p) * Un, W[5] * Un])

    def macro(self):
        m, P, R = self.m, self.p, self.p.R
        Z = P.Z_rot
        dtimp = self.cfl_imp() * self.dt
        self.dtimp = dtimp
        r = np.zeros(self.F)
        for f, (a, b) in enumerate(m.face_cell):
            if b >= 0:
                Wm = 0.5 * (self.W[a] + self.W[b])
                dl = np.linalg.norm(m.cell_center[b] - m.cell_center[a])
            else:
                Wm = self.W[a]
                dl = 2 * np.linalg.norm(m.face_center[f] - m.cell_center[a])
            rho, U, T, Ttr, Trot = _prim(Wm, R)
            mu = P.mu_ref * (Ttr / P.T_ref) ** P.omega_vis
            r[f] = abs(U @ m.face_normal[f]) + np.sqrt(1.4 * R * T) + 2 * mu / (rho * dl)
        dW = np.zeros((self.N, 6))
        tau_n = [self.tau(_prim(w, R)[0], _prim(w, R)[3]) for w in self.W]
        seq = self.order + self.order[::-1]
        for _ in range(P.n_macro_sgs):
            for i in seq:
                Wc = self.W[i] + dW[i]
                rho, U, T, Ttr, Trot = _prim(Wc, R)
                tau = tau_n[i]
                Di = 1.0 / dtimp[i]
                lhs = np.zeros(6)
                for f in self.faces_of[i]:
                    a, b = m.face_cell[f]
                    j = b if a == i else a
                    A_V = m.face_area[f] / m.cell_volume[i]
                    Di += 0.5 * A_V * r[f]
                    if j < 0:
                        continue
                    n = m.face_normal[f] * (1.0 if a == i else -1.0)
                    jac = self.euler(self.W[j] + dW[j], n) - self.euler(self.W[j], n)
                    lhs += 0.5 * A_V * (jac - r[f] * dW[j])
                res = -self.macroF[i].copy()
                res[5] += (rho * R * T - self.W[i, 5]) / (Z * tau)
                diag = np.full(6, Di)
                diag[5] += 1.0 / (Z * tau)
                cand = (res - lhs) / diag
                r2, _, _, Ttr2, Trot2 = _prim(self.W[i] + cand, R)
                if r2 > 0 and Ttr2 > 0 and Trot2 > 0:
                    dW[i] = cand
        self.Wt = self.W + dW
        self.taut = np.array([self.tau(_prim(w, R)[0], _prim(w, R)[3]) for w in self.Wt])

    # -- Step 5 -------------------------------------------------------------------------
    def micro(self):
        m, P = self.m, self.p
        self.eqt = np.stack([self.equilibrium(self.Wt[i], self.q[i]) for i in range(self.N)], axis=1)
        self.res = (self.eqt - self.phi) / self.taut[None, :, None] - self.microF
        dphi = np.zeros((2, self.N, self.K))
        seq = self.order + self.order[::-1]
        for _ in range(P.n_micro_sgs):
            for i in seq:
                Dii = 1.0 / self.dtimp[i] + 1.0 / self.taut[i]
                off = np.zeros((2, self.K))
                for f in self.faces_of[i]:
                    a, b = m.face_cell[f]
                    j = b if a == i else a
                    n = m.face_normal[f] * (1.0 if a == i else -1.0)
                    un = self.u @ n
                    A_V = m.face_area[f] / m.cell_volume[i]
                    Dii = Dii + 0.5 * A_V * un * (1 + np.sign(un))
                    if j >= 0:
                        off += 0.5 * A_V * un * (1 - np.sign(un)) * dphi[:, j]
                dphi[:, i] = (self.res[:, i] - off) / Dii
        self.dphi = dphi

    # -- Step 6 -------------------------------------------------------------------------
    def update(self):
        P, R = self.p, self.p.R
        Z = P.Z_rot
        Wold = self.W.copy()
        self.phi = self.phi + self.dphi
        for i in range(self.N):
            rho, U, T, Ttr, Trot = _prim(self.Wt[i], R)
            d = self.phi[:, i] - self.eqt[:, i]
            c = self.u - U
            c2 = (c * c).sum(1)
            self.W[i, 0] = self.w @ d[0] + self.Wt[i, 0]
            self.W[i, 1:4] = (self.w * d[0]) @ self.u + self.Wt[i, 1:4]
            self.W[i, 4] = self.w @ (0.5 * (self.u ** 2).sum(1) * d[0] + d[1]) + self.Wt[i, 4]
            self.W[i, 5] = self.w @ d[1] + rho * R * ((1 - 1 / Z) * Trot + T / Z)
            qtr = 0.5 * ((self.w * c2 * d[0]) @ c) + self.q[i, :3] * (1 - (1 - P.omega0) / Z) / 3
            qrot = (self.w * d[1]) @ c + self.q[i, 3:] * (1 - P.delta) * (1 - (1 - P.omega1) / Z)
            self.q[i] = np.concatenate([qtr, qrot])
        num = np.abs(self.W - Wold).sum(0)
        mom = np.linalg.norm(Wold[:, 1:4], axis=1).sum()
        den = np.array([np.abs(Wold[:, 0]).sum(), mom, mom, mom,
                        np.abs(Wold[:, 4]).sum(), np.abs(Wold[:, 5]).sum()])
        self.iter += 1
        return num / np.maximum(den, 1e-300)

    def iterate(self):
        self.gradient()
        self.faces()
        self.fluxes()
        self.macro()
        self.micro()
        return self.update()
