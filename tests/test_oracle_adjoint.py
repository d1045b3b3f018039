"""Pins of the steady-residual / adjoint oracle (oracle/adjoint.py, plain PyTorch CPU).

The restatement of R(X; p) is checked against the C oracle's independent
restatement of the same steps (flux, gradient, wall sums), against the fixed point
of the C oracle's iteration (R = 0 at a converged state), against conservation
(closed cavity), and the adjoint total derivative against central finite
differences of re-converged C-oracle steady states.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from oracle.adjoint import DRAG, HEAT, Steady
from paper_2303_10846_gb300 import inputs as I
from tests.workloads import tiny_cavity, tiny_tet


def lid_farfield():
    """Tiny cavity whose lid is an (inflowing, sheared) farfield boundary."""
    wl = tiny_cavity()
    wl.bcs = [wl.bcs[0], I.BC(I.BC_FARFIELD, 1.05, (0.15, 0.02, -0.03), 1.1)]
    return wl


def _second_order(wl):
    wl.params = dataclasses.replace(wl.params, first_order_iters=0)
    return wl


def _state(o, st):
    return (torch.as_tensor(o.get(O.BUF_PHI)), torch.as_tensor(o.get(O.BUF_W)),
            torch.as_tensor(o.get(O.BUF_Q)))


def _tet_sutherland():
    wl = tiny_tet(n_gh=4)
    wl.params = dataclasses.replace(wl.params, viscosity_law=1, sutherland_c=0.4)
    return wl


@pytest.mark.parametrize("make", [tiny_cavity, lambda: tiny_tet(n_gh=4), _tet_sutherland],
                         ids=["cavity", "tet", "tet-sutherland"])
def test_flux_and_gradient_match_c_oracle(make):
    wl = _second_order(make())
    o = O.Oracle(wl)
    o.iterate(3)
    st = Steady(wl)
    phi, _, _ = _state(o, st)
    o.step("gradient"); o.step("faces"); o.step("fluxes")
    Fc = o.get(O.BUF_MICRO_F)
    Gc = o.get(O.BUF_GRAD)
    Ft, _ = st.micro_flux(phi, st.p0())
    Gt = st.gradient(phi).permute(0, 3, 1, 2).numpy()
    assert np.max(np.abs(Ft.numpy() - Fc)) <= 1e-12 * np.max(np.abs(Fc))
    assert np.max(np.abs(Gt - Gc)) <= 1e-12 * np.max(np.abs(Gc))


def test_objectives_match_c_oracle_wall_sums():
    wl = _second_order(tiny_tet(n_gh=4))
    o = O.Oracle(wl)
    o.iterate(3)
    st = Steady(wl)
    phi, _, _ = _state(o, st)
    _, force, heat = o.surface()
    Jh = float(st.objective(phi, st.p0(), HEAT))
    Jd = float(st.objective(phi, st.p0(), DRAG))
    e = st.drag_direction()
    assert abs(Jh - heat) <= 1e-12 * abs(heat)
    assert abs(Jd - force @ e) <= 1e-12 * abs(force @ e)


@pytest.fixture(scope="module")
def converged_lid_farfield():
    wl = lid_farfield()
    o = O.Oracle(wl)
    rc, n, res = o.iterate(3000, 1e-14)
    assert rc == 0 and res.max() < 1e-13
    st = Steady(wl)
    return wl, o, st


def test_residual_vanishes_at_the_iteration_fixed_point(converged_lid_farfield):
    """R is the fixed-point residual of the scheme: zero at a converged iterate."""
    wl, o, st = converged_lid_farfield
    phi, W, q = _state(o, st)
    Rp, RW, Rq = st.residual(phi, W, q, st.p0())
    Fm, _ = st.micro_flux(phi, st.p0())
    assert float(Rp.abs().max()) < 1e-11 * float(Fm.abs().max())
    assert float(RW.abs().max()) < 1e-12 * float(W.abs().max())
    assert float(Rq.abs().max()) < 1e-12 * float(W.abs().max())
    # and not zero away from it
    Rp2, _, _ = st.residual(phi * 1.001, W, q, st.p0())
    assert float(Rp2.abs().max()) > 1e-6 * float(Fm.abs().max())


def test_closed_cavity_conserves_energy_and_momentum():
    """All-wall cavity at steady state: the total energy and momentum fluxes through
    the walls vanish, so J_heat = 0 and its T_w derivative is 0."""
    wl = tiny_cavity()
    o = O.Oracle(wl)
    rc, n, res = o.iterate(3000, 1e-14)
    st = Steady(wl)
    phi, W, q = _state(o, st)
    x = st.pack(phi, W, q)
    scale = float(W[:, 4].abs().max())
    lam, J, dJdp = st.adjoint_dense(x, HEAT)
    assert abs(J) < 1e-12 * scale
    assert abs(float(dJdp[0])) < 1e-10 * scale


@pytest.mark.parametrize("lim,h,law", [(0, 1e-6, 0), (1, 1e-7, 0), (2, 1e-6, 0), (0, 1e-6, 1)])
def test_vjp_is_the_transpose_of_the_finite_difference_jvp(lim, h, law):
    """<v, J u> by central differences equals <J^T v, u> (the limiter's min/max kinks
    are crossed by the wider steps, hence the smaller step with the limiter on); law 1
    takes Sutherland's viscosity, whose temperature slope enters through tau."""
    wl = tiny_tet(n_gh=4)
    wl.params = dataclasses.replace(wl.params, first_order_iters=0, limiter=lim,
                                    viscosity_law=law, sutherland_c=0.4)
    o = O.Oracle(wl)
    o.iterate(3)
    st = Steady(wl)
    x = st.pack(*_state(o, st))
    g = torch.Generator().manual_seed(5)
    u = torch.randn(x.shape, generator=g, dtype=torch.float64) * x.abs()
    v = torch.randn(x.shape, generator=g, dtype=torch.float64)
    p = st.p0()
    Ju = (st.R_flat(x + h * u, p) - st.R_flat(x - h * u, p)) / (2 * h)
    vt, _ = st.vjp(x, v, p)
    lhs, rhs = float(v @ Ju), float(vt @ u)
    assert abs(lhs - rhs) <= 1e-6 * abs(lhs)


def _converged_J(make, ip, h, start):
    """(J_heat, J_drag) of the C-oracle steady state with parameter ip shifted by h."""
    wl = make()
    if ip == 0:
        wl.bcs = [dataclasses.replace(b, T=b.T + h) if b.kind == I.BC_WALL else b for b in wl.bcs]
    else:
        b = wl.bcs[1]
        arr = [b.rho, *b.U, b.T]
        arr[ip - 1] += h
        wl.bcs = [wl.bcs[0], I.BC(I.BC_FARFIELD, arr[0], tuple(arr[1:4]), arr[4])]
    o = O.Oracle(wl)
    o.set_state(*start)
    rc, n, res = o.iterate(3000, 1e-15)
    assert rc == 0 and res.max() < 1e-14
    st = Steady(wl)
    phi = torch.as_tensor(o.get(O.BUF_PHI))
    return np.array([float(st.objective(phi, st.p0(), HEAT)), float(st.objective(phi, st.p0(), DRAG))])


def test_adjoint_total_derivative_matches_finite_differences(converged_lid_farfield):
    """dJ/dp = dJ/dp|_X + lam^T dR/dp (dense adjoint) against central differences of
    fully re-converged steady states, h = 1e-6 (truncation ~h^2, convergence error
    ~1e-15/h): agreement to 1e-7 of max |dJ/dp|."""
    wl, o, st = converged_lid_farfield
    x = st.pack(*_state(o, st))
    start = (o.get(O.BUF_W), o.get(O.BUF_Q), o.get(O.BUF_PHI))
    A = st.jacobian(x).numpy()
    h = 1e-6
    fd = np.array([(_converged_J(lid_farfield, ip, h, start) - _converged_J(lid_farfield, ip, -h, start))
                   / (2 * h) for ip in range(6)])
    for col, which in enumerate((HEAT, DRAG)):
        J, jx, jp = st.objective_grad(x, which)
        lam = torch.as_tensor(np.linalg.solve(A.T, -jx.numpy()))
        _, rp = st.vjp(x, lam)
        dJdp = (jp + rp).numpy()
        assert np.max(np.abs(fd[:, col] - dJdp)) <= 1e-7 * np.max(np.abs(dJdp)), (which, fd[:, col], dJdp)


def test_frozen_limiter_operator():
    """Limiter freezing: iterations before the freeze are unchanged; afterwards the C
    oracle reconstructs with the stored limiter values, which the restated operator
    reproduces when given them (and the stored values are in [0, 1])."""
    def make(frz):
        wl = tiny_tet(n_gh=4)
        wl.params = dataclasses.replace(wl.params, first_order_iters=0, limiter_freeze=frz)
        return wl
    o1, o2 = O.Oracle(make(12)), O.Oracle(make(0))
    o1.iterate(11); o2.iterate(11)
    assert np.array_equal(o1.get(O.BUF_PHI), o2.get(O.BUF_PHI))
    o1.iterate(20)
    L = o1.get(O.BUF_LSTORE)
    assert L.min() >= 0.0 and L.max() <= 1.0 and L.min() < 1.0
    phi = torch.as_tensor(o1.get(O.BUF_PHI))
    o1.step("gradient"); o1.step("faces"); o1.step("fluxes")
    Fc = o1.get(O.BUF_MICRO_F)
    wl = make(12)
    Ff, _ = Steady(wl, L_frozen=L).micro_flux(phi, Steady(wl).p0())
    Fl, _ = Steady(wl).micro_flux(phi, Steady(wl).p0())
    assert np.max(np.abs(Ff.numpy() - Fc)) <= 1e-12 * np.max(np.abs(Fc))
    assert np.max(np.abs(Fl.numpy() - Fc)) > 1e-9 * np.max(np.abs(Fc))
