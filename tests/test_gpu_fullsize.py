"""Parity at the benchmark's full size: the Ma-5 sphere, N = 61,911 tetrahedra, K = 3,033
velocities, iterated in the benchmark's launch configuration (the CUDA graph of one
iteration), FP64 and mixed precision.  The oracle cannot run the whole case in a test,
so it checks sampled outputs one at a time (interface kernel per face from the GPU's
own inputs, micro residual per cell) and the tests check properties that hold at any
size (mixed vs FP64 surface quantities, bitwise repeatability).

Tolerances: FP64 1e-10 relative to the scale of the summed terms (the micro flux and
the residual are small differences of large terms).  Mixed: 2e-5,
because the GPU works in FP32 (relative rounding 6e-8, interface state from
float-float moments), while the oracle is fed the FP32 values widened to FP64.
"""
import numpy as np
import pytest

import oracle as O
from paper_2303_10846_gb300 import inputs as I
from tests import patch as PT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sphere():
    return I.sphere_workload()


def _solver(wl, prec, debug=False, macro32=False):
    from paper_2303_10846_gb300.rykov import Solver
    return Solver(wl, prec, debug=debug, macro32=macro32)


TOLS = {"fp64": 1e-10, "mixed": 2e-5}


def _rows_of(s, name, rows):
    rows = np.asarray(rows, np.int64)
    return s.debug_rows(name, rows)


def check_recon_patches(s, wl, prec, faces, phi_rows, W, q):
    """Reconstructed face values phi(x_ij - u s_ij) (Eq. flux_solve_phi_phi: gradient,
    limiter, upwind choice) of sampled interior faces against the oracle run on a
    two-ring patch around the face's cells, fed the GPU's own phi rows (widened to
    FP64 in mixed precision).  In mixed precision the upwind choice is taken on the
    FP32 value of u.n: velocities with |u.n| < 1e-5 |u| are left out there."""
    K = wl.dvs.K
    u = wl.dvs.u
    tol = TOLS[prec]
    phi0_gpu = _rows_of(s, "FACE", faces)
    for t, f in enumerate(faces):
        a, b = wl.mesh.face_cell[f]
        pw, g2l, fidx = PT.patch_workload(wl, [a, b], 2)
        P = np.array(sorted(g2l, key=g2l.get))
        phi = np.stack([phi_rows[int(g)] for g in P], axis=1)          # [2, n, K]
        op = O.Oracle(pw)
        op.set_state(W[P], q[P], phi.reshape(-1))
        op.step("gradient")
        op.step("faces")
        ref = op.get(O.BUF_FACE0).reshape(2, pw.mesh.n_face, K)[:, PT.local_face(fidx, f)]
        op.close()
        keep = np.ones(K, bool)
        if prec == "mixed":
            un = u @ wl.mesh.face_normal[f]
            keep = np.abs(un) > 1e-5 * np.linalg.norm(u, axis=1)
        for fd in range(2):
            sc = np.max(np.abs(phi[fd]))
            err = np.max(np.abs(phi0_gpu[fd, t, keep] - ref[fd, keep]))
            assert err <= tol * sc, f"face {f} field {fd}: {err / sc:.3e}"


def check_last_sweep_patches(s, wl, prec, cells, phi_n, q_n, Wt, taut, cfl):
    """The last point update of the micro PR-SGS (Eq. implicit_mic_final_equ) and the
    Step-6 update (Eqs. solve_rho - solve_qrot) of sampled cells of colour 0 (the last
    colour of the last, backward, sweep, so the neighbours' final increments are the
    ones it read) against the oracle on a one-ring patch fed the GPU's own Res,
    neighbour increments, W~, tau~, q^n and phi^n."""
    m = wl.mesh
    K = wl.dvs.K
    tol = TOLS[prec]
    csr = PT.cell_faces(m)
    nb = {int(i): PT.neighbours(m, csr, int(i)) for i in cells}
    rows = sorted(set(int(i) for i in cells) | set(j for v in nb.values() for j in v))
    res = dict(zip(rows, np.moveaxis(_rows_of(s, "RES", rows), 1, 0)))
    dphi = dict(zip(rows, np.moveaxis(_rows_of(s, "DPHI", rows), 1, 0)))
    phi1 = dict(zip(cells, np.moveaxis(_rows_of(s, "PHI", cells), 1, 0)))
    W1, q1 = s.debug_get("W"), s.debug_get("Q")
    u, w = wl.dvs.u, wl.dvs.w
    for i in cells:
        i = int(i)
        pw, g2l, _ = PT.patch_workload(wl, [i], 1, cfl_imp=cfl)
        P = np.array(sorted(g2l, key=g2l.get))
        n, li = len(P), g2l[i]
        z = np.zeros((2, K))
        op = O.Oracle(pw)
        op.set_state(W1[P], q_n[P], np.stack([phi_n[i] if g == i else z for g in P], 1).reshape(-1))
        op.put(O.BUF_RES, np.stack([res.get(int(g), z) for g in P], 1).reshape(-1))
        op.put(O.BUF_DPHI, np.stack([dphi.get(int(g), z) if g != i else z for g in P], 1).reshape(-1))
        op.put(O.BUF_WT, Wt[P].reshape(-1))
        op.put(O.BUF_TAUT, taut[P])
        op.micro_point(li, False, 0)
        d_o = op.get(O.BUF_DPHI).reshape(2, n, K)[:, li]
        sc_d = max(np.max(np.abs(dphi[j])) for j in [i] + nb[i])
        assert np.max(np.abs(dphi[i] - d_o)) <= tol * sc_d, f"cell {i} increment"
        op.update_cell(li)
        p_o = op.get(O.BUF_PHI).reshape(2, n, K)[:, li]
        assert np.max(np.abs(phi1[i] - p_o)) <= tol * np.max(np.abs(phi_n[i])), f"cell {i} phi"
        W_o = op.get(O.BUF_W).reshape(n, 6)[li]
        q_o = op.get(O.BUF_Q).reshape(n, 6)[li]
        op.close()
        # scales of the Step-6 sums: |W~| per row (momentum rows: rho |U~| + the thermal
        # speed rho sqrt(R T~)), and for q the summed magnitudes w |c|^3 |g| of the
        # velocity sum (a cancelling sum near equilibrium)
        rho = Wt[i, 0]
        R = wl.params.R
        Tsc = Wt[i, 4] / (2.5 * rho * R)
        msc = np.linalg.norm(Wt[i, 1:4]) + rho * np.sqrt(R * Tsc)
        scW = np.array([rho, msc, msc, msc, abs(Wt[i, 4]), abs(Wt[i, 5])])
        assert np.all(np.abs(W1[i] - W_o) <= tol * scW), f"cell {i} W"
        cvec = u - Wt[i, 1:4] / rho
        c2 = np.sum(cvec ** 2, axis=1)
        qsc = max(0.5 * np.sum(w * c2 ** 1.5 * np.abs(phi1[i][0])), np.sum(w * np.sqrt(c2) * np.abs(phi1[i][1])))
        assert np.max(np.abs(q1[i] - q_o)) <= tol * qsc, f"cell {i} q"


def check_sampled(s, wl, prec, n_iter, debug, n_faces=48, n_cells=48, seed=2024,
                  n_recon=6, n_last=6):
    """Iterate n_iter times (graph path), then step through one more iteration and
    check sampled interior faces (the reconstruction against the oracle on a patch;
    the interface kernel from the GPU's own phi(x_f - u s)), sampled cells (micro flux
    by its definition from the face values, first-sweep residual with the oracle's
    equilibrium at (W~, q^n)) and sampled colour-0 cells (last micro point update and
    Step-6 update against the oracle on a patch)."""
    from paper_2303_10846_gb300 import rykov as RK
    m = wl.mesh
    tol = TOLS[prec]
    s.iterate(n_iter)
    rng = np.random.default_rng(seed)
    interior = np.nonzero(m.face_cell[:, 1] >= 0)[0]
    faces = np.sort(rng.choice(interior, n_faces, replace=False))
    cells = np.sort(rng.choice(m.n_cell, n_cells, replace=False))
    rfaces = faces[:n_recon]
    csr = PT.cell_faces(m)
    rcells = sorted(set(int(g) for f in rfaces for g in PT.grow(m, csr, m.face_cell[f], 2)))
    phi_r = dict(zip(rcells, np.moveaxis(_rows_of(s, "PHI", rcells), 1, 0)))
    W0, q0 = s.debug_get("W"), s.debug_get("Q")
    s.step(RK.STEP_RECON)
    check_recon_patches(s, wl, prec, rfaces, phi_r, W0, q0)
    phi0 = s.debug_rows("FACE", faces)
    s.step(RK.STEP_FACES)
    phif = s.debug_rows("FACE", faces)
    fst = s.debug_get("FSTATE") if debug else None
    sf = s.debug_get("S")
    u, w = wl.dvs.u, wl.dvs.w
    for j, f in enumerate(faces):
        st, gf, hf = O.interface(wl.params, u, w, phi0[0, j], phi0[1, j], sf[f])
        sc = max(np.max(np.abs(gf)), np.max(np.abs(hf)))
        assert np.max(np.abs(phif[0, j] - gf)) <= tol * sc, f"face {f} g"
        assert np.max(np.abs(phif[1, j] - hf)) <= tol * sc, f"face {f} h"
        if fst is not None:
            for idx in (0, 4, 5, 6, 7):             # rho, T, T_tr, T_rot, tau
                assert abs(fst[f, idx] - st[idx]) <= tol * abs(st[idx]), f"face {f} state {idx}"
            qs = max(np.max(np.abs(st[8:14])), 1e-300)
            assert np.max(np.abs(fst[f, 8:14] - st[8:14])) <= 10 * tol * qs + 1e-14, f"face {f} q"
    s.step(RK.STEP_FLUXES)
    phi = s.debug_rows("PHI", cells)
    q_n = s.debug_get("Q")
    # the micro flux is a small difference of large face terms: errors are measured on
    # the scale of the terms (sum of their magnitudes), as for any cancelling sum
    Fd = np.zeros((2, len(cells), wl.dvs.K))
    Fs = np.zeros(len(cells))
    for j, i in enumerate(cells):
        fl = np.nonzero((m.face_cell[:, 0] == i) | (m.face_cell[:, 1] == i))[0]
        vals = s.debug_rows("FACE", fl)
        mag = np.zeros((2, wl.dvs.K))
        for t, f in enumerate(fl):
            sg = 1.0 if m.face_cell[f, 0] == i else -1.0
            term = m.face_area[f] * sg * (u @ m.face_normal[f]) * vals[:, t] / m.cell_volume[i]
            Fd[:, j] += term
            mag += np.abs(term)
        Fs[j] = np.max(mag)
    if debug:
        F = s.debug_rows("MICRO_F", cells)
        for j, i in enumerate(cells):
            assert np.max(np.abs(F[:, j] - Fd[:, j])) <= tol * Fs[j], f"cell {i} flux"
    s.step(RK.STEP_MACRO)
    Wt = s.debug_get("WT")
    taut = s.debug_get("TAUT")
    lcells = np.sort(rng.choice(np.nonzero(m.cell_colour == 0)[0], n_last, replace=False))
    phi_n = dict(zip(lcells, np.moveaxis(_rows_of(s, "PHI", lcells), 1, 0)))
    dt = s.debug_get("DT")
    cfl = dt[lcells[0], 1] / dt[lcells[0], 0]
    s.step(RK.STEP_MICRO)
    check_last_sweep_patches(s, wl, prec, lcells, phi_n, q_n, Wt, taut, cfl)
    res = s.debug_rows("RES", cells)
    R = wl.params.R
    for j, i in enumerate(cells):
        W = Wt[i]
        rho = W[0]
        U = W[1:4] / rho
        ke = 0.5 * rho * U @ U
        T = (W[4] - ke) / (2.5 * rho * R)
        Trot = W[5] / (rho * R)
        Ttr = (W[4] - ke - W[5]) / (1.5 * rho * R)
        stt = O.make_state(rho, U, T, Ttr, Trot, q_n[i, :3], q_n[i, 3:])
        G, H = O.equilibrium(wl.params, stt, u)
        coll = np.stack([(G - phi[0, j]) / taut[i], (H - phi[1, j]) / taut[i]])
        sc = max(np.max(np.abs(phi[:, j])) / taut[i], Fs[j])
        assert np.max(np.abs(res[:, j] - (coll - Fd[:, j]))) <= tol * sc, f"cell {i} residual"


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sampled_faces_and_cells_at_full_size(sphere, prec):
    """Sphere, the bench workload, past the first-order start."""
    s = _solver(sphere, prec, debug=True)
    check_sampled(s, sphere, prec, 12, True)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_capsule_sampled(prec):
    """Capsule at 25 degrees angle of attack, Mach 10, Kn 0.01: ~205k tetrahedra x ~6,000
    velocities (the capsule configuration, checked at its full size)."""
    wl = I.capsule_workload()
    s = _solver(wl, prec, debug=(prec == "mixed"))
    check_sampled(s, wl, prec, 12, prec == "mixed", n_faces=32, n_cells=32)


def test_scale_case_sampled():
    """Scale case: sphere-cone, ~520k tetrahedra x ~7,900 velocities in mixed precision
    (about 190 GB of device arrays), one second-order iteration checked on samples."""
    wl = I.cone_scale_workload()
    wl.params.first_order_iters = 0
    s = _solver(wl, "mixed", debug=False)
    check_sampled(s, wl, "mixed", 1, False, n_faces=24, n_cells=24)


def test_mixed_matches_fp64_on_the_surface_at_full_size(sphere):
    """Accuracy target of the mixed form: wall pressure, heat flux and drag
    within 1e-5 (relative to their largest values) of the FP64 form after the same
    iterations from the same state."""
    s64 = _solver(sphere, "fp64")
    s32 = _solver(sphere, "mixed")
    s64.iterate(40)
    s32.iterate(40)
    p64, f64, h64 = s64.surface()
    p32, f32, h32 = s32.surface()
    assert np.max(np.abs(p32[:, 0] - p64[:, 0])) <= 1e-5 * np.max(np.abs(p64[:, 0]))     # p_w
    assert np.max(np.abs(p32[:, 4] - p64[:, 4])) <= 1e-5 * np.max(np.abs(p64[:, 4]))     # q_w
    e = np.asarray(sphere.ref["U"]) / np.linalg.norm(sphere.ref["U"])
    assert abs(f32 @ e - f64 @ e) <= 1e-5 * abs(f64 @ e)                                 # drag
    assert abs(h32 - h64) <= 1e-5 * np.max(np.abs(p64[:, 4])) * np.sum(sphere.mesh.face_area[
        np.nonzero(sphere.mesh.face_cell[:, 1] == -1)[0]])
    # integrated loads: C_D, and C_L, C_m (near zero at zero incidence) on the C_D scale
    a32, a64 = s32.aero(), s64.aero()
    assert np.max(np.abs(a32[6:9] - a64[6:9])) <= 1e-5 * abs(a64[6])


def test_full_size_iterations_are_bitwise_repeatable(sphere):
    s = _solver(sphere, "mixed")
    s.iterate(25)
    W1, q1, _ = s.moments()
    s.set_state_prim(sphere.prim0)
    s.iterate(25)
    W2, q2, _ = s.moments()
    assert np.array_equal(W1, W2) and np.array_equal(q1, q2)


def test_cooperative_macro_solve_is_bitwise_identical_at_full_size(sphere, monkeypatch):
    """The cooperative macro PR-SGS (grid barriers between colour phases) gives the same
    iterates as the per-colour launches on the full sphere (mixed context with the FP64
    macro solve, the one that has a cooperative form)."""
    a = _solver(sphere, "mixed")
    a.iterate(15)
    Wa, qa, _ = a.moments()
    monkeypatch.setenv("RYKOV_COOP", "1")
    b = _solver(sphere, "mixed")
    b.iterate(15)
    Wb, qb, _ = b.moments()
    assert np.array_equal(Wa, Wb) and np.array_equal(qa, qb)


def test_macro_phase_launch_overlap_is_bitwise_identical_at_full_size(sphere, monkeypatch):
    """The FP32 macro phases launched with and without programmatic serialisation
    (RYKOV_PDL) give the same iterates on the full sphere."""
    out = []
    for flag in ("0", "1"):
        monkeypatch.setenv("RYKOV_PDL", flag)
        s = _solver(sphere, "mixed", macro32=True)
        s.iterate(15)
        out.append(s.moments()[:2])
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_staged_micro_sweeps_are_bitwise_identical_at_full_size(sphere, monkeypatch):
    """Staged and direct row loads in the micro sweeps give the same iterates on the
    full sphere (mixed precision, the bench configuration)."""
    out = []
    for flag in ("0", "7", "12"):
        monkeypatch.setenv("RYKOV_STAGED", flag)
        s = _solver(sphere, "mixed")
        s.iterate(15)
        out.append(s.moments()[:2])
        s.close()
    for W, q in out[1:]:
        assert np.array_equal(out[0][0], W) and np.array_equal(out[0][1], q)


def test_long_mixed_run_stays_finite(sphere):
    """300 mixed-precision iterations from the initial field (past the point where the
    distribution tails reach the FP32 subnormal range): the residual stays finite and
    falls below 1e-4."""
    s = _solver(sphere, "mixed")
    rc, n, res = s.iterate(300)
    assert rc == 0 and n == 300
    assert np.all(np.isfinite(res)) and np.max(res) < 1e-4


def test_sphere_mixed_converges_to_1e_6(sphere):
    """The bench workload reaches the residual 1e-6 in mixed precision from the initial
    field (about 100 iterations with the implicit CFL of 50)."""
    s = _solver(sphere, "mixed")
    rc, n, res = s.iterate(300, tol=1e-6)
    assert rc == 0 and np.max(res) < 1e-6 and n < 300


def test_macro_fp32_converges_like_the_fp64_macro_solve(sphere):
    """The FP32 delta-form macro solve of mixed contexts against the FP64 one, both from
    the initial field to the residual 1e-6: the same number of iterations within 3, and
    the converged wall pressure, heat flux and C_D within 1e-5 (relative to their
    largest values)."""
    out = []
    for m32 in (False, True):
        s = _solver(sphere, "mixed", macro32=m32)
        rc, n, res = s.iterate(300, tol=1e-6)
        assert rc == 0 and np.max(res) < 1e-6
        out.append((n, s.surface()[0], s.aero()))
        s.close()
    (n64, p64, a64), (n32, p32, a32) = out
    assert abs(n32 - n64) <= 3
    for c in (0, 4):                                 # p_w, q_w
        assert np.max(np.abs(p32[:, c] - p64[:, c])) <= 1e-5 * np.max(np.abs(p64[:, c]))
    assert abs(a32[6] - a64[6]) <= 1e-5 * abs(a64[6])


def test_mixed_adjoint_fp32_arithmetic_at_full_size(sphere, monkeypatch):
    """The adjoint of the mixed sphere with FP32 per-velocity arithmetic against the same
    context with FP64 arithmetic (RYKOV_ADJ_FP64=1): the heat objective to 1e-6, its
    gradient and dR/dp^T v to 1e-4; the VJP applied to that gradient to 1e-4 in the
    2-norm per block and 3e-3 in the max norm (single entries of the phi block carry
    FP32 cancellation: measured 1.8e-3)."""
    s = _solver(sphere, "mixed")
    s.iterate(150)
    s.bind_adjoint(1)
    monkeypatch.setenv("RYKOV_ADJ_FP64", "1")
    J64, g64, dp64 = s.objective("heat")
    out64, pp64 = s.vjp(g64)
    monkeypatch.delenv("RYKOV_ADJ_FP64")
    J32, g32, dp32 = s.objective("heat")
    out32, pp32 = s.vjp(g64)
    n1 = 2 * s.N * s.K
    assert abs(J32 - J64) <= 1e-6 * abs(J64)
    rel = lambda a, b: float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    rel2 = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    assert rel(g32, g64) < 1e-4 and rel(dp32, dp64) < 1e-4
    for a, b in ((out32[:n1], out64[:n1]), (out32[n1:], out64[n1:])):
        assert rel2(a, b) < 1e-4 and rel(a, b) < 3e-3
    assert rel(pp32, pp64) < 1e-4
