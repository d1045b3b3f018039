"""Thin Python binding of librykov (include/rykov.h).

Argument marshalling only: every step of the implicit iteration runs in the CUDA
kernels of librykov.so.  PyTorch supplies the device workspace (one uint8 CUDA
tensor) and the stream.  The module-level functions carry the C names; ``Solver``
bundles the usual call sequence.  There is no CPU fallback: importing works
anywhere, but creating a solver requires the compiled library and a CUDA device.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

RK_OK, RK_EINVAL, RK_ENOMEM, RK_ECUDA, RK_EDEVICE, RK_EDIVERGED, RK_ETIMEOUT, RK_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7
RK_FP64, RK_MIXED = 0, 1
RK_DEBUG = 0x100
RK_MACRO_FP32 = 0x200
RK_WALL, RK_FARFIELD = 0, 1
STEP_RECON, STEP_FACES, STEP_FLUXES, STEP_MACRO, STEP_MICRO = range(5)
BUF = dict(PHI=0, W=1, Q=2, FACE=4, FSTATE=6, MICRO_F=7, MACRO_F=8, WT=9, RES=10, DPHI=11,
           DT=12, S=13, TAUT=14)

# names of every exported entry point (checked by the ABI test)
EXPORTS = ["rk_version", "rk_create", "rk_destroy", "rk_last_error", "rk_upload_mesh",
           "rk_upload_dvs", "rk_set_params", "rk_set_bc", "rk_dims", "rk_workspace_size",
           "rk_bind_workspace", "rk_set_state_prim", "rk_set_state", "rk_get_distribution",
           "rk_implicit_iterate", "rk_residual", "rk_moments", "rk_surface", "rk_step",
           "rk_debug_get", "rk_profile", "rk_profile_get", "rk_residual_noalloc", "rk_aero",
           "rk_noalloc_last_error", "rk_state_len", "rk_adjoint_workspace_size",
           "rk_bind_adjoint_workspace", "rk_get_state", "rk_put_state", "rk_steady_residual",
           "rk_vjp", "rk_objective", "rk_adjoint_solve", "rk_adjoint_get", "rk_debug_rows",
           "rk_peak_flops"]
RK_OBJ_HEAT, RK_OBJ_DRAG = 0, 1
OBJECTIVES = {"heat": RK_OBJ_HEAT, "drag": RK_OBJ_DRAG}
PROF_CLASSES = ["recon", "face_interior", "face_boundary", "fluxes", "macro_sgs",
                "micro_sweep_first", "micro_sweep_mid", "micro_sweep_last", "update"]


class RkParams(C.Structure):
    _fields_ = [("R", C.c_double), ("Z_rot", C.c_double), ("omega_vis", C.c_double),
                ("mu_ref", C.c_double), ("T_ref", C.c_double), ("omega0", C.c_double),
                ("omega1", C.c_double), ("delta", C.c_double), ("cfl_s", C.c_double),
                ("cfl_imp", C.c_double), ("cfl_imp0", C.c_double), ("cfl_ramp", C.c_double),
                ("lim_k", C.c_double), ("n_micro_sgs", C.c_int32), ("n_macro_sgs", C.c_int32),
                ("limiter", C.c_int32), ("first_order_iters", C.c_int32),
                ("limiter_freeze", C.c_int32), ("viscosity_law", C.c_int32),
                ("sutherland_c", C.c_double)]


_lib = None


def load(path: str | None = None):
    """Load librykov.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.build()
    L = C.CDLL(path)
    vp, i64, i32, dp, sz = C.c_void_p, C.c_int64, C.c_int32, C.c_double, C.c_size_t
    P = C.POINTER
    sig = {
        "rk_version": ([], C.c_int),
        "rk_create": ([P(vp), C.c_int, C.c_size_t], C.c_int),
        "rk_destroy": ([vp], C.c_int),
        "rk_last_error": ([vp], C.c_char_p),
        "rk_upload_mesh": ([vp, i64, i64, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "rk_upload_dvs": ([vp, i64, vp, vp], C.c_int),
        "rk_set_params": ([vp, P(RkParams)], C.c_int),
        "rk_set_bc": ([vp, i32, i32, dp, vp, dp], C.c_int),
        "rk_dims": ([vp, vp], C.c_int),
        "rk_workspace_size": ([vp, P(sz)], C.c_int),
        "rk_bind_workspace": ([vp, vp, sz], C.c_int),
        "rk_set_state_prim": ([vp, vp, vp, C.c_int], C.c_int),
        "rk_set_state": ([vp, vp, vp, vp, C.c_int], C.c_int),
        "rk_get_distribution": ([vp, vp, C.c_int], C.c_int),
        "rk_implicit_iterate": ([vp, i32, dp, P(i32), vp], C.c_int),
        "rk_residual": ([vp, vp], C.c_int),
        "rk_moments": ([vp, vp, vp, vp, C.c_int], C.c_int),
        "rk_surface": ([vp, dp, vp, dp, vp, vp, vp], C.c_int),
        "rk_aero": ([vp, dp, vp, vp, dp, dp, vp, vp], C.c_int),
        "rk_step": ([vp, C.c_int], C.c_int),
        "rk_debug_get": ([vp, C.c_int, vp, i64], C.c_int),
        "rk_profile": ([vp, C.c_int], C.c_int),
        "rk_profile_get": ([vp, vp, vp], C.c_int),
        "rk_residual_noalloc": ([vp, vp, i64, vp, C.c_size_t], C.c_int),
        "rk_noalloc_last_error": ([], C.c_char_p),
        "rk_state_len": ([vp, P(i64)], C.c_int),
        "rk_adjoint_workspace_size": ([vp, i32, P(sz)], C.c_int),
        "rk_bind_adjoint_workspace": ([vp, i32, vp, sz], C.c_int),
        "rk_get_state": ([vp, vp, C.c_int], C.c_int),
        "rk_put_state": ([vp, vp, C.c_int], C.c_int),
        "rk_steady_residual": ([vp, vp, C.c_int], C.c_int),
        "rk_vjp": ([vp, vp, vp, vp, C.c_int], C.c_int),
        "rk_objective": ([vp, C.c_int, vp, vp, vp, C.c_int], C.c_int),
        "rk_adjoint_solve": ([vp, C.c_int, i32, dp, P(i32), vp, vp, vp], C.c_int),
        "rk_adjoint_get": ([vp, vp, C.c_int], C.c_int),
        "rk_debug_rows": ([vp, C.c_int, vp, i64, vp], C.c_int),
        "rk_peak_flops": ([C.c_int, C.c_size_t, vp, P(dp)], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


class RykovError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"librykov error {code}: {msg}")
        self.code = code


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def make_params(p) -> RkParams:
    d = p.as_dict() if hasattr(p, "as_dict") else dict(p)
    return RkParams(**{k: d[k] for k, _ in RkParams._fields_})


# ---- C names ------------------------------------------------------------------------
def rk_version():
    return load().rk_version()


def rk_create(precision: int, stream: int):
    h = C.c_void_p()
    rc = load().rk_create(C.byref(h), int(precision), int(stream))
    if rc:
        raise RykovError(rc, "rk_create failed")
    return h


def rk_residual_noalloc(W_new, W_old, n_cell: int, res_out, stream: int) -> int:
    """Residual of one step from two device states into a device output, without
    any device allocation (see include/rykov.h).  Arguments are CUDA tensors."""
    return load().rk_residual_noalloc(_ptr(W_new), _ptr(W_old), int(n_cell), _ptr(res_out),
                                      int(stream))


def peak_tflops(kind: str = "fp64", stream=None) -> float:
    """FMA throughput of the current device in TFLOP/s (rk_peak_flops), "fp64" or "fp32"."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = C.c_double()
    rc = load().rk_peak_flops(0 if kind == "fp64" else 1, st.cuda_stream, _ptr(sink), C.byref(out))
    if rc != RK_OK:
        raise RykovError(rc, "rk_peak_flops failed")
    return float(out.value)


class Solver:
    """One solver context on the current CUDA device and stream.

    wl: a workload (mesh, dvs, params, bcs, prim0) from ``inputs``;
    precision: "fp64" or "mixed"; macro32: mixed contexts solve the macro PR-SGS in
    FP32 delta form (RK_MACRO_FP32) instead of FP64."""

    def __init__(self, wl, precision: str = "fp64", stream=None, debug: bool = False,
                 params=None, macro32: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("librykov needs a CUDA device (no CPU path exists)")
        self.torch = torch
        self.L = load()
        self.wl = wl
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        prec = ((RK_FP64 if precision == "fp64" else RK_MIXED) | (RK_DEBUG if debug else 0)
                | (RK_MACRO_FP32 if macro32 else 0))
        self.h = rk_create(prec, self.stream.cuda_stream)
        m, d = wl.mesh, wl.dvs
        self._mesh = [_c(m.face_cell, np.int64), _c(m.face_normal, np.float64),
                      _c(m.face_area, np.float64), _c(m.face_center, np.float64),
                      _c(m.cell_center, np.float64), _c(m.cell_volume, np.float64),
                      _c(m.cell_colour, np.int32)]
        self._check(self.L.rk_upload_mesh(self.h, m.n_cell, m.n_face, *[_ptr(a) for a in self._mesh]))
        u, w = _c(d.u, np.float64), _c(d.w, np.float64)
        self._check(self.L.rk_upload_dvs(self.h, d.K, _ptr(u), _ptr(w)))
        self.set_params(params if params is not None else wl.params)
        for b, bc in enumerate(wl.bcs):
            U = _c(bc.U, np.float64)
            self._check(self.L.rk_set_bc(self.h, b, int(bc.kind), float(bc.rho), _ptr(U), float(bc.T)))
        dims = np.zeros(6, np.int64)
        self._check(self.L.rk_dims(self.h, _ptr(dims)))
        self.N, self.F, self.K, self.Kp, self.C, self.n_wall = (int(x) for x in dims)
        nbytes = C.c_size_t()
        self._check(self.L.rk_workspace_size(self.h, C.byref(nbytes)))
        self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device="cuda")
        self._check(self.L.rk_bind_workspace(self.h, _ptr(self.workspace), int(nbytes.value)))
        self.set_state_prim(wl.prim0)

    def _check(self, rc):
        if rc != RK_OK:
            msg = self.L.rk_last_error(self.h)
            raise RykovError(rc, msg.decode() if msg else "")
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.L.rk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        self._params = make_params(p)
        self._check(self.L.rk_set_params(self.h, C.byref(self._params)))

    def set_state_prim(self, prim, q=None):
        if hasattr(prim, "data_ptr"):
            self._check(self.L.rk_set_state_prim(self.h, _ptr(prim), _ptr(q), 1))
        else:
            pr = _c(prim, np.float64)
            qq = _c(q, np.float64) if q is not None else None
            self._check(self.L.rk_set_state_prim(self.h, _ptr(pr), _ptr(qq), 0))

    def iterate(self, n: int, tol: float = 0.0):
        done = C.c_int32(0)
        res = np.zeros(6)
        rc = self.L.rk_implicit_iterate(self.h, int(n), float(tol), C.byref(done), _ptr(res))
        if rc not in (RK_OK, RK_EDIVERGED):
            self._check(rc)
        return rc, int(done.value), res

    def step(self, which: int):
        self._check(self.L.rk_step(self.h, int(which)))

    def debug_get(self, name: str):
        shapes = dict(PHI=(2, self.N, self.K), RES=(2, self.N, self.K), DPHI=(2, self.N, self.K),
                      MICRO_F=(2, self.N, self.K), FACE=(2, self.F, self.K), W=(self.N, 6),
                      Q=(self.N, 6), MACRO_F=(self.N, 6), WT=(self.N, 6), FSTATE=(self.F, 16),
                      DT=(self.N, 3), S=(self.F,), TAUT=(self.N,))
        shp = shapes[name]
        out = np.empty(int(np.prod(shp)))
        self._check(self.L.rk_debug_get(self.h, BUF[name], _ptr(out), out.size))
        return out.reshape(shp)

    def debug_rows(self, name: str, rows):
        """rows of PHI / RES / DPHI / MICRO_F (cells) or FACE (faces): [2, n, K]."""
        rows = _c(rows, np.int64)
        out = np.empty((2, len(rows), self.K))
        self._check(self.L.rk_debug_rows(self.h, BUF[name], _ptr(rows), len(rows), _ptr(out)))
        return out

    def moments(self):
        W = np.empty((self.N, 6)); q = np.empty((self.N, 6)); T3 = np.empty((self.N, 3))
        self._check(self.L.rk_moments(self.h, _ptr(W), _ptr(q), _ptr(T3), 0))
        return W, q, T3

    def surface(self, rho_inf=None, U_inf=None, T_inf=None):
        ref = self.wl.ref
        rho_inf = ref["rho"] if rho_inf is None else rho_inf
        U = _c(ref["U"] if U_inf is None else U_inf, np.float64)
        T_inf = ref["T"] if T_inf is None else T_inf
        per = np.zeros((max(self.n_wall, 1), 8)); force = np.zeros(3); heat = np.zeros(1)
        self._check(self.L.rk_surface(self.h, float(rho_inf), _ptr(U), float(T_inf), _ptr(per),
                                      _ptr(force), _ptr(heat)))
        return per[:self.n_wall], force, float(heat[0])

    def aero(self, x_ref=(0.0, 0.0, 0.0), S_ref=1.0, L_ref=1.0, lift_dir=(0.0, 0.0, 1.0),
             rho_inf=None, U_inf=None):
        """[F(3), M(3), C_D, C_L, C_m, L/D] of the current state (rk_aero)."""
        ref = self.wl.ref
        rho_inf = ref["rho"] if rho_inf is None else rho_inf
        U = _c(ref["U"] if U_inf is None else U_inf, np.float64)
        x = _c(x_ref, np.float64)
        e = _c(lift_dir, np.float64)
        out = np.zeros(10)
        self._check(self.L.rk_aero(self.h, float(rho_inf), _ptr(U), _ptr(x), float(S_ref),
                                   float(L_ref), _ptr(e), _ptr(out)))
        return out

    def get_distribution(self):
        torch = self.torch
        dt = torch.float64 if self.precision == "fp64" else torch.float32
        out = torch.empty((2, self.N, self.Kp), dtype=dt, device="cuda")
        self._check(self.L.rk_get_distribution(self.h, _ptr(out), 1))
        return out

    def profile(self, enable: bool = True):
        self._check(self.L.rk_profile(self.h, int(bool(enable))))

    def profile_get(self):
        """Per kernel class: (summed device ms, launches) and the total launch count."""
        ms = np.zeros(len(PROF_CLASSES))
        cnt = np.zeros(len(PROF_CLASSES) + 1, np.int64)
        self._check(self.L.rk_profile_get(self.h, _ptr(ms), _ptr(cnt)))
        return ({n: (float(ms[i]), int(cnt[i])) for i, n in enumerate(PROF_CLASSES)},
                int(cnt[-1]))

    def residual(self):
        res = np.zeros(6)
        self._check(self.L.rk_residual(self.h, _ptr(res)))
        return res

    # ---- adjoint of the steady residual ---------------------------------------------
    def bind_adjoint(self, krylov_dim: int = 20):
        """Allocate (torch) and bind the adjoint workspace; krylov_dim = GMRES restart."""
        torch = self.torch
        nbytes = C.c_size_t()
        self._check(self.L.rk_adjoint_workspace_size(self.h, int(krylov_dim), C.byref(nbytes)))
        self.adj_workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device="cuda")
        self._check(self.L.rk_bind_adjoint_workspace(self.h, int(krylov_dim), _ptr(self.adj_workspace),
                                                     int(nbytes.value)))
        n = C.c_int64()
        self._check(self.L.rk_state_len(self.h, C.byref(n)))
        self.state_len = int(n.value)

    def _vec(self, x):
        """(pointer, on_device) of a packed state vector (numpy or CUDA tensor)."""
        if hasattr(x, "data_ptr"):
            return _ptr(x), 1
        return _ptr(x), 0

    def get_state(self):
        x = np.empty(self.state_len)
        self._check(self.L.rk_get_state(self.h, _ptr(x), 0))
        return x

    def put_state(self, x):
        x = x if hasattr(x, "data_ptr") else _c(x, np.float64)
        p, dev = self._vec(x)
        self._check(self.L.rk_put_state(self.h, p, dev))

    def steady_residual(self):
        r = np.empty(self.state_len)
        self._check(self.L.rk_steady_residual(self.h, _ptr(r), 0))
        return r

    def vjp(self, v):
        """(dR/dX)^T v and (dR/dp)^T v at the current state."""
        v = v if hasattr(v, "data_ptr") else _c(v, np.float64)
        out = np.empty(self.state_len) if not hasattr(v, "data_ptr") else self.torch.empty_like(v)
        pp = np.zeros(6)
        pv, dev = self._vec(v)
        self._check(self.L.rk_vjp(self.h, pv, _ptr(out), _ptr(pp), dev))
        return out, pp

    def objective(self, which="heat"):
        """J, dJ/dX (packed) and the explicit dJ/dp at the current state."""
        J = np.zeros(1); g = np.empty(self.state_len); dp = np.zeros(6)
        self._check(self.L.rk_objective(self.h, OBJECTIVES[which], _ptr(J), _ptr(g), _ptr(dp), 0))
        return float(J[0]), g, dp

    def adjoint_solve(self, which="heat", max_iter: int = 500, tol: float = 1e-10):
        """Adjoint solve at the current state: (iterations, relative residual, J, dJ/dp)."""
        it = C.c_int32(0); rr = np.zeros(1); J = np.zeros(1); dp = np.zeros(6)
        self._check(self.L.rk_adjoint_solve(self.h, OBJECTIVES[which], int(max_iter), float(tol),
                                            C.byref(it), _ptr(rr), _ptr(J), _ptr(dp)))
        return int(it.value), float(rr[0]), float(J[0]), dp

    def adjoint_get(self):
        lam = np.empty(self.state_len)
        self._check(self.L.rk_adjoint_get(self.h, _ptr(lam), 0))
        return lam

    def set_boundary_params(self, p):
        """Apply p = (T_w shift, rho_inf, U_inf[3], T_inf) to the boundary conditions of
        the workload (walls: T + p[0]; farfields: (p[1], p[2:5], p[5]))."""
        p = [float(x) for x in p]
        for b, bc in enumerate(self.wl.bcs):
            if bc.kind == RK_WALL:
                U = _c(bc.U, np.float64)
                self._check(self.L.rk_set_bc(self.h, b, RK_WALL, float(bc.rho), _ptr(U), float(bc.T) + p[0]))
            else:
                U = _c(p[2:5], np.float64)
                self._check(self.L.rk_set_bc(self.h, b, RK_FARFIELD, p[1], _ptr(U), p[5]))


def steady_objective(solver: Solver, p, which="heat", n_iter: int = 2000, tol: float = 1e-12,
                     adj_iter: int = 500, adj_tol: float = 1e-10):
    """J(X*(p)) of the converged steady state as a differentiable torch function of
    the boundary parameters p (6 doubles: T_w shift, rho_inf, U_inf, T_inf): forward =
    implicit iterations to convergence; backward = the adjoint solve (dJ/dp)."""
    import torch

    class _SteadyJ(torch.autograd.Function):
        @staticmethod
        def forward(ctx, pt):
            solver.set_boundary_params(pt.detach().cpu().numpy())
            rc, done, res = solver.iterate(n_iter, tol)
            if rc != RK_OK:
                raise RykovError(rc, "steady_objective: the iteration diverged")
            it, rel, J, dJdp = solver.adjoint_solve(which, adj_iter, adj_tol)
            ctx.save_for_backward(torch.as_tensor(dJdp, dtype=pt.dtype))
            return pt.new_tensor(J)

        @staticmethod
        def backward(ctx, gout):
            (dJdp,) = ctx.saved_tensors
            return gout * dJdp.to(gout.device)

    return _SteadyJ.apply(p)
