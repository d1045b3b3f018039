"""Python access to the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: the oracle exists to check the CUDA library.  Only the
tests, the smoke check and the benchmark's CPU-baseline/reference legs may import
this package; the library itself never does.

The oracle is compiled with gcc on first use (``build()``); it shares no code with
the CUDA path.  Inputs come from ``paper_2303_10846_gb300.inputs`` (seeded
generators, no method arithmetic).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

BUF_PHI, BUF_W, BUF_Q, BUF_GRAD, BUF_FACE, BUF_FACE0, BUF_FSTATE, BUF_MICRO_F, \
    BUF_MACRO_F, BUF_WT, BUF_RES, BUF_DPHI, BUF_DT, BUF_S, BUF_TAUT, BUF_LSTORE = range(16)


class OrcParams(C.Structure):
    _fields_ = [("R", C.c_double), ("Z_rot", C.c_double), ("omega_vis", C.c_double),
                ("mu_ref", C.c_double), ("T_ref", C.c_double), ("omega0", C.c_double),
                ("omega1", C.c_double), ("delta", C.c_double), ("cfl_s", C.c_double),
                ("cfl_imp", C.c_double), ("cfl_imp0", C.c_double), ("cfl_ramp", C.c_double),
                ("lim_k", C.c_double),
                ("n_micro_sgs", C.c_int32), ("n_macro_sgs", C.c_int32),
                ("limiter", C.c_int32), ("first_order_iters", C.c_int32),
                ("limiter_freeze", C.c_int32), ("viscosity_law", C.c_int32),
                ("sutherland_c", C.c_double)]


class OrcState(C.Structure):
    _fields_ = [("rho", C.c_double), ("U", C.c_double * 3), ("T", C.c_double),
                ("Ttr", C.c_double), ("Trot", C.c_double), ("qtr", C.c_double * 3),
                ("qrot", C.c_double * 3)]


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    with _lock:
        if (not force and os.path.exists(_SO)
                and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
            return _SO
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", src, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        P = C.POINTER
        L.orc_create.restype = vp
        L.orc_create.argtypes = [P(OrcParams)]
        L.orc_destroy.argtypes = [vp]
        L.orc_set_mesh.argtypes = [vp, i64, i64, vp, vp, vp, vp, vp, vp, vp]
        L.orc_set_dvs.argtypes = [vp, i64, vp, vp]
        L.orc_set_bc.argtypes = [vp, i32, i32, dp, vp, dp]
        L.orc_set_params.argtypes = [vp, P(OrcParams)]
        L.orc_prepare.argtypes = [vp]
        L.orc_set_state_prim.argtypes = [vp, vp, vp]
        L.orc_set_state.argtypes = [vp, vp, vp, vp]
        L.orc_iterate.argtypes = [vp, i32, dp, P(i32), vp]
        for n in ("gradient", "faces", "fluxes", "macro", "micro"):
            getattr(L, f"orc_step_{n}").argtypes = [vp]
        L.orc_step_update.argtypes = [vp, vp]
        L.orc_micro_point.argtypes = [vp, i64, C.c_int, i32]
        L.orc_update_cell.argtypes = [vp, i64]
        L.orc_buffer_len.restype = i64
        L.orc_buffer_len.argtypes = [vp, C.c_int]
        L.orc_get.argtypes = [vp, C.c_int, vp]
        L.orc_put.argtypes = [vp, C.c_int, vp]
        L.orc_n_wall_faces.restype = i64
        L.orc_n_wall_faces.argtypes = [vp]
        L.orc_surface.argtypes = [vp, dp, vp, dp, vp, vp, vp]
        L.orc_aero.argtypes = [vp, dp, vp, vp, dp, dp, vp, vp]
        L.orc_equilibrium.argtypes = [P(OrcParams), P(OrcState), i64, vp, vp, vp]
        L.orc_equilibrium_parts.argtypes = [P(OrcParams), P(OrcState), i64, vp, vp, vp, vp, vp]
        L.orc_interface.argtypes = [P(OrcParams), i64, vp, vp, vp, vp, dp, vp, vp, vp]
        L.orc_euler_flux.argtypes = [P(OrcParams), vp, vp, vp]
        L.orc_spectral_radius.restype = dp
        L.orc_spectral_radius.argtypes = [P(OrcParams), vp, vp, dp]
        L.orc_venkat.restype = dp
        L.orc_venkat.argtypes = [dp, dp, dp]
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def make_params(p) -> OrcParams:
    d = p.as_dict() if hasattr(p, "as_dict") else dict(p)
    return OrcParams(**{k: d[k] for k, _ in OrcParams._fields_})


def make_state(rho, U, T, Ttr, Trot, qtr=(0, 0, 0), qrot=(0, 0, 0)) -> OrcState:
    s = OrcState()
    s.rho, s.T, s.Ttr, s.Trot = rho, T, Ttr, Trot
    for d in range(3):
        s.U[d], s.qtr[d], s.qrot[d] = U[d], qtr[d], qrot[d]
    return s


# ---------------------------------------------------------------------------------
# pure functions
# ---------------------------------------------------------------------------------
def equilibrium(params, state: OrcState, u):
    u = _c(u, np.float64); K = len(u)
    G = np.empty(K); H = np.empty(K)
    pp = make_params(params)
    lib().orc_equilibrium(C.byref(pp), C.byref(state), K, _ptr(u), _ptr(G), _ptr(H))
    return G, H


def equilibrium_parts(params, state: OrcState, u):
    u = _c(u, np.float64); K = len(u)
    out = [np.empty(K) for _ in range(4)]
    pp = make_params(params)
    lib().orc_equilibrium_parts(C.byref(pp), C.byref(state), K, _ptr(u), *[_ptr(o) for o in out])
    return out


def interface(params, u, w, g0, h0, s):
    u = _c(u, np.float64); w = _c(w, np.float64)
    g0 = _c(g0, np.float64); h0 = _c(h0, np.float64)
    K = len(w)
    st = np.empty(16); gf = np.empty(K); hf = np.empty(K)
    pp = make_params(params)
    lib().orc_interface(C.byref(pp), K, _ptr(u), _ptr(w), _ptr(g0), _ptr(h0), float(s),
                        _ptr(st), _ptr(gf), _ptr(hf))
    return st, gf, hf


def euler_flux(params, W, n):
    W = _c(W, np.float64); n = _c(n, np.float64); G = np.empty(6)
    pp = make_params(params)
    lib().orc_euler_flux(C.byref(pp), _ptr(W), _ptr(n), _ptr(G))
    return G


def spectral_radius(params, Wm, n, dl):
    Wm = _c(Wm, np.float64); n = _c(n, np.float64)
    pp = make_params(params)
    return lib().orc_spectral_radius(C.byref(pp), _ptr(Wm), _ptr(n), float(dl))


def venkat(d1, d2, eps2):
    return lib().orc_venkat(float(d1), float(d2), float(eps2))


# ---------------------------------------------------------------------------------
# solver context
# ---------------------------------------------------------------------------------
class Oracle:
    """FP64 CPU restatement of the implicit iteration on one workload."""

    def __init__(self, wl, params=None):
        L = lib()
        self.wl = wl
        self.params = params if params is not None else wl.params
        self._pp = make_params(self.params)
        self.h = L.orc_create(C.byref(self._pp))
        m, d = wl.mesh, wl.dvs
        self.N, self.F, self.K = m.n_cell, m.n_face, d.K
        self._keep = [_c(m.face_cell, np.int64), _c(m.face_normal, np.float64),
                      _c(m.face_area, np.float64), _c(m.face_center, np.float64),
                      _c(m.cell_center, np.float64), _c(m.cell_volume, np.float64),
                      _c(m.cell_colour, np.int32)]
        rc = L.orc_set_mesh(self.h, self.N, self.F, *[_ptr(a) for a in self._keep])
        if rc:
            raise RuntimeError(f"orc_set_mesh failed ({rc})")
        u, w = _c(d.u, np.float64), _c(d.w, np.float64)
        if L.orc_set_dvs(self.h, self.K, _ptr(u), _ptr(w)):
            raise RuntimeError("orc_set_dvs failed")
        for b, bc in enumerate(wl.bcs):
            U = _c(bc.U, np.float64)
            L.orc_set_bc(self.h, b, int(bc.kind), float(bc.rho), _ptr(U), float(bc.T))
        rc = L.orc_prepare(self.h)
        if rc:
            raise RuntimeError(f"orc_prepare failed ({rc})")
        self.set_state_prim(wl.prim0)

    def close(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state_prim(self, prim, q=None):
        prim = _c(prim, np.float64)
        qq = _c(q, np.float64) if q is not None else None
        rc = lib().orc_set_state_prim(self.h, _ptr(prim), _ptr(qq) if qq is not None else None)
        if rc:
            raise RuntimeError("orc_set_state_prim failed")

    def set_state(self, W, q=None, phi=None):
        W = _c(W, np.float64)
        qq = _c(q, np.float64) if q is not None else None
        ph = _c(phi, np.float64) if phi is not None else None
        lib().orc_set_state(self.h, _ptr(W), _ptr(qq) if qq is not None else None,
                            _ptr(ph) if ph is not None else None)

    def iterate(self, n: int, tol: float = 0.0):
        done = C.c_int32(0)
        res = np.zeros(6)
        rc = lib().orc_iterate(self.h, int(n), float(tol), C.byref(done), _ptr(res))
        return rc, int(done.value), res

    def step(self, name: str):
        L = lib()
        if name == "update":
            res = np.zeros(6)
            L.orc_step_update(self.h, _ptr(res))
            return res
        getattr(L, f"orc_step_{name}")(self.h)
        return None

    _SHAPES = {
        BUF_PHI: lambda s: (2, s.N, s.K), BUF_W: lambda s: (s.N, 6), BUF_Q: lambda s: (s.N, 6),
        BUF_GRAD: lambda s: (2, 3, s.N, s.K), BUF_FACE: lambda s: (2, s.F, s.K),
        BUF_FACE0: lambda s: (2, s.F, s.K), BUF_FSTATE: lambda s: (s.F, 16),
        BUF_MICRO_F: lambda s: (2, s.N, s.K), BUF_MACRO_F: lambda s: (s.N, 6),
        BUF_WT: lambda s: (s.N, 6), BUF_RES: lambda s: (2, s.N, s.K),
        BUF_DPHI: lambda s: (2, s.N, s.K), BUF_DT: lambda s: (s.N, 3), BUF_S: lambda s: (s.F,),
        BUF_TAUT: lambda s: (s.N,), BUF_LSTORE: lambda s: (2, s.N, s.K),
    }

    def micro_point(self, cell: int, first_forward: bool = False, colour: int = 0):
        """One point update of the micro PR-SGS for one cell (orc_micro_point)."""
        lib().orc_micro_point(self.h, int(cell), int(bool(first_forward)), int(colour))

    def update_cell(self, cell: int):
        """Step 6 (update and compensation) for one cell (orc_update_cell)."""
        lib().orc_update_cell(self.h, int(cell))

    def get(self, which: int) -> np.ndarray:
        n = lib().orc_buffer_len(self.h, which)
        out = np.empty(n)
        if lib().orc_get(self.h, which, _ptr(out)):
            raise RuntimeError("orc_get failed")
        return out.reshape(self._SHAPES[which](self))

    def put(self, which: int, arr):
        arr = _c(arr, np.float64).ravel()
        if lib().orc_put(self.h, which, _ptr(arr)):
            raise RuntimeError("orc_put failed")

    def surface(self, rho_inf=None, U_inf=None, T_inf=None):
        ref = self.wl.ref
        rho_inf = ref["rho"] if rho_inf is None else rho_inf
        U_inf = ref["U"] if U_inf is None else U_inf
        T_inf = ref["T"] if T_inf is None else T_inf
        nw = lib().orc_n_wall_faces(self.h)
        per = np.zeros((max(nw, 1), 8))
        force = np.zeros(3)
        heat = np.zeros(1)
        U = _c(U_inf, np.float64)
        lib().orc_surface(self.h, float(rho_inf), _ptr(U), float(T_inf), _ptr(per),
                          _ptr(force), _ptr(heat))
        return per[:nw], force, float(heat[0])

    def aero(self, x_ref=(0.0, 0.0, 0.0), S_ref=1.0, L_ref=1.0, lift_dir=(0.0, 0.0, 1.0),
             rho_inf=None, U_inf=None):
        """[F(3), M(3), C_D, C_L, C_m, L/D] of the current state (orc_aero)."""
        ref = self.wl.ref
        rho_inf = ref["rho"] if rho_inf is None else rho_inf
        U = _c(ref["U"] if U_inf is None else U_inf, np.float64)
        x = _c(x_ref, np.float64)
        e = _c(lift_dir, np.float64)
        out = np.zeros(10)
        rc = lib().orc_aero(self.h, float(rho_inf), _ptr(U), _ptr(x), float(S_ref), float(L_ref),
                            _ptr(e), _ptr(out))
        if rc:
            raise ValueError(f"orc_aero failed ({rc})")
        return out
