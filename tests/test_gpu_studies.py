"""Angle-of-attack sweeps and DVS-criterion studies through the library (GPU), checked
against the FP64 oracle driven through the same boundary changes."""
import dataclasses
import math

import numpy as np
import pytest

import oracle as O
from paper_2303_10846_gb300 import inputs as I
from paper_2303_10846_gb300 import studies as S
from tests import workloads as TW

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def _tet():
    return TW.tiny_tet(lim=1, first_order_iters=1, cfl_imp=20.0)


def test_aoa_sweep_matches_oracle_fp64():
    """Two angles (5 and 15 degrees in the x-z plane), five iterations each from the
    turned initial field: the GPU's loads equal the oracle's on the same turned
    workloads (freestream, initial field and velocity space turned together)."""
    wl = _tet()
    kw = dict(x_ref=(0.1, 0.0, -0.05), S_ref=0.8, L_ref=1.2)
    recs = S.aoa_sweep(wl, (5.0, 15.0), precision="fp64", n_iter=5, tol=0.0, **kw)
    U0 = np.asarray(wl.ref["U"], float)
    for r, a in zip(recs, (5.0, 15.0)):
        wa = S.turned_workload(wl, a)
        U, el = S.freestream_at(U0, a)
        assert np.allclose(wa.ref["U"], U)
        o = O.Oracle(wa)
        o.iterate(5)
        ref = o.aero(lift_dir=el, U_inf=U, **kw)
        assert r["iterations"] == 5
        got = np.array(r["force"] + r["moment"] + [r["C_D"], r["C_L"], r["C_m"]])
        exp = ref[:9]
        assert np.max(np.abs(got[:3] - exp[:3])) < TOL64 * np.max(np.abs(exp[:3]))
        assert np.max(np.abs(got[3:6] - exp[3:6])) < TOL64 * np.max(np.abs(exp[3:6]))
        assert np.max(np.abs(got[6:9] - exp[6:9])) < TOL64 * np.max(np.abs(exp[6:9]))
    assert abs(recs[1]["C_L"] - recs[0]["C_L"]) > 1e-3 * abs(recs[0]["C_D"])


def test_dvs_study_runs_variants():
    """Two variants of the DVS criterion (outer radius 3 and 4 sqrt(R T0), no refined
    balls) on the small sphere mesh: each runs its iterations with finite loads, and
    the residual has fallen well below its start."""
    base = _tet()

    def make(radius_factor):
        wl = _tet()
        U = wl.ref["U"]
        dvs = I.unstructured_dvs(U, 1.0, 1.2, U[0] / math.sqrt(1.4 * I.R_GAS), True, target=300,
                                 radius_factor=radius_factor, refine=False)
        return dataclasses.replace(wl, dvs=dvs)

    recs = S.dvs_study(make, [dict(radius_factor=3.0), dict(radius_factor=4.0)], precision="fp64",
                       n_iter=150, tol=1e-9)
    assert recs[0]["K"] != base.dvs.K and recs[1]["K"] > 0
    for r in recs:
        assert 0 < r["iterations"] <= 150 and r["residual"] < 1e-4
        assert np.isfinite(r["C_D"]) and np.isfinite(r["heat"]) and r["C_D"] > 0
