"""The allocation-free residual entry point (rk_residual_noalloc) against the
residual that rk_implicit_iterate reports, through the C ABI, on two implicit steps
in a row, and against a NumPy restatement of the residual definition at its size
limit and at a size that is not a multiple of its 256-cell blocks.  This file sorts
last so that a run stopping at the first failure has already run every other test."""
import os
import re

import numpy as np
import pytest

from tests import workloads as TW

pytestmark = pytest.mark.gpu

TOL = 1e-10          # the FP64 parity tolerance of the other GPU tests
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _limit():
    with open(os.path.join(ROOT, "include", "rykov.h")) as f:
        return int(re.search(r"#define RK_NOALLOC_MAX_CELLS (\d+)", f.read()).group(1))


def _residual(Wn, Wo):
    """The residual definition written out: sum |W_new - W_old| / sum |W_old| per
    component, the momentum rows over sum |rho U|."""
    num = np.abs(Wn - Wo).sum(axis=0)
    mom = np.sqrt((Wo[:, 1:4] ** 2).sum(axis=1)).sum()
    den = np.array([np.abs(Wo[:, 0]).sum(), mom, mom, mom, np.abs(Wo[:, 4]).sum(), np.abs(Wo[:, 5]).sum()])
    return num / den


def test_residual_noalloc_matches_iterate_residual_twice():
    import torch
    from paper_2303_10846_gb300.rykov import RK_OK, Solver, rk_residual_noalloc

    wl = TW.tiny_tet(lim=1, cfl_imp=20.0)
    s = Solver(wl, "fp64")
    stream = s.stream.cuda_stream
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        W_old = torch.from_numpy(s.moments()[0]).cuda()
        rc, n, res_ref = s.iterate(1)
        assert rc == RK_OK and n == 1
        W_new = torch.from_numpy(s.moments()[0]).cuda()
        torch.cuda.synchronize()
        assert rk_residual_noalloc(W_new, W_old, s.N, out, stream) == RK_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - res_ref) / np.abs(res_ref)) < TOL


@pytest.mark.parametrize("n", ["limit", 300001])
def test_residual_noalloc_many_blocks(n):
    """Seeded random states over many 256-cell blocks (all 4,096 at the size limit),
    two calls in a row on the shared scratch, against the residual written out."""
    import torch
    from paper_2303_10846_gb300.rykov import RK_OK, rk_residual_noalloc

    n = _limit() if n == "limit" else n
    rng = np.random.default_rng(n)
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    for rep in range(2):
        Wo = rng.uniform(0.5, 2.0, (n, 6))
        Wo[:, 1:4] = rng.normal(0.0, 1.0, (n, 3))
        Wn = Wo * (1.0 + rng.normal(0.0, 1e-3 * (rep + 1), (n, 6)))
        a, b = torch.from_numpy(Wn).cuda(), torch.from_numpy(Wo).cuda()
        torch.cuda.synchronize()
        assert rk_residual_noalloc(a, b, n, out, 0) == RK_OK
        torch.cuda.synchronize()
        ref = _residual(Wn, Wo)
        assert np.max(np.abs(out.cpu().numpy() - ref) / ref) < 1e-12


def test_residual_noalloc_rejects_bad_arguments():
    import torch
    from paper_2303_10846_gb300.rykov import RK_EINVAL, RK_OK, load, rk_residual_noalloc

    limit = _limit()
    W = torch.ones((limit, 6), dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    assert rk_residual_noalloc(W, W, limit + 1, out, 0) == RK_EINVAL
    assert b"exceeds" in load().rk_noalloc_last_error()
    assert rk_residual_noalloc(W, W, 0, out, 0) == RK_EINVAL
    assert rk_residual_noalloc(W, W, 4, None, 0) == RK_EINVAL
    assert rk_residual_noalloc(W, W, limit, out, 0) == RK_OK          # the limit itself
    torch.cuda.synchronize()
    assert load().rk_noalloc_last_error() == b""
    assert np.all(out.cpu().numpy() == 0.0)
