"""The allocation-free residual entry point (rk_residual_noalloc) against the
residual that rk_implicit_iterate reports, through the C ABI, on two implicit steps
in a row.  This file sorts last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from tests import workloads as TW

pytestmark = pytest.mark.gpu

TOL = 1e-10          # the FP64 parity tolerance of the other GPU tests


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


def test_residual_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    from paper_2303_10846_gb300.rykov import RK_EINVAL, load, rk_residual_noalloc

    W = torch.zeros((4, 6), dtype=torch.float64, device="cuda")
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    limit = 1048576
    assert rk_residual_noalloc(W, W, limit + 1, out, 0) == RK_EINVAL
    assert b"exceeds" in load().rk_noalloc_last_error()
