"""sgf_rayleigh_noalloc: the Rayleigh extraction for callers that cannot allocate during the call
(for example code running while a CUDA stream is captured into a graph, or a process held to a
device-memory budget fixed in advance). It keeps its scratch in a static device array instead of
calling cudaMalloc, so it must give the same B_n and efficiencies as sgf_rayleigh, call after call,
even though every call reuses the array left behind by the previous one.

This file is collected last on purpose: it runs alone in a fresh process and after every other
test, and a failure here cannot hide an earlier one.
"""
import numpy as np
import pytest

from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")
torch = pytest.importorskip("torch")


def test_noalloc_rayleigh_matches_allocating_entry_point_on_two_calls():
    # a workload away from Wood anomalies: there every propagating/evanescent decision is well
    # posed (at an exact anomaly beta_n is the square root of a rounding-level number)
    par = I.wl_deep_corrugation_neumann_small(N=1024, nx=32)
    op = sgf.Operator(par, precision=64)
    mu = torch.from_numpy(I.random_density(par["N"], 11)).cuda()
    n_lo, n_hi = -6, 3  # propagating modes -3..0 plus evanescent ones
    B_ref, eff_ref, err_ref = sgf.sgf_rayleigh(op.ctx, mu.data_ptr(), n_lo, n_hi)
    # a second density, so that the second call cannot pass by reading stale scratch
    mu2 = torch.from_numpy(I.random_density(par["N"], 3)).cuda()
    B2_ref, eff2_ref, err2_ref = sgf.sgf_rayleigh(op.ctx, mu2.data_ptr(), n_lo, n_hi)
    for m, (Br, er, xr) in ((mu, (B_ref, eff_ref, err_ref)), (mu2, (B2_ref, eff2_ref, err2_ref))):
        B, eff, err = sgf.sgf_rayleigh_noalloc(op.ctx, m.data_ptr(), n_lo, n_hi)
        assert np.max(np.abs(B - Br)) <= 1e-12 * np.max(np.abs(Br))
        assert np.max(np.abs(eff - er)) <= 1e-12
        assert abs(err - xr) <= 1e-12
    # the range limit is reported as an error, not silently truncated
    with pytest.raises(sgf.SgfError) as e:
        sgf.sgf_rayleigh_noalloc(op.ctx, mu.data_ptr(), 0, 2000)
    assert e.value.status == 1
    op.close()
