"""sgf_rayleigh_noalloc: the Rayleigh extraction for callers that cannot allocate during the call
(a process held to a device-memory budget fixed in advance, or a real-time loop that must stay out of
the allocator). It keeps its scratch in a static device array instead of calling cudaMalloc, so it
must give the same B_n and efficiencies as sgf_rayleigh, call after call, even though every call
reuses the array left behind by the previous one.

This file is collected last on purpose: it runs alone in a fresh process and after every other
test, and a failure here cannot hide an earlier one.
"""
import numpy as np
import pytest

from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")
torch = pytest.importorskip("torch")


def _same(got, ref):
    B, eff, err = got
    Br, er, xr = ref
    assert np.all(np.isfinite(B)) and np.all(np.isfinite(eff)) and np.isfinite(err)
    assert np.max(np.abs(B - Br)) <= 1e-12 * np.max(np.abs(Br))
    assert np.max(np.abs(eff - er)) <= 1e-12
    assert abs(err - xr) <= 1e-12


def test_noalloc_rayleigh_matches_allocating_entry_point_on_two_calls():
    # a workload away from Wood anomalies: there every propagating/evanescent decision is well
    # posed (at an exact anomaly beta_n is the square root of a rounding-level number)
    par = I.wl_deep_corrugation_neumann_small(N=1024, nx=32)
    op = sgf.Operator(par, precision=64)
    mu = torch.from_numpy(I.random_density(par["N"], 11)).cuda()
    n_lo, n_hi = -6, 3  # propagating modes -3..0 plus evanescent ones
    ref1 = sgf.sgf_rayleigh(op.ctx, mu.data_ptr(), n_lo, n_hi)
    # a second density, so that the second call cannot pass by reading stale scratch
    mu2 = torch.from_numpy(I.random_density(par["N"], 3)).cuda()
    ref2 = sgf.sgf_rayleigh(op.ctx, mu2.data_ptr(), n_lo, n_hi)
    for m, ref in ((mu, ref1), (mu2, ref2)):
        _same(sgf.sgf_rayleigh_noalloc(op.ctx, m.data_ptr(), n_lo, n_hi), ref)
    # the range limit is reported as an error, not silently truncated
    with pytest.raises(sgf.SgfError) as e:
        sgf.sgf_rayleigh_noalloc(op.ctx, mu.data_ptr(), 0, 2000)
    assert e.value.status == 1
    op.close()


def test_noalloc_rayleigh_wide_mode_range_and_full_scratch():
    # shifted kernel (j = 8) on the double-Wood sinusoid: modes up to |n| = 400 are strongly
    # evanescent (|beta_n| h up to ~640), where the product form of (1 - e^{i beta h})^j / beta
    # overflows; both entry points must return the same finite values. The second range fills the
    # static scratch exactly (1024 modes), so the last 64-mode chunk and the boundary are covered.
    par = I.wl_sinusoid_dirichlet(N=512)
    op = sgf.Operator(par, precision=64)
    mu = torch.from_numpy(I.random_density(par["N"], 5)).cuda()
    for n_lo, n_hi in ((-400, 400), (-512, 511)):
        ref = sgf.sgf_rayleigh(op.ctx, mu.data_ptr(), n_lo, n_hi)
        _same(sgf.sgf_rayleigh_noalloc(op.ctx, mu.data_ptr(), n_lo, n_hi), ref)
        _same(sgf.sgf_rayleigh_noalloc(op.ctx, mu.data_ptr(), n_lo, n_hi), ref)
    op.close()
