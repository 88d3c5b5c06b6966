"""The cell-size autotuner (sgf_autotune_cells): it keeps the fastest candidate that builds,
reports the others, and leaves an operator that agrees with the oracle's Algorithm 3 built with
the parameters it chose (1e-10, the FP64 parity bound of the forward map)."""
import numpy as np
import pytest

from oracle import accel as ac
from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")


def test_autotune_keeps_fastest_built_candidate_and_matches_oracle():
    par = I.wl_sinusoid_dirichlet(N=512)
    op = sgf.Operator(par)
    cands = [8, 16, 24, 32, 64]  # 24 does not divide N = 512: rejected
    best, ms = sgf.sgf_autotune_cells(op.ctx, cands, reps=10)
    built = ms > 0
    assert not built[cands.index(24)]
    assert built.sum() >= 3
    assert best == cands[int(np.argmin(np.where(built, ms, np.inf)))]
    P = sgf.sgf_get_params(op.ctx)
    assert P.nx == best
    dx = par["d"] / par["N"]
    par2 = dict(par, nx=best, ny=P.ny, hmin=P.hmin, Ma=P.Ma, a_s=P.Ma * dx, gamma=0.5 * P.Ma * dx, h=P.h,
                L=par["d"] / best)
    mu = I.random_density(par["N"], 3)
    y = np.zeros_like(mu)
    sgf.sgf_apply_host(op.ctx, mu, y)
    op.close()
    ref = ac.Accel(par2).apply(mu)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-10


def test_autotune_deep_corrugation_builds_every_candidate_and_keeps_accuracy():
    # the N = 16384 benchmark workload (j = 0): 32, 64 and 128 cell columns all build (box, window
    # and grid re-derived per candidate; large cells tile the near-operator build). Timed alone, 64
    # columns are fastest but reach an energy error of 4.3e-8 only; the accuracy-aware tuner keeps
    # the fastest candidate below the configuration's target (1e-8), and its solve meets it.
    torch = pytest.importorskip("torch")
    par = I.wl_deep_corrugation_neumann()
    op = sgf.Operator(par, precision=32)
    cands = [32, 64, 128]
    best_t, ms_t = sgf.sgf_autotune_cells(op.ctx, cands, reps=20)
    assert np.all(ms_t > 0), ms_t
    st, best, ms, eps = sgf.sgf_autotune(op.ctx, cands, 1e-8, reps=20)
    assert st == 0 and np.all(ms > 0), (st, ms, eps)
    i = cands.index(best)
    assert abs(eps[i]) < 1e-8
    assert all(ms[i] <= ms[c] for c in range(len(cands)) if abs(eps[c]) < 1e-8)
    x = torch.zeros(par["N"], dtype=torch.complex128, device="cuda")
    st, its, rr = sgf.sgf_solve(op.ctx, 1e-12, 4000, x.data_ptr())
    _, _, e = sgf.sgf_rayleigh(op.ctx, x.data_ptr(), -40, 40)
    op.close()
    assert st == 0 and rr <= 1e-12, (best, st, its, rr)
    assert abs(e) < 1e-8, (best, e, ms, eps)
