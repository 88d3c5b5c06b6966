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
