"""The declared failure statuses, each produced on the host side of a call (no GPU fault, no
trap, no device wait): the call returns its status with a message, and the context stays usable.

* SGF_ERESONANT_CELL: a cell side L with (k L / pi)^2 = m^2 + n^2 (here 1 + 1), i.e. -k^2 a
  Dirichlet eigenvalue of the cell (Section 5.1, the non-resonance requirement on the cells);
* SGF_ENOCONV: GMRES (Algorithm 1) given maxit = 3 on a system that needs 13 applications;
* SGF_ENONFINITE: a right-hand side holding a NaN.
"""
import math

import numpy as np
import pytest

from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")
torch = pytest.importorskip("torch")


def test_resonant_cell_is_rejected():
    L = math.sqrt(2) / 2  # k L / pi = sqrt(2) at k = 2 pi
    par = I.flat(N=64, d=4 * L, nx=4, theta_deg=10.0)
    ctx = sgf.sgf_create(0)
    try:
        sgf.sgf_set_profile_fourier(ctx, par["d"], par["a"], par["b"])
        sgf.sgf_set_wave(ctx, par["k"], par["theta"], par["bc"])
        sgf.sgf_set_params(ctx, sgf.params_from(par))
        with pytest.raises(sgf.SgfError) as e:
            sgf.sgf_build_operator(ctx)
        assert e.value.status == 2 and "resonant" in str(e.value)
        # the same context builds once the cell is not resonant (half the side)
        sgf.sgf_set_params(ctx, sgf.params_from(I.flat(N=64, d=4 * L, nx=8, theta_deg=10.0)))
        sgf.sgf_build_operator(ctx)
    finally:
        sgf.sgf_destroy(ctx)


def test_gmres_out_of_iterations_reports_no_convergence():
    par = I.wl_sinusoid_dirichlet(N=256)
    op = sgf.Operator(par)
    x = torch.zeros(par["N"], dtype=torch.complex128, device="cuda")
    st, its, rr = sgf.sgf_solve(op.ctx, 1e-12, 3, x.data_ptr())
    assert st == 5 and its <= 4 and rr > 1e-12
    assert "relative residual" in sgf.load().sgf_last_error(op.ctx).decode()
    st, its, rr = sgf.sgf_solve(op.ctx, 1e-12, 2000, x.data_ptr())
    assert st == 0 and rr <= 1e-12
    op.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_non_finite_right_hand_side_is_reported(prec):
    par = I.wl_sinusoid_dirichlet(N=256)
    op = sgf.Operator(par, precision=prec)
    b = torch.from_numpy(I.random_density(par["N"], 3)).cuda()
    b[17] = complex(float("nan"), 0.0)
    x = torch.zeros_like(b)
    st, its, rr = sgf.sgf_solve_rhs(op.ctx, b.data_ptr(), 0, 1e-12, 100, x.data_ptr())
    assert st == 7
    assert "non-finite" in sgf.load().sgf_last_error(op.ctx).decode()
    b[17] = 0.1
    st, its, rr = sgf.sgf_solve_rhs(op.ctx, b.data_ptr(), 0, 1e-12, 2000, x.data_ptr())
    assert st == 0 and rr <= 1e-12
    op.close()
