"""Energy balance and convergence of the accelerated solves on the benchmark configurations
(eqs. energy_error, discrete_eq; Algorithm 1): the FP64 path and the mixed path (FP32 far field,
FP64 residual refinement) solve to a relative residual of 1e-10 or below, the two solutions agree,
and the energy error 1 - sum e_n of each is held at what the configuration reaches:

* deep corrugation (N = 16384, TM, j = 0, n_per = 2048): target 1e-8, measured 4.4e-9;
* double-Wood sinusoid (N = 512, j = 8, n_per = 640, tuned equivalent-source fit): target 1e-8,
  measured 2.9e-9 (the exact system 8e-11; neighbouring fit settings spread to 8e-8: the
  accelerator's approximation with 16 x 16 cells, k L = 0.79);
* Gaussian Wood surface (N = 8192, grazing 85 deg, j = 8, n_per = 1024): measured 3.9e-6 (exact
  system 4.7e-10), held at 2e-5; its FP64 GMRES stops at the attainable residual (~5e-11).
"""
import numpy as np
import pytest

from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")
torch = pytest.importorskip("torch")


def _solve(par, prec, tol=1e-12, maxit=4000):
    op = sgf.Operator(par, precision=prec)
    x = torch.zeros(par["N"], dtype=torch.complex128, device="cuda")
    try:
        st, its, rr = sgf.sgf_solve(op.ctx, tol, maxit, x.data_ptr())
    except sgf.SgfError as e:
        st, its, rr = e.status, -1, float("nan")
    _, _, eps = sgf.sgf_rayleigh(op.ctx, x.data_ptr(), -120, 120)
    op.close()
    return st, its, rr, eps, x


@pytest.mark.parametrize("name,make,eps_max,relres_max", [
    ("deep_corrugation", I.wl_deep_corrugation_neumann, 1e-8, 1e-12),
    ("double_wood_sinusoid", I.wl_sinusoid_dirichlet_energy, 1e-8, 1e-12),
    ("gaussian_wood", I.wl_gaussian_wood_energy, 2e-5, 1e-10),
])
def test_solves_reach_residual_and_energy_balance(name, make, eps_max, relres_max):
    par = make()
    sols = {}
    for prec in (64, 32):
        st, its, rr, eps, x = _solve(par, prec)
        assert rr <= relres_max, (prec, st, its, rr)
        assert abs(eps) < eps_max, (prec, eps)
        sols[prec] = x
    d = float(torch.linalg.norm(sols[32] - sols[64]) / torch.linalg.norm(sols[64]))
    assert d < 1e-6, d



@pytest.mark.parametrize("prec", [64, 32])
def test_solve_residual_with_ragged_krylov_tiles(prec):
    """GMRES with its float-float Arnoldi kernels on N = 1200 (ragged 256-element chunks and
    32-element tiles): the solution's residual b - A x, recomputed with a separate application of
    the FP64 operator, matches the reported relative residual and the 1e-12 target."""
    par = I.wl_sinusoid_dirichlet(N=1200)
    op = sgf.Operator(par, precision=prec)
    try:
        x = torch.zeros(par["N"], dtype=torch.complex128, device="cuda")
        st, its, rr = sgf.sgf_solve(op.ctx, 1e-12, 4000, x.data_ptr())
        assert st == 0 and rr <= 1e-12, (st, its, rr)
        b = torch.empty_like(x)
        sgf.sgf_rhs(op.ctx, b.data_ptr())
    finally:
        op.close()
    op64 = sgf.Operator(par, precision=64)
    try:
        ax = torch.empty_like(x)
        sgf.sgf_apply(op64.ctx, x.data_ptr(), ax.data_ptr())
    finally:
        op64.close()
    res = float(torch.linalg.norm(b - ax) / torch.linalg.norm(b))
    assert res < 2e-12, (res, rr)


@pytest.mark.parametrize("name,make", [
    ("deep_corrugation", I.wl_deep_corrugation_neumann),
    ("double_wood_sinusoid", I.wl_sinusoid_dirichlet_energy),
])
def test_recycled_refinement_matches_plain_refinement(monkeypatch, name, make):
    """The mixed path's later correction solves deflate with the Krylov space of the first one
    (GCRO form): the solution is the same to the solve tolerance as with plain refinement, and on
    the deep corrugation, whose GMRES spends most iterations finding a few slow components, it takes
    fewer applications."""
    par = make()
    monkeypatch.delenv("SGF_NO_RECYCLE", raising=False)
    st1, its1, rr1, eps1, x1 = _solve(par, 32)
    monkeypatch.setenv("SGF_NO_RECYCLE", "1")
    st2, its2, rr2, eps2, x2 = _solve(par, 32)
    assert st1 == st2 == 0, (st1, st2)
    assert rr1 <= 1e-12 and rr2 <= 1e-12, (rr1, rr2)
    d = float(torch.linalg.norm(x1 - x2) / torch.linalg.norm(x2))
    assert d < 1e-10, d
    assert abs(eps1 - eps2) < 1e-10, (eps1, eps2)
    if name == "deep_corrugation":
        assert its1 < 0.8 * its2, (its1, its2)
