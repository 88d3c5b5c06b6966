"""The gradient of an efficiency with respect to the profile's Fourier coefficients (sgf_gradient):
against the oracle's derivative by definition (central differences of dense solves of the
accelerated operator and of the exact system), between precisions, and at full size as a
directional derivative of the GPU's own solves.

Tolerances: the oracle's difference quotient with eps = 1e-6 carries ~2e-6 (relative to the largest
component) of rounding noise, the GPU's node-local differences ~1e-7; we require 2e-5 of the largest
component. Against the exact system the accelerator's approximation (1e-4 level) decides: 2e-3.
"""
import numpy as np
import pytest

from oracle import gradient as og
from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")
torch = pytest.importorskip("torch")

COEFFS = [("a", 0), ("a", 1), ("b", 2), ("a", 3)]


def _solve(op, tol=1e-12):
    mu = torch.zeros(op.par["N"], dtype=torch.complex128, device="cuda")
    st, its, rr = sgf.sgf_solve(op.ctx, tol, 3000, mu.data_ptr())
    assert st == 0
    return mu


def _gpu_gradient(par, precision=64, n=0):
    op = sgf.Operator(par, precision=precision)
    mu = _solve(op)
    M = len(par["a"]) - 1
    ga, gb, Bn, en, its = sgf.sgf_gradient(op.ctx, mu.data_ptr(), n, M)
    _, eff, _ = sgf.sgf_rayleigh(op.ctx, mu.data_ptr(), n, n)
    op.close()
    return ga, gb, en, float(eff[0])


def _pick(ga, gb):
    return np.array([ga[m] if k == "a" else gb[m] for k, m in COEFFS])


@pytest.mark.parametrize("bc", [0, 1])
def test_gradient_matches_oracle_difference_quotients(bc):
    par = I.wl_harmonic_gradient_small(bc=bc)
    ga, gb, en, en_ray = _gpu_gradient(par)
    assert abs(en - en_ray) < 1e-12
    assert gb[0] == 0.0
    got = _pick(ga, gb)
    ref = og.efficiency_gradient_fd(par, 0, COEFFS, 1e-6, "accel")
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) < 2e-5 * scale, (got, ref)
    ex = og.efficiency_gradient_fd(par, 0, COEFFS, 1e-6, "exact")
    assert np.max(np.abs(got - ex)) < 2e-3 * scale
    # moving the whole surface up leaves e_0 of the exact system unchanged (a phase of B_0 only)
    assert abs(ex[0]) < 1e-6 * scale


def test_gradient_mixed_precision_matches_fp64():
    par = I.wl_harmonic_gradient_small()
    ga, gb, _, _ = _gpu_gradient(par, 64)
    ma, mb, _, _ = _gpu_gradient(par, 32)
    scale = max(np.max(np.abs(ga)), np.max(np.abs(gb)))
    assert max(np.max(np.abs(ma - ga)), np.max(np.abs(mb - gb))) < 1e-5 * scale


def test_gradient_full_size_directional_derivative():
    # the 128-coefficient workload (N = 4096): g . u against the difference quotient of e_0 along u
    par = I.wl_harmonic_gradient()
    ga, gb, en, _ = _gpu_gradient(par)
    assert np.all(np.isfinite(ga)) and np.all(np.isfinite(gb))
    rng = np.random.default_rng(5)
    ua, ub = rng.standard_normal(len(ga)), rng.standard_normal(len(gb))
    ub[0] = 0.0
    nrm = np.sqrt(np.sum(ua**2) + np.sum(ub**2))
    ua, ub = ua / nrm, ub / nrm
    eps = 1e-6
    vals = []
    for sg in (1.0, -1.0):
        p2 = dict(par, a=par["a"] + sg * eps * ua, b=par["b"] + sg * eps * ub)
        op = sgf.Operator(p2)
        mu = _solve(op)
        _, eff, _ = sgf.sgf_rayleigh(op.ctx, mu.data_ptr(), 0, 0)
        op.close()
        vals.append(float(eff[0]))
    fd = (vals[0] - vals[1]) / (2 * eps)
    dd = float(np.dot(ga, ua) + np.dot(gb, ub))
    assert abs(dd - fd) < 1e-4 * np.sqrt(np.sum(ga**2) + np.sum(gb**2)), (dd, fd)


def test_autograd_function_matches_gradient_and_difference_quotient():
    from paper_1707_04950_gb300.autograd import efficiency

    par = I.wl_harmonic_gradient_small()
    a = torch.tensor(par["a"], dtype=torch.float64, requires_grad=True)
    b = torch.tensor(par["b"], dtype=torch.float64, requires_grad=True)
    e = efficiency(a, b, par, 0)
    e.backward()
    ga, gb, en, _ = _gpu_gradient(par)
    assert abs(float(e) - en) < 1e-12
    assert np.max(np.abs(a.grad.numpy() - ga)) < 1e-7 * np.max(np.abs(ga))
    assert np.max(np.abs(b.grad.numpy() - gb)) < 1e-7 * np.max(np.abs(ga))
    # the forward map of the Function, differenced along a1
    eps = 1e-6
    da = torch.zeros_like(a)
    da[1] = eps
    with torch.no_grad():
        ep = efficiency(a + da, b, par, 0)
        em = efficiency(a - da, b, par, 0)
    fd = float(ep - em) / (2 * eps)
    assert abs(fd - ga[1]) < 2e-5 * np.max(np.abs(ga))


@pytest.mark.parametrize("bc", [0, 1])
def test_analytic_node_derivatives_match_difference_quotients(bc):
    # sgf_gradient (derivative factors built analytically) against sgf_gradient_fd (the same factors
    # rebuilt at moved node positions and differenced): the differences carry the rebuilt factors'
    # rounding divided by 2 eps (measured up to 2e-5 of the largest component; the analytic values are
    # the closer to the oracle's difference quotients of the dense solves), so 1e-4
    par = I.wl_harmonic_gradient_small(bc=bc)
    op = sgf.Operator(par)
    mu = _solve(op)
    M = len(par["a"]) - 1
    ga, gb, _, _, _ = sgf.sgf_gradient(op.ctx, mu.data_ptr(), 0, M)
    fa, fb, _, _, _ = sgf.sgf_gradient(op.ctx, mu.data_ptr(), 0, M, fd=True)
    op.close()
    scale = max(np.max(np.abs(fa)), np.max(np.abs(fb)))
    assert max(np.max(np.abs(ga - fa)), np.max(np.abs(gb - fb))) < 1e-4 * scale, (ga, fa, gb, fb)
