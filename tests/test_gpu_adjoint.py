"""Parity of the adjoint map A^H (sgf_apply with transpose_conj = 1) and of the adjoint GMRES solve
(sgf_solve_rhs) with the oracle's conjugate-transposed accelerated matrix, per-term adjoint
identities <A x, y> = <x, A^H y> on the GPU at small and full size, and the mixed-precision adjoint
against the FP64 one.

Tolerances follow the forward map: the FP64 adjoint evaluates the same operator as the oracle in
another order. The least-squares factors built on each side (condition ~1e6 after the Tikhonov
term) differ at rounding times condition, which leaves the two operators ~1e-10 apart at the Wood
configuration in some directions (the forward map measures 7e-11 there); compared element by
element (largest difference over the largest reference element) we require 1e-9. The
mixed adjoint carries the FP32 far-field error (1e-5); an
identity between the GPU's own forward and adjoint maps holds to rounding (1e-12 FP64; the two
mixed maps round differently, 1e-6).
"""
import numpy as np
import pytest

from oracle import accel as ac
from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")
torch = pytest.importorskip("torch")

CASES = {
    "sinusoid_dirichlet_wood_n512": lambda: I.wl_sinusoid_dirichlet(N=512),
    "sinusoid_dirichlet_ragged_n400": lambda: I.wl_sinusoid_dirichlet(N=400),
    "deep_neumann_n1024": lambda: I.wl_deep_corrugation_neumann_small(N=1024, nx=32),
}

_mat = {}


def _matrix(name):
    """Dense accelerated operator of the oracle (Algorithm 3 applied to the identity)."""
    if name not in _mat:
        _mat[name] = ac.Accel(CASES[name]()).matrix()
    return _mat[name]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _maxrel(a, b):
    """Largest element-wise difference over the largest reference element."""
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _apply(op, x, adj, mask=None):
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()
    yt = torch.empty_like(xt)
    if mask is not None:
        sgf.sgf_debug_mask(op.ctx, mask)
    try:
        sgf.sgf_apply(op.ctx, xt.data_ptr(), yt.data_ptr(), 1, adj)
    finally:
        if mask is not None:
            sgf.sgf_debug_mask(op.ctx, 15)
    torch.cuda.synchronize()
    return yt.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_fp64_matches_oracle(name):
    par = CASES[name]()
    A = _matrix(name)
    v = I.random_density(par["N"], 9)
    op = sgf.Operator(par, precision=64)
    got = _apply(op, v, 1)
    op.close()
    assert _maxrel(got, A.conj().T @ v) < 1e-9  # element-wise; the forward map's tolerance


@pytest.mark.parametrize("name", ["sinusoid_dirichlet_wood_n512", "deep_neumann_n1024"])
@pytest.mark.parametrize("prec", [64, 32])
def test_adjoint_every_convolution_variant_matches_oracle(name, prec):
    # the adjoint Y convolution and X passes in every launch variant (forced; see the forward test)
    par = CASES[name]()
    ref = _matrix(name).conj().T @ I.random_density(par["N"], 9)
    v = I.random_density(par["N"], 9)
    op = sgf.Operator(par, precision=prec)
    errs = {}
    for c in (1, 2, 3):
        for vpt in (8, 16):
            sgf.sgf_debug_force_variants(op.ctx, c, vpt)
            errs[(c, vpt)] = _maxrel(_apply(op, v, 1), ref)
    op.close()
    assert max(errs.values()) < (1e-9 if prec == 64 else 5e-5), errs


@pytest.mark.parametrize("name", ["sinusoid_dirichlet_wood_n512", "deep_neumann_n1024"])
@pytest.mark.parametrize("mask", [1, 2, 4, 8, 15])
def test_adjoint_identity_per_term(name, mask):
    # each term of the forward map (far field, near field, modes, identity) against its own adjoint
    par = CASES[name]()
    x = I.random_density(par["N"], 3)
    y = I.random_density(par["N"], 4)
    op = sgf.Operator(par, precision=64)
    Ax = _apply(op, x, 0, mask)
    Ahy = _apply(op, y, 1, mask)
    op.close()
    if mask == 4 and not np.any(Ax):
        assert not np.any(Ahy)  # no completion modes in this configuration
        return
    lhs, rhs = np.vdot(y, Ax), np.vdot(Ahy, x)
    assert abs(lhs - rhs) < 1e-12 * np.linalg.norm(Ax) * np.linalg.norm(y)


def test_adjoint_mixed_matches_fp64():
    par = CASES["deep_neumann_n1024"]()
    v = I.random_density(par["N"], 5)
    o64 = sgf.Operator(par, precision=64)
    o32 = sgf.Operator(par, precision=32)
    a64, a32 = _apply(o64, v, 1), _apply(o32, v, 1)
    o64.close()
    o32.close()
    assert _rel(a32, a64) < 1e-5


@pytest.mark.parametrize("prec", [64, 32])
def test_adjoint_full_size_deep_corrugation(prec):
    # the N = 16384 Neumann workload: forward/adjoint identity of the GPU maps; mixed against FP64
    par = I.wl_deep_corrugation_neumann()
    x = I.random_density(par["N"], 7)
    y = I.random_density(par["N"], 8)
    op = sgf.Operator(par, precision=prec)
    Ax, Ahy = _apply(op, x, 0), _apply(op, y, 1)
    op.close()
    assert np.all(np.isfinite(Ahy))
    tol = 1e-12 if prec == 64 else 1e-6
    assert abs(np.vdot(y, Ax) - np.vdot(Ahy, x)) < tol * np.linalg.norm(Ax) * np.linalg.norm(y)
    if prec == 32:
        o64 = sgf.Operator(par, precision=64)
        a64 = _apply(o64, y, 1)
        o64.close()
        assert _rel(Ahy, a64) < 1e-5


@pytest.mark.parametrize("prec", [64, 32])
def test_adjoint_solve_matches_dense_solve(prec):
    name = "sinusoid_dirichlet_wood_n512"
    par = CASES[name]()
    A = _matrix(name)
    b = I.random_density(par["N"], 12)
    ref = np.linalg.solve(A.conj().T, b)
    op = sgf.Operator(par, precision=prec)
    bt = torch.from_numpy(b).cuda()
    xt = torch.empty_like(bt)
    st, its, rr = sgf.sgf_solve_rhs(op.ctx, bt.data_ptr(), 1, 1e-12, 2000, xt.data_ptr())
    op.close()
    assert st == 0 and rr <= 1e-12
    assert _rel(xt.cpu().numpy(), ref) < (1e-8 if prec == 64 else 1e-6)
    # the forward solve on the same right-hand side through the same entry point
    op = sgf.Operator(par, precision=64)
    st, its, rr = sgf.sgf_solve_rhs(op.ctx, bt.data_ptr(), 0, 1e-12, 2000, xt.data_ptr())
    op.close()
    assert st == 0
    assert _rel(xt.cpu().numpy(), np.linalg.solve(A, b)) < 1e-8
