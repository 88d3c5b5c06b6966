"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same seeded inputs.

Tolerances: the FP64 path computes the same arithmetic as the oracle's Algorithm 3 in a different
order (FFT instead of direct convolution sums, folded spectral series, fused near operator). Outputs
are compared element by element, as the largest difference over the largest reference element. The
least-squares factors of the equivalent sources are built on each side (condition ~1e6 after the
Tikhonov term), so they differ at rounding x condition and single elements of the far field differ
by up to 3.6e-10 (deep Neumann case; 1e-11 to 1e-10 elsewhere): we require 1e-9 element-wise (a wrong
row or a wrapped column moves an element by 1e-3 or more). The mixed path runs the projection, FFT
convolution and interpolation in FP32 complex; we require 1e-5 per application and 1e-6 after FP64
refinement of a solve (element-wise: 5e-5 per application).
"""
import math

import numpy as np
import pytest

from oracle import accel as ac, direct as dr
from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _maxrel(a, b):
    """Largest element-wise difference over the largest reference element."""
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


FP64_ELEM = 1e-9  # element-wise FP64 parity (see the module docstring)


def _apply(op, mu, mask=None):
    if mask is not None:
        sgf.sgf_debug_mask(op.ctx, mask)
    y = np.zeros_like(mu)
    sgf.sgf_apply_host(op.ctx, np.ascontiguousarray(mu), y)
    if mask is not None:
        sgf.sgf_debug_mask(op.ctx, 15)
    return y


_cache = {}


def _oracle(name, par):
    if name not in _cache:
        _cache[name] = ac.Accel(par)
    return _cache[name]


def _far_oracle(acc, st):
    """sum_t I_q[i,t] phi^all(x_t): the interpolated global-convolution term alone."""
    out = np.zeros(acc.N, complex)
    ctr = np.array([acc.L / 2, acc.L / 2])
    for q in acc.cells:
        idx = np.array(acc.cell_nodes[q])
        phi = np.array([st["phi_all"][(q, t)] for t in range(len(acc.samp_ori))])
        rel = np.stack([acc.x[idx], acc.f[idx]], 1) - (acc.corner(*q) + ctr)
        if acc.bc == 0:
            Bn = acc.fb_basis(rel)
        else:
            nuh = np.stack([-acc.f1[idx], np.ones(len(idx))], 1) / acc.s[idx][:, None]
            Bn = acc.fb_basis(rel, nuh)
        out[idx] = Bn @ (acc.pinv_fb @ phi)
    return out


CASES = {
    "sinusoid_dirichlet_wood_n512": lambda: I.wl_sinusoid_dirichlet(N=512),
    "sinusoid_dirichlet_ragged_n400": lambda: I.wl_sinusoid_dirichlet(N=400),
    "deep_neumann_n1024": lambda: I.wl_deep_corrugation_neumann_small(N=1024, nx=32),
    # eta = 1e3 puts all five propagating modes (n = -3..1, two of them at the Wood anomaly) in the
    # completion set: more modes than the far-field kernel's four warps
    "sinusoid_dirichlet_five_modes_n512": lambda: I.wl_sinusoid_dirichlet(N=512, eta=1e3),
}


@pytest.mark.parametrize("name", ["sinusoid_dirichlet_wood_n512", "deep_neumann_n1024"])
def test_kernel_table_matches_oracle(name):
    par = CASES[name]()
    acc = _oracle(name, par)
    op = sgf.Operator(par)
    for lam, key in ((0, "H"), (1, "V")):
        mono, dip, nr = acc.tab[key]
        Px = mono.shape[0]
        Py = int(op.info["PyH" if lam == 0 else "PyV"])
        for kind, ref in ((0, mono), (1, dip)):
            got = sgf.sgf_debug_table(op.ctx, lam, kind, (Px, Py))
            iy = np.arange(-(nr - 1), nr) % Py
            g = got[:, iy]
            err = np.max(np.abs(g - ref)) / np.max(np.abs(ref))
            assert err < 1e-10, f"{key} kind {kind}: {err:.3e}"
    op.close()


@pytest.mark.parametrize("name", list(CASES))
def test_apply_fp64_matches_oracle(name):
    par = CASES[name]()
    acc = _oracle(name, par)
    mu = I.random_density(par["N"], 7)
    y_ref, st = acc.apply(mu, return_stages=True)
    op = sgf.Operator(par, precision=64)
    y = _apply(op, mu)
    # stage checks localise a failure: far field, near operator (+ singular), modes, identity
    far = _apply(op, mu, 1)
    near = _apply(op, mu, 2)
    modes = _apply(op, mu, 4)
    far_ref = _far_oracle(acc, st)
    near_ref = st["reg"] - far_ref + st["sing"]
    # element-wise stage errors on the scale of the largest output element (the near and mode terms
    # are small parts of it; at a Wood anomaly beta_n of the grazing mode is the square root of a
    # rounding-level number)
    scale = np.max(np.abs(y_ref))
    e_far, e_near, e_mod = (np.max(np.abs(far - far_ref)) / scale, np.max(np.abs(near - near_ref)) / scale,
                            np.max(np.abs(modes - st["modes"])) / scale)
    op.close()
    assert e_far < FP64_ELEM, f"far {e_far:.3e}"
    assert e_near < FP64_ELEM, f"near {e_near:.3e}"
    assert e_mod < FP64_ELEM, f"modes {e_mod:.3e}"
    assert _maxrel(y, y_ref) < FP64_ELEM


# Every launch variant of the grid convolution the full-size operator can take: the Y convolution
# with 16 values per thread in registers (1), the same with a global scratch for its partial
# product (2, taken by the FP64 V grid of the N = 16384 workload), 8 values per thread (3); the X
# passes with 8 or 16 values per thread (16 on the largest grids). Forced on the small cases.
VARIANTS = [(c, v) for c in (1, 2, 3) for v in (8, 16)]


@pytest.mark.parametrize("name", ["sinusoid_dirichlet_wood_n512", "deep_neumann_n1024"])
@pytest.mark.parametrize("prec", [64, 32])
def test_every_convolution_variant_matches_oracle(name, prec):
    par = CASES[name]()
    acc = _oracle(name, par)
    mu = I.random_density(par["N"], 7)
    y_ref = acc.apply(mu)
    op = sgf.Operator(par, precision=prec)
    errs = {}
    for c, v in VARIANTS:
        sgf.sgf_debug_force_variants(op.ctx, c, v)
        errs[(c, v)] = _maxrel(_apply(op, mu), y_ref)
    sgf.sgf_debug_force_variants(op.ctx, 0, 0)
    errs["auto"] = _maxrel(_apply(op, mu), y_ref)
    op.close()
    # mixed: the FP32 far field, element-wise 1.0e-5 to 1.5e-5 on the deep Neumann case for every
    # variant and for the per-launch choice alike
    tol = FP64_ELEM if prec == 64 else 5e-5
    assert max(errs.values()) < tol, errs


@pytest.mark.parametrize("name", ["sinusoid_dirichlet_wood_n512", "sinusoid_dirichlet_five_modes_n512"])
def test_apply_mixed_precision_matches_oracle(name):
    """Mixed forward map against the oracle, applied several times to the same density: every
    application matches (the first after the build as well as later ones), so no term reads
    storage that the application itself did not write."""
    par = CASES[name]()
    mu = I.random_density(par["N"], 8)
    y_ref = _oracle(name, par).apply(mu)
    op = sgf.Operator(par, precision=32)
    ys = [_apply(op, mu) for _ in range(4)]
    op.close()
    for y in ys:
        assert np.all(np.isfinite(y))
        assert _maxrel(y, y_ref) < 1e-5


def test_multiple_rhs_and_linearity():
    par = CASES["sinusoid_dirichlet_wood_n512"]()
    op = sgf.Operator(par, precision=64)
    m1, m2 = I.random_density(par["N"], 1), I.random_density(par["N"], 2)
    both = np.ascontiguousarray(np.concatenate([m1, m2]))
    out = np.zeros_like(both)
    sgf.sgf_apply_host(op.ctx, both, out, 2)
    y1, y2 = _apply(op, m1), _apply(op, m2)
    y12 = _apply(op, np.ascontiguousarray(2.0 * m1 - 1j * m2))
    op.close()
    # the scatter of equivalent sources sums duplicates with atomics: equal up to rounding order
    assert _rel(out[: par["N"]], y1) < 1e-14 and _rel(out[par["N"]:], y2) < 1e-14
    assert _rel(y12, 2.0 * y1 - 1j * y2) < 1e-13


def _solve(op, tol=1e-12, maxit=2000):
    torch = pytest.importorskip("torch")
    mu = torch.zeros(op.par["N"], dtype=torch.complex128, device="cuda")
    st, its, rr = sgf.sgf_solve(op.ctx, tol, maxit, mu.data_ptr())
    return st, its, rr, mu.cpu().numpy()


def test_flat_surface_solve_closed_form():
    for bc in (0, 1):
        par = I.flat(N=256, d=1.0, theta_deg=20.0, bc=bc, nx=8, n_per=80)
        op = sgf.Operator(par)
        st, its, rr, mu = _solve(op)
        assert st == 0 and rr < 1e-12
        al, be = dr.wave(par)
        x = dr.nodes(par)[0]
        q = (1 - np.exp(1j * be * par["h"])) ** par["j"]
        c = -1 / (q / 2) if bc == 0 else 1j * be / (-q / 2)
        # the closed form solves the exact system; the accelerated one (oracle: 4.2e-5 Dirichlet,
        # 5.1e-6 Neumann relative to |c|) differs by the accelerator's approximation
        assert np.max(np.abs(mu - c * np.exp(1j * al * x))) < 1e-4 * abs(c)
        torch = pytest.importorskip("torch")
        B, eff, eps = sgf.sgf_rayleigh(op.ctx, torch.from_numpy(mu).cuda().data_ptr(), 0, 0)
        assert abs(B[0] - (-1 if bc == 0 else 1)) < 1e-7
        op.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_solve_rayleigh_energy_against_oracle(prec):
    torch = pytest.importorskip("torch")
    par = I.wl_sinusoid_dirichlet(N=256)
    op = sgf.Operator(par, precision=prec)
    st, its, rr, mu = _solve(op)
    assert st == 0 and rr < 1e-12
    # Rayleigh kernel parity on the GPU solution
    U, _ = dr.mode_sets(par)
    B, eff, eps = sgf.sgf_rayleigh(op.ctx, torch.from_numpy(mu).cuda().data_ptr(), int(U.min()), int(U.max()))
    n, Bo, effo, epso = dr.rayleigh(par, mu)
    assert np.max(np.abs(B - Bo)) < 1e-12 * np.max(np.abs(Bo))
    # against the exact Nystrom solution: the accelerator error bounds the difference
    mu_ex = np.linalg.solve(dr.assemble(par), dr.rhs(par))
    _, Bex, _, eps_ex = dr.rayleigh(par, mu_ex)
    assert np.max(np.abs(B - Bex)) < 1e-4
    assert abs(eps) < 1e-4
    op.close()


def test_mixed_solve_matches_fp64_solve():
    par = I.wl_sinusoid_dirichlet(N=512)
    o64 = sgf.Operator(par, precision=64)
    o32 = sgf.Operator(par, precision=32)
    _, _, rr64, m64 = _solve(o64)
    _, its32, rr32, m32 = _solve(o32)
    o64.close()
    o32.close()
    assert rr32 < 1e-12
    assert _rel(m32, m64) < 1e-6


def test_error_codes():
    par = I.wl_sinusoid_dirichlet(N=512)
    ctx = sgf.sgf_create(0)
    try:
        with pytest.raises(sgf.SgfError) as e:
            sgf.sgf_build_operator(ctx)
        assert e.value.status == 10  # SGF_ESTATE: nothing set
        sgf.sgf_set_profile_fourier(ctx, par["d"], par["a"], par["b"])
        sgf.sgf_set_wave(ctx, par["k"], par["theta"], par["bc"])
        p = sgf.params_from(par)
        p.N = 500  # not a multiple of nx
        sgf.sgf_set_params(ctx, p)
        with pytest.raises(sgf.SgfError) as e:
            sgf.sgf_build_operator(ctx)
        assert e.value.status == 1
        p = sgf.params_from(par)
        p.Ma = 40  # singular window beyond the cell side
        sgf.sgf_set_params(ctx, p)
        with pytest.raises(sgf.SgfError) as e:
            sgf.sgf_build_operator(ctx)
        assert e.value.status == 4
        p = sgf.params_from(par)
        p.h = 0.5 * par["L"] / par["p"] * 66  # 2h on a grid lag
        sgf.sgf_set_params(ctx, p)
        with pytest.raises(sgf.SgfError) as e:
            sgf.sgf_build_operator(ctx)
        assert e.value.status in (3, 4)
        y = np.zeros(par["N"], complex)
        with pytest.raises(sgf.SgfError) as e:
            sgf.sgf_apply_host(ctx, y.copy(), y)
        assert e.value.status == 10
    finally:
        sgf.sgf_destroy(ctx)


@pytest.mark.parametrize("prec", [64, 32])
def test_full_size_deep_corrugation_sampled_rows(prec):
    # the headline workload (N = 16384, 128 x 257 cells, Neumann): sampled rows against the exact
    # operator (the accelerator's approximation error bounds the difference) and the two precisions
    # against each other
    par = I.wl_deep_corrugation_neumann()
    mu = I.random_density(par["N"], 7)
    op = sgf.Operator(par, precision=prec)
    y = _apply(op, mu)
    op.close()
    assert np.all(np.isfinite(y))
    rows = np.array([3, 4100, 8191, 12000])
    yr = dr.apply_rows(par, mu, rows)
    scale = np.max(np.abs(yr))
    # the accelerator's approximation (j = 0, n_per = 2048, ls_reg = 1e-8): measured 3.7e-8 (FP64)
    # and 1.0e-6 (mixed, FP32 far field) element-wise
    assert np.max(np.abs(y[rows] - yr)) < (1e-7 if prec == 64 else 3e-6) * scale
    if prec == 32:
        o64 = sgf.Operator(par, precision=64)
        y64 = _apply(o64, mu)
        o64.close()
        assert _rel(y, y64) < 1e-5


def test_full_size_gaussian_wood_sampled_rows():
    # the rough-surface Wood workload (N = 8192, period 40, theta = 85 deg, k at the n = -80 Wood
    # anomaly): sampled rows against the exact operator (measured 1e-6, the accelerator's
    # approximation; bound 1e-5) and the mixed path against the FP64 path
    par = I.wl_gaussian_wood()
    mu = I.random_density(par["N"], 7)
    o64 = sgf.Operator(par, precision=64)
    y = _apply(o64, mu)
    o64.close()
    rows = np.array([5, 2000, 4100, 7000])
    yr = dr.apply_rows(par, mu, rows)
    assert np.max(np.abs(y[rows] - yr)) < 1e-5 * np.max(np.abs(yr))
    o32 = sgf.Operator(par, precision=32)
    y32 = _apply(o32, mu)
    o32.close()
    assert _rel(y32, y) < 1e-5
