"""Pins of the accelerated-operator oracle (Section 5 of Bruno & Maas, Algorithms 2-3) against the
exact Nystrom operator, the equivalent-source validity statement (E1/E2 setting of Section 5.2-5.3)
and the Dirichlet-problem reconstruction inside a cell."""
import math

import numpy as np
import pytest

from oracle import accel as ac, direct as dr, green as gr
from paper_1707_04950_gb300 import inputs as I


def _relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# Accelerated vs exact operator (the accelerator's approximation error, not rounding): measured
# 9.0e-7 (Dirichlet, double Wood sinusoid, N = 128) and 5.4e-7 (Neumann, deep shape, N = 192); the
# pins hold them at 5e-6. A local set missing one cell row moves them to 2.7e-2 and 8.1e-3, and so
# does a dipole kernel of the wrong sign on one orientation (test_planted_mistakes_fail_the_pins).
ACCEL_VS_EXACT = 5e-6


def _dirichlet_case():
    par = I.wl_sinusoid_dirichlet(N=128)
    return par, I.random_density(128, 7)


def _neumann_case():
    par = I.wl_deep_corrugation_neumann_small(N=192, nx=24)
    return par, I.random_density(192, 11)


def test_accelerated_matches_exact_operator_dirichlet_wood():
    # the accelerated forward map approximates (1/2 I + D^dx) of the exact system
    par, mu = _dirichlet_case()
    y_exact = dr.assemble(par) @ mu
    y = ac.Accel(par).apply(mu)
    assert _relerr(y, y_exact) < ACCEL_VS_EXACT


def test_accelerated_matches_exact_operator_neumann_deep():
    par, mu = _neumann_case()
    y_exact = dr.assemble(par) @ mu
    y = ac.Accel(par).apply(mu)
    assert _relerr(y, y_exact) < ACCEL_VS_EXACT


def _drop_top_row(orig):
    def rows(self, cy_r):
        r = set(orig(self, cy_r))
        if r:
            r.discard(max(r))
        return r
    return rows


@pytest.mark.parametrize("case", ["dirichlet", "neumann"])
@pytest.mark.parametrize("mistake", ["local_set_row", "dipole_sign_V"])
def test_planted_mistakes_fail_the_pins(monkeypatch, case, mistake):
    # a plausible mistake planted in the oracle's Algorithm 2/3 must move the accelerated operator
    # far outside the accelerated-vs-exact pin
    par, mu = _dirichlet_case() if case == "dirichlet" else _neumann_case()
    y_exact = dr.assemble(par) @ mu
    if mistake == "local_set_row":
        monkeypatch.setattr(ac.Accel, "rows_of_Sj", _drop_top_row(ac.Accel.rows_of_Sj))
        acc = ac.Accel(par)
    else:
        # the V dipole kernel of the periodised table with the wrong sign (the least-squares fit
        # keeps the right one)
        orig_tables = ac.Accel._tables

        def tables(self):
            orig_tables(self)
            mono, dip, nr = self.tab["V"]
            self.tab["V"] = (mono, -dip, nr)
        monkeypatch.setattr(ac.Accel, "_tables", tables)
        acc = ac.Accel(par)
    assert _relerr(acc.apply(mu), y_exact) > 100 * ACCEL_VS_EXACT


def test_mode_and_singular_parts_are_the_exact_ones():
    # EvalSingular and EvalModes of Algorithm 3 are the exact operators of Section 4.3
    par = I.wl_sinusoid_dirichlet(N=128)
    mu = I.random_density(128, 3)
    A, parts = dr.assemble(par, return_parts=True)
    _, st = ac.Accel(par).apply(mu, return_stages=True)
    assert _relerr(st["sing"], parts["sing"] @ mu) < 1e-14
    assert _relerr(st["modes"], parts["modes"] @ mu) < 1e-14


def _square(ctr, side, n=160):
    t = np.linspace(0, 1, n, endpoint=False)
    h = side / 2
    return np.concatenate([
        np.stack([ctr[0] - h + 2 * h * t, ctr[1] - h + 0 * t], 1),
        np.stack([ctr[0] + h + 0 * t, ctr[1] - h + 2 * h * t], 1),
        np.stack([ctr[0] + h - 2 * h * t, ctr[1] + h + 0 * t], 1),
        np.stack([ctr[0] - h + 0 * t, ctr[1] + h - 2 * h * t], 1)])


@pytest.mark.parametrize("shifted", [False, True])
def test_equivalent_sources_valid_outside_validity_region(shifted):
    # k = 10, L = 0.3 (the setting of the paper's validity figures): a smooth curve of surface
    # sources in one cell; the monopole+dipole equivalent sources reproduce its field outside S_q
    # (and, with shifted Green functions, outside the shifted validity region S_j^q)
    prof = I.sinusoid(3.0, 0.03)
    par = I.make_params(prof, 10.0, 10.0, 0, 100, nx=10, ny=1, hmin=-0.15, j=2, h0=0.2)
    acc = ac.Accel(par)
    q = (4, 0)
    idx = np.array(acc.cell_nodes[q])
    mu = I.random_density(par["N"], 5)
    c0 = acc.corner(*q)
    psi_c = acc.true_field(acc.coll_rel + c0, idx) @ mu[idx]
    ctr = c0 + acc.L / 2
    k, j, h = acc.k, acc.j, acc.h
    for lam in ("H", "V"):
        dens = acc.pinv_eq[lam] @ psi_c
        ys = acc.src_rel[lam] + c0
        nu = acc.nu[lam]
        pts = _square(ctr, 4 * acc.L)
        if shifted:
            pts = pts[pts[:, 1] > ctr[1] - 1.5 * acc.L]   # above the shifted copies of S_q
        X = pts[:, 0][:, None] - ys[:, 0][None, :]
        Y = pts[:, 1][:, None] - ys[:, 1][None, :]
        if shifted:
            Gm = gr.Gj(k, j, h, X, Y)
            ax, ay = gr.gradGj(k, j, h, X, Y)
            Xl = pts[:, 0][:, None] - acc.x[idx][None, :]
            Yl = pts[:, 1][:, None] - acc.f[idx][None, :]
            bx, by = gr.gradGj(k, j, h, Xl, Yl)
            ref = ((acc.f1[idx][None, :] * bx - by) * acc.dx) @ mu[idx]
        else:
            Gm = gr.G0(k, X, Y)
            ax, ay = gr.gradG0(k, X, Y)
            ref = acc.true_field(pts, idx) @ mu[idx]
        phi = Gm @ dens[:acc.neq] + (-(nu[0] * ax + nu[1] * ay)) @ dens[acc.neq:]
        # the paper reports < 1e-12 for its (unprinted) layout; with p = 8, e = 1 and surface nodes
        # spanning the whole cell this layout reaches a few 1e-6
        assert np.max(np.abs(phi - ref)) < 1e-5 * np.max(np.abs(ref))


def test_cell_reconstruction_of_exterior_field():
    # the Dirichlet-problem reconstruction (eqs. planewave, plwave_QR) recovers, inside c^q, a
    # Helmholtz field radiated from outside S_q from its values on the cell-boundary samples
    par = I.wl_sinusoid_dirichlet(N=128)
    acc = ac.Accel(par)
    L, k = acc.L, acc.k
    src = np.array([[2.1 * L, 0.3 * L], [-1.2 * L, 1.9 * L], [0.5 * L, -1.6 * L]])
    amp = np.array([1.0, 0.7 - 0.2j, -0.4j])

    def field(P):
        return sum(a * gr.G0(k, P[:, 0] - s[0], P[:, 1] - s[1]) for a, s in zip(amp, src))

    ctr = np.array([L / 2, L / 2])
    w = acc.pinv_fb @ field(acc.samp_rel)
    rng = np.random.default_rng(1)
    inner = rng.uniform(0, L, (200, 2))
    got = acc.fb_basis(inner - ctr) @ w
    ref = field(inner)
    assert np.max(np.abs(got - ref)) < 2e-5 * np.max(np.abs(ref))


def test_dense_matrix_and_adjoint_match_the_forward_map():
    # matrix() applies Algorithm 3 to the identity; its columns must reproduce apply() on any
    # density, and the adjoint built from it satisfies <A x, y> = <x, A^H y> against apply()
    par = I.wl_sinusoid_dirichlet(N=128)
    acc = ac.Accel(par)
    A = acc.matrix()
    x = I.random_density(par["N"], 3)
    y = I.random_density(par["N"], 4)
    Ax = acc.apply(x)
    assert _relerr(A @ x, Ax) < 1e-11
    Ahy = acc.apply_adjoint(y, A)
    lhs = np.vdot(y, Ax)
    rhs = np.vdot(Ahy, x)
    assert abs(lhs - rhs) < 1e-11 * np.linalg.norm(Ax) * np.linalg.norm(y)
    # a block of columns runs column by column
    X = np.stack([x, y], 1)
    assert _relerr(acc.apply(X)[:, 1], acc.apply(y)) < 1e-11  # BLAS summation order only
