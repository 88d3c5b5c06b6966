"""Pins of the exact Nystrom oracle (Sections 2 and 4 of Bruno & Maas) against closed forms,
textbook perturbation theory, the energy-balance identity and independent quadrature."""
import math
import warnings

import numpy as np
import pytest
from scipy import integrate

from oracle import direct as dr, green as gr
from paper_1707_04950_gb300 import inputs as I


def test_log_quadrature_weights_against_adaptive_quadrature():
    # int_{-a}^{a} ln(4 sin^2(pi x/(2a))) phi(x) dx for a smooth phi vanishing at +-a with all
    # derivatives, versus adaptive quadrature that resolves the log singularity at 0
    # superalgebraic convergence: 48 -> 96 -> 192 nodes per period
    errs = []
    for M in (24, 48, 96):
        dx = 0.24 / M
        a = M * dx
        s, r = dr.kress_weights(M, dx)

        def phi(x):
            return gr.S_window(np.array([x]), 0.1 * a, a)[0] * math.cos(1.7 * x / a) * math.exp(0.4 * x / a)

        f = lambda x: math.log(4 * math.sin(math.pi * x / (2 * a)) ** 2) * phi(x)
        kw = dict(limit=400, epsabs=1e-15, epsrel=1e-14)
        with np.errstate(all="ignore"):
            ref = integrate.quad(f, -a, 0, **kw)[0] + integrate.quad(f, 0, a, **kw)[0]
        got = float(np.sum(r * np.array([phi(v) for v in s * dx])))
        errs.append(abs(got - ref) / abs(ref))
    assert errs[0] < 1e-8 and errs[1] < 1e-9 and errs[2] < 1e-12


def test_log_quadrature_exact_on_trigonometric_polynomials():
    # textbook: int_0^{2pi} ln(4 sin^2(t/2)) cos(m t) dt = -2 pi/m (m >= 1), 0 (m = 0); mapped to
    # period 2a this is -2a/m. The full 2M-point rule is exact up to degree M-1.
    M, dx = 16, 0.02
    a = M * dx
    s, r = dr.kress_weights(M, dx)
    # the excluded node s = M carries cos(pi m) times its weight; add it from the symmetric formula
    rM = -2 * dx * sum(math.cos(math.pi * m) / m for m in range(1, M)) - dx / M * (-1.0) ** M
    for m in range(0, M):
        got = float(np.sum(r * np.cos(math.pi * m * s / M))) + rM * math.cos(math.pi * m)
        ref = 0.0 if m == 0 else -2 * a / m
        assert abs(got - ref) < 1e-12


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("j", [0, 8])
def test_flat_surface_closed_form(bc, j):
    # f = 0: mu = c e^{i alpha x}; Dirichlet c = -1/[(1-e^{i beta h})^j/2 + d 1_{U^eta}(0)],
    # B_0 = -1; Neumann c = i beta/[-(1-e^{i beta h})^j/2 + i beta d 1_{U^eta}(0)], B_0 = +1
    par = I.flat(N=64, d=1.0, theta_deg=20.0, bc=bc, nx=8, j=j, n_per=80)
    A = dr.assemble(par)
    mu = np.linalg.solve(A, dr.rhs(par))
    al, be = dr.wave(par)
    x = dr.nodes(par)[0]
    _, Ue = dr.mode_sets(par)
    q = (1 - np.exp(1j * be * par["h"])) ** j
    ind = float(0 in Ue)
    c = -1 / (q / 2 + par["d"] * ind) if bc == 0 else 1j * be / (-q / 2 + 1j * be * par["d"] * ind)
    assert np.max(np.abs(mu - c * np.exp(1j * al * x))) < 1e-12 * abs(c)
    n, B, e, eps = dr.rayleigh(par, mu)
    B0 = B[list(n).index(0)]
    assert abs(B0 - (-1 if bc == 0 else 1)) < 1e-12
    assert abs(eps) < 1e-12


def test_small_amplitude_first_order_perturbation():
    # f = eps cos(2 pi x/d), Dirichlet: B_0 = -1 + O(eps^2), B_{+-1} = i beta eps + O(eps^2)
    # (the B_0 defect is a true second-order term: its ratio to eps^2 is the same at both eps)
    ratio = []
    for eps in (1e-3, 1e-4):
        prof = I.sinusoid(1.0, eps)
        par = I.make_params(prof, 2 * math.pi, 20.0, 0, 96, nx=8, ny=1, hmin=-1.0 / 16, j=0, n_per=400)
        mu = np.linalg.solve(dr.assemble(par), dr.rhs(par))
        n, B, _, _ = dr.rayleigh(par, mu, -1, 1)
        _, be = dr.wave(par)
        ratio.append(abs(B[1] + 1) / eps**2)
        for t in (0, 2):
            assert abs(B[t] - 1j * be * eps) < 0.2 * eps**2
    assert ratio[0] < 30 and abs(ratio[1] / ratio[0] - 1) < 1e-3


def test_kr_diagonal_is_the_limit_of_the_off_diagonal_kernel():
    # K_r(x, x') -> f''/(4 pi (1+f'^2)) + sum_m w_m (i k/4) H1(k m h) as x' -> x (Dirichlet)
    par = I.wl_sinusoid_dirichlet(N=128)
    k, j, h, a_s = par["k"], par["j"], par["h"], par["a_s"]
    x0 = 0.37
    f, f1, f2 = dr.profile(par, np.array([x0]))
    w = gr.binom_weights(j)
    diag = f2[0] / (4 * math.pi * (1 + f1[0] ** 2)) + sum(w[m] * 0.25j * k * gr.sp.hankel1(1, k * m * h) for m in range(1, j + 1))
    vals = []
    for t in (2e-3, 1e-3, 5e-4):
        xl = np.array([x0 - t])
        fl, f1l, _ = dr.profile(par, xl)
        X, Y = t, f[0] - fl[0]
        ax, ay = gr.gradGj(k, j, h, np.array([X]), np.array([Y]))
        kern = f1l[0] * ax[0] - ay[0]
        r = math.hypot(X, Y)
        ks = -k * gr.sp.j1(k * r) / r / (4 * math.pi) * (Y - f1l[0] * X)
        vals.append(kern - ks * math.log(4 * math.sin(math.pi * X / (2 * a_s)) ** 2))
    # Richardson: K_r is smooth, error O(t)
    lim = 2 * vals[2] - vals[1]
    assert abs(lim - diag) < 2e-5 * abs(diag) + 1e-6


def test_energy_balance_at_double_wood_anomaly_converges_with_window():
    # sinusoid at a double Wood anomaly (beta_1 = beta_-3 = 0): the energy error of the
    # perfectly conducting grating falls with the smooth-truncation length A (Lemma lemma_app_1)
    errs = []
    for n_per in (20, 80):
        par = I.wl_sinusoid_dirichlet(N=64, n_per=n_per)
        mu = np.linalg.solve(dr.assemble(par), dr.rhs(par))
        errs.append(abs(dr.rayleigh(par, mu)[3]))
    assert errs[1] < errs[0] / 50
    assert errs[1] < 2e-7


def test_shift_invariance_of_rayleigh_coefficients():
    # away from Wood, B_n does not depend on the shift order j or on h (only mu does)
    prof = I.sinusoid(1.0, 0.15)
    base = dict(nx=8, ny=4, hmin=-0.25)
    res = []
    for j, h0, nper in ((0, 0.5, 800), (8, 0.5, 120), (8, 0.4, 120)):
        par = I.make_params(prof, 2 * math.pi, 20.0, 0, 96, j=j, h0=h0, n_per=nper, **base)
        mu = np.linalg.solve(dr.assemble(par), dr.rhs(par))
        res.append(dr.rayleigh(par, mu, -1, 0)[1])
    assert np.max(np.abs(res[1] - res[0])) < 1e-7
    assert np.max(np.abs(res[2] - res[0])) < 1e-7
