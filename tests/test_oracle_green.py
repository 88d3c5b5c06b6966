"""Pins of the oracle's Green-function layer against closed forms, identities and independent sums.

Sections 2-3 of Bruno & Maas: free-space G (eq. free_space), classical spectral G^qper
(eq. quasi_per_rayleigh), shifted G_j (eq. shifted_green_function), lattice and spectral forms of
G~_j^qper (eqs. shifted_periodic_green_function, shifted_quasi_per_rayleigh,
shifted_periodic_green_function_spectral), the Wood-safe rewrite (eq. betan_taylor), window S.
"""
import math

import mpmath
import numpy as np
import pytest

from oracle import green as gr

K = 2 * math.pi
D = 2.0
TH = math.radians(20.0)
AL = K * math.sin(TH)
H = 0.5017361111111112


def test_hankel_against_mpmath():
    # scipy's H0/H1 (used by the oracle) against arbitrary-precision Bessel functions
    for z in (1e-3, 0.37, 1.0, 4.2, 17.5, 63.0):
        for n in (0, 1):
            ref = complex(mpmath.besselj(n, z) + 1j * mpmath.bessely(n, z))
            got = complex(gr.sp.hankel1(n, z))
            assert abs(got - ref) <= 1e-13 * abs(ref)


def test_free_space_gradient_by_finite_differences():
    X, Y, e = 0.31, -0.22, 1e-6
    gx, gy = gr.gradG0(K, np.array([X]), np.array([Y]))
    fx = (gr.G0(K, X + e, Y) - gr.G0(K, X - e, Y)) / (2 * e)
    fy = (gr.G0(K, X, Y + e) - gr.G0(K, X, Y - e)) / (2 * e)
    assert abs(gx[0] - fx) < 1e-8 and abs(gy[0] - fy) < 1e-8


def _pts():
    X = np.array([0.3, -0.7, 0.9, 0.05])
    Y = np.array([0.2, -0.3, 0.45, -1.3])
    return X, Y


@pytest.mark.parametrize("j,nper,tol", [(0, 1500, 1e-9), (1, 400, 1e-10), (8, 200, 1e-11)])
def test_spectral_equals_windowed_spatial_sum(j, nper, tol):
    # two independent representations of the same lattice sum agree where both converge
    # (the unshifted sum decays like |X|^{-1/2}, so its smooth truncation needs a longer window)
    X, Y = _pts()
    if j == 0:
        Y = np.abs(Y) + 0.1
    a = gr.gtilde_spectral(K, AL, D, j, H, X, Y, 40.0)
    b = gr.gtilde_spatial_centered(K, AL, D, j, H, X, Y, nper * D, 0.5)
    for u, v in zip(a, b):
        assert np.max(np.abs(u - v) / np.abs(u)) < tol


def test_shifted_equals_combination_of_classical_rayleigh():
    # away from Wood: G~_j(X,Y) = sum_m w_m G^qper(X, Y + m h), with G^qper summed here directly
    X, Y = _pts()
    j = 8
    w = gr.binom_weights(j)
    n = np.arange(-400, 401)
    an = AL + 2 * math.pi * n / D
    bn = np.where(K * K - an * an >= 0, np.sqrt(np.abs(K * K - an * an)) + 0j, 1j * np.sqrt(np.abs(an * an - K * K)))
    ref = np.zeros(len(X), complex)
    for m in range(j + 1):
        t = Y + m * H
        ref += w[m] * np.sum(1j / (2 * D * bn[None, :]) * np.exp(1j * an[None, :] * X[:, None] + 1j * bn[None, :] * np.abs(t)[:, None]), axis=1)
    g, _, _ = gr.gtilde_spectral(K, AL, D, j, H, X, Y, 40.0)
    assert np.max(np.abs(g - ref) / np.abs(ref)) < 1e-12


def test_quasi_periodicity_and_y_symmetry():
    X, Y = _pts()
    g1, _, _ = gr.gtilde_spectral(K, AL, D, 8, H, X + D, Y, 40.0)
    g0, _, _ = gr.gtilde_spectral(K, AL, D, 8, H, X, Y, 40.0)
    assert np.max(np.abs(g1 - np.exp(1j * AL * D) * g0)) < 1e-13 * np.max(np.abs(g0))
    Yp = np.abs(Y) + 0.05
    a, _, _ = gr.gtilde_spectral(K, AL, D, 0, H, X, Yp, 40.0)
    b, _, _ = gr.gtilde_spectral(K, AL, D, 0, H, X, -Yp, 40.0)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(a))


def test_binomial_identity_and_closed_form_above():
    # sum_m w_m e^{i beta (Y + m h)} = e^{i beta Y}(1 - e^{i beta h})^j  ->  for Y > 0 the spectral
    # coefficients equal i/(2 d beta)(1 - e^{i beta h})^j e^{i beta Y}
    j = 8
    n = np.arange(-30, 31)
    Y = np.array([0.4, 1.3])
    c, cy = gr.spectral_coeffs(K, AL, D, j, H, Y, n)
    bn = gr.beta_n(K, AL, D, n)
    ref = 1j / (2 * D * bn[None, :]) * (1 - np.exp(1j * bn * H))[None, :] ** j * np.exp(1j * bn[None, :] * Y[:, None])
    assert np.max(np.abs(c - ref) / np.abs(ref)) < 1e-12
    refy = -(1 - np.exp(1j * bn * H))[None, :] ** j * np.exp(1j * bn[None, :] * Y[:, None]) / (2 * D)
    assert np.max(np.abs(cy - refy) / np.abs(refy)) < 1e-12


def test_Qj_matches_definition_and_limit():
    b = np.array([0.7, 2.3, 1e-2, 0.9j, 3j])
    for j in (1, 2, 8):
        ref = (1 - np.exp(1j * b * H)) ** j / b
        assert np.max(np.abs(gr.Qj(b, H, j) - ref) / np.abs(ref)) < 1e-10
    # limit beta -> 0: (−i beta h)^j / beta -> 0 for j >= 2, -i h for j = 1
    assert abs(gr.Qj(np.array([0j]), H, 8)[0]) == 0.0
    assert abs(gr.Qj(np.array([0j]), H, 1)[0] - (-1j * H)) < 1e-15


def test_wood_safe_rewrite_agrees_with_direct_form():
    # eq. betan_taylor is an exact rewrite: compare against the direct m-sum at small but
    # non-zero beta, computed in extended precision
    j = 8
    Y = -1.37  # between shifted poles
    for kk in (AL + 2 * math.pi / D * 1 + 1e-3, AL + 2 * math.pi / D * 1 - 1e-3):
        n = np.array([-1])
        c, _ = gr.spectral_coeffs(kk, AL, D, j, H, np.array([Y]), n)
        an = mpmath.mpf(AL) - 2 * mpmath.pi / D
        q = mpmath.mpf(kk) ** 2 - an**2
        bn = mpmath.sqrt(q) if q > 0 else 1j * mpmath.sqrt(-q)
        s = sum((-1) ** m * math.comb(j, m) * mpmath.exp(1j * bn * abs(Y + m * H)) for m in range(j + 1))
        ref = complex(1j / (2 * D * bn) * s)
        assert abs(c[0, 0] - ref) < 1e-11 * abs(ref)


def test_wood_behaviour_classical_diverges_shifted_finite():
    # at alpha_1 -> k the classical coefficient 1/beta_1 blows up; the j = 8 one stays bounded
    X, Y = np.array([0.3]), np.array([0.4])
    vals0, vals8 = [], []
    for eps in (1e-3, 1e-5, 1e-7):
        kk = abs(AL + 2 * math.pi / D) + eps
        vals0.append(abs(gr.gtilde_spectral(kk, AL, D, 0, H, X, Y, 40.0)[0][0]))
        vals8.append(abs(gr.gtilde_spectral(kk, AL, D, 8, H, X, Y, 40.0)[0][0]))
    assert vals0[2] > 10 * vals0[0]
    assert max(vals8) / min(vals8) < 1.01


def test_window_properties():
    g, a = 0.3, 0.7
    x = np.linspace(-1, 1, 2001)
    s = gr.S_window(x, g, a)
    assert np.all(s[np.abs(x) <= g] == 1.0) and np.all(s[np.abs(x) >= a] == 0.0)
    assert np.all(np.diff(s[x >= 0]) <= 1e-15)
    # all derivatives vanish at the ends: S ~ exp(-c/(a-|x|)) decays faster than any power
    assert gr.S_window(np.array([a - 1e-3]), g, a)[0] < 1e-100
    assert 1 - gr.S_window(np.array([g + 1e-3]), g, a)[0] < 1e-100


def test_hybrid_switch_is_continuous_across_delta_min():
    # the hybrid evaluation must agree on both sides of the spectral/spatial switch
    par = {"k": K, "d": D, "j": 8, "h": H, "theta": TH, "n_per": 200, "c_win": 0.5,
           "delta_min": D / 64, "spec_exp": 40.0}
    X = np.array([0.4, 0.4])
    Y = np.array([-H + D / 64 * 1.001, -H + D / 64 * 0.999])
    g, _, _ = gr.gtilde_hybrid(par, X, Y)
    assert abs(g[0] - g[1]) < 1e-3 * abs(g[0])
    a = gr.gtilde_spectral(K, AL, D, 8, H, X[1:], Y[1:], 40.0)[0][0]
    assert abs(a - g[1]) < 1e-10 * abs(a)
