"""Green functions of the shifted quasi-periodic method (Sections 2-3 of Bruno & Maas).

Conventions: lags X = x - x', Y = y - y'. G(X,Y) = (i/4) H0^(1)(k r) (eq. free_space).
Shifted G_j = sum_{m=0..j} (-1)^m C(j,m) G(X, Y + m h) (eq. shifted_green_function).
Lattice sum with phase e^{-i alpha p d} (eq. shifted_periodic_green_function; the printed classical
lattice sum carries the opposite phase sign, a slip: the spectral form fixes e^{-i alpha p d}).
Windowed lattice sums multiply the window after differentiation (the window of the truncated
operator acts on the already differentiated kernel, eq. DAdx_def).
"""
from __future__ import annotations

import math
import numpy as np
from scipy import special as sp


def binom_weights(j):
    """w_m = (-1)^m C(j,m), m = 0..j."""
    return np.array([(-1) ** m * math.comb(j, m) for m in range(j + 1)], dtype=float)


# ------------------------------------------------------------------ free space (eq. free_space)

def G0(k, X, Y):
    r = np.hypot(X, Y)
    return 0.25j * sp.hankel1(0, k * r)


def gradG0(k, X, Y):
    """(dG/dX, dG/dY) = (i/4)(-k H1(kr)) (X, Y)/r."""
    r = np.hypot(X, Y)
    c = -0.25j * k * sp.hankel1(1, k * r) / r
    return c * X, c * Y


def Gj(k, j, h, X, Y, skip_m0=False):
    w = binom_weights(j)
    out = 0j * np.asarray(X, float)
    for m in range(0 if not skip_m0 else 1, j + 1):
        out = out + w[m] * G0(k, X, Y + m * h)
    return out


def gradGj(k, j, h, X, Y, skip_m0=False):
    w = binom_weights(j)
    gx = 0j * np.asarray(X, float)
    gy = 0j * np.asarray(X, float)
    for m in range(0 if not skip_m0 else 1, j + 1):
        ax, ay = gradG0(k, X, Y + m * h)
        gx = gx + w[m] * ax
        gy = gy + w[m] * ay
    return gx, gy


# ------------------------------------------------------------------ windows (eq. S_def)

def S_window(x, gamma, a):
    """S_{gamma,a}(x): 1 on |x|<=gamma, exp(2 e^{-1/u}/(u-1)) with u=(|x|-gamma)/(a-gamma), 0 beyond a."""
    x = np.abs(np.asarray(x, float))
    out = np.zeros_like(x)
    out[x <= gamma] = 1.0
    mid = (x > gamma) & (x < a)
    u = (x[mid] - gamma) / (a - gamma)
    out[mid] = np.exp(2.0 * np.exp(-1.0 / u) / (u - 1.0))
    return out


# ------------------------------------------------------------------ Rayleigh wavenumbers (eq. alpha_beta_def)

def alpha_n(k, theta, d, n):
    return k * math.sin(theta) + 2 * math.pi * np.asarray(n, float) / d


def beta_n(k, alpha, d, n):
    """beta_n = sqrt(k^2 - alpha_n^2) (positive) for propagating n, i sqrt(alpha_n^2 - k^2) otherwise."""
    an = alpha + 2 * math.pi * np.asarray(n, float) / d
    q = k * k - an * an
    return np.where(q >= 0, np.sqrt(np.abs(q)) + 0j, 1j * np.sqrt(np.abs(q)))


def csinc(z):
    """sin(z)/z for complex z (series below |z| < 1e-3)."""
    z = np.asarray(z, complex)
    out = np.empty_like(z)
    small = np.abs(z) < 1e-3
    zs = z[small]
    out[small] = 1 - zs * zs / 6 + zs**4 / 120
    zl = z[~small]
    out[~small] = np.sin(zl) / zl
    return out


def Qj(beta, h, j):
    """(1 - e^{i beta h})^j / beta. Where |beta h| < 1 it is written as
    (-2i)^j e^{i j beta h/2} sin^{j-1}(beta h/2) (h/2) sinc(beta h/2), so that the beta -> 0 limit
    (Wood anomaly) is evaluated exactly (Section 3.2, eq. betan_taylor); elsewhere the quotient itself
    is well conditioned, while the factors of the rewrite overflow for strongly evanescent modes."""
    beta = np.asarray(beta, complex)
    if j == 0:
        return 1.0 / beta
    out = np.empty(beta.shape, complex)
    small = np.abs(beta * h) < 1.0
    half = beta[small] * h / 2
    out[small] = (-2j) ** j * np.exp(1j * j * half) * np.sin(half) ** (j - 1) * (h / 2) * csinc(half)
    b = beta[~small]
    out[~small] = (1.0 - np.exp(1j * b * h)) ** j / b
    return out


# ------------------------------------------------------------------ shifted spectral series (Sec. 3.2)

def spectral_range(k, alpha, d, delta, spec_exp):
    """Integer range [n_lo, n_hi] outside which |e^{i beta_n delta}| < e^{-spec_exp}."""
    T = math.sqrt(k * k + (spec_exp / delta) ** 2)
    n_hi = int(math.ceil((T - alpha) * d / (2 * math.pi)))
    n_lo = int(math.floor((-T - alpha) * d / (2 * math.pi)))
    return n_lo, n_hi


def spectral_coeffs(k, alpha, d, j, h, Y, n):
    """c_n(Y) of G~ = sum_n c_n e^{i alpha_n X} (eq. shifted_quasi_per_rayleigh) and the Y-derivative
    coefficients cy_n(Y) = -1/(2d) sum_m w_m sgn(Y+mh) e^{i beta_n |Y+mh|}.
    Y: (P,) array; n: (T,) integer array. Returns arrays (P, T).
    Near beta_n = 0 the m-sum is rewritten per eq. betan_taylor (exact rewrite, used where
    |beta_n| (|Y| + j h) < 1 so that no growing exponential is multiplied by a cancelling sum)."""
    Y = np.asarray(Y, float)[:, None]
    beta = beta_n(k, alpha, d, n)[None, :]
    w = binom_weights(j)
    S0 = 0j * (Y + beta.real)
    S1 = 0j * (Y + beta.real)
    for m in range(j + 1):
        t = Y + m * h
        em = np.exp(1j * beta * np.abs(t))
        S0 = S0 + w[m] * em
        S1 = S1 + w[m] * np.sign(t) * em
    with np.errstate(divide="ignore", invalid="ignore"):
        c = 1j / (2 * d * beta) * S0
    cy = -S1 / (2 * d)
    if j >= 1:
        safe = np.abs(beta) * (np.abs(Y) + j * h) < 1.0
        if np.any(safe):
            bb = np.broadcast_to(beta, safe.shape)[safe]
            YY = np.broadcast_to(Y, safe.shape)[safe]
            acc = np.exp(1j * bb * YY) * Qj(bb, h, j)
            for m in range(j + 1):
                t = YY + m * h
                neg = t < 0
                if np.any(neg):
                    acc = acc - np.where(neg, 2j * w[m] * t * csinc(bb * t), 0)
            c[safe] = 1j / (2 * d) * acc
    return c, cy


def gtilde_spectral(k, alpha, d, j, h, X, Y, spec_exp=40.0, delta=None):
    """G~_j^qper and its gradient by the shifted spectral series, at points (X, Y)."""
    X = np.atleast_1d(np.asarray(X, float))
    Y = np.atleast_1d(np.asarray(Y, float))
    if delta is None:
        delta = float(np.min(np.abs(Y[:, None] + h * np.arange(j + 1)[None, :])))
    n_lo, n_hi = spectral_range(k, alpha, d, delta, spec_exp)
    n = np.arange(n_lo, n_hi + 1)
    c, cy = spectral_coeffs(k, alpha, d, j, h, Y, n)
    an = alpha + 2 * math.pi * n / d
    ex = np.exp(1j * X[:, None] * an[None, :])
    g = np.sum(c * ex, axis=1)
    gx = np.sum(1j * an[None, :] * c * ex, axis=1)
    gy = np.sum(cy * ex, axis=1)
    return g, gx, gy


def gtilde_spatial_centered(k, alpha, d, j, h, X, Y, A, c_win, puncture=None):
    """Windowed lattice sum sum_p e^{-i alpha p d} S_{cA,A}(X+pd) G_j(X+pd, Y) and its gradient
    (eq. Gq_limit with the window applied after differentiation), for X in [-d/2, d/2).
    puncture: boolean mask of points whose (p=0, m=0) term is dropped (the self term of the
    punctured Green functions at coincident points, eq. phi_def / phi_jq_def)."""
    X = np.atleast_1d(np.asarray(X, float))
    Y = np.atleast_1d(np.asarray(Y, float))
    P = int(math.ceil(A / d)) + 1
    w = binom_weights(j)
    g = np.zeros(X.shape, complex)
    gx = np.zeros(X.shape, complex)
    gy = np.zeros(X.shape, complex)
    for p in range(-P, P + 1):
        Xp = X + p * d
        sw = S_window(Xp, c_win * A, A)
        if not np.any(sw > 0):
            continue
        ph = np.exp(-1j * alpha * p * d)
        for m in range(j + 1):
            Ym = Y + m * h
            if p == 0 and m == 0 and puncture is not None and np.any(puncture):
                ok = ~puncture
                val = np.zeros(X.shape, complex)
                vx = np.zeros(X.shape, complex)
                vy = np.zeros(X.shape, complex)
                val[ok] = G0(k, Xp[ok], Ym[ok])
                vx[ok], vy[ok] = gradG0(k, Xp[ok], Ym[ok])
            else:
                val = G0(k, Xp, Ym)
                vx, vy = gradG0(k, Xp, Ym)
            fac = ph * sw * w[m]
            g += fac * val
            gx += fac * vx
            gy += fac * vy
    return g, gx, gy


def reduce_x(X, d):
    """X = X' + q d with X' in [-d/2, d/2)."""
    q = np.floor((np.asarray(X, float) + d / 2) / d)
    return X - q * d, q


def gtilde_hybrid(par, X, Y, puncture=None):
    """Hybrid spatial/spectral evaluation of G~_j^qper and its gradient (Sections 3.2, 4.2.3):
    spectral series where delta = min_m |Y + m h| >= delta_min, windowed spatial sum otherwise.
    The spatial branch reduces X to [-d/2, d/2) and applies the quasi-periodic phase e^{i alpha q d}."""
    k, d, j, h = par["k"], par["d"], par["j"], par["h"]
    alpha = k * math.sin(par["theta"])
    A = par["n_per"] * d
    X = np.atleast_1d(np.asarray(X, float))
    Y = np.atleast_1d(np.asarray(Y, float))
    delta = np.min(np.abs(Y[:, None] + h * np.arange(j + 1)[None, :]), axis=1)
    spec = delta >= par["delta_min"]
    g = np.zeros(X.shape, complex)
    gx = np.zeros(X.shape, complex)
    gy = np.zeros(X.shape, complex)
    if np.any(spec):
        idx = np.nonzero(spec)[0]
        # chunk by delta so that each chunk's term range is set by its smallest delta
        order = idx[np.argsort(delta[idx])]
        for s in range(0, len(order), 2048):
            ch = order[s:s + 2048]
            a, b, c = gtilde_spectral(k, alpha, d, j, h, X[ch], Y[ch], par["spec_exp"], float(delta[ch].min()))
            g[ch], gx[ch], gy[ch] = a, b, c
    if np.any(~spec):
        idx = np.nonzero(~spec)[0]
        Xr, q = reduce_x(X[idx], d)
        pun = None if puncture is None else np.asarray(puncture)[idx]
        for s in range(0, len(idx), 4096):
            sl = slice(s, s + 4096)
            a, b, c = gtilde_spatial_centered(k, alpha, d, j, h, Xr[sl], Y[idx][sl], A, par["c_win"],
                                              None if pun is None else pun[sl])
            ph = np.exp(1j * alpha * q[sl] * d)
            g[idx[sl]], gx[idx[sl]], gy[idx[sl]] = ph * a, ph * b, ph * c
    return g, gx, gy
