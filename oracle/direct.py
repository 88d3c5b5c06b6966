"""The exact (unaccelerated) Nystrom system of Bruno & Maas, Section 4, and Rayleigh extraction.

(sigma/2 I + D^dx) mu = rhs,  D^dx = D~_sing + D~_reg + D_M   (eqs. D_deltax, discrete_eq)

Dirichlet (TE, the paper's case): double layer, sigma = +1, rhs = -u^inc, per-node weight dx with
the unnormalised source normal nu_l = (-f'_l, 1) (equivalently unit normal times ds_l).
Neumann (TM, "treated analogously" in the paper, derived here): single layer with target normal
derivative, sigma = -1, rhs = -d u^inc/d nu_hat, kernel nu_hat_i . grad_X G_j, weight s_l dx.

D~_sing  eq. local_mat with the Martensen-Kussmaul split (eqs. descomp-kr_def): K_s is the exact
         coefficient of ln r^2 in the m = 0 term; the log argument is read as pi(x-x')/(2a) (window
         support 2a) and R_il are the trigonometric log-quadrature weights for period 2a
         (R. Kress, Linear Integral Equations, trigonometric interpolatory quadrature);
         W_il = dx (trapezoid).
D~_reg   eqs. D_ns / G_jq_s: kernel dG~/dnu - sum_{p=-1..1} e^{-i alpha p d} S^f_p dG_j/dnu(X+pd, Y),
         S^f the distance-based window; G~ by the hybrid evaluation.
D_M      eq. D_M_deltax with the phases restored: sum_{n in U^eta} e^{i alpha_n x_i + i beta_n f_i}
         sum_l e^{-i alpha_n x_l - i beta_n f_l} mu_l ds_l.
U^eta    eq. M_eta, restricted to |beta_n| <= k (modes the shifts can cancel: propagating, grazing,
         weakly evanescent; far-evanescent modes have |1/beta_n| < eta without any cancellation).
"""
from __future__ import annotations

import math
import numpy as np
from scipy import special as sp

from . import green as gr


def nodes(par):
    """x_l = l dx (l = 1..N) and f, f', f'' from the Fourier coefficients."""
    N, d = par["N"], par["d"]
    x = d / N * np.arange(1, N + 1)
    f, f1, f2 = profile(par, x)
    return x, f, f1, f2


def profile(par, x):
    d = par["d"]
    a, b = par["a"], par["b"]
    x = np.asarray(x, float)
    f = np.full(x.shape, float(a[0]))
    f1 = np.zeros(x.shape)
    f2 = np.zeros(x.shape)
    for m in range(1, len(a)):
        w = 2 * math.pi * m / d
        c, s = np.cos(w * x), np.sin(w * x)
        f += a[m] * c + b[m] * s
        f1 += w * (-a[m] * s + b[m] * c)
        f2 += -w * w * (a[m] * c + b[m] * s)
    return f, f1, f2


def wave(par):
    k, th = par["k"], par["theta"]
    return k * math.sin(th), k * math.cos(th)


def rhs(par):
    """Dirichlet: -u^inc; Neumann: -d u^inc / d nu_hat = i (alpha f' + beta)/s u^inc (eq. fist_eq)."""
    x, f, f1, _ = nodes(par)
    al, be = wave(par)
    uinc = np.exp(1j * (al * x - be * f))
    if par["bc"] == 0:
        return -uinc
    s = np.sqrt(1 + f1 * f1)
    return 1j * (al * f1 + be) / s * uinc


def mode_sets(par):
    """Propagating set U (k^2 - alpha_n^2 > 0) and completion set U^eta (eq. M_eta)."""
    k, d, j, h = par["k"], par["d"], par["j"], par["h"]
    al, _ = wave(par)
    nlo = int(math.floor((-math.sqrt(2) * k - al) * d / (2 * math.pi))) - 1
    nhi = int(math.ceil((math.sqrt(2) * k - al) * d / (2 * math.pi))) + 1
    n = np.arange(nlo, nhi + 1)
    an = al + 2 * math.pi * n / d
    bn = gr.beta_n(k, al, d, n)
    U = n[(k * k - an * an) > 0]
    q = np.abs(gr.Qj(bn, h, j))
    Ueta = n[(q < par["eta"]) & (np.abs(bn) <= k)]
    return U, Ueta


def kress_weights(M, dx):
    """r_s, s = -(M-1)..(M-1): weights for the integral of ln(4 sin^2(pi X/(2a))) phi over a
    period 2a = 2 M dx sampled at spacing dx, X = s dx."""
    s = np.arange(-(M - 1), M)
    m = np.arange(1, M)
    r = -2 * dx * np.sum(np.cos(np.pi * np.outer(s, m) / M) / m[None, :], axis=1) - dx / M * (-1.0) ** s
    return s, r


def _kernel_dnu(par, gx, gy, f1_src, f1_tgt, s_src, s_tgt):
    """Per-dx kernel from a gradient (dG/dX, dG/dY) at X = x_tgt - x_src."""
    if par["bc"] == 0:
        return f1_src * gx - gy
    return (-f1_tgt * gx + gy) / s_tgt * s_src


def reg_matrix(par, rows=None):
    """Dense matrix of D~_reg (eqs. D_ns, G_jq_s): all N rows, or the target rows given."""
    N, d, k, j, h = par["N"], par["d"], par["k"], par["j"], par["h"]
    dx = d / N
    al, _ = wave(par)
    x, f, f1, f2 = nodes(par)
    s = np.sqrt(1 + f1 * f1)
    a_s, gam = par["a_s"], par["gamma"]
    rows = np.arange(N) if rows is None else np.asarray(rows)
    I, K = np.meshgrid(rows, np.arange(N), indexing="ij")
    X = (x[I] - x[K]).ravel()
    Y = (f[I] - f[K]).ravel()
    diag = (I == K).ravel()
    g, gx, gy = gr.gtilde_hybrid(par, X, Y, puncture=diag)
    for p in (-1, 0, 1):
        Xp = X + p * d
        r = np.hypot(Xp, Y)
        sf = gr.S_window(r, gam, a_s)
        sel = sf > 0
        if not np.any(sel):
            continue
        skip = diag & (p == 0)
        ax = np.zeros(X.shape, complex)
        ay = np.zeros(X.shape, complex)
        ok = sel & ~skip
        ax[ok], ay[ok] = gr.gradGj(k, j, h, Xp[ok], Y[ok])
        sk = sel & skip
        if np.any(sk):
            ax[sk], ay[sk] = gr.gradGj(k, j, h, Xp[sk], Y[sk], skip_m0=True)
        ph = np.exp(-1j * al * p * d)
        gx = gx - ph * sf * ax
        gy = gy - ph * sf * ay
    kreg = _kernel_dnu(par, gx, gy, f1[K].ravel(), f1[I].ravel(), s[K].ravel(), s[I].ravel())
    return (dx * kreg).reshape(len(rows), N)


def assemble_rows(par, rows):
    """Rows `rows` of the dense matrix (sigma/2 I + D_sing + D_reg + D_M) (eq. discrete_eq), as a
    len(rows) x N block: the same parts as assemble(), restricted to the given targets."""
    rows = np.asarray(rows)
    A = reg_matrix(par, rows).astype(complex)
    r, c, v = sing_triplets(par, rows)
    pos = {int(t): n for n, t in enumerate(rows)}
    np.add.at(A, (np.array([pos[int(t)] for t in r]), c), v)
    T, S = modes_factors(par)
    A += T[rows] @ S
    sigma = 0.5 if par["bc"] == 0 else -0.5
    A[np.arange(len(rows)), rows] += sigma
    return A


def apply_rows(par, mu, rows):
    """Rows `rows` of (sigma/2 I + D^dx) mu of the exact system, without assembling the matrix."""
    rows = np.asarray(rows)
    y = reg_matrix(par, rows) @ mu
    r, c, v = sing_triplets(par, rows)
    pos = {int(t): n for n, t in enumerate(rows)}
    np.add.at(y, np.array([pos[int(t)] for t in r]), v * mu[c])
    T, S = modes_factors(par)
    y += T[rows] @ (S @ mu)
    sigma = 0.5 if par["bc"] == 0 else -0.5
    return y + sigma * mu[rows]


def sing_triplets(par, rows=None):
    """D~_sing (eq. local_mat) as (rows, cols, values) triplets for all target rows (or the given
    ones); columns wrapped by quasi-periodicity mu_{l+N} = e^{i alpha d} mu_l (eq. quasiper_disc)."""
    N, d, k, j, h = par["N"], par["d"], par["k"], par["j"], par["h"]
    dx = d / N
    al, _ = wave(par)
    x, f, f1, f2 = nodes(par)
    s = np.sqrt(1 + f1 * f1)
    ii = np.arange(N) if rows is None else np.asarray(rows)
    x, f, f1, f2, s = x[ii], f[ii], f1[ii], f2[ii], s[ii]
    a_s, gam = par["a_s"], par["gamma"]
    M = par["Ma"]
    ss, rw = kress_weights(M, dx)
    w = gr.binom_weights(j)
    hk = sum(w[m] * 0.25j * k * sp.hankel1(1, k * m * h) for m in range(1, j + 1))
    out_r, cols, vals = [], [], []
    for si, rs in zip(ss, rw):
        ll = ii - si                      # unwrapped source index (0-based)
        lw = np.mod(ll, N)
        wrap = np.floor_divide(ll, N)
        xl = dx * (ll + 1)
        fl, f1l, _ = profile(par, xl)
        sl = np.sqrt(1 + f1l * f1l)
        Xs = x - xl
        Ys = f - fl
        r = np.hypot(Xs, Ys)
        sf = gr.S_window(r, gam, a_s)
        ph = np.exp(1j * al * d * wrap)
        if si == 0:
            kr = f2 / (4 * math.pi * (1 + f1 * f1)) + (hk if par["bc"] == 0 else -hk)
            val = dx * kr * sf
        else:
            ax, ay = gr.gradGj(k, j, h, Xs, Ys)
            kern = _kernel_dnu(par, ax, ay, f1l, f1, sl, s)
            j1r = k * sp.j1(k * r) / r
            if par["bc"] == 0:
                ks = -j1r / (4 * math.pi) * (Ys - f1l * Xs)
            else:
                ks = j1r / (4 * math.pi) * (-f1 * Xs + Ys) / s * sl
            lg = np.log(4 * np.sin(math.pi * Xs / (2 * a_s)) ** 2)
            kr = kern - ks * lg
            val = (rs * ks + dx * kr) * sf
        out_r.append(ii)
        cols.append(lw)
        vals.append(val * ph)
    return np.concatenate(out_r), np.concatenate(cols), np.concatenate(vals)


def modes_factors(par):
    """D_M = T @ S with T [N x |U^eta|] (target factors) and S [|U^eta| x N] (source factors)."""
    N, d, k = par["N"], par["d"], par["k"]
    dx = d / N
    al, _ = wave(par)
    x, f, f1, _ = nodes(par)
    s = np.sqrt(1 + f1 * f1)
    _, Ueta = mode_sets(par)
    T = np.zeros((N, len(Ueta)), complex)
    S = np.zeros((len(Ueta), N), complex)
    for t, n in enumerate(Ueta):
        an = al + 2 * math.pi * n / d
        bn = complex(gr.beta_n(k, al, d, np.array([n]))[0])
        tgt = np.exp(1j * (an * x + bn * f))
        if par["bc"] == 1:
            tgt = tgt * (1j * an * (-f1) + 1j * bn) / s
        T[:, t] = tgt
        S[t, :] = np.exp(-1j * (an * x + bn * f)) * s * dx
    return T, S


def assemble(par, return_parts=False):
    """Dense N x N matrix of (sigma/2 I + D_sing + D_reg + D_M) (eq. discrete_eq)."""
    N = par["N"]
    Areg = reg_matrix(par)
    r, c, v = sing_triplets(par)
    Asing = np.zeros((N, N), complex)
    np.add.at(Asing, (r, c), v)
    T, S = modes_factors(par)
    Amod = T @ S
    sigma = 0.5 if par["bc"] == 0 else -0.5
    A = sigma * np.eye(N) + Asing + Areg + Amod
    if return_parts:
        return A, {"sing": Asing, "reg": Areg, "modes": Amod}
    return A


def solve(par, A=None):
    if A is None:
        A = assemble(par)
    return np.linalg.solve(A, rhs(par))


def rayleigh(par, mu, n_lo=None, n_hi=None):
    """B_n of u^s = sum_n B_n e^{i alpha_n x + i beta_n y} above the surface (eq. rayexp), from the
    spectral form of G~ for Y > 0 (eq. shifted_periodic_green_function_spectral) and M^eta;
    efficiencies e_n = (beta_n/beta)|B_n|^2 and energy error eps = 1 - sum_{n in U} e_n."""
    N, d, k, j, h = par["N"], par["d"], par["k"], par["j"], par["h"]
    dx = d / N
    al, be = wave(par)
    x, f, f1, _ = nodes(par)
    s = np.sqrt(1 + f1 * f1)
    U, Ueta = mode_sets(par)
    if n_lo is None:
        n_lo, n_hi = int(U.min()), int(U.max())
    n = np.arange(n_lo, n_hi + 1)
    B = np.zeros(len(n), complex)
    for t, nn in enumerate(n):
        an = al + 2 * math.pi * nn / d
        bn = complex(gr.beta_n(k, al, d, np.array([nn]))[0])
        q = complex(gr.Qj(np.array([bn]), h, j)[0])
        ph = np.exp(-1j * (an * x + bn * f))
        ind = 1.0 if nn in set(Ueta.tolist()) else 0.0
        if par["bc"] == 0:
            wgt = (bn - an * f1) * q / (2 * d) + s * ind
        else:
            wgt = s * (1j * q / (2 * d) + ind)
        B[t] = dx * np.sum(mu * ph * wgt)
    bnv = gr.beta_n(k, al, d, n)
    prop = np.isin(n, U)
    eff = np.where(prop, bnv.real / be * np.abs(B) ** 2, 0.0)
    eps = 1.0 - float(np.sum(eff[prop]))
    return n, B, eff, eps
