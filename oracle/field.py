"""Scattered field off the surface: test infrastructure (only tests, the smoke check and the
benchmark's CPU baseline use this package).

Once the density mu solves the Nystrom system, the scattered field at any point above the surface
is the representation of eq. int_eq_dirichlet discretised at the nodes with the same trapezoid
weights as the operator (the remark after Algorithm 3 evaluates it with a modified Algorithm 3):

  Dirichlet: u^s(x, y) = dx sum_l [ (f'_l dG~/dX - dG~/dY) + s_l M^eta ](x - x_l, y - f_l) mu_l
             (double layer, unnormalised source normal nu_l = (-f'_l, 1));
  Neumann:   u^s(x, y) = dx sum_l s_l [ G~ + M^eta ](x - x_l, y - f_l) mu_l (single layer).

G~ = G~_j^qper by the hybrid evaluation (spectral series away from the shifted images, windowed
lattice sums near them), M^eta the completion modes (eq. M_eta). The trapezoid rule is spectrally
accurate for targets a few node spacings off the surface; closer targets see the near-singular
integrand and lose accuracy (the paper gives no special quadrature there).

field_rayleigh is the same sum written mode by mode with the Y > 0 spectral form of G~ (eq.
shifted_periodic_green_function_spectral): valid for targets above every node, and the form the
GPU path uses above its cell box.
"""
from __future__ import annotations

import math
import numpy as np

from . import direct as dr
from . import green as gr


def incident(par, pts):
    """u^inc = e^{i (alpha x - beta y)} (eq. fist_eq)."""
    al, be = dr.wave(par)
    pts = np.asarray(pts, float).reshape(-1, 2)
    return np.exp(1j * (al * pts[:, 0] - be * pts[:, 1]))


def _mode_values(par, X, Y):
    """M^eta(X, Y) = sum_{n in U^eta} e^{i alpha_n X + i beta_n Y}."""
    k, d = par["k"], par["d"]
    al, _ = dr.wave(par)
    _, Ueta = dr.mode_sets(par)
    out = np.zeros(np.shape(X), complex)
    for n in Ueta:
        an = al + 2 * math.pi * n / d
        bn = complex(gr.beta_n(k, al, d, np.array([n]))[0])
        out += np.exp(1j * (an * X + bn * Y))
    return out


def field_direct(par, mu, pts, total=False):
    """u^s (plus u^inc when total) at the points pts [n, 2] from the density mu [N]: the discretised
    representation by its definition, one G~ evaluation per (target, node) pair."""
    N, d = par["N"], par["d"]
    dx = d / N
    x, f, f1, _ = dr.nodes(par)
    s = np.sqrt(1 + f1 * f1)
    pts = np.asarray(pts, float).reshape(-1, 2)
    mu = np.asarray(mu, complex)
    out = np.zeros(len(pts), complex)
    for t, (xt, yt) in enumerate(pts):
        X = xt - x
        Y = yt - f
        g, gx, gy = gr.gtilde_hybrid(par, X, Y)
        M = _mode_values(par, X, Y)
        if par["bc"] == 0:
            kern = f1 * gx - gy + s * M
        else:
            kern = s * (g + M)
        out[t] = dx * np.sum(kern * mu)
    if total:
        out = out + incident(par, pts)
    return out


def field_rayleigh(par, mu, pts, n_lo, n_hi):
    """The same field for targets above every node, mode by mode: for Y > 0 every shifted image lies
    below the target, G~ = sum_n (i/(2d)) Q_j(beta_n) e^{i alpha_n X + i beta_n Y} with
    Q_j = (1 - e^{i beta_n h})^j / beta_n, so u^s = sum_n e^{i alpha_n x} sum_l w_ln e^{i beta_n (y - f_l)}
    e^{-i alpha_n x_l} mu_l, summed over n_lo..n_hi (the caller picks the range from the height)."""
    N, d, k, j, h = par["N"], par["d"], par["k"], par["j"], par["h"]
    dx = d / N
    al, _ = dr.wave(par)
    x, f, f1, _ = dr.nodes(par)
    s = np.sqrt(1 + f1 * f1)
    _, Ueta = dr.mode_sets(par)
    ue = set(Ueta.tolist())
    pts = np.asarray(pts, float).reshape(-1, 2)
    assert np.all(pts[:, 1] > f.max()), "Rayleigh form only above every node"
    mu = np.asarray(mu, complex)
    out = np.zeros(len(pts), complex)
    for n in range(n_lo, n_hi + 1):
        an = al + 2 * math.pi * n / d
        bn = complex(gr.beta_n(k, al, d, np.array([n]))[0])
        q = complex(gr.Qj(np.array([bn]), h, j)[0])
        ind = 1.0 if n in ue else 0.0
        if par["bc"] == 0:
            # -(d/dY) and f' (d/dX) of the mode, times i/(2d) Q_j, plus the completion mode
            w = (bn - an * f1) * q / (2 * d) + s * ind
        else:
            w = s * (1j * q / (2 * d) + ind)
        E = np.exp(1j * (an * (pts[:, 0][:, None] - x[None, :]) + bn * (pts[:, 1][:, None] - f[None, :])))
        out += dx * (E @ (w * mu))
    return out
