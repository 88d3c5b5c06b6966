"""Pins of the gradient oracle (central difference quotients of e_n over dense solves) by symmetries
of the exact scattering problem, independent of any GPU code:

* vertical translation f -> f + c changes every B_n by a phase only, so de_0/da_0 = 0;
* horizontal translation f(x) -> f(x - s) also changes B_n by a phase only, so the derivative of
  e_0 along the coefficient direction (da_m, db_m) = (-w_m b_m, w_m a_m), w_m = 2 pi m / d,
  vanishes (up to the discretisation: the nodes do not move with the profile);
* at normal incidence an even profile (cosines only) has e_0(b_m = +s) = e_0(b_m = -s) by mirror
  symmetry, so de_0/db_m = 0, while de_0/da_m does not vanish.
A difference quotient with a wrong sign, a wrong step or a wrong coefficient index fails at least
one of them.
"""
import math

import numpy as np
import pytest

from oracle import gradient as og
from paper_1707_04950_gb300 import inputs as I


def _eff(par, n=0):
    return og.efficiency(par, n, "exact")[0]


@pytest.mark.slow
def test_vertical_and_horizontal_translation_leave_e0_unchanged():
    # 3 harmonics, period 2, Dirichlet, 20 deg; measured at N = 128: de_0/da_0 = -1.1e-8,
    # de_0/da_1 = 4.06, derivative along the translation tangent -2.6e-8 (|u| = 0.40)
    par = I.wl_harmonic_gradient_small(N=128, nx=8)
    g = og.efficiency_gradient_fd(par, 0, [("a", 0), ("a", 1)], 1e-6, "exact")
    scale = np.max(np.abs(g[1:]))
    assert scale > 1e-3  # the profile coefficients do move e_0
    assert abs(g[0]) < 2e-8 * scale
    # along the tangent of the horizontal translation
    d = par["d"]
    M = len(par["a"]) - 1
    w = 2 * math.pi * np.arange(M + 1) / d
    ua, ub = -w * par["b"], w * par["a"]
    eps = 1e-5
    ep = _eff(dict(par, a=par["a"] + eps * ua, b=par["b"] + eps * ub))
    em = _eff(dict(par, a=par["a"] - eps * ua, b=par["b"] - eps * ub))
    dd = (ep - em) / (2 * eps)
    unorm = math.sqrt(float(np.sum(ua**2) + np.sum(ub**2)))
    assert abs(dd) < 1e-7 * scale * unorm


@pytest.mark.slow
def test_mirror_symmetry_at_normal_incidence():
    # measured at N = 128: de_0/da_1 = -7.65, de_0/db_1 = 1.7e-10, de_0/db_2 = -1.1e-10
    prof = {"d": 2.3, "a": np.array([0.0, 0.08, 0.03]), "b": np.zeros(3)}  # even profile, no Wood
    par = I.make_params(prof, 2 * math.pi, 0.0, 0, 128, nx=8, j=0)
    g = og.efficiency_gradient_fd(par, 0, [("a", 1), ("b", 1), ("b", 2)], 1e-6, "exact")
    assert abs(g[0]) > 1.0
    assert max(abs(g[1]), abs(g[2])) < 1e-9 * abs(g[0])
