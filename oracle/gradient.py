"""Reference derivatives of the efficiencies e_n = (beta_n/beta)|B_n|^2 (eqs. rayexp, energy_error)
with respect to the profile's Fourier coefficients. Test infrastructure only.

The derivative is taken by its definition, as a central difference quotient of e_n at the
coefficient moved by +-eps, where e_n comes from a dense solve of either the accelerated operator
(Algorithm 3 assembled column by column by accel.Accel.matrix) or the exact Nystrom system of
Section 4 (direct.assemble). For the accelerated operator the cell assignment of the nodes must not
change between the three profiles (the operator is a different approximation in another
assignment); a change raises.
"""
from __future__ import annotations

import numpy as np

from . import accel as ac
from . import direct as dr


def efficiency(par, n, operator="accel"):
    """e_n of the dense solution, with the cell assignment used (None for the exact system)."""
    if operator == "accel":
        acc = ac.Accel(par)
        A = acc.matrix()
        cells = {q: list(v) for q, v in acc.cell_nodes.items()}
    else:
        A = dr.assemble(par)
        cells = None
    mu = np.linalg.solve(A, dr.rhs(par))
    ns, _, eff, _ = dr.rayleigh(par, mu, n, n)
    return float(eff[0]), cells


def moved(par, kind, m, delta):
    """Parameters with coefficient kind ('a' or 'b') m moved by delta (all else unchanged)."""
    p2 = dict(par)
    arr = np.array(par[kind], dtype=float).copy()
    arr[m] += delta
    p2[kind] = arr
    return p2


def efficiency_gradient_fd(par, n, coeffs, eps=1e-6, operator="accel"):
    """[(e_n(c + eps) - e_n(c - eps)) / (2 eps) for each (kind, m) in coeffs]."""
    base = efficiency(par, n, operator)[1]
    out = []
    for kind, m in coeffs:
        vals = []
        for sg in (1.0, -1.0):
            e, cells = efficiency(moved(par, kind, m, sg * eps), n, operator)
            if cells != base:
                raise RuntimeError(f"cell assignment changed for {kind}{m} {sg * eps:+g}")
            vals.append(e)
        out.append((vals[0] - vals[1]) / (2 * eps))
    return np.array(out)
