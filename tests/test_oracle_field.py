"""Pins of the oracle's scattered field off the surface (oracle/field.py, Accel.field), each against
something other than the formula itself:

* a flat surface, where the reflected wave is known in closed form (-1 Dirichlet, +1 Neumann);
* the boundary condition: extrapolated along the normal to the surface, the total field of a
  solved density vanishes (Dirichlet) or has zero normal derivative (Neumann);
* the mode-by-mode Rayleigh form above every node (a different formula for the same sum);
* the Helmholtz equation and quasi-periodicity of the field;
* the accelerated field (Algorithm 3 at off-surface targets) against the direct sum, within the
  accelerator's approximation (1e-5 of the field measured; 2e-4 required).
"""
import math

import numpy as np
import pytest

from oracle import accel as ac, direct as dr, field as fl
from paper_1707_04950_gb300 import inputs as I

_sol = {}


def _neumann_sinusoid():
    return I.make_params(I.sinusoid(2.0, 0.25), 2 * np.pi, 30.0, 1, 256, nx=16, ny=16, hmin=-1.0)


CASES = {"dirichlet_wood": lambda: I.wl_sinusoid_dirichlet(N=256), "neumann": _neumann_sinusoid}


def _solved(name):
    if name not in _sol:
        par = CASES[name]()
        _sol[name] = (par, dr.solve(par))
    return _sol[name]


def _targets(par, n, seed, margin=0.05):
    """Random targets over three periods, between the surface (plus a margin) and the box top."""
    top = par["hmin"] + par["ny"] * par["L"]
    rng = np.random.default_rng(seed)
    P = np.stack([rng.uniform(-par["d"], 2 * par["d"], n), rng.uniform(-0.25, top - 1e-3, n)], 1)
    return P[P[:, 1] > dr.profile(par, P[:, 0])[0] + margin]


@pytest.mark.parametrize("bc", [0, 1])
def test_flat_surface_reflects_the_incident_wave(bc):
    par = I.flat(N=64, d=1.0, theta_deg=20.0, bc=bc, nx=8)
    mu = dr.solve(par)
    al, be = dr.wave(par)
    pts = np.array([[0.13, 0.3], [0.77, 0.05], [0.5, 1.3], [-0.4, 0.6]])
    ref = (-1.0 if bc == 0 else 1.0) * np.exp(1j * (al * pts[:, 0] + be * pts[:, 1]))
    assert np.max(np.abs(fl.field_direct(par, mu, pts) - ref)) < 1e-9
    assert np.max(np.abs(fl.field_direct(par, mu, pts, total=True) - ref - fl.incident(par, pts))) < 1e-9


def _normal_line(par, i, mu):
    x, f, f1, _ = dr.nodes(par)
    nrm = np.array([-f1[i], 1.0]) / math.hypot(f1[i], 1.0)
    ds = np.arange(3, 9) * par["d"] / par["N"]
    P = np.array([[x[i], f[i]]]) + ds[:, None] * nrm[None, :]
    return ds, fl.field_direct(par, mu, P, total=True)


def _poly_coef(ds, u, k):
    return np.polyfit(ds, u.real, 5)[k] + 1j * np.polyfit(ds, u.imag, 5)[k]


def test_dirichlet_total_field_vanishes_on_the_surface():
    # the configuration is a double Wood anomaly: without the completion modes the limit is O(1)
    par, mu = _solved("dirichlet_wood")
    for i in (5, 37, 200):
        ds, u = _normal_line(par, i, mu)
        assert abs(_poly_coef(ds, u, -1)) < 1e-3 * np.max(np.abs(u)), i


def test_neumann_normal_derivative_vanishes_on_the_surface():
    # the extrapolated derivative is less accurate than a value: 2e-2 of k |u| (measured 6e-3)
    par, mu = _solved("neumann")
    for i in (5, 37, 100):
        ds, u = _normal_line(par, i, mu)
        assert abs(_poly_coef(ds, u, -2)) < 2e-2 * par["k"] * np.max(np.abs(u)), i


@pytest.mark.parametrize("name", list(CASES))
def test_rayleigh_form_matches_the_direct_sum(name):
    par, mu = _solved(name)
    fmax = dr.nodes(par)[1].max()
    pts = np.array([[0.1, fmax + 0.3], [1.1, fmax + 0.15], [-1.7, fmax + 0.6], [3.3, fmax + 1.0]])
    ud = fl.field_direct(par, mu, pts)
    ur = fl.field_rayleigh(par, mu, pts, -60, 60)
    assert np.max(np.abs(ud - ur)) < 1e-11 * np.max(np.abs(ud))


def test_field_solves_helmholtz_and_is_quasi_periodic():
    par, mu = _solved("dirichlet_wood")
    xt, yt, hh = 0.6, 0.35, 1e-3
    Q = np.array([[xt, yt], [xt + hh, yt], [xt - hh, yt], [xt, yt + hh], [xt, yt - hh]])
    u = fl.field_direct(par, mu, Q)
    lap = (u[1] + u[2] + u[3] + u[4] - 4 * u[0]) / hh**2
    k2u = par["k"] ** 2 * u[0]
    assert abs(lap + k2u) < 1e-4 * abs(k2u)  # second-order differences: (k h)^2 / 12 ~ 3e-6
    al, _ = dr.wave(par)
    v = fl.field_direct(par, mu, np.array([[0.3, 0.4], [0.3 + par["d"], 0.4], [0.3 - 2 * par["d"], 0.4]]))
    assert abs(v[1] - np.exp(1j * al * par["d"]) * v[0]) < 1e-12 * abs(v[0])
    assert abs(v[2] - np.exp(-2j * al * par["d"]) * v[0]) < 1e-12 * abs(v[0])


@pytest.mark.parametrize("name", list(CASES))
def test_accelerated_field_matches_the_direct_sum(name):
    par, mu = _solved(name)
    P = _targets(par, 14, 1 if name == "neumann" else 2)
    ua = ac.Accel(par).field(mu, P)
    ud = fl.field_direct(par, mu, P)
    assert np.max(np.abs(ua - ud)) < 2e-4 * np.max(np.abs(ud))
