"""sgf_suggest_params (host only, CPU): the suggested parameters satisfy every constraint of the
accelerated build, detect Wood configurations, grow monotonically with the digits asked for, and
reach the target energy balance with the oracle's exact system (the discretisation they choose; the
accelerator's own approximation comes on top and is not part of this check).
"""
import math

import numpy as np
import pytest

from oracle import direct as dr
from paper_1707_04950_gb300 import build as _build
from paper_1707_04950_gb300 import inputs as I
from paper_1707_04950_gb300 import sgf


@pytest.fixture(scope="module", autouse=True)
def _library():
    _build.build()  # host-only entry point: the library loads without a GPU


THETA_LITTROW = math.degrees(math.asin(1 / 3))
COMPOSITE = {"d": 2 * math.pi, "a": np.zeros(5), "b": -0.25 * np.array([0.0, 1.0, 1 / 2, 1 / 3, 1 / 4])}


def _littrow(H_over_d):
    return {"d": 2 * math.pi, "a": np.zeros(2), "b": np.array([0.0, H_over_d * math.pi])}


CASES = {  # profile, k, theta (deg), bc, Wood?
    "sinusoid_double_wood_dirichlet": (I.sinusoid(2.0, 0.25), 2 * math.pi, 30.0, 0, True),
    "sinusoid_double_wood_neumann": (I.sinusoid(2.0, 0.25), 2 * math.pi, 30.0, 1, True),
    "littrow_quarter_wood_k3": (_littrow(0.25), 3.0, THETA_LITTROW, 0, True),
    "littrow_half_k2.5": (_littrow(0.5), 2.5, THETA_LITTROW, 0, False),
    "harmonic_neumann": (I.harmonic_surface(2.0, 3, 0.05, 4), 2 * math.pi, 20.0, 1, False),
    "composite_k20": (COMPOSITE, 20.0, 45.0, 0, False),
    "composite_wood": (COMPOSITE, 6 / (1 - math.sin(math.radians(45))), 45.0, 0, True),
    "deep_corrugation": (I.sinusoid(10.0, 10.0), 2 * math.pi, 45.0, 1, False),
    "littrow_deep_wood_k9": (_littrow(1.0), 9.0, THETA_LITTROW, 0, True),
    "gaussian_rough": (I.gaussian_surface(10.0, 0.5, 2.0, 5000), 2 * math.pi, 40.0, 0, False),
}


def _suggest(name, tol, converged=None):
    prof, k, th, bc, _ = CASES[name]
    try:
        p = sgf.sgf_suggest_params(prof["d"], prof["a"], prof["b"], k, math.radians(th), bc, tol)
        ok = True
    except sgf.SgfError as e:  # SGF_ENOCONV: the lattice-sum check did not reach tol/10
        assert e.status == 5 and e.params.n_per == 16384
        p, ok = e.params, False
    if converged is not None:
        converged.append(ok)
    par = {f: getattr(p, f) for f, _ in sgf.sgf_params._fields_}
    d = prof["d"]
    par.update(d=d, a=np.asarray(prof["a"], float), b=np.asarray(prof["b"], float), k=k, theta=math.radians(th), bc=bc,
               L=d / par["nx"], a_s=par["Ma"] * d / par["N"])
    par["gamma"] = 0.5 * par["a_s"]
    return par


def _pow2(n):
    return n > 0 and n & (n - 1) == 0


@pytest.mark.parametrize("name", list(CASES))
def test_suggestion_satisfies_the_build_constraints(name):
    par = _suggest(name, 1e-8)
    N, nx, p, L = par["N"], par["nx"], par["p"], par["L"]
    assert N % nx == 0 and _pow2(nx) and _pow2(nx * p)
    assert par["a_s"] < L and 2 <= par["Ma"]
    x, f, f1, _ = dr.nodes(par)
    assert par["h"] > par["a_s"] * np.max(np.abs(f1))  # shifted images clear of the singular window
    cy = np.ceil((f - par["hmin"]) / L) - 1
    assert cy.min() >= 0 and cy.max() < par["ny"]  # every node inside the cell box
    for m in range(1, par["j"] + 1):  # shifted poles off the grid lags
        r = m * par["h"] / (L / p)
        assert abs(r - round(r)) > 1e-6
    t = (par["k"] * L / math.pi) ** 2  # non-resonant cell
    assert all(abs(t - (m * m + n * n)) > 1e-3 for m in range(1, 40) for n in range(1, 40))
    assert 4 * (p + 1) <= 64 and 8 <= par["n_per"] <= 20000


@pytest.mark.parametrize("name", list(CASES))
def test_shifts_chosen_at_wood_anomalies(name):
    assert (_suggest(name, 1e-6)["j"] == 8) == CASES[name][4]


@pytest.mark.parametrize("name", ["sinusoid_double_wood_dirichlet", "littrow_half_k2.5", "composite_wood"])
def test_more_digits_more_work(name):
    ok = []
    a, b = _suggest(name, 1e-4, ok), _suggest(name, 1e-10, ok)
    assert b["N"] >= a["N"] and b["n_per"] >= a["n_per"]
    assert b["N"] > a["N"]
    # the composite surface at its Wood wavenumber needs more than 16384 periods for 1e-11 (the
    # lattice sum converges like A^-3.5 there): the suggestion says so instead of returning OK
    assert ok == [True, name != "composite_wood"]


@pytest.mark.parametrize("name,tol", [
    ("sinusoid_double_wood_dirichlet", 1e-6), ("sinusoid_double_wood_neumann", 1e-6),
    ("littrow_quarter_wood_k3", 1e-6), ("littrow_half_k2.5", 1e-6), ("harmonic_neumann", 1e-6),
    ("littrow_half_k2.5", 1e-8), ("harmonic_neumann", 1e-8), ("sinusoid_double_wood_neumann", 1e-8),
])
def test_energy_balance_at_suggested_parameters(name, tol):
    # measured: 1.6e-8 ... 4.2e-7 at 1e-6; 7.7e-9 ... 5.7e-8 at 1e-8
    par = _suggest(name, tol)
    mu = dr.solve(par)
    eps = abs(dr.rayleigh(par, mu, -60, 60)[3])
    assert eps < 10 * tol, (name, tol, par["N"], eps)


def test_argument_errors():
    prof = I.sinusoid(2.0, 0.25)
    for tol in (0.0, 1e-15, 0.5):
        with pytest.raises(sgf.SgfError) as e:
            sgf.sgf_suggest_params(prof["d"], prof["a"], prof["b"], 2 * math.pi, 0.3, 0, tol)
        assert e.value.status == 1
    with pytest.raises(sgf.SgfError):
        sgf.sgf_suggest_params(prof["d"], prof["a"], prof["b"], 2 * math.pi, 2.0, 0, 1e-6)  # |theta| >= pi/2
