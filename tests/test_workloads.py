"""The synthetic workloads that stand in for the paper's tables (CPU): the golden rows are read as
the paper states them (d = 2 pi so that d / lambda = k; Littrow mount sin(theta) = 1/3; H / lambda as
printed), Wood rows are Wood anomalies (some alpha_n = +-k) and non-Wood rows are not.
"""
import math
import os

import numpy as np
import pytest

from oracle import direct as dr
from paper_1707_04950_gb300 import inputs as I

HERE = os.path.dirname(__file__)


def _rows(name):
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", name)) if ln.strip() and not ln.startswith("#")]
    return [[float(v) for v in r] for r in rows]


def _min_beta_over_k(par):
    k, d = par["k"], par["d"]
    al, _ = dr.wave(par)
    n = np.arange(-200, 201)
    an = al + 2 * math.pi * n / d
    return float(np.min(np.abs(k * k - an * an))) / (k * k)


def test_littrow_rows_read_as_printed():
    rows = _rows("sinusoid_littrow_energy_error.txt")
    assert len(rows) == 36
    for Hd, Hl, dl, N, hl, n_per, _, _, _ in rows:
        par = I.wl_littrow(Hd, dl, int(N), hl, int(n_per))
        lam = 2 * math.pi / par["k"]
        H = 2 * np.max(np.abs(par["b"]))
        assert abs(H / lam - Hl) < 0.006  # the printed H / lambda (two decimals)
        assert abs(par["d"] / lam - dl) < 1e-12
        assert abs(math.sin(par["theta"]) - 1 / 3) < 1e-15
        wood = _min_beta_over_k(par) < 1e-12
        assert wood == (hl > 0), (Hd, dl)
        if hl > 0:
            assert par["j"] == 8 and abs(par["h"] / lam - hl) < 1e-12
            # the singular window stays below the shifted images of the steepest node
            assert par["h"] > par["a_s"] * math.pi * H / par["d"]
        else:
            assert par["j"] == 0
        assert 2 <= par["Ma"] < par["N"] / 2


@pytest.mark.parametrize("wood", [False, True])
def test_composite_rows_read_as_printed(wood):
    for N, n_per, _, _ in _rows("composite_surface_energy_error.txt"):
        par = I.wl_composite(int(N), int(n_per), wood=wood)
        x, f, f1, _ = dr.nodes(par)
        assert abs((f.max() - f.min()) - 0.763) < 2e-3  # the printed peak-to-trough height
        assert (_min_beta_over_k(par) < 1e-12) == wood
        if wood:
            assert par["j"] == 8 and par["h"] == 0.16 and par["h"] > par["a_s"] * np.max(np.abs(f1))


@pytest.mark.parametrize("r", [2, 4])
def test_repeated_corrugation_is_the_benchmark_shape(r):
    """The longer-surface workload repeats the benchmark corrugation: the same profile values at the
    same abscissae, node spacing, cell size and box, r times the period and the nodes, and no mode
    of the longer period sits at a Wood anomaly."""
    base = I.wl_deep_corrugation_neumann()
    rep = I.wl_deep_corrugation_neumann_periods(r)
    assert rep["N"] == r * base["N"] and rep["nx"] == r * base["nx"] and rep["d"] == r * base["d"]
    x = np.linspace(0.0, base["d"], 257)
    f0 = I.profile_eval_host({"d": base["d"], "a": base["a"], "b": base["b"]}, x)
    f1 = I.profile_eval_host({"d": rep["d"], "a": rep["a"], "b": rep["b"]}, x)
    assert np.max(np.abs(f1 - f0)) < 1e-12
    assert rep["d"] / rep["N"] == pytest.approx(base["d"] / base["N"])
    assert rep["d"] / rep["nx"] == pytest.approx(base["d"] / base["nx"])
    assert rep["ny"] == base["ny"] and rep["hmin"] == pytest.approx(base["hmin"])
    assert _min_beta_over_k(rep) > 1e-3
