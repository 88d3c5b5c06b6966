"""The scattered field off the surface (sgf_field) against the oracle: inside the cell box against
the oracle's Algorithm 3 at off-surface targets (the same accelerated sum, FP64), above the box
against the Rayleigh form and the direct sum; solved densities against the flat-surface closed form;
argument and edge cases.

Tolerances: inside the box the two sides evaluate the same FP64 operations in another order, with
least-squares factors built separately (condition ~1e6 after the Tikhonov term, as for the forward
map, whose parity measures 7e-11). Off the surface the field is smaller than the convolved values
it is fitted from (phi^all and phi^int cancel in the local subtraction), so the same absolute
rounding is larger relative to it: measured 4e-10 of the largest value; we require 1e-9. Above
the box both sides sum the same exact series: 1e-11 off Wood anomalies. At a Wood anomaly
beta_n = sqrt(k^2 - alpha_n^2) of the anomalous mode is a square root of a rounding-level number,
so the one-ulp difference between the two sides' alpha = k sin(theta) moves it by ~1e-8, and its
completion mode e^{i alpha_n x + i beta_n (y - f)} carries that into the field (measured 1.3e-9 of
the largest value): 1e-8 there. Against the direct (unaccelerated) sum the accelerator's
approximation decides: 2e-4.
"""
import numpy as np
import pytest

from oracle import accel as ac, direct as dr, field as fl
from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")
torch = pytest.importorskip("torch")

CASES = {
    "sinusoid_dirichlet_wood_n512": lambda: I.wl_sinusoid_dirichlet(N=512),
    "deep_neumann_n1024": lambda: I.wl_deep_corrugation_neumann_small(N=1024, nx=32),
}
_acc = {}


def _accel(name):
    if name not in _acc:
        _acc[name] = ac.Accel(CASES[name]())
    return _acc[name]


def _targets(par, n, seed, margin=0.02, above=0):
    """Targets over three periods between the surface (plus a margin) and the box top, and `above`
    more between the box top and one period higher."""
    top = par["hmin"] + par["ny"] * par["L"]
    rng = np.random.default_rng(seed)
    P = np.stack([rng.uniform(-par["d"], 2 * par["d"], 4 * n), rng.uniform(par["hmin"], top, 4 * n)], 1)
    P = P[P[:, 1] > dr.profile(par, P[:, 0])[0] + margin][:n]
    Q = np.stack([rng.uniform(-par["d"], 2 * par["d"], above), top + rng.uniform(0, par["d"], above)], 1)
    return np.concatenate([P, Q])


def _field(op, mu, P, total=False):
    mt = torch.from_numpy(np.ascontiguousarray(mu, dtype=np.complex128)).cuda()
    ut = torch.full((len(P),), complex("nan"), dtype=torch.complex128, device="cuda")
    sgf.sgf_field(op.ctx, mt.data_ptr(), P, ut.data_ptr(), total)
    torch.cuda.synchronize()
    return ut.cpu().numpy()


@pytest.mark.parametrize("name", list(CASES))
def test_field_in_the_box_matches_oracle_algorithm3(name):
    # a random density: the map mu -> u^s is linear, parity needs no solve; targets over several
    # cells per row, three periods, and cells without nodes
    A = _accel(name)
    par = A.par
    mu = I.random_density(par["N"], 11)
    P = _targets(par, 40, 3)
    op = sgf.Operator(par, precision=64)
    got = _field(op, mu, P)
    got_t = _field(op, mu, P, total=True)
    op.close()
    ref = A.field(mu, P)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) < 1e-9 * scale
    assert np.max(np.abs(got_t - ref - fl.incident(par, P))) < 1e-9 * max(scale, 1.0)


@pytest.mark.parametrize("name", list(CASES))
def test_field_above_the_box_matches_rayleigh_form(name):
    par = CASES[name]()
    mu = I.random_density(par["N"], 12)
    P = _targets(par, 0, 4, above=12)
    top = par["hmin"] + par["ny"] * par["L"]
    P = np.concatenate([P, [[0.37, top], [par["d"] * 5 + 0.1, top + 0.5]]])  # at the box top; period 5
    op = sgf.Operator(par, precision=64)
    got = _field(op, mu, P)
    op.close()
    fmax = dr.nodes(par)[1].max()
    n_c = int(np.ceil((37.0 / (P[:, 1].min() - fmax) + par["k"] + np.pi / par["d"]) * par["d"] / (2 * np.pi))) + 1
    n0 = int(round(-par["k"] * np.sin(par["theta"]) * par["d"] / (2 * np.pi)))
    ref = fl.field_rayleigh(par, mu, P, n0 - n_c, n0 + n_c)
    tol = 1e-8 if name.startswith("sinusoid_dirichlet_wood") else 1e-11
    assert np.max(np.abs(got - ref)) < tol * np.max(np.abs(ref))
    # and the direct definition at two of them
    dref = fl.field_direct(par, mu, P[:2])
    assert np.max(np.abs(got[:2] - dref)) < 10 * tol * np.max(np.abs(dref))


@pytest.mark.parametrize("prec", [64, 32])
def test_solved_field_against_direct_sum_and_closed_form(prec):
    # Dirichlet at a double Wood anomaly: the GPU solve and field against the oracle's dense solve
    # and direct field (the accelerator's approximation); a flat surface against the reflected wave
    par = I.wl_sinusoid_dirichlet(N=256)
    op = sgf.Operator(par, precision=prec)
    mu = torch.zeros(par["N"], dtype=torch.complex128, device="cuda")
    assert sgf.sgf_solve(op.ctx, 1e-12, 2000, mu.data_ptr())[0] == 0
    P = _targets(par, 16, 5, margin=0.05, above=4)
    got = _field(op, mu.cpu().numpy(), P)
    op.close()
    ref = fl.field_direct(par, dr.solve(par), P)
    assert np.max(np.abs(got - ref)) < 2e-4 * np.max(np.abs(ref))
    flat = I.flat(N=256, d=1.0, theta_deg=20.0, bc=0, nx=8, n_per=80)
    op = sgf.Operator(flat, precision=prec)
    mu = torch.zeros(256, dtype=torch.complex128, device="cuda")
    assert sgf.sgf_solve(op.ctx, 1e-12, 2000, mu.data_ptr())[0] == 0
    P = np.array([[0.1, 0.02], [0.6, 0.05], [1.7, 0.2], [0.3, 0.9]])
    got = _field(op, mu.cpu().numpy(), P, total=True)
    op.close()
    al, be = dr.wave(flat)
    exact = np.exp(1j * (al * P[:, 0] - be * P[:, 1])) - np.exp(1j * (al * P[:, 0] + be * P[:, 1]))
    assert np.max(np.abs(got - exact)) < 1e-4


def test_field_argument_errors_and_empty_call():
    par = I.wl_sinusoid_dirichlet(N=256)
    op = sgf.Operator(par)
    mu = torch.from_numpy(I.random_density(256, 1)).cuda()
    u = torch.zeros(4, dtype=torch.complex128, device="cuda")
    sgf.sgf_field(op.ctx, mu.data_ptr(), np.zeros((0, 2)), u.data_ptr())  # nothing to do
    x, f, _, _ = dr.nodes(par)
    for bad in ([[0.3, par["hmin"] - 0.1]], [[np.nan, 0.5]], [[x[7], f[7]]]):  # below, NaN, on a node
        with pytest.raises(sgf.SgfError) as e:
            sgf.sgf_field(op.ctx, mu.data_ptr(), np.array(bad), u.data_ptr())
        assert e.value.status == 1
    op.close()


def test_full_size_deep_corrugation_sampled_targets():
    # the N = 16384 Neumann workload (128 x 256 cells): targets in the grooves, in empty cells and
    # above the box against the oracle's direct sum and Rayleigh form for a random density
    par = I.wl_deep_corrugation_neumann()
    mu = I.random_density(par["N"], 13)
    rng = np.random.default_rng(6)
    xs = rng.uniform(0, par["d"], 3)
    P = np.stack([xs, dr.profile(par, xs)[0] + 0.3], 1)  # 0.3 above the surface (4 cells)
    top = par["hmin"] + par["ny"] * par["L"]
    P = np.concatenate([P, [[2.5, top - 0.01], [7.0, top + 0.2]]])
    op = sgf.Operator(par, precision=32)
    got = _field(op, mu, P)
    op.close()
    ref = fl.field_direct(par, mu, P)
    assert np.max(np.abs(got - ref)) < 2e-4 * np.max(np.abs(ref))
    assert abs(got[-1] - ref[-1]) < 1e-10 * abs(ref[-1])
