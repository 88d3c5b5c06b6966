"""The exact Nystrom system of the deep corrugation (depth/period 2, TM) under the reading the
benchmark uses: the periodic Green function without shifts (j = 0), as the paper does for its deep
non-Wood gratings (Section 6, Table deep_gratings, "G^qper_0 eval.").

What pins it: on this shape the unshifted exact system is well conditioned and its energy balance
(eq. energy_error) converges with N, while the shifted kernel (j = 8, h ~ lambda/2) makes the same
exact system nearly singular (Section 6.1: shifted sources close to a deep surface cause
ill-conditioning). The condition grows like |1 - e^{ikh}|^j-scaled images of vertically separated
node pairs; measured on the period-10 benchmark geometry (N = 1024): j = 0 4.7e2, j = 2 9.8e3,
j = 4 8.3e6, j = 8 (h = lambda) 5.0e9. So the stalled GMRES of the shifted formulation there is a
property of the exact system, not of the accelerator.
"""
import numpy as np
import pytest

from oracle import direct as dr
from paper_1707_04950_gb300 import inputs as I


def _solve(par):
    A = dr.assemble(par)
    mu = np.linalg.solve(A, dr.rhs(par))
    return A, dr.rayleigh(par, mu)[3]


@pytest.mark.slow
def test_unshifted_deep_corrugation_is_well_conditioned_and_converges_in_N():
    # period 2, depth 4 (the small parity shape); measured: cond 96, eps -1.8e-6 (N = 256) and
    # 2.3e-7 (N = 384)
    A, e256 = _solve(I.wl_deep_corrugation_neumann_small(N=256, nx=16, j=0, n_per=160))
    assert np.linalg.cond(A) < 2e2
    assert abs(e256) < 1e-5
    _, e384 = _solve(I.wl_deep_corrugation_neumann_small(N=384, nx=16, j=0, n_per=160))
    assert abs(e384) < abs(e256) / 4


@pytest.mark.slow
def test_shifted_kernel_makes_the_deep_exact_system_nearly_singular():
    # same shape, j = 8 at h ~ lambda/2: measured cond 1.35e7 and eps 0.14 at N = 256
    par = I.wl_deep_corrugation_neumann_small(N=256, nx=16, j=8, n_per=40)
    A = dr.assemble(par)
    assert np.linalg.cond(A) > 1e6
