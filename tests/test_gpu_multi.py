"""Several densities through one operator in one pass (sgf_apply with nrhs > 1): the projection,
near rows and reconstruction read the operator data once for up to 8 columns, and the X passes and
Y convolutions run all columns' grids per launch. Each column must equal the single-density map
(FP64: the same arithmetic up to the order of the atomic scatter, 1e-12; mixed: the FP32 far field
summed in another order, whose element-wise error against the oracle is already 1.0e-5 to 1.5e-5 on
the deep Neumann case, so 5e-5) and the oracle's Algorithm 3 on a block of columns (the
element-wise parity bounds of the single map: 1e-9 FP64, 5e-5 mixed). 11 columns cross a pass
boundary.
"""
import numpy as np
import pytest

from oracle import accel as ac
from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")
torch = pytest.importorskip("torch")

CASES = {
    "sinusoid_dirichlet_wood_n512": lambda: I.wl_sinusoid_dirichlet(N=512),
    "deep_neumann_n1024": lambda: I.wl_deep_corrugation_neumann_small(N=1024, nx=32),
}
_acc = {}


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _block(par, nr, seed0=40):
    return np.stack([I.random_density(par["N"], seed0 + r) for r in range(nr)], 1)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [64, 32])
def test_columns_match_single_applications_and_oracle(name, prec):
    par = CASES[name]()
    nr = 11
    X = _block(par, nr)
    op = sgf.Operator(par, precision=prec)
    xt = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()  # column r at offset r N
    yt = torch.empty_like(xt)
    sgf.sgf_apply(op.ctx, xt.data_ptr(), yt.data_ptr(), nr, 0)
    Y = yt.cpu().numpy().T
    Y1 = np.zeros_like(X)
    for r in range(nr):
        y1 = torch.empty_like(xt[r])
        sgf.sgf_apply(op.ctx, xt[r].data_ptr(), y1.data_ptr(), 1, 0)
        Y1[:, r] = y1.cpu().numpy()
    op.close()
    assert _maxrel(Y, Y1) < (1e-12 if prec == 64 else 5e-5)
    if name not in _acc:
        _acc[name] = ac.Accel(par)
    ref = _acc[name].apply(X)
    assert _maxrel(Y, ref) < (1e-9 if prec == 64 else 5e-5)
