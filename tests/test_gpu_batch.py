"""Batches of independent problems (sgf_batch_*): the batched forward map against each problem's own
sgf_apply and against the oracle, the lockstep batched GMRES against single solves and against the
flat-surface closed form at several incidence angles, and the batch's argument checks.

Tolerances: a batch runs each problem's captured forward map unchanged, so outputs agree with the
single-problem path up to the summation order of the atomic scatter (1e-13). Solutions agree with
single solves to the solver tolerance times the condition number (1e-9 FP64; 1e-6 mixed).
"""
import numpy as np
import pytest

from oracle import accel as ac, direct as dr
from paper_1707_04950_gb300 import inputs as I

pytestmark = pytest.mark.gpu

sgf = pytest.importorskip("paper_1707_04950_gb300.sgf")
torch = pytest.importorskip("torch")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def _single_apply(op, x):
    xt, yt = _dev(x), torch.empty(len(x), dtype=torch.complex128, device="cuda")
    sgf.sgf_apply(op.ctx, xt.data_ptr(), yt.data_ptr(), 1, 0)
    torch.cuda.synchronize()
    return yt.cpu().numpy()


def _problems():
    return [(I.wl_sinusoid_dirichlet(N=512), 64),
            (I.wl_sinusoid_dirichlet(N=400), 64),
            (I.wl_deep_corrugation_neumann_small(N=1024, nx=32), 32)]


def test_batch_apply_matches_single_applies_and_oracle():
    probs = _problems()
    ops = [sgf.Operator(par, precision=prec) for par, prec in probs]
    xs = [_dev(I.random_density(op.par["N"], 20 + p)) for p, op in enumerate(ops)]
    ys = [torch.empty_like(x) for x in xs]
    b = sgf.sgf_batch_create([op.ctx for op in ops])
    try:
        sgf.sgf_batch_apply(b, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys])
        torch.cuda.synchronize()
        # a second launch with the outputs as inputs: the per-call pointer tables are rebound
        zs = [torch.empty_like(x) for x in xs]
        sgf.sgf_batch_apply(b, [y.data_ptr() for y in ys], [z.data_ptr() for z in zs])
        torch.cuda.synchronize()
    finally:
        sgf.sgf_batch_destroy(b)
    for (_, prec), op, x, y, z in zip(probs, ops, xs, ys, zs):
        # FP64: rounding order of the atomic scatter only; mixed: the FP32 scatter's rounding order,
        # amplified by the far-field/local-subtraction cancellation (the mixed path's own error)
        tol = 1e-13 if prec == 64 else 1e-5
        ref = _single_apply(op, x.cpu().numpy())
        assert _rel(y.cpu().numpy(), ref) < tol
        assert _rel(z.cpu().numpy(), _single_apply(op, ref)) < 100 * tol
    par = ops[0].par
    ref = ac.Accel(par).apply(xs[0].cpu().numpy())
    assert _rel(ys[0].cpu().numpy(), ref) < 1e-10
    for op in ops:
        op.close()


def _single_solve(op):
    mu = torch.zeros(op.par["N"], dtype=torch.complex128, device="cuda")
    st, its, rr = sgf.sgf_solve(op.ctx, 1e-12, 2000, mu.data_ptr())
    assert st == 0
    return mu.cpu().numpy()


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_solve_matches_single_solves(mixed):
    probs = [(I.wl_sinusoid_dirichlet(N=512), 64), (I.wl_sinusoid_dirichlet(N=256), 64),
             (I.flat(N=256, d=1.0, theta_deg=20.0, bc=1, nx=8, n_per=80), 64)]
    if mixed:
        probs = [(par, 32) for par, _ in probs]
    ops = [sgf.Operator(par, precision=prec) for par, prec in probs]
    mus = [torch.zeros(op.par["N"], dtype=torch.complex128, device="cuda") for op in ops]
    b = sgf.sgf_batch_create([op.ctx for op in ops])
    try:
        st, its, rr = sgf.sgf_batch_solve(b, 1e-12, 2000, [m.data_ptr() for m in mus])
        msg = sgf.load().sgf_batch_last_error(b)
    finally:
        sgf.sgf_batch_destroy(b)
    assert st == 0, (msg, its, rr)
    assert np.all(rr <= 1e-12) and all(i > 0 for i in its)
    for op, m in zip(ops, mus):
        ref = _single_solve(op)
        assert _rel(m.cpu().numpy(), ref) < (1e-6 if mixed else 1e-9)
        op.close()


def test_batch_of_angles_flat_surface_closed_form():
    # one surface, several incidence angles (independent problems): mu = c e^{i alpha x} with the
    # closed-form c of the shifted system on a flat surface, within the accelerator's error
    angles = [5.0, 20.0, 35.0, 50.0]
    pars = [I.flat(N=256, d=1.0, theta_deg=t, bc=0, nx=8, n_per=80) for t in angles]
    ops = [sgf.Operator(par) for par in pars]
    mus = [torch.zeros(256, dtype=torch.complex128, device="cuda") for _ in ops]
    b = sgf.sgf_batch_create([op.ctx for op in ops])
    try:
        st, its, rr = sgf.sgf_batch_solve(b, 1e-12, 2000, [m.data_ptr() for m in mus])
    finally:
        sgf.sgf_batch_destroy(b)
    assert st == 0
    for par, op, m in zip(pars, ops, mus):
        al, be = dr.wave(par)
        x = dr.nodes(par)[0]
        _, Ueta = dr.mode_sets(par)
        q = (1 - np.exp(1j * be * par["h"])) ** par["j"]
        c = -1 / (q / 2 + (par["d"] if 0 in set(np.atleast_1d(Ueta).tolist()) else 0.0))
        assert np.max(np.abs(m.cpu().numpy() - c * np.exp(1j * al * x))) < 1e-4 * abs(c)
        op.close()


def test_batch_argument_errors():
    par = I.wl_sinusoid_dirichlet(N=256)
    op = sgf.Operator(par)
    with pytest.raises(sgf.SgfError) as e:
        sgf.sgf_batch_create([])
    assert e.value.status == 1
    with pytest.raises(sgf.SgfError) as e:
        sgf.sgf_batch_create([op.ctx, op.ctx])  # the same problem twice
    assert e.value.status == 1
    ctx = sgf.sgf_create(0)
    try:
        with pytest.raises(sgf.SgfError) as e:
            sgf.sgf_batch_create([op.ctx, ctx])  # not built
        assert e.value.status == 10
    finally:
        sgf.sgf_destroy(ctx)
    b = sgf.sgf_batch_create([op.ctx])
    try:
        with pytest.raises(sgf.SgfError) as e:
            sgf.sgf_batch_apply(b, [0], [0])
        assert e.value.status == 1
    finally:
        sgf.sgf_batch_destroy(b)
    op.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_angle_batch_shares_the_near_operator(prec):
    # one surface at several incidence angles: the batch applies one shared near-field pass (the
    # blocks differ only by the phase of their period copy) and must agree with each problem's own
    # forward map up to summation order (FP64 1e-12; mixed: the FP32 far field's rounding, 1e-5);
    # ten angles exercise more than one group of eight in the shared kernel
    thetas = [30.0, 10.0, 45.0, 60.0, 5.0, 20.0, 35.0, 50.0, 15.0, 25.0] if prec == 64 else [30.0, 10.0, 45.0]
    pars = [I.make_params(I.sinusoid(2.0, 0.25), 2 * np.pi, t, 0, 512, nx=16, ny=16, hmin=-1.0) for t in thetas]
    ops = [sgf.Operator(par, precision=prec) for par in pars]
    xs = [_dev(I.random_density(512, 40 + p)) for p in range(len(ops))]
    ys = [torch.empty_like(x) for x in xs]
    import os

    os.environ["SGF_BATCH_SHARED"] = "1"  # force the shared form (creation otherwise keeps the faster)
    os.environ["SGF_BATCH_MULTI"] = "0"
    try:
        b = sgf.sgf_batch_create([op.ctx for op in ops])
    finally:
        del os.environ["SGF_BATCH_SHARED"]
        del os.environ["SGF_BATCH_MULTI"]
    try:
        assert sgf.sgf_batch_shared_near(b) == 1
        sgf.sgf_batch_apply(b, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys])
        torch.cuda.synchronize()
        mus = [torch.zeros(512, dtype=torch.complex128, device="cuda") for _ in ops]
        # 1e-11: at 35 degrees the system's attainable relative residual is ~1.2e-12
        st, its, rr = sgf.sgf_batch_solve(b, 1e-11, 2000, [m.data_ptr() for m in mus])
    finally:
        sgf.sgf_batch_destroy(b)
    assert st == 0 and np.all(rr <= 1e-11)
    tol = 1e-12 if prec == 64 else 1e-5
    for op, x, y, m in zip(ops, xs, ys, mus):
        assert _rel(y.cpu().numpy(), _single_apply(op, x.cpu().numpy())) < tol
        ref = torch.zeros(512, dtype=torch.complex128, device="cuda")
        assert sgf.sgf_solve(op.ctx, 1e-11, 2000, ref.data_ptr())[0] == 0
        assert _rel(m.cpu().numpy(), ref.cpu().numpy()) < (1e-8 if prec == 64 else 1e-6)
        op.close()
    # problems on different surfaces do not share
    o1, o2 = sgf.Operator(I.wl_sinusoid_dirichlet(N=512)), sgf.Operator(I.wl_sinusoid_dirichlet(N=400))
    b = sgf.sgf_batch_create([o1.ctx, o2.ctx])
    try:
        assert not sgf.sgf_batch_shared_near(b)
    finally:
        sgf.sgf_batch_destroy(b)
    o1.close()
    o2.close()


def _maxrel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("prec", [64, 32])
def test_angle_batch_multi_column_form(prec):
    # one surface at ten incidence angles in the multi-column form (two passes of at most eight
    # columns): the first problem's P, near operator and reconstruction rows serve every angle, with
    # each angle's twists, spectra and mode factors. Every angle must match its own forward map
    # (FP64 1e-11 element-wise: the alpha phases are formed as a product of the first angle's and a
    # relative one; mixed: the FP32 far field's summation order, 5e-5) and the oracle's Algorithm 3
    # built for that angle (1e-9 / 5e-5 element-wise)
    import os

    thetas = [30.0, 10.0, 45.0, 60.0, 5.0, 20.0, 35.0, 50.0, 15.0, 25.0]
    pars = [I.make_params(I.sinusoid(2.0, 0.25), 2 * np.pi, t, 0, 512, nx=16, ny=16, hmin=-1.0) for t in thetas]
    ops = [sgf.Operator(par, precision=prec) for par in pars]
    xs = [_dev(I.random_density(512, 60 + p)) for p in range(len(ops))]
    ys = [torch.empty_like(x) for x in xs]
    os.environ["SGF_BATCH_MULTI"] = "1"
    try:
        b = sgf.sgf_batch_create([op.ctx for op in ops])
    finally:
        del os.environ["SGF_BATCH_MULTI"]
    try:
        assert sgf.sgf_batch_shared_near(b) == 2
        sgf.sgf_batch_apply(b, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys])
        torch.cuda.synchronize()
        mus = [torch.zeros(512, dtype=torch.complex128, device="cuda") for _ in ops]
        st, its, rr = sgf.sgf_batch_solve(b, 1e-11, 2000, [m.data_ptr() for m in mus])
    finally:
        sgf.sgf_batch_destroy(b)
    assert st == 0 and np.all(rr <= 1e-11)
    tol = 1e-11 if prec == 64 else 5e-5
    for p, (op, x, y, m) in enumerate(zip(ops, xs, ys, mus)):
        yh = y.cpu().numpy()
        assert _maxrel(yh, _single_apply(op, x.cpu().numpy())) < tol, p
        if p in (0, 3, 9):
            ref = ac.Accel(pars[p]).apply(x.cpu().numpy())
            assert _maxrel(yh, ref) < (1e-9 if prec == 64 else 5e-5), p
        sol = torch.zeros(512, dtype=torch.complex128, device="cuda")
        assert sgf.sgf_solve(op.ctx, 1e-11, 2000, sol.data_ptr())[0] == 0
        assert _rel(m.cpu().numpy(), sol.cpu().numpy()) < (1e-8 if prec == 64 else 1e-6)
        op.close()
