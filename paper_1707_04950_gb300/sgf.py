"""ctypes binding of the sgf C ABI (include/sgf.h): argument marshalling only.

Every function keeps the C name. Device buffers are passed as integer addresses (for example
`tensor.data_ptr()` of a torch complex128 CUDA tensor); host buffers as numpy arrays. The binding
raises SgfError on any non-zero status and never falls back to another implementation: if the
library is not built, loading fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsgf.so")

STATUS = {0: "SGF_OK", 1: "SGF_EINVAL", 2: "SGF_ERESONANT_CELL", 3: "SGF_EPOLE_ON_GRID", 4: "SGF_EWINDOW",
          5: "SGF_ENOCONV", 6: "SGF_EBREAKDOWN", 7: "SGF_ENONFINITE", 8: "SGF_ETIMEOUT", 9: "SGF_ECUDA",
          10: "SGF_ESTATE"}

EXPORTED = ["sgf_create", "sgf_destroy", "sgf_last_error", "sgf_set_profile_fourier", "sgf_set_wave",
            "sgf_set_params", "sgf_build_operator", "sgf_apply", "sgf_apply_host", "sgf_rhs", "sgf_solve", "sgf_solve_rhs",
            "sgf_rayleigh", "sgf_rayleigh_noalloc", "sgf_field", "sgf_build_exact", "sgf_select_operator",
            "sgf_exact_matrix", "sgf_suggest_params", "sgf_gradient", "sgf_gradient_fd", "sgf_get_params", "sgf_autotune_cells", "sgf_info", "sgf_set_profiling", "sgf_stage_times", "sgf_debug_mask", "sgf_debug_table",
            "sgf_debug_force_variants", "sgf_autotune",
            "sgf_batch_create", "sgf_batch_destroy", "sgf_batch_last_error", "sgf_batch_apply", "sgf_batch_solve",
            "sgf_batch_shared_near"]


class SgfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class sgf_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("j", ctypes.c_int), ("h", ctypes.c_double), ("n_per", ctypes.c_int),
                ("c_win", ctypes.c_double), ("Ma", ctypes.c_int), ("eta", ctypes.c_double),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("hmin", ctypes.c_double), ("p", ctypes.c_int),
                ("e", ctypes.c_int), ("n_coll", ctypes.c_int), ("n_fb", ctypes.c_int),
                ("delta_min", ctypes.c_double), ("spec_exp", ctypes.c_double), ("precision", ctypes.c_int),
                ("ls_reg", ctypes.c_double)]


_lib = None


def load():
    """Load libsgf.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"sgf library not built: {LIB_PATH} (run python -m paper_1707_04950_gb300.build)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, d, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
    sig = {
        "sgf_create": [ctypes.POINTER(vp), i, vp],
        "sgf_set_profile_fourier": [vp, d, i, dp, dp],
        "sgf_set_wave": [vp, d, d, i],
        "sgf_set_params": [vp, ctypes.POINTER(sgf_params)],
        "sgf_build_operator": [vp],
        "sgf_apply": [vp, vp, vp, i, i],
        "sgf_apply_host": [vp, vp, vp, i],
        "sgf_rhs": [vp, vp],
        "sgf_solve": [vp, d, i, vp, ctypes.POINTER(i), dp],
        "sgf_solve_rhs": [vp, vp, i, d, i, vp, ctypes.POINTER(i), dp],
        "sgf_rayleigh": [vp, vp, i, i, dp, dp, dp],
        "sgf_field": [vp, vp, ctypes.c_long, dp, vp, i],
        "sgf_build_exact": [vp],
        "sgf_suggest_params": [d, i, dp, dp, d, d, i, d, i, ctypes.POINTER(sgf_params)],
        "sgf_select_operator": [vp, i],
        "sgf_exact_matrix": [vp, vp],
        "sgf_rayleigh_noalloc": [vp, vp, i, i, dp, dp, dp],
        "sgf_gradient": [vp, vp, i, d, i, dp, dp, dp, dp, ctypes.POINTER(i)],
        "sgf_gradient_fd": [vp, vp, i, d, i, dp, dp, dp, dp, ctypes.POINTER(i)],
        "sgf_get_params": [vp, ctypes.POINTER(sgf_params)],
        "sgf_autotune_cells": [vp, ctypes.POINTER(i), i, i, ctypes.POINTER(i), dp],
        "sgf_autotune": [vp, ctypes.POINTER(i), i, i, d, ctypes.POINTER(i), dp, dp],
        "sgf_info": [vp, dp],
        "sgf_set_profiling": [vp, i],
        "sgf_stage_times": [vp, dp],
        "sgf_debug_mask": [vp, i],
        "sgf_debug_table": [vp, i, i, vp],
        "sgf_debug_force_variants": [vp, i, i],
        "sgf_batch_create": [ctypes.POINTER(vp), i, ctypes.POINTER(vp), vp],
        "sgf_batch_apply": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp)],
        "sgf_batch_solve": [vp, d, i, ctypes.POINTER(vp), ctypes.POINTER(i), dp],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.sgf_destroy.argtypes = [vp]
    lib.sgf_destroy.restype = None
    lib.sgf_last_error.argtypes = [vp]
    lib.sgf_last_error.restype = ctypes.c_char_p
    lib.sgf_batch_destroy.argtypes = [vp]
    lib.sgf_batch_destroy.restype = None
    lib.sgf_batch_last_error.argtypes = [vp]
    lib.sgf_batch_last_error.restype = ctypes.c_char_p
    lib.sgf_batch_shared_near.argtypes = [vp]
    lib.sgf_batch_shared_near.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(ctx, st):
    if st != 0:
        msg = load().sgf_last_error(ctx)
        raise SgfError(st, msg.decode() if msg else "")


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# ------------------------------------------------------------------ C-named wrappers
def sgf_create(device=0, stream=0):
    lib = load()
    ctx = ctypes.c_void_p()
    st = lib.sgf_create(ctypes.byref(ctx), int(device), ctypes.c_void_p(stream or None))
    _check(ctx, st)
    return ctx


def sgf_destroy(ctx):
    load().sgf_destroy(ctx)


def sgf_set_profile_fourier(ctx, d, a, b):
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    assert a.shape == b.shape
    _check(ctx, load().sgf_set_profile_fourier(ctx, float(d), len(a) - 1, _dptr(a), _dptr(b)))


def sgf_set_wave(ctx, k, theta, bc):
    _check(ctx, load().sgf_set_wave(ctx, float(k), float(theta), int(bc)))


def sgf_set_params(ctx, p: sgf_params):
    _check(ctx, load().sgf_set_params(ctx, ctypes.byref(p)))


def sgf_build_operator(ctx):
    _check(ctx, load().sgf_build_operator(ctx))


def sgf_apply(ctx, mu_ptr, out_ptr, nrhs=1, transpose_conj=0):
    _check(ctx, load().sgf_apply(ctx, ctypes.c_void_p(mu_ptr), ctypes.c_void_p(out_ptr), int(nrhs), int(transpose_conj)))


def sgf_apply_host(ctx, mu, out, nrhs=1):
    assert mu.dtype == np.complex128 and out.dtype == np.complex128
    assert mu.flags.c_contiguous and out.flags.c_contiguous
    _check(ctx, load().sgf_apply_host(ctx, mu.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p),
                                      int(nrhs)))


def sgf_apply_host_ptr(ctx, mu_host_ptr, out_host_ptr, nrhs=1):
    """sgf_apply_host on raw host addresses (e.g. pinned torch CPU tensors)."""
    _check(ctx, load().sgf_apply_host(ctx, ctypes.c_void_p(mu_host_ptr), ctypes.c_void_p(out_host_ptr), int(nrhs)))


def sgf_rhs(ctx, out_ptr):
    _check(ctx, load().sgf_rhs(ctx, ctypes.c_void_p(out_ptr)))


def sgf_solve(ctx, tol, maxit, mu_ptr):
    its = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    st = load().sgf_solve(ctx, float(tol), int(maxit), ctypes.c_void_p(mu_ptr), ctypes.byref(its), ctypes.byref(rr))
    return st, its.value, rr.value


def sgf_solve_rhs(ctx, rhs_ptr, transpose_conj, tol, maxit, x_ptr):
    its = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    st = load().sgf_solve_rhs(ctx, ctypes.c_void_p(rhs_ptr), int(transpose_conj), float(tol), int(maxit),
                              ctypes.c_void_p(x_ptr), ctypes.byref(its), ctypes.byref(rr))
    return st, its.value, rr.value


def sgf_rayleigh(ctx, mu_ptr, n_lo, n_hi):
    n = n_hi - n_lo + 1
    B = np.zeros(2 * n)
    eff = np.zeros(n)
    err = np.zeros(1)
    _check(ctx, load().sgf_rayleigh(ctx, ctypes.c_void_p(mu_ptr), int(n_lo), int(n_hi), _dptr(B), _dptr(eff), _dptr(err)))
    return B[0::2] + 1j * B[1::2], eff, float(err[0])


def sgf_field(ctx, mu_ptr, xy, u_ptr, total=False):
    """Scattered (total=True: total) field at the points xy [n, 2] (host array) into u_ptr (device
    complex128 [n])."""
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64).reshape(-1, 2))
    _check(ctx, load().sgf_field(ctx, ctypes.c_void_p(mu_ptr), len(xy), _dptr(xy), ctypes.c_void_p(u_ptr),
                                 1 if total else 0))


def sgf_suggest_params(d, a, b, k, theta, bc, tol, precision=64):
    """Suggested sgf_params for a profile (cosine/sine coefficients a, b), a wave and a target
    accuracy (host only). Returns the ctypes record."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    p = sgf_params()
    st = load().sgf_suggest_params(float(d), len(a) - 1, _dptr(a), _dptr(b), float(k), float(theta), int(bc),
                                   float(tol), int(precision), ctypes.byref(p))
    if st == 5:  # SGF_ENOCONV: the record is filled; the error carries it
        e = SgfError(st, f"sgf_suggest_params: the windowed lattice sums do not reach {tol:g} by n_per = 16384")
        e.params = p
        raise e
    if st != 0:
        raise SgfError(st, "sgf_suggest_params: argument out of range")
    return p


def sgf_build_exact(ctx):
    _check(ctx, load().sgf_build_exact(ctx))


def sgf_select_operator(ctx, exact):
    _check(ctx, load().sgf_select_operator(ctx, 1 if exact else 0))


def sgf_exact_matrix(ctx, A_ptr):
    _check(ctx, load().sgf_exact_matrix(ctx, ctypes.c_void_p(A_ptr)))


def sgf_gradient(ctx, mu_ptr, n, M, tol=1e-12, maxit=2000, fd=False):
    """d e_n / d(a_m, b_m), m = 0..M (M = number of profile harmonics); returns (grad_a, grad_b, B_n,
    e_n, adjoint iterations). fd=True calls sgf_gradient_fd (difference-quotient node derivatives)."""
    ga = np.zeros(M + 1)
    gb = np.zeros(M + 1)
    B = np.zeros(2)
    en = np.zeros(1)
    its = ctypes.c_int(0)
    fn = load().sgf_gradient_fd if fd else load().sgf_gradient
    _check(ctx, fn(ctx, ctypes.c_void_p(mu_ptr), int(n), float(tol), int(maxit), _dptr(B), _dptr(en), _dptr(ga),
                   _dptr(gb), ctypes.byref(its)))
    return ga, gb, B[0] + 1j * B[1], float(en[0]), its.value


def sgf_get_params(ctx):
    p = sgf_params()
    _check(ctx, load().sgf_get_params(ctx, ctypes.byref(p)))
    return p


def sgf_autotune_cells(ctx, nx_list, reps=20):
    """Returns (best nx, per-candidate ms per application or minus the build status)."""
    arr = (ctypes.c_int * len(nx_list))(*[int(x) for x in nx_list])
    best = ctypes.c_int(0)
    ms = np.zeros(len(nx_list))
    _check(ctx, load().sgf_autotune_cells(ctx, arr, len(nx_list), int(reps), ctypes.byref(best), _dptr(ms)))
    return best.value, ms


def sgf_autotune(ctx, nx_list, eps_tol, reps=20):
    """Accuracy-aware tuning: returns (status, best nx, ms per application, energy error per
    candidate). Status 5 (SGF_ENOCONV): no candidate reached eps_tol; the most accurate is kept."""
    arr = (ctypes.c_int * len(nx_list))(*[int(x) for x in nx_list])
    best = ctypes.c_int(0)
    ms = np.zeros(len(nx_list))
    eps = np.zeros(len(nx_list))
    st = load().sgf_autotune(ctx, arr, len(nx_list), int(reps), float(eps_tol), ctypes.byref(best), _dptr(ms),
                             _dptr(eps))
    if st not in (0, 5):
        _check(ctx, st)
    return st, best.value, ms, eps


def sgf_rayleigh_noalloc(ctx, mu_ptr, n_lo, n_hi):
    """sgf_rayleigh without allocation (static device scratch, at most 1024 modes per call)."""
    n = n_hi - n_lo + 1
    B = np.zeros(2 * n)
    eff = np.zeros(n)
    err = np.zeros(1)
    _check(ctx, load().sgf_rayleigh_noalloc(ctx, ctypes.c_void_p(mu_ptr), int(n_lo), int(n_hi), _dptr(B), _dptr(eff),
                                            _dptr(err)))
    return B[0::2] + 1j * B[1::2], eff, float(err[0])


def _bcheck(batch, st):
    if st != 0:
        msg = load().sgf_batch_last_error(batch)
        raise SgfError(st, msg.decode() if msg else "")


def _ptrs(seq):
    return (ctypes.c_void_p * len(seq))(*[ctypes.c_void_p(int(x)) for x in seq])


def sgf_batch_create(ctxs, stream=0):
    lib = load()
    b = ctypes.c_void_p()
    arr = (ctypes.c_void_p * len(ctxs))(*[c.value if isinstance(c, ctypes.c_void_p) else c for c in ctxs])
    st = lib.sgf_batch_create(ctypes.byref(b), len(ctxs), arr, ctypes.c_void_p(stream or None))
    if st != 0:
        msg = lib.sgf_batch_last_error(b)
        lib.sgf_batch_destroy(b)
        raise SgfError(st, msg.decode() if msg else "")
    return b


def sgf_batch_destroy(batch):
    load().sgf_batch_destroy(batch)


def sgf_batch_shared_near(batch):
    """The batch's form: 0 child graphs, 1 shared near pass, 2 multi-column (sgf.h)."""
    return int(load().sgf_batch_shared_near(batch))


def sgf_batch_apply(batch, mu_ptrs, out_ptrs):
    _bcheck(batch, load().sgf_batch_apply(batch, _ptrs(mu_ptrs), _ptrs(out_ptrs)))


def sgf_batch_solve(batch, tol, maxit, mu_ptrs):
    n = len(mu_ptrs)
    its = (ctypes.c_int * n)()
    rr = np.zeros(n)
    st = load().sgf_batch_solve(batch, float(tol), int(maxit), _ptrs(mu_ptrs), its, _dptr(rr))
    return st, list(its), rr


INFO_KEYS = ["N", "n_occ", "nnz", "PxH", "nrowH", "PyH", "PxV", "nrowV", "PyV", "neq", "nfit", "nb", "nm",
             "bytes64", "bytes32", "launches", "graphs", "maxW", "maxnq", "twlog",
             "build_ms", "build_tables_ms", "build_ls_ms", "build_near_ms"]


def sgf_info(ctx):
    v = np.zeros(24)
    _check(ctx, load().sgf_info(ctx, _dptr(v)))
    return dict(zip(INFO_KEYS, v.tolist()))


def sgf_set_profiling(ctx, on):
    _check(ctx, load().sgf_set_profiling(ctx, int(on)))


def sgf_stage_times(ctx):
    v = np.zeros(8)
    _check(ctx, load().sgf_stage_times(ctx, _dptr(v)))
    return v


def sgf_debug_mask(ctx, mask):
    _check(ctx, load().sgf_debug_mask(ctx, int(mask)))


def sgf_debug_force_variants(ctx, conv_variant, fftx_vpt):
    _check(ctx, load().sgf_debug_force_variants(ctx, int(conv_variant), int(fftx_vpt)))


def sgf_debug_table(ctx, lam, kind, shape):
    out = np.zeros(shape, dtype=np.complex128)
    _check(ctx, load().sgf_debug_table(ctx, int(lam), int(kind), out.ctypes.data_as(ctypes.c_void_p)))
    return out


# ------------------------------------------------------------------ convenience
def params_from(par, precision=None) -> sgf_params:
    """C parameter record from a workload dictionary (paper_1707_04950_gb300.inputs)."""
    return sgf_params(N=par["N"], j=par["j"], h=par["h"], n_per=par["n_per"], c_win=par["c_win"], Ma=par["Ma"],
                      eta=par["eta"], nx=par["nx"], ny=par["ny"], hmin=par["hmin"], p=par["p"], e=par["e"],
                      n_coll=par["n_coll"], n_fb=par["n_fb"], delta_min=par["delta_min"],
                      spec_exp=par["spec_exp"], precision=int(precision or par["precision"]),
                      ls_reg=par["ls_reg"])


class Operator:
    """One built operator: sgf_create + setters + sgf_build_operator on a workload dictionary."""

    def __init__(self, par, device=0, stream=0, precision=None):
        self.par = par
        self.ctx = sgf_create(device, stream)
        try:
            sgf_set_profile_fourier(self.ctx, par["d"], par["a"], par["b"])
            sgf_set_wave(self.ctx, par["k"], par["theta"], par["bc"])
            sgf_set_params(self.ctx, params_from(par, precision))
            sgf_build_operator(self.ctx)
        except Exception:
            sgf_destroy(self.ctx)
            self.ctx = None
            raise
        self.info = sgf_info(self.ctx)

    def close(self):
        if self.ctx is not None:
            sgf_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
