"""Seeded synthetic workloads: surface profiles, incidences, accelerator parameters and densities.

This module is shared by the CUDA path's tests/bench and by the CPU oracle. It holds no arithmetic
of the scattering method itself: it only builds profile Fourier coefficients, picks the numerical
parameters of a run (cell grid, shift h, windows, ...) by the rules stated below, and draws random
complex densities. Both sides receive the resulting dictionary as input.

Profile convention: f(x) = a[0] + sum_{m>=1} a[m] cos(2 pi m x / d) + b[m] sin(2 pi m x / d).

Parameter rules (readings of the paper where it prints no value):
  * nodes x_l = l*dx, l = 1..N, dx = d/N (Section 4.2: x_0 = 0, x_N = d);
  * singular window a = floor(0.75 L / dx) dx (a < L, Remark a_cond), gamma = a/2, large window
    flat fraction c = 1/2 and A = n_per * d (Section 4.2.2);
  * shift h = (round(h0/dg) + 1/(j+1)) dg with dg = L/p the finest grid lag in Y: every shifted
    pole m h (1 <= m <= j) then stays at least dg/(j+1) away from a lag of the equivalent-source
    grids (Section 3.1 poles P_j); a half-integer offset would put 2h, 4h, ... on the grid;
  * spectral/spatial switch distance delta_min = d/64 (Section 3.2, estimate of the spectral decay);
  * eta = 1e-3 for the mode completion M^eta (Section 3.1);
  * ls_reg = 1e-6: Tikhonov weight (relative to |A|_F) of the equivalent-source least squares.
"""
from __future__ import annotations

import math
import numpy as np

DIRICHLET = 0
NEUMANN = 1


def profile_eval_host(prof, x):
    """f, f', f'' of a Fourier profile at points x (used only to choose the cell box)."""
    d = prof["d"]
    a = np.asarray(prof["a"], float)
    b = np.asarray(prof["b"], float)
    x = np.asarray(x, float)
    f = np.full_like(x, a[0])
    for m in range(1, len(a)):
        w = 2 * math.pi * m / d
        f += a[m] * np.cos(w * x) + b[m] * np.sin(w * x)
    return f


def sinusoid(d, amp, phase="cos"):
    a = np.zeros(2)
    b = np.zeros(2)
    if phase == "cos":
        a[1] = amp
    else:
        b[1] = amp
    return {"d": float(d), "a": a, "b": b}


def gaussian_surface(d, rms, corr_len, seed):
    """Gaussian random periodic surface with correlation exp(-x^2/lc^2).

    Spectrum W(K) = rms^2 lc /(2 sqrt(pi)) exp(-K^2 lc^2/4); complex amplitudes
    F_m = sqrt(pi W(K_m)/d) (g1 + i g2), F_{-m} = conj(F_m), F_0 = 0, |m| <= ceil(6 d /(pi lc)).
    Returned as cosine/sine coefficients a_m = 2 Re F_m, b_m = -2 Im F_m.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    M = int(math.ceil(6 * d / (math.pi * corr_len)))
    m = np.arange(1, M + 1)
    K = 2 * math.pi * m / d
    W = rms**2 * corr_len / (2 * math.sqrt(math.pi)) * np.exp(-(K**2) * corr_len**2 / 4)
    g = rng.standard_normal((M, 2))
    F = np.sqrt(math.pi * W / d) * (g[:, 0] + 1j * g[:, 1])
    a = np.zeros(M + 1)
    b = np.zeros(M + 1)
    a[1:] = 2 * F.real
    b[1:] = -2 * F.imag
    return {"d": float(d), "a": a, "b": b}


def harmonic_surface(d, n_harm, scale, seed):
    """sum_{m=1..n_harm} c_m cos + s_m sin with c_m, s_m ~ N(0, (scale/m)^2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = np.arange(1, n_harm + 1)
    g = rng.standard_normal((n_harm, 2))
    a = np.zeros(n_harm + 1)
    b = np.zeros(n_harm + 1)
    a[1:] = g[:, 0] * scale / m
    b[1:] = g[:, 1] * scale / m
    return {"d": float(d), "a": a, "b": b}


def make_params(prof, k, theta_deg, bc, N, *, j=8, h0=0.5, n_per=40, nx, ny=None, hmin=None,
                p=8, e=1, n_coll=200, n_fb=12, eta=1e-3, delta_min=None, spec_exp=40.0,
                c_win=0.5, precision=64, ls_reg=1e-6, h=None):
    """Assemble the full parameter record of one scattering problem. The shift h is h0 moved off the
    accelerator's grid lags unless given exactly (the dense operator has no grid)."""
    d = prof["d"]
    dx = d / N
    L = d / nx
    xs = dx * np.arange(1, N + 1)
    f = profile_eval_host(prof, xs)
    fmin, fmax = float(f.min()), float(f.max())
    if hmin is None:
        hmin = fmin - 0.5 * L
    if ny is None:
        ny = int(math.floor((fmax - hmin) / L)) + 1
    assert hmin < fmin and hmin + ny * L >= fmax, "cell box does not contain the profile"
    Ma = int(math.floor(0.75 * L / dx + 1e-9))
    a_s = Ma * dx
    dg = L / p
    if h is None:
        h = (round(h0 / dg) + 1.0 / (j + 1)) * dg
    if delta_min is None:
        delta_min = d / 64.0
    theta = math.radians(theta_deg)
    return {
        "d": d, "a": np.asarray(prof["a"], float), "b": np.asarray(prof["b"], float),
        "k": float(k), "theta": theta, "bc": int(bc), "N": int(N),
        "j": int(j), "h": float(h), "n_per": int(n_per), "c_win": float(c_win),
        "Ma": Ma, "a_s": float(a_s), "gamma": 0.5 * a_s, "eta": float(eta),
        "nx": int(nx), "ny": int(ny), "L": float(L), "hmin": float(hmin),
        "p": int(p), "e": int(e), "n_coll": int(n_coll), "n_fb": int(n_fb),
        "delta_min": float(delta_min), "spec_exp": float(spec_exp), "precision": int(precision),
        "ls_reg": float(ls_reg),
    }


# --------------------------------------------------------------------------------------------
# Named workloads (sizes and shapes of the paper's test problems; all synthetic)
# --------------------------------------------------------------------------------------------

def wl_sinusoid_dirichlet(N=512, nx=16, **kw):
    """Perfectly conducting sinusoid y = 0.25 cos(pi x), d = 2, k = 2 pi, theta = 30 deg
    (double Wood anomaly: alpha_n = pi (1 + n), beta_1 = beta_-3 = 0), 16x16 cells on [-1, 1)."""
    prof = sinusoid(2.0, 0.25)
    ny = kw.pop("ny", nx)
    hmin = kw.pop("hmin", -1.0)
    return make_params(prof, 2 * math.pi, 30.0, DIRICHLET, N, nx=nx, ny=ny, hmin=hmin, **kw)


def wl_sinusoid_dirichlet_energy(N=512, **kw):
    """The double-Wood sinusoid (wl_sinusoid_dirichlet) at the settings of its energy-balance run:
    n_per = 640 (the windowed sums converge like A^-3.5 at the anomaly, Lemma lemma_app_1: energy
    error of the exact system 2.1e-6 at n_per = 40, 1.3e-8 at 160, 8e-11 at 640) and the
    equivalent-source fit with e = 2 extra points per side end, n_coll = 196 collocation points
    and Tikhonov weight 1e-10: measured accelerated energy error -2.9e-9. The neighbouring settings
    (e in {1, 2, 3}, ls_reg in 3e-11..3e-10, n_coll in {160, 196, 200}) give 3e-9..8e-8, and
    e = 1 with ls_reg = 1e-6 4.4e-6: at 16 x 16 cells (k L = 0.79) the equivalent-source fit
    limits the accelerated operator to ~1e-8."""
    kw.setdefault("n_per", 640)
    kw.setdefault("ls_reg", 1e-10)
    kw.setdefault("e", 2)
    kw.setdefault("n_coll", 196)
    return wl_sinusoid_dirichlet(N=N, **kw)


def wl_gaussian_wood_energy(N=8192, **kw):
    """The Gaussian Wood surface (wl_gaussian_wood) at the settings of its energy-balance run:
    n_per = 1024 (the paper's scaling d n_per ~ 4e4 for its grazing rough surfaces), Tikhonov weight
    1e-10 and n_fb = 14 (measured accelerated energy error 3.9e-6; exact system 4.7e-10)."""
    kw.setdefault("n_per", 1024)
    kw.setdefault("ls_reg", 1e-10)
    kw.setdefault("n_fb", 14)
    return wl_gaussian_wood(N=N, **kw)


def wl_deep_corrugation_neumann(N=16384, nx=128, **kw):
    """Deep sinusoidal corrugation, depth/period = 2, period 10 (wavelength 1), TM (Neumann),
    theta = 45 deg, 128 cell columns (L = 10/128); one extra cell row so that half-open cells hold
    both the crest and the trough node.

    Away from Wood anomalies (the nearest, n = 3 and n = -17, have |beta_n| = 0.75 and 0.74) the
    unshifted periodic Green function is used (j = 0), as in the paper's deep-grating runs (Section 6,
    Table deep_gratings: "G^qper_0 eval."); Section 6.1 warns that shifted sources close to a deep
    surface make the system ill-conditioned. The j = 0 windowed lattice sum converges slowly here
    (n_per = 640: 3e-8, 1280: 5e-11 next to Y = 0), so n_per = 2048 (the parameter rule for 1e-8).
    Pass j = 8 (and n_per = 40) for the shifted kernel on the same geometry."""
    prof = sinusoid(10.0, 10.0)
    kw.setdefault("j", 0)
    kw.setdefault("n_per", 2048)
    # Tikhonov weight of the equivalent-source fit: measured energy error of the solution 7.2e-7
    # (1e-6), 9.9e-9 (1e-7), 4.4e-9 (1e-8), 4.9e-9 (1e-9), 7.4e-9 (1e-10)
    kw.setdefault("ls_reg", 1e-8)
    return make_params(prof, 2 * math.pi, 45.0, NEUMANN, N, nx=nx, **kw)


def wl_deep_corrugation_neumann_periods(r, **kw):
    """The deep corrugation repeated r times in one period of 10 r (N = 16384 r nodes, 128 r cell
    columns: the same shape, cell size and points per wavelength, r times the surface)."""
    a = np.zeros(r + 1)
    a[r] = 10.0
    prof = {"d": 10.0 * r, "a": a, "b": np.zeros(r + 1)}
    kw.setdefault("j", 0)
    kw.setdefault("n_per", 2048)
    kw.setdefault("ls_reg", 1e-8)
    return make_params(prof, 2 * math.pi, 45.0, NEUMANN, 16384 * r, nx=128 * r, **kw)


def wl_deep_corrugation_neumann_small(N=1024, nx=32, **kw):
    """Same shape as the deep corrugation (depth/period = 2) at period 2: the small parity case."""
    prof = sinusoid(2.0, 2.0)
    return make_params(prof, 2 * math.pi, 45.0, NEUMANN, N, nx=nx, **kw)


def wl_gaussian_wood(N=8192, nx=64, seed=2, **kw):
    """Gaussian rough surface rms 0.5, correlation length 2, period 40, theta = 85 deg at the
    Wood wavenumber k = 2 pi 80 /(40 (1 + sin 85 deg)) (alpha_-80 = -k)."""
    prof = gaussian_surface(40.0, 0.5, 2.0, seed)
    th = 85.0
    k = 2 * math.pi * 80 / (40.0 * (1 + math.sin(math.radians(th))))
    return make_params(prof, k, th, DIRICHLET, N, nx=nx, **kw)


def wl_gaussian_angles(i, N=2048, d=10.0, nx=32, surface_seed=5000, **kw):
    """One of the 64 problems of the multi-problem workload: Gaussian rough surface (rms 0.5,
    correlation length 2, period d), k = 2 pi, Dirichlet, incidence theta_i = 89 deg i / 63,
    i = 0..63 (theta = 0 is a Wood configuration for integer d)."""
    prof = gaussian_surface(d, 0.5, 2.0, surface_seed)
    return make_params(prof, 2 * math.pi, 89.0 * i / 63.0, DIRICHLET, N, nx=nx, **kw)


# The batched sweep: Gaussian rough surfaces (rms 0.5, correlation length 2) of periods 10, 25, 50,
# 100 with N = 2048, 4096, 8192, 16384, four surfaces per period (seeds 5000 + 4 i + s), each at 64
# incidence angles theta = 89 deg i / 63 (k = 2 pi) and at 16 Wood wavenumbers: for theta_w = 5 w
# deg (w = 1..16) the order n = -round(d (1 + sin theta_w)) meets alpha_n = -k exactly at
# k = 2 pi |n| / (d (1 + sin theta_w)). Cells: n_x the smallest power of two with L <= 0.45 lambda.
SWEEP_SURFACES = ((10.0, 2048), (25.0, 4096), (50.0, 8192), (100.0, 16384))


def sweep_nx(d, lam=1.0):
    nx = 4
    while d / nx > 0.45 * lam:
        nx *= 2
    return nx


def wl_sweep_angle(period_index, surface, i, **kw):
    """Problem i (0..63) of the angle sweep on surface `surface` (0..3) of period SWEEP_SURFACES[period_index]."""
    d, N = SWEEP_SURFACES[period_index]
    prof = gaussian_surface(d, 0.5, 2.0, 5000 + 4 * period_index + surface)
    return make_params(prof, 2 * math.pi, 89.0 * i / 63.0, DIRICHLET, N, nx=sweep_nx(d), **kw)


def wl_sweep_wood(period_index, surface, w, **kw):
    """Wood problem w (1..16) of the sweep: theta_w = 5 w deg at the wavenumber where alpha_n = -k."""
    d, N = SWEEP_SURFACES[period_index]
    prof = gaussian_surface(d, 0.5, 2.0, 5000 + 4 * period_index + surface)
    th = 5.0 * w
    n = -round(d * (1 + math.sin(math.radians(th))))
    k = 2 * math.pi * abs(n) / (d * (1 + math.sin(math.radians(th))))
    return make_params(prof, k, th, DIRICHLET, N, nx=sweep_nx(d, 2 * math.pi / k), **kw)


def wl_harmonic_gradient(N=4096, d=20.0, n_harm=64, scale=0.05, nx=64, seed=4, **kw):
    """Gradient workload: sum_{m <= 64} c_m cos + s_m sin with c_m, s_m ~ N(0, (0.05/m)^2), period 20,
    k = 2 pi, theta = 20 deg, Dirichlet; the efficiency e_0 is differentiated with respect to the
    128 coefficients."""
    prof = harmonic_surface(d, n_harm, scale, seed)
    return make_params(prof, 2 * math.pi, 20.0, DIRICHLET, N, nx=nx, **kw)


def wl_harmonic_gradient_small(N=256, d=2.0, n_harm=3, scale=0.05, nx=8, seed=4, bc=DIRICHLET, **kw):
    """The same kind of surface at period 2 with 3 harmonics: the small gradient parity case."""
    prof = harmonic_surface(d, n_harm, scale, seed)
    return make_params(prof, 2 * math.pi, 20.0, bc, N, nx=nx, **kw)


def wl_composite(N, n_per, wood=False, nx=32, **kw):
    """Composite surface f = -(sin x + sin 2x / 2 + sin 3x / 3 + sin 4x / 4) / 4, d = 2 pi, theta =
    45 deg, Dirichlet (the convergence study of Section 6.1): k = 20 with the unshifted Green function
    (j = 0), or the Wood wavenumber k = 6 / (1 - sin 45 deg) with j = 8 and h = 0.16. 32 cell columns
    keep the singular window a = 0.75 L below h / max|f'| (max|f'| = 1)."""
    prof = {"d": 2 * math.pi, "a": np.zeros(5), "b": -0.25 * np.array([0.0, 1.0, 1 / 2, 1 / 3, 1 / 4])}
    if wood:
        k = 6.0 / (1.0 - math.sin(math.radians(45.0)))
        kw.setdefault("j", 8)
        kw.setdefault("h", 0.16)
    else:
        k = 20.0
        kw.setdefault("j", 0)
    return make_params(prof, k, 45.0, DIRICHLET, N, n_per=n_per, nx=nx, **kw)


def wl_littrow(H_over_d, d_over_lambda, N, h_over_lambda, n_per, **kw):
    """Sinusoid f = (H/2) sin(2 pi x / d) in the Littrow mount of order -1 (sin theta = 1/3),
    Dirichlet, d = 2 pi so that k = d / lambda (the sinusoid tables of Section 6.2): j = 0 when
    h_over_lambda is 0 (non-Wood rows), else j = 8 with h = h_over_lambda lambda. For the dense
    operator: singular window a = min(lambda/2, 0.4 d), below 0.9 h / max|f'| when shifted."""
    d = 2 * math.pi
    k = float(d_over_lambda)
    lam = d / k
    H = H_over_d * d
    prof = {"d": d, "a": np.zeros(2), "b": np.array([0.0, H / 2])}
    shifted = h_over_lambda > 0
    a = min(0.5 * lam, 0.4 * d)
    if shifted:
        a = min(a, 0.9 * h_over_lambda * lam / (math.pi * H / d))
    par = make_params(prof, k, math.degrees(math.asin(1.0 / 3.0)), DIRICHLET, N, j=8 if shifted else 0,
                      h=h_over_lambda * lam if shifted else 0.5, n_per=n_per, nx=4, hmin=-H, ny=8, **kw)
    dx = d / N
    par["Ma"] = max(2, int(a / dx))
    par["a_s"] = par["Ma"] * dx
    par["gamma"] = 0.5 * par["a_s"]
    return par


def accel_table_params(prof, k, theta_deg, N, j, h, n_per, lam, maxslope, ls_reg=1e-10):
    """Accelerator parameters for one row of the paper's convergence and grating tables (Section
    6): cells of side L <= 0.45 lambda (n_x a power of two, at least 4), N rounded up to a multiple
    of n_x, the singular window a = 0.75 L, or less with shifts so that a max|f'| < 0.9 h."""
    d = prof["d"]
    nx = 4
    while d / nx > 0.45 * lam:
        nx *= 2
    N = int(math.ceil(N / nx) * nx)
    par = make_params(prof, k, theta_deg, DIRICHLET, N, nx=nx, j=j, h=h, n_per=n_per, ls_reg=ls_reg)
    dx = d / N
    a = 0.75 * par["L"]
    if j > 0:
        a = min(a, 0.9 * h / maxslope)
    if a / dx < 2:
        raise ValueError(f"N = {N} gives fewer than two nodes in the singular window of {nx} cells")
    par["Ma"] = int(a / dx)
    par["a_s"] = par["Ma"] * dx
    par["gamma"] = 0.5 * par["a_s"]
    return par


def flat(N=64, d=1.0, k=2 * math.pi, theta_deg=20.0, bc=DIRICHLET, nx=8, **kw):
    prof = {"d": float(d), "a": np.zeros(1), "b": np.zeros(1)}
    kw.setdefault("hmin", -0.5 * d / nx)
    kw.setdefault("ny", 1)
    return make_params(prof, k, theta_deg, bc, N, nx=nx, **kw)


def random_density(N, seed, dtype=np.complex128):
    """Complex normal density vector, normalised to unit 2-norm."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    v /= np.linalg.norm(v)
    return v.astype(dtype)
