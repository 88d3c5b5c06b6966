"""Shifted equivalent-source acceleration, Section 5 of Bruno & Maas: Algorithm 2 (initialisation)
and Algorithm 3 (forward map), step by step in the paper's order and notation.

Readings (where the paper prints no detail):
  * cells c^q = (a1, b1] x (a2, b2] of side L, column cx = ceil(x/L) - 1 (integer arithmetic on
    the node index), row cy = ceil((f - h_min)/L) - 1 (Remark cell_def);
  * Lambda^H_q: points (a1 + s L/p, a2 + b L), Lambda^V_q: (a1 + b L, a2 + s L/p), s = -e..p+e,
    b = 0, 1 (sides extended by e points per end, ~20% more points for p = 8, e = 1); dipole
    normals (0, 1) for H and (1, 0) for V; n_eq = 2 (p + 1 + 2e) sources per orientation;
  * n_coll collocation points equispaced on the boundary of S_q (3L x 3L), offset by half a
    spacing from its lower-left corner; least squares by Householder QR (eq. eq_source_point) with a
    Tikhonov term ls_reg |A|_F |xi|: the collocation matrix has condition ~1e13 for the layouts
    used, so the plain solution's near-null components are set by rounding and, carried through the
    local subtraction, make the operator depend on rounding at the 1e-5 level;
  * punctured Green functions drop only the m = 0 (and, for the periodised kernel, p = 0) self
    term at coincident points, in both Phi~_j^qper and Phi_j, so phi^all - phi^int removes the
    local cells' equivalent sources exactly (eqs. phi_def, phi_jq_def, psi_na_sum);
  * the plane-wave Dirichlet reconstruction (eq. planewave, plwave_QR) is realised in the
    Fourier-Bessel basis J_n(k rho) e^{i n theta}, |n| <= n_fb, about the cell centre: by the
    Jacobi-Anger expansion n_plw = 2 n_fb + 1 equispaced plane waves span the same functions up to
    aliased orders |n| >= n_plw, while the plane-wave matrix itself is numerically singular for
    cells of a fraction of a wavelength; samples are the cell-boundary points of the H grid (top and
    bottom sides) and the V grid (left and right sides), corners entering twice (eq. combine_psi_pna);
  * LocalFFT (eq. small_convolution_grid) is evaluated by its direct sum;
  * GlobalFFT (eq. large_convolution_per_grid) is evaluated by its direct sum over the merged grid
    sources with the kernel table of Algorithm 2 on the lag grid;
  * Neumann (TM): the true field of a cell is the single layer sum mu_l G(x - y_l) ds_l, the
    reconstruction is differentiated along the unit target normal.
"""
from __future__ import annotations

import math
import numpy as np
from scipy import special as sp
from scipy.linalg import solve_triangular

from . import green as gr
from . import direct as dr


def _qr_pinv(A, reg=0.0):
    """Least-squares solution operator of A by Householder QR; with reg > 0 the Tikhonov-regularised
    problem min |A x - b|^2 + (reg |A|_F)^2 |x|^2, i.e. QR of [A; reg |A|_F I] restricted to b."""
    m, n = A.shape
    if reg > 0:
        A = np.concatenate([A, reg * np.linalg.norm(A) * np.eye(n)], axis=0)
    Q, R = np.linalg.qr(A, mode="reduced")
    return solve_triangular(R, Q.conj().T)[:, :m]


class Accel:
    """Algorithm 2 in the constructor, Algorithm 3 in apply()."""

    def __init__(self, par):
        self.par = par
        N, d, k = par["N"], par["d"], par["k"]
        self.N, self.d, self.k = N, d, k
        self.j, self.h = par["j"], par["h"]
        self.alpha, self.beta = dr.wave(par)
        self.dx = d / N
        self.L, self.nx, self.ny, self.hmin = par["L"], par["nx"], par["ny"], par["hmin"]
        self.p, self.e = par["p"], par["e"]
        self.delta = self.L / self.p
        self.neq = 2 * (self.p + 1 + 2 * self.e)
        self.bc = par["bc"]
        self.x, self.f, self.f1, self.f2 = dr.nodes(par)
        self.s = np.sqrt(1 + self.f1**2)
        self._geometry()
        self._eq_source_ls()
        self._fb_ls()
        self._tables()
        self.sing = dr.sing_triplets(par)
        self.modes = dr.modes_factors(par)

    # ------------------------------------------------------------------ geometry (Sec. 5.1)
    def _geometry(self):
        N, nx = self.N, self.nx
        i1 = np.arange(1, N + 1)
        self.cx = (i1 * nx + N - 1) // N - 1
        self.cy = np.ceil((self.f - self.hmin) / self.L).astype(int) - 1
        assert np.all((self.cy >= 0) & (self.cy < self.ny)), "profile leaves the cell box"
        self.cell_nodes = {}
        for i in range(N):
            self.cell_nodes.setdefault((int(self.cx[i]), int(self.cy[i])), []).append(i)
        self.cells = sorted(self.cell_nodes.keys(), key=lambda c: (c[1], c[0]))
        # relative equivalent-source layout (w.r.t. the lower-left corner (a1, a2) of the cell)
        sgrid = np.arange(-self.e, self.p + self.e + 1)
        self.src_rel = {}
        self.src_idx = {}
        pts_h, pts_v, idx_h, idx_v = [], [], [], []
        for b in (0, 1):
            for s in sgrid:
                pts_h.append((s * self.delta, b * self.L))
                idx_h.append((int(s), b))          # grid offset (ix = cx p + s, iy = cy + b)
                pts_v.append((b * self.L, s * self.delta))
                idx_v.append((b, int(s)))          # grid offset (ix = cx + b, iy = cy p + s + e)
        self.src_rel["H"] = np.array(pts_h)
        self.src_rel["V"] = np.array(pts_v)
        self.src_idx["H"] = idx_h
        self.src_idx["V"] = idx_v
        self.nu = {"H": np.array([0.0, 1.0]), "V": np.array([1.0, 0.0])}
        # collocation points on the boundary of S_q = [-L, 2L]^2 (relative to (a1, a2))
        nc = self.par["n_coll"]
        per = 12 * self.L
        t = (np.arange(nc) + 0.5) * per / nc
        side = np.minimum((t // (3 * self.L)).astype(int), 3)
        u = t - side * 3 * self.L
        L = self.L
        cxy = np.zeros((nc, 2))
        cxy[side == 0] = np.stack([-L + u[side == 0], -L + 0 * u[side == 0]], 1)
        cxy[side == 1] = np.stack([2 * L + 0 * u[side == 1], -L + u[side == 1]], 1)
        cxy[side == 2] = np.stack([2 * L - u[side == 2], 2 * L + 0 * u[side == 2]], 1)
        cxy[side == 3] = np.stack([-L + 0 * u[side == 3], 2 * L - u[side == 3]], 1)
        self.coll_rel = cxy
        # cell-boundary samples: H bottom, H top, V left, V right (s = 0..p)
        samp, sori, sidx = [], [], []
        for b in (0, 1):
            for s in range(self.p + 1):
                samp.append((s * self.delta, b * L)); sori.append("H"); sidx.append((s, b))
        for b in (0, 1):
            for s in range(self.p + 1):
                samp.append((b * L, s * self.delta)); sori.append("V"); sidx.append((b, s))
        self.samp_rel = np.array(samp)
        self.samp_ori = sori
        self.samp_idx = sidx
        # local sets L(q) (eqs. S_jq_hat, S_jq, small_convolution): r with c^q inside S_j^r
        self.mh_over_L = np.array([m * self.h / self.L for m in range(self.j + 1)])

    def corner(self, cx, cy):
        return np.array([cx * self.L, self.hmin + cy * self.L])

    def rows_of_Sj(self, cy_r):
        """Cell rows c with c intersecting S^r - m h e_2 for some m (half-open cells)."""
        rows = set()
        for m, sh in enumerate(self.mh_over_L):
            lo, hi = cy_r - 2 - sh, cy_r + 2 - sh          # open interval of admissible rows
            for c in range(int(math.floor(lo)) + 1, int(math.ceil(hi))):
                if lo < c < hi:
                    rows.add(c)
        return rows

    def local_cells(self, q):
        """r = (cx_r, cy_r) in the infinite strip (cx_r unwrapped) with c^q in S_j^r, occupied only."""
        cxq, cyq = q
        out = []
        for dxc in (-1, 0, 1):
            cxr = cxq + dxc
            ref = cxr % self.nx
            for cyr in range(self.ny):
                if (ref, cyr) not in self.cell_nodes:
                    continue
                if cyq in self.rows_of_Sj(cyr):
                    out.append((cxr, cyr))
        return out

    # ------------------------------------------------------------------ Algorithm 2: QR factors
    def _eq_source_ls(self):
        k = self.k
        self.pinv_eq = {}
        for lam in ("H", "V"):
            src = self.src_rel[lam]
            X = self.coll_rel[:, 0][:, None] - src[:, 0][None, :]
            Y = self.coll_rel[:, 1][:, None] - src[:, 1][None, :]
            gx, gy = gr.gradG0(k, X, Y)
            nu = self.nu[lam]
            A = np.concatenate([gr.G0(k, X, Y), -(nu[0] * gx + nu[1] * gy)], axis=1)
            self.pinv_eq[lam] = _qr_pinv(A, self.par.get("ls_reg", 0.0))

    def fb_basis(self, rel, nu=None):
        """Fourier-Bessel functions about the cell centre at points rel (relative to the centre),
        or their derivative along the unit vectors nu."""
        n = np.arange(-self.par["n_fb"], self.par["n_fb"] + 1)
        k = self.k
        rho0 = self.L / math.sqrt(2)
        nrm = (k * rho0 / 2) ** np.abs(n) / sp.factorial(np.abs(n))
        r = np.hypot(rel[:, 0], rel[:, 1])
        th = np.arctan2(rel[:, 1], rel[:, 0])

        def Z(m):
            return sp.jv(m[None, :], k * r[:, None]) * np.exp(1j * m[None, :] * th[:, None])

        if nu is None:
            return Z(n) / nrm[None, :]
        dZx = (k / 2) * (Z(n - 1) - Z(n + 1))
        dZy = (1j * k / 2) * (Z(n + 1) + Z(n - 1))
        return (nu[:, 0][:, None] * dZx + nu[:, 1][:, None] * dZy) / nrm[None, :]

    def _fb_ls(self):
        ctr = np.array([self.L / 2, self.L / 2])
        B = self.fb_basis(self.samp_rel - ctr)
        self.pinv_fb = _qr_pinv(B)

    # ------------------------------------------------------------------ Algorithm 2: G~ on the lag grid
    def grid_geom(self, lam):
        """(dx_grid, dy_grid, P_x, number of rows) of Pi_lambda^per."""
        if lam == "H":
            return self.delta, self.L, self.nx * self.p, self.ny + 1
        return self.L, self.delta, self.nx, self.ny * self.p + 1 + 2 * self.e

    def _tables(self):
        """Twisted periodised kernels T[ix, iy_lag] = e^{-i alpha X} (G~, -dG~/dnu) at X = ix dxg
        reduced to [-d/2, d/2) by the integer lag, Y = iy_lag dyg (Remark large_FFT_eval)."""
        par = self.par
        k, d, j, h, al = self.k, self.d, self.j, self.h, self.alpha
        A = par["n_per"] * d
        self.tab = {}
        for lam in ("H", "V"):
            dxg, dyg, Px, nr = self.grid_geom(lam)
            ix = np.arange(Px)
            iy = np.arange(-(nr - 1), nr)
            IX, IY = np.meshgrid(ix, iy, indexing="ij")
            IXr = np.where(IX >= Px // 2, IX - Px, IX)       # integer reduction
            Xr = (IXr * dxg).ravel()
            Y = (IY * dyg).ravel()
            pun = ((IX == 0) & (IY == 0)).ravel()
            delta = np.min(np.abs(Y[:, None] + h * np.arange(j + 1)[None, :]), axis=1)
            spec = delta >= par["delta_min"]
            g = np.zeros(Xr.shape, complex)
            gx = np.zeros(Xr.shape, complex)
            gy = np.zeros(Xr.shape, complex)
            # spectral rows: one term range per lag row
            for yv in np.unique(Y[spec]):
                sel = spec & (Y == yv)
                dl = float(np.min(np.abs(yv + h * np.arange(j + 1))))
                a, b, c = gr.gtilde_spectral(k, al, d, j, h, Xr[sel], Y[sel], par["spec_exp"], dl)
                g[sel], gx[sel], gy[sel] = a, b, c
            if np.any(~spec):
                sel = ~spec
                a, b, c = gr.gtilde_spatial_centered(k, al, d, j, h, Xr[sel], Y[sel], A, par["c_win"], pun[sel])
                g[sel], gx[sel], gy[sel] = a, b, c
            tw = np.exp(-1j * al * Xr)
            nu = self.nu[lam]
            mono = (tw * g).reshape(IX.shape)
            dip = (tw * -(nu[0] * gx + nu[1] * gy)).reshape(IX.shape)
            self.tab[lam] = (mono, dip, nr)

    def kernel(self, lam, dix, diy):
        """(Phi~, d Phi~/dn_y) at integer lag (dix, diy): e^{i alpha X} T[dix mod P_x, diy]."""
        dxg, dyg, Px, nr = self.grid_geom(lam)
        mono, dip, _ = self.tab[lam]
        ph = np.exp(1j * self.alpha * dix * dxg)
        return ph * mono[np.mod(dix, Px), diy + nr - 1], ph * dip[np.mod(dix, Px), diy + nr - 1]

    # ------------------------------------------------------------------ per-node true field kernel
    def true_field(self, pts, nodes_idx, shift=0.0):
        """psi(x) = sum_l mu_l K(x, y_l) w_l for unit mu: matrix [len(pts), len(nodes)]."""
        k = self.k
        xl = self.x[nodes_idx] + shift
        X = pts[:, 0][:, None] - xl[None, :]
        Y = pts[:, 1][:, None] - self.f[nodes_idx][None, :]
        if self.bc == 0:
            gx, gy = gr.gradG0(k, X, Y)
            return (self.f1[nodes_idx][None, :] * gx - gy) * self.dx
        return gr.G0(k, X, Y) * (self.s[nodes_idx] * self.dx)[None, :]

    # ------------------------------------------------------------------ Algorithm 3 steps
    def _eq_densities(self, mu):
        """EqSources (eq. eq_source_point): densities of every occupied reference cell."""
        dens = {}
        for q in self.cells:
            idx = np.array(self.cell_nodes[q])
            pts = self.coll_rel + self.corner(*q)
            psi = self.true_field(pts, idx) @ mu[idx]
            for lam in ("H", "V"):
                dens[(q, lam)] = self.pinv_eq[lam] @ psi
        return dens

    def _merge(self, dens, shape):
        """GlobalEqSMerge (eq. sum_eqsources): duplicates summed on Pi^per, quasi-periodic wrap."""
        al, d = self.alpha, self.d
        merged = {"H": {}, "V": {}}
        for q in self.cells:
            cxq, cyq = q
            for lam in ("H", "V"):
                dxg, dyg, Px, nr = self.grid_geom(lam)
                v = dens[(q, lam)]
                for t, (o1, o2) in enumerate(self.src_idx[lam]):
                    if lam == "H":
                        ixr, iy = cxq * self.p + o1, cyq + o2
                    else:
                        ixr, iy = cxq + o1, cyq * self.p + o2 + self.e
                    wrap = ixr // Px
                    ph = np.exp(-1j * al * d * wrap)
                    key = (ixr - wrap * Px, iy)
                    a = merged[lam].setdefault(key, np.zeros((2,) + shape, complex))
                    a[0] += v[t] * ph
                    a[1] += v[self.neq + t] * ph
        return merged

    def _sample_grid(self, q, t):
        """Grid indices (ix unwrapped, iy) of sample t of cell q."""
        cxq, cyq = q
        o1, o2 = self.samp_idx[t]
        if self.samp_ori[t] == "H":
            return cxq * self.p + o1, cyq + o2
        return cxq + o1, cyq * self.p + o2 + self.e

    def _phi_all(self, merged, cells):
        """GlobalFFT (eq. large_convolution_per_grid), by its direct sum on the sample points of the
        given cells (any cells of the box, occupied or not)."""
        phi_all = {}
        for lam in ("H", "V"):
            keys = list(merged[lam].keys())
            if not keys:
                continue
            gx_ = np.array([kk[0] for kk in keys])
            gy_ = np.array([kk[1] for kk in keys])
            xi = np.array([merged[lam][kk][0] for kk in keys])
            ze = np.array([merged[lam][kk][1] for kk in keys])
            for q in cells:
                ts = [t for t in range(len(self.samp_ori)) if self.samp_ori[t] == lam]
                for t in ts:
                    six, siy = self._sample_grid(q, t)
                    km, kd = self.kernel(lam, six - gx_, siy - gy_)
                    phi_all[(q, t)] = km @ xi + kd @ ze
        return phi_all

    def _phi_int(self, dens, cells, shape):
        """LocalEqSMerge + LocalFFT (eqs. sum_eqsources_local, small_convolution_grid): phi^int on the
        sample points of the given cells from the equivalent sources of their local cells."""
        k, d, j, h, al = self.k, self.d, self.j, self.h, self.alpha
        phi_int = {}
        for q in cells:
            loc = self.local_cells(q)
            for t in range(len(self.samp_ori)):
                lam = self.samp_ori[t]
                x_t = self.samp_rel[t] + self.corner(*q)
                acc = np.zeros(shape, complex)
                for (cxr, cyr) in loc:
                    ref = cxr % self.nx
                    wrap = (cxr - ref) // self.nx
                    v = dens[((ref, cyr), lam)] * np.exp(1j * al * d * wrap)
                    ys = self.src_rel[lam] + self.corner(cxr, cyr)
                    X = x_t[0] - ys[:, 0]
                    Y = x_t[1] - ys[:, 1]
                    same = (np.abs(X) < 1e-12 * self.L) & (np.abs(Y) < 1e-12 * self.L)
                    Xs = np.where(same, 1.0, X)
                    Ys = np.where(same, 0.0, Y)
                    Gv = gr.Gj(k, j, h, Xs, Ys)
                    ax, ay = gr.gradGj(k, j, h, Xs, Ys)
                    if np.any(same):
                        g1 = gr.Gj(k, j, h, X[same], Y[same], skip_m0=True)
                        b1, b2 = gr.gradGj(k, j, h, X[same], Y[same], skip_m0=True)
                        Gv[same], ax[same], ay[same] = g1, b1, b2
                    nu = self.nu[lam]
                    dG = -(nu[0] * ax + nu[1] * ay)
                    acc = acc + Gv @ v[:self.neq] + dG @ v[self.neq:]
                phi_int[(q, t)] = acc
        return phi_int

    # ------------------------------------------------------------------ Algorithm 3
    def apply(self, mu, return_stages=False):
        """Algorithm 3 on one density mu [N] or on a block of columns mu [N, R] (column by column;
        every step is linear in mu)."""
        par = self.par
        k, d, j, h, al = self.k, self.d, self.j, self.h, self.alpha
        mu = np.asarray(mu, complex)
        st = {}
        dens = self._eq_densities(mu)
        st["dens"] = dens
        merged = self._merge(dens, mu.shape[1:])
        phi_all = self._phi_all(merged, self.cells)
        st["phi_all"] = phi_all
        phi_int = self._phi_int(dens, self.cells, mu.shape[1:])
        st["phi_int"] = phi_int

        out = np.zeros(mu.shape, complex)
        ctr = np.array([self.L / 2, self.L / 2])
        for q in self.cells:
            idx = np.array(self.cell_nodes[q])
            # LocalSubtract + Combine-lambda (eqs. psi_na_sum, combine_psi_pna)
            phi_ni = np.array([phi_all[(q, t)] - phi_int[(q, t)] for t in range(len(self.samp_ori))])
            # PlaneWaveWeights (eq. plwave_QR)
            wq = self.pinv_fb @ phi_ni
            # NonIntersecting (eq. planewave) at the nodes of c^q
            rel = np.stack([self.x[idx], self.f[idx]], 1) - (self.corner(*q) + ctr)
            if self.bc == 0:
                Bn = self.fb_basis(rel)
            else:
                nuh = np.stack([-self.f1[idx], np.ones(len(idx))], 1) / self.s[idx][:, None]
                Bn = self.fb_basis(rel, nuh)
            psi_ni = Bn @ wq
            # Intersecting (eq. final_correction_0): exact sum over nodes of the local cells
            psi_int = np.zeros((len(idx),) + mu.shape[1:], complex)
            for (cxr, cyr) in self.local_cells(q):
                ref = cxr % self.nx
                wrap = (cxr - ref) // self.nx
                lidx = np.array(self.cell_nodes[(ref, cyr)])
                mul = mu[lidx] * np.exp(1j * al * d * wrap)
                X = self.x[idx][:, None] - (self.x[lidx][None, :] + wrap * d)
                Y = self.f[idx][:, None] - self.f[lidx][None, :]
                r = np.hypot(X, Y)
                sf = gr.S_window(r, par["gamma"], par["a_s"])
                use = sf < 1.0
                ax = np.zeros(X.shape, complex)
                ay = np.zeros(X.shape, complex)
                ax[use], ay[use] = gr.gradGj(k, j, h, X[use], Y[use])
                kern = dr._kernel_dnu(par, ax, ay, self.f1[lidx][None, :], self.f1[idx][:, None],
                                      self.s[lidx][None, :], self.s[idx][:, None])
                psi_int += ((1 - sf) * kern * self.dx) @ mul
            # EvalRegular (eq. final_correction)
            out[idx] += psi_ni + psi_int
        st["reg"] = out.copy()

        # EvalSingular (eq. local_mat), EvalModes (eq. D_M_deltax), AddOperators (eq. discrete_eq)
        r_, c_, v_ = self.sing
        sing = np.zeros(mu.shape, complex)
        np.add.at(sing, r_, v_.reshape((-1,) + (1,) * (mu.ndim - 1)) * mu[c_])
        T, S = self.modes
        modes = T @ (S @ mu)
        sigma = 0.5 if self.bc == 0 else -0.5
        y = sigma * mu + sing + out + modes
        if return_stages:
            st["sing"], st["modes"] = sing, modes
            return y, st
        return y

    # ------------------------------------------------------------------ field off the surface
    def target_cell(self, xr, y):
        """Cell (cx, cy) holding a target of the reference period inside the box (the last column and
        row also take the box's right and top edges)."""
        cx = min(int(math.floor(xr / self.L)), self.nx - 1)
        cy = min(int(math.floor((y - self.hmin) / self.L)), self.ny - 1)
        return cx, cy

    def field(self, mu, pts, total=False):
        """Scattered field at points of the cell box by Algorithm 3 with targets off the surface (the
        remark after Algorithm 3: the steps of eqs. final_correction_0 and planewave evaluated at the
        targets). Each target is reduced to the reference period, x = x_r + w d with x_r in [0, d);
        in its cell the Fourier-Bessel fit of phi^ni = phi^all - phi^int gives the field of the
        non-local sources, the nodes of the local cells add theirs exactly (plain trapezoid sum with
        G_j; targets are off the surface), the completion modes add M^eta, and the quasi-periodic
        phase e^{i alpha d w} restores the target's period."""
        k, d, j, h, al = self.k, self.d, self.j, self.h, self.alpha
        mu = np.asarray(mu, complex)
        pts = np.asarray(pts, float).reshape(-1, 2)
        w = np.floor(pts[:, 0] / d)
        xr = pts[:, 0] - w * d
        y = pts[:, 1]
        top = self.hmin + self.ny * self.L
        assert np.all((y >= self.hmin) & (y < top)), "targets outside the cell box"
        tc = [self.target_cell(a, b) for a, b in zip(xr, y)]
        cells = sorted(set(tc), key=lambda c: (c[1], c[0]))
        dens = self._eq_densities(mu)
        merged = self._merge(dens, ())
        phi_all = self._phi_all(merged, cells)
        phi_int = self._phi_int(dens, cells, ())
        T, S = self.modes
        msum = S @ mu
        _, Ueta = dr.mode_sets(self.par)
        ctr = np.array([self.L / 2, self.L / 2])
        out = np.zeros(len(pts), complex)
        for n_t, q in enumerate(tc):
            phi_ni = np.array([phi_all[(q, t)] - phi_int[(q, t)] for t in range(len(self.samp_ori))])
            wq = self.pinv_fb @ phi_ni
            rel = np.array([[xr[n_t], y[n_t]]]) - (self.corner(*q) + ctr)
            far = (self.fb_basis(rel) @ wq)[0]
            near = 0j
            for (cxr, cyr) in self.local_cells(q):
                ref = cxr % self.nx
                wrap = (cxr - ref) // self.nx
                lidx = np.array(self.cell_nodes[(ref, cyr)])
                mul = mu[lidx] * np.exp(1j * al * d * wrap)
                X = xr[n_t] - (self.x[lidx] + wrap * d)
                Y = y[n_t] - self.f[lidx]
                if self.bc == 0:
                    ax, ay = gr.gradGj(k, j, h, X, Y)
                    kern = self.f1[lidx] * ax - ay
                else:
                    kern = gr.Gj(k, j, h, X, Y) * self.s[lidx]
                near += self.dx * np.sum(kern * mul)
            modes = 0j
            for t, n in enumerate(Ueta):
                an = al + 2 * math.pi * n / d
                bn = complex(gr.beta_n(k, al, d, np.array([n]))[0])
                modes += np.exp(1j * (an * xr[n_t] + bn * y[n_t])) * msum[t]
            out[n_t] = (far + near + modes) * np.exp(1j * al * d * w[n_t])
        if total:
            al_, be_ = dr.wave(self.par)
            out = out + np.exp(1j * (al_ * pts[:, 0] - be_ * pts[:, 1]))
        return out

    def matrix(self):
        """The accelerated operator as a dense N x N matrix: Algorithm 3 applied to the identity."""
        return self.apply(np.eye(self.N, dtype=complex))

    def apply_adjoint(self, v, A=None):
        """The adjoint (conjugate transpose) of the accelerated operator applied to v [N] or [N, R]:
        plain definition, from the dense matrix (pass A = matrix() to reuse it)."""
        if A is None:
            A = self.matrix()
        return A.conj().T @ np.asarray(v, complex)
