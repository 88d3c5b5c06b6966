// Device kernels of the sgf library.
//
// Initialisation (Algorithm 2 of Bruno & Maas, all FP64):
//   k_profile        nodes and profile derivatives (Section 4.2)
//   k_build_coll     collocation matrix of the equivalent-source least squares (eq. eq_source_point)
//   k_build_fb       cell-reconstruction matrix on the cell-boundary samples (eq. plwave_QR)
//   k_qr_pinv        Householder QR least-squares operator R^{-1} Q^H of a small matrix (one block)
//   k_build_P        per-cell projection matrices P_q = pinv_eq * T_q (EqSources as a linear map)
//   k_build_I        per-node reconstruction rows (PlaneWaveWeights + NonIntersecting)
//   k_table_spec     periodised kernel rows by the shifted spectral series, folded mod P_x
//                    (eq. shifted_quasi_per_rayleigh, Remark large_FFT_eval)
//   k_table_spat     periodised kernel rows near shifted poles by the windowed lattice sum,
//                    warp-reduced over periods (eq. Gq_limit)
//   k_phi_off        free-space shifted kernel between cell samples and local equivalent sources,
//                    per relative cell offset (the q-independent local grid, eq. pi_q_hat)
//   k_near           block-sparse near operator: exact intersecting sum (eq. final_correction_0),
//                    singular quadrature (eq. local_mat) and the local equivalent-source
//                    subtraction (eqs. small_convolution, psi_na_sum) folded into one matrix
//   k_modes          separable factors of D_M (eq. D_M_deltax)
// Forward map (Algorithm 3), templated on the far-field precision T:
//   k_project        EqSources + GlobalEqSMerge (scatter with the quasi-periodic twist) + mode sums
//   k_fft_x/k_conv_y GlobalFFT (sgf_fft.cuh)
//   k_interp_near    Combine-lambda + NonIntersecting + Intersecting + EvalSingular + EvalModes +
//                    AddOperators
#include "sgf_internal.h"
#include "sgf_fft.cuh"

// ============================================================== profile
__global__ void k_profile(const double* __restrict__ coef, int M, double d, int N, double* x, double* f,
                          double* f1, double* f2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const double* a = coef;
  const double* b = coef + (M + 1);
  double fv = a[0], d1 = 0, d2 = 0;
  for (int m = 1; m <= M; ++m) {
    long mm = ((long)m * (long)(i + 1)) % N;  // 2 pi m x/d = 2 pi m (i+1)/N
    double s, c;
    sincospi(2.0 * (double)mm / (double)N, &s, &c);
    double w = 2.0 * SGF_PI * m / d;
    fv += a[m] * c + b[m] * s;
    d1 += w * (-a[m] * s + b[m] * c);
    d2 += -w * w * (a[m] * c + b[m] * s);
  }
  x[i] = d * (double)(i + 1) / (double)N;
  f[i] = fv;
  f1[i] = d1;
  f2[i] = d2;
}

cudaError_t launch_profile(sgf_ctx* c) {
  int M = (int)c->fa.size() - 1;
  k_profile<<<ceil_div(c->N, 256), 256, 0, c->stream>>>(c->d_coef, M, c->d, c->N, c->d_x, c->d_f, c->d_f1, c->d_f2);
  return cudaGetLastError();
}

// ============================================================== least-squares matrices
// A[lam] is n_coll x 2 neq, column-major (lda = n_coll + 2 neq): monopole columns G(x_t - y_s), dipole
// columns d/dnu_y G = -nu . grad G(x_t - y_s), nu = (0,1) for H and (1,0) for V.
__global__ void k_build_coll(double k, int ncoll, int neq, const double* __restrict__ coll_rel,
                             const double* __restrict__ src_rel, zd* A) {
  const long lda = ncoll + 2 * neq;  // room for the Tikhonov rows
  int lam = blockIdx.y;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ncoll * neq) return;
  int t = idx % ncoll, s = idx / ncoll;
  double X = coll_rel[2 * t] - src_rel[(lam * neq + s) * 2];
  double Y = coll_rel[2 * t + 1] - src_rel[(lam * neq + s) * 2 + 1];
  GreenVal g;
  g.g = zd(0, 0); g.gx = zd(0, 0); g.gy = zd(0, 0);
  green0_add(k, X, Y, 1.0, true, g);
  zd* Al = A + (long)lam * lda * 2 * neq;
  Al[(long)s * lda + t] = g.g;
  Al[(long)(neq + s) * lda + t] = lam == 0 ? -g.gy : -g.gx;
}

// B is n_fit x nb column-major: b_n(x_t - centre), n = -n_fb..n_fb, scaled by (k rho0/2)^|n|/|n|!
__global__ void k_build_fb(double k, double L, int nfit, int nfb, const double* __restrict__ samp_rel, zd* B) {
  int nb = 2 * nfb + 1;
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nfit * nb) return;
  int t = idx % nfit, bi = idx / nfit;
  int n = bi - nfb;
  double X = samp_rel[2 * t] - 0.5 * L, Y = samp_rel[2 * t + 1] - 0.5 * L;
  double r = hypot(X, Y), th = atan2(Y, X);
  double krho0 = k * L / sqrt(2.0);
  B[(long)bi * nfit + t] = (1.0 / fb_norm(n, krho0)) * fb_Z(n, k * r, th);
}

cudaError_t launch_build_matrices(sgf_ctx* c, zd* d_Acoll, zd* d_Bfb, const double* d_coll_rel,
                                  const double* d_src_rel, const double* d_samp_rel) {
  int nc = c->prm.n_coll, neq = c->neq;
  dim3 g1(ceil_div((long)nc * neq, 128), 2);
  k_build_coll<<<g1, 128, 0, c->stream>>>(c->k, nc, neq, d_coll_rel, d_src_rel, d_Acoll);
  k_build_fb<<<ceil_div((long)c->nfit * c->nb, 128), 128, 0, c->stream>>>(c->k, c->L, c->nfit, c->prm.n_fb, d_samp_rel,
                                                                          d_Bfb);
  return cudaGetLastError();
}

// ============================================================== Householder QR least squares
// Tikhonov augmentation of a column-major m0 x n matrix stored with leading dimension m0 + n:
// rows m0..m0+n-1 become reg |A|_F I (one block).
__global__ void k_augment(zd* A, int m0, int n, double reg) {
  __shared__ double red[256];
  const int lda = m0 + n;
  double part = 0;
  for (int idx = threadIdx.x; idx < m0 * n; idx += blockDim.x) part += abs2(A[(long)(idx / m0) * lda + idx % m0]);
  red[threadIdx.x] = part;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double s = reg * sqrt(red[0]);
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    int c = idx / n, r = idx % n;
    A[(long)c * lda + m0 + r] = zd(r == c ? s : 0.0, 0);
  }
}

// One block. A (m x n, column-major) is overwritten by the Householder vectors; pinv (n x m_out,
// row-major: pinv[s*m_out + t]) = the first m_out columns of R^{-1} Q^H. scratch: n*n (R) + n
// (alpha) + m*m (work) entries.
__global__ void k_qr_pinv(zd* A, int m, int n, int m_out, zd* pinv, zd* scratch) {
  __shared__ double red[256];
  zd* R = scratch;
  zd* alph = scratch + (long)n * n;
  zd* E = alph + n;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int c = 0; c < n; ++c) {
    zd* col = A + (long)c * m;
    double part = 0;
    for (int i = c + tid; i < m; i += nt) part += abs2(col[i]);
    red[tid] = part;
    __syncthreads();
    for (int o = nt / 2; o > 0; o >>= 1) {
      if (tid < o) red[tid] += red[tid + o];
      __syncthreads();
    }
    double xn2 = red[0];
    __syncthreads();
    zd x0 = col[c];
    double ax0 = sqrt(abs2(x0));
    double xn = sqrt(xn2);
    zd ph = ax0 > 0 ? zd(x0.re / ax0, x0.im / ax0) : zd(1, 0);
    zd al = -xn * ph;
    zd v0 = x0 - al;
    double vn2 = xn2 - ax0 * ax0 + abs2(v0);
    double inv = vn2 > 0 ? 1.0 / sqrt(vn2) : 0.0;
    __syncthreads();
    for (int i = c + tid; i < m; i += nt) col[i] = (i == c ? v0 : col[i]) * inv;
    if (tid == 0) alph[c] = al;
    __syncthreads();
    for (int cc = c + 1 + tid; cc < n; cc += nt) {
      zd* cl = A + (long)cc * m;
      zd dot(0, 0);
      for (int i = c; i < m; ++i) dot += mulc(cl[i], col[i]);  // v^H a
      for (int i = c; i < m; ++i) cl[i] -= 2.0 * (col[i] * dot);
    }
    __syncthreads();
  }
  for (int r = tid; r < n * n; r += nt) {
    int i = r / n, jj = r % n;
    R[r] = (jj > i) ? A[(long)jj * m + i] : (jj == i ? alph[i] : zd(0, 0));
  }
  __syncthreads();
  for (int t = tid; t < m_out; t += nt) {
    zd* e = E + (long)t * m;
    for (int i = 0; i < m; ++i) e[i] = zd(i == t ? 1.0 : 0.0, 0);
    for (int c = 0; c < n; ++c) {
      const zd* v = A + (long)c * m;
      zd dot(0, 0);
      for (int i = c; i < m; ++i) dot += mulc(e[i], v[i]);
      for (int i = c; i < m; ++i) e[i] -= 2.0 * (v[i] * dot);
    }
    for (int i = n - 1; i >= 0; --i) {
      zd s = e[i];
      for (int jj = i + 1; jj < n; ++jj) s -= R[(long)i * n + jj] * e[jj];
      e[i] = cdiv(s, R[(long)i * n + i]);
    }
    for (int i = 0; i < n; ++i) pinv[(long)i * m_out + t] = e[i];
  }
}

// augment: A is stored with leading dimension m_out + n and gets the Tikhonov rows (reg may be 0).
cudaError_t launch_qr_pinv(sgf_ctx* c, zd* A, int m_out, int n, bool augment, double reg, zd* pinv, zd* scratch) {
  int mt = augment ? m_out + n : m_out;
  if (mt > 256) return cudaErrorInvalidValue;
  if (augment) k_augment<<<1, 256, 0, c->stream>>>(A, m_out, n, reg);
  k_qr_pinv<<<1, 256, 0, c->stream>>>(A, mt, n, m_out, pinv, scratch);
  return cudaGetLastError();
}

// ============================================================== projection matrices P_q
// Block per occupied cell, warp per node: T_t = true-field kernel at collocation point t, then
// P[lam][s][l] = sum_t pinv_eq[lam][s][t] T_t.
struct GeoArgs {
  double k, alpha, d, dx, L, hmin, gam, a_s;
  int N, j, bc, p, neq, nfit, ncoll, nb, nfb, Ma, nx;
  double h;
  // 0: the factors themselves. Otherwise their derivative with respect to the nodes' own position:
  // 1 d/df, 2 d/df' (for the near operator of the target node, 3 d/df, 4 d/df' of the source node)
  int dmode;
};

__global__ void k_build_P(GeoArgs g, const int* __restrict__ cell_start, const int* __restrict__ node_idx,
                          const int* __restrict__ occ_cx, const int* __restrict__ occ_cy,
                          const double* __restrict__ x, const double* __restrict__ f, const double* __restrict__ f1,
                          const double* __restrict__ coll_rel, const zd* __restrict__ pinv_eq, zd* P) {
  extern __shared__ unsigned char smem_raw[];
  zd* buf = reinterpret_cast<zd*>(smem_raw);
  const int q = blockIdx.x;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = blockDim.x / 32;
  const int s0 = cell_start[q], nq = cell_start[q + 1] - s0;
  const double cx = occ_cx[q] * g.L, cy = g.hmin + occ_cy[q] * g.L;
  zd* T = buf + warp * g.ncoll;
  const int nout = 4 * g.neq;
  zd* Pq = P + (long)nout * s0;
  for (int l = warp; l < nq; l += nw) {
    int nid = node_idx[s0 + l];
    double xl = x[nid], fl = f[nid], sl = sqrt(1 + f1[nid] * f1[nid]);
    for (int t = lane; t < g.ncoll; t += 32) {
      double X = cx + coll_rel[2 * t] - xl, Y = cy + coll_rel[2 * t + 1] - fl;
      if (g.dmode == 0) {
        GreenVal gv;
        gv.g = zd(0, 0); gv.gx = zd(0, 0); gv.gy = zd(0, 0);
        green0_add(g.k, X, Y, 1.0, g.bc == 1, gv);
        T[t] = g.bc == 0 ? g.dx * (f1[nid] * gv.gx - gv.gy) : (sl * g.dx) * gv.g;
      } else {  // the node is the source: dY/df_l = -1
        GreenHess hv;
        hv.g = hv.gx = hv.gy = hv.gxy = hv.gyy = zd(0, 0);
        green0_hess_add(g.k, X, Y, 1.0, hv);
        const double f1l = f1[nid];
        if (g.bc == 0)
          T[t] = g.dmode == 1 ? g.dx * (hv.gyy - f1l * hv.gxy) : g.dx * hv.gx;
        else
          T[t] = g.dmode == 1 ? (-sl * g.dx) * hv.gy : (f1l / sl * g.dx) * hv.g;
      }
    }
    __syncwarp();
    for (int o = lane; o < nout; o += 32) {
      int lam = o / (2 * g.neq), s = o % (2 * g.neq);
      const zd* pr = pinv_eq + ((long)lam * 2 * g.neq + s) * g.ncoll;
      zd acc(0, 0);
      for (int t = 0; t < g.ncoll; ++t) acc += pr[t] * T[t];
      Pq[(long)l * nout + o] = acc;
    }
    __syncwarp();
  }
}

static GeoArgs geo_args(sgf_ctx* c) {
  GeoArgs g;
  g.k = c->k; g.alpha = c->alpha; g.d = c->d; g.dx = c->dx; g.L = c->L; g.hmin = c->prm.hmin;
  g.gam = c->gam; g.a_s = c->a_s; g.N = c->N; g.j = c->prm.j; g.bc = c->bc; g.p = c->prm.p; g.neq = c->neq;
  g.nfit = c->nfit; g.ncoll = c->prm.n_coll; g.nb = c->nb; g.nfb = c->prm.n_fb; g.Ma = c->prm.Ma; g.nx = c->prm.nx;
  g.h = c->prm.h;
  g.dmode = 0;
  return g;
}


cudaError_t launch_build_P_geo(sgf_ctx* c, const zd* pinv_eq, const double* d_coll_rel, const double* f,
                              const double* f1, zd* P, int dmode) {
  GeoArgs g = geo_args(c);
  g.dmode = dmode;
  size_t sm = (size_t)8 * g.ncoll * sizeof(zd);
  cudaFuncSetAttribute(k_build_P, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_build_P<<<c->n_occ, 256, sm, c->stream>>>(g, c->d_cell_start, c->d_node_idx, c->d_occ_cx, c->d_occ_cy, c->d_x, f, f1,
                                                d_coll_rel, pinv_eq, P);
  return cudaGetLastError();
}
cudaError_t launch_build_P(sgf_ctx* c, const zd* pinv_eq, const double* d_coll_rel) {
  return launch_build_P_geo(c, pinv_eq, d_coll_rel, c->d_f, c->d_f1, c->o64.P, 0);
}

// ============================================================== reconstruction rows I
// Thread per node (cell order): E_b = basis (Dirichlet) or its unit-normal derivative (Neumann)
// at the node relative to the cell centre; I[t] = sum_b E_b pinv_fb[b][t]; Ip[t] = I[t] e^{i alpha x_t}.
__global__ void k_build_I(GeoArgs g, const int* __restrict__ node_cell, const int* __restrict__ node_idx,
                          const int* __restrict__ occ_cx, const int* __restrict__ occ_cy, const double* __restrict__ x,
                          const double* __restrict__ f, const double* __restrict__ f1,
                          const double* __restrict__ samp_rel, const zd* __restrict__ pinv_fb, zd* Iplain, zd* Ip) {
  int pos = blockIdx.x * blockDim.x + threadIdx.x;
  if (pos >= g.N) return;
  int q = node_cell[pos];
  int nid = node_idx[pos];
  double cxl = occ_cx[q] * g.L, cyl = g.hmin + occ_cy[q] * g.L;
  double X = x[nid] - (cxl + 0.5 * g.L), Y = f[nid] - (cyl + 0.5 * g.L);
  double r = hypot(X, Y), th = atan2(Y, X), kr = g.k * r;
  double krho0 = g.k * g.L / sqrt(2.0);
  double sn = sqrt(1 + f1[nid] * f1[nid]);
  double nux = -f1[nid] / sn, nuy = 1.0 / sn;
  zd E[64];
  for (int bi = 0; bi < g.nb; ++bi) {
    int n = bi - g.nfb;
    double inv = 1.0 / fb_norm(n, krho0);
    zd zm = fb_Z(n - 1, kr, th), zp = fb_Z(n + 1, kr, th);
    zd dzx = (0.5 * g.k) * (zm - zp);           // d/dX of J_n(k rho) e^{i n theta}
    zd dzy = zd(0, 0.5 * g.k) * (zp + zm);      // d/dY
    if (g.dmode == 0) {
      E[bi] = g.bc == 0 ? inv * fb_Z(n, kr, th) : inv * (nux * dzx + nuy * dzy);
    } else if (g.bc == 0) {  // the node's own height moves the sample point: d/dY; f' does not enter
      E[bi] = g.dmode == 1 ? inv * dzy : zd(0, 0);
    } else if (g.dmode == 1) {
      zd zm2 = fb_Z(n - 2, kr, th), zp2 = fb_Z(n + 2, kr, th), z0 = fb_Z(n, kr, th);
      zd dyx = zd(0, 0.25 * g.k * g.k) * (zm2 - zp2);            // d2/dYdX
      zd dyy = (-0.25 * g.k * g.k) * (zm2 + 2.0 * z0 + zp2);    // d2/dY2
      E[bi] = inv * (nux * dyx + nuy * dyy);
    } else {  // d(unit normal)/df' = (-1, -f')/s^3
      const double s3 = sn * sn * sn;
      E[bi] = inv * ((-1.0 / s3) * dzx + (-f1[nid] / s3) * dzy);
    }
  }
  for (int t = 0; t < g.nfit; ++t) {
    zd acc(0, 0);
    for (int bi = 0; bi < g.nb; ++bi) acc += E[bi] * pinv_fb[(long)bi * g.nfit + t];
    Iplain[(long)pos * g.nfit + t] = acc;
    double xt = cxl + samp_rel[2 * t];
    Ip[(long)pos * g.nfit + t] = acc * expi(g.alpha * xt);
  }
}

cudaError_t launch_build_I_geo(sgf_ctx* c, const zd* pinv_fb, zd* d_Iplain, const double* d_samp_rel, const double* f,
                              const double* f1, zd* Ip, int dmode) {
  GeoArgs g = geo_args(c);
  g.dmode = dmode;
  k_build_I<<<ceil_div(c->N, 64), 64, 0, c->stream>>>(g, c->d_node_cell, c->d_node_idx, c->d_occ_cx, c->d_occ_cy, c->d_x,
                                                       f, f1, d_samp_rel, pinv_fb, d_Iplain, Ip);
  return cudaGetLastError();
}
cudaError_t launch_build_I(sgf_ctx* c, const zd* pinv_fb, zd* d_Iplain, const double* d_samp_rel) {
  return launch_build_I_geo(c, pinv_fb, d_Iplain, d_samp_rel, c->d_f, c->d_f1, c->o64.Ip, 0);
}

// ============================================================== periodised kernel table
struct TabArgs {
  double k, alpha, d, h, dxg, dyg, delta_min, spec_exp, A, cwin;
  int j, Px, logPx, Py, nrow, lam;
};

// Block per lag row iy_lag in [-(nrow-1), nrow-1] whose delta >= delta_min: writes
// Tx[kx][iy_cyc] = Px * sum_{n = kx mod Px} coefficient (the X transform of the twisted row).
__global__ void k_table_spec(TabArgs a, const double* __restrict__ binw, zd* Txm, zd* Txd) {
  const int iyl = (int)blockIdx.x - (a.nrow - 1);
  const double Y = iyl * a.dyg;
  const double dl = row_delta(Y, a.j, a.h);
  if (dl < a.delta_min) return;
  double T = sqrt(a.k * a.k + (a.spec_exp / dl) * (a.spec_exp / dl));
  long n_hi = (long)ceil((T - a.alpha) * a.d / (2 * SGF_PI));
  long n_lo = (long)floor((-T - a.alpha) * a.d / (2 * SGF_PI));
  const int iyc = ((iyl % a.Py) + a.Py) % a.Py;
  for (int kx = threadIdx.x; kx < a.Px; kx += blockDim.x) {
    // n = kx + t Px within [n_lo, n_hi]
    long t0 = (long)ceil((double)(n_lo - kx) / a.Px), t1 = (long)floor((double)(n_hi - kx) / a.Px);
    zd Fm(0, 0), Fd(0, 0);
    for (long t = t0; t <= t1; ++t) {
      int n = (int)(kx + t * a.Px);
      zd c, cy;
      double an;
      spec_coef(a.k, a.alpha, a.d, a.j, a.h, Y, n, binw, c, cy, an);
      Fm += c;
      Fd += (a.lam == 0) ? -cy : zd(0, -an) * c;
    }
    Txm[(long)kx * a.Py + iyc] = (double)a.Px * Fm;
    Txd[(long)kx * a.Py + iyc] = (double)a.Px * Fd;
  }
}

// Warp per lag point (ix, iy_lag) of a row with delta < delta_min: windowed lattice sum over
// periods p (lanes), X reduced to [-d/2, d/2) by the integer lag, window after differentiation,
// the (p = 0, m = 0) term dropped at lag (0, 0). Writes the twisted values to Tl[ix][iy_cyc].
__global__ void k_table_spat(TabArgs a, const double* __restrict__ binw, zd* Tlm, zd* Tld) {
  const int lane = threadIdx.x % 32;
  const long wid = ((long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
  const long npts = (long)a.Px * (2 * a.nrow - 1);
  if (wid >= npts) return;
  const int ix = (int)(wid % a.Px);
  const int iyl = (int)(wid / a.Px) - (a.nrow - 1);
  const double Y = iyl * a.dyg;
  if (row_delta(Y, a.j, a.h) >= a.delta_min) return;
  const int ixr = ix >= a.Px / 2 ? ix - a.Px : ix;
  const double Xr = ixr * a.dxg;
  const bool punct = (ix == 0 && iyl == 0);
  const int P = (int)ceil(a.A / a.d) + 1;
  zd g(0, 0), gx(0, 0), gy(0, 0);
  for (int p = -P + lane; p <= P; p += 32) {
    double xp = Xr + p * a.d;
    double S = window_S(xp, a.cwin * a.A, a.A);
    if (S <= 0) continue;
    GreenVal gv = green_j(a.k, a.j, a.h, xp, Y, punct && p == 0, true, binw);
    zd ph = expi(-a.alpha * p * a.d);
    g += (S * ph) * gv.g;
    gx += (S * ph) * gv.gx;
    gy += (S * ph) * gv.gy;
  }
  g = warp_sum(g);
  gx = warp_sum(gx);
  gy = warp_sum(gy);
  if (lane == 0) {
    zd tw = expi(-a.alpha * Xr);
    const int iyc = ((iyl % a.Py) + a.Py) % a.Py;
    Tlm[(long)ix * a.Py + iyc] = tw * g;
    Tld[(long)ix * a.Py + iyc] = tw * (a.lam == 0 ? -gy : -gx);
  }
}

__global__ void k_add_scale(zd* dst, const zd* src, long n, double s) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = s * (dst[i] + src[i]);
}
__global__ void k_scale(zd* dst, long n, double s) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = s * dst[i];
}
__global__ void k_to_f32(const zd* __restrict__ s, zf* __restrict__ d, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = zf((float)s[i].re, (float)s[i].im);
}
// Full-circle table tw[i] = e^{-2 pi i i / 2^twlog}, i < 2^twlog.
__global__ void k_twiddles(zd* tw, int twlog) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int n = 1 << twlog;
  if (i >= n) return;
  double s, c;
  sincospi(-2.0 * i / n, &s, &c);
  tw[i] = zd(c, s);
}

__global__ void k_split_ff(const zd* __restrict__ s, float4* __restrict__ d, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = cff_from(s[i]);
}
cudaError_t launch_split_ff(const zd* src, float4* dst, long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_split_ff<<<ceil_div(n, 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(const zd* src, zf* dst, long n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_to_f32<<<ceil_div(n, 256), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

static size_t fftx_smem(int Px, int ty, size_t esz) { return ((size_t)splen(Px * ty) + Px) * esz; }
// Rows per block of the X passes: at least 16 contiguous bytes per column read, enough blocks for
// two waves of the 152 SMs where the row count allows; threads = Px * ty / 16 (16 values each).
static int fftx_ty(int Px, int nrow, size_t esz) {
  int tmax = 8192 / Px;
  int tcoal = (int)((16 + esz - 1) / esz);
  int ttarget = (nrow + 303) / 304;
  int ty = std::max(tcoal, ttarget);
  if (ty > tmax) ty = tmax;
  if (ty < 1) ty = 1;
  return ty;
}
// Threads for one contiguous FFT of length Py = 2^la 3^lb when a thread holds at most vpt values
// (vpt = 16: 15 with radix-3 stages; vpt = 8: 6 with radix-3 stages), a multiple of 32, >= 64.
static int conv_threads(int Py, int vpt, int lb) {
  int per = lb > 0 ? (vpt == 16 ? 15 : 6) : vpt;
  int t = (Py + per - 1) / per;
  t = (t + 31) / 32 * 32;
  return t < 64 ? 64 : t;
}
static int fftx_threads(int Px, int ty, int vpt) {
  int t = (Px * ty + vpt - 1) / vpt;
  t = (t + 31) / 32 * 32;
  return t < 64 ? 64 : t;
}
// Registers per thread of a kernel, looked up once per kernel.
static int func_regs(const void* f) {
  cudaFuncAttributes fa;
  return cudaFuncGetAttributes(&fa, f) == cudaSuccess ? fa.numRegs : 255;
}
template <typename T, int VPT>
static int fftx_regs() {
  static const int r = func_regs((const void*)k_fft_x<T, VPT>);
  return r;
}

// X passes: 8 values per thread (twice the threads of the 16-value variant, shorter per-thread
// chains in each stage) whenever the block stays within 1024 threads and the register file.
template <typename T>
static cudaError_t run_fft_x(cplx<T>* g, const Orient& o, int nrow, int narr, const cplx<T>* tw, int twlog, int dir,
                             cudaStream_t s, long arr_stride = 0) {
  int ty = fftx_ty(o.Px, nrow, sizeof(cplx<T>));
  size_t sm = fftx_smem(o.Px, ty, sizeof(cplx<T>));
  dim3 grid(ceil_div(nrow, ty), narr);
  if (arr_stride == 0) arr_stride = (long)o.Px * nrow;
  int t8 = fftx_threads(o.Px, ty, 8);
  const bool fits8 = t8 <= 1024 && (long)fftx_regs<T, 8>() * t8 <= 65536;
  if (o.force_vpt ? o.force_vpt == 8 : fits8) {
    cudaFuncSetAttribute(k_fft_x<T, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_fft_x<T, 8><<<grid, t8, sm, s>>>(g, o.logPx, nrow, ty, arr_stride, tw, twlog, dir);
  } else {
    cudaFuncSetAttribute(k_fft_x<T, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_fft_x<T, 16><<<grid, fftx_threads(o.Px, ty, 16), sm, s>>>(g, o.logPx, nrow, ty, arr_stride, tw, twlog, dir);
  }
  return cudaGetLastError();
}

cudaError_t launch_tables(sgf_ctx* c) {
  cudaError_t e;
  for (int lam = 0; lam < 2; ++lam) {
    const Orient& o = c->og[lam];
    TabArgs a;
    a.k = c->k; a.alpha = c->alpha; a.d = c->d; a.h = c->prm.h; a.dxg = o.dxg; a.dyg = o.dyg;
    a.delta_min = c->prm.delta_min; a.spec_exp = c->prm.spec_exp; a.A = c->prm.n_per * c->d; a.cwin = c->prm.c_win;
    a.j = c->prm.j; a.Px = o.Px; a.logPx = o.logPx; a.Py = o.Py; a.nrow = o.nrow; a.lam = lam;
    long n = (long)o.Px * o.Py;
    zd* Txm = c->d_Tx[lam][0];
    zd* Txd = c->d_Tx[lam][1];
    zd* Tlm = c->o64.Khat[lam][0];  // lag-space scratch, overwritten below by the spectra
    zd* Tld = c->o64.Khat[lam][1];
    cudaMemsetAsync(Txm, 0, n * sizeof(zd), c->stream);
    cudaMemsetAsync(Txd, 0, n * sizeof(zd), c->stream);
    cudaMemsetAsync(Tlm, 0, n * sizeof(zd), c->stream);
    cudaMemsetAsync(Tld, 0, n * sizeof(zd), c->stream);
    k_table_spec<<<2 * o.nrow - 1, 256, 0, c->stream>>>(a, c->d_binw, Txm, Txd);
    long npts = (long)o.Px * (2 * o.nrow - 1);
    k_table_spat<<<ceil_div(npts * 32, 256), 256, 0, c->stream>>>(a, c->d_binw, Tlm, Tld);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // X transform of the spatial rows (the arrays are [Px][Py]: Py "rows" of Px points)
    if ((e = run_fft_x<double>(Tlm, o, o.Py, 1, c->o64.tw, c->twlog, -1, c->stream)) != cudaSuccess) return e;
    if ((e = run_fft_x<double>(Tld, o, o.Py, 1, c->o64.tw, c->twlog, -1, c->stream)) != cudaSuccess) return e;
    k_add_scale<<<ceil_div(n, 256), 256, 0, c->stream>>>(Txm, Tlm, n, 1.0);
    k_add_scale<<<ceil_div(n, 256), 256, 0, c->stream>>>(Txd, Tld, n, 1.0);
    // Y transform into the spectra, scaled by 1/(Px Py)
    cudaMemcpyAsync(Tlm, Txm, n * sizeof(zd), cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(Tld, Txd, n * sizeof(zd), cudaMemcpyDeviceToDevice, c->stream);
    size_t sm = (size_t)splen(o.Py) * sizeof(zd);
    cudaFuncSetAttribute(k_fft_y_full<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int ty_threads = conv_threads(o.Py, 16, o.lb);
    k_fft_y_full<double><<<o.Px, ty_threads, sm, c->stream>>>(Tlm, o.Py, o.la, o.lb, c->o64.twy[lam], -1);
    k_fft_y_full<double><<<o.Px, ty_threads, sm, c->stream>>>(Tld, o.Py, o.la, o.lb, c->o64.twy[lam], -1);
    double sc = 1.0 / ((double)o.Px * o.Py);
    k_scale<<<ceil_div(n, 256), 256, 0, c->stream>>>(Tlm, n, sc);
    k_scale<<<ceil_div(n, 256), 256, 0, c->stream>>>(Tld, n, sc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (c->o32.Khat[lam][0]) {
      launch_to_f32(Tlm, c->o32.Khat[lam][0], n, c->stream);
      launch_to_f32(Tld, c->o32.Khat[lam][1], n, c->stream);
    }
  }
  return cudaGetLastError();
}

__global__ void k_twiddles_n(zd* tw, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double sn, cs;
  sincospi(-2.0 * i / n, &sn, &cs);
  tw[i] = zd(cs, sn);
}

cudaError_t launch_twiddles(sgf_ctx* c) {
  int n = 1 << c->twlog;
  k_twiddles<<<ceil_div(n, 256), 256, 0, c->stream>>>(c->o64.tw, c->twlog);
  if (c->o32.tw) launch_to_f32(c->o64.tw, c->o32.tw, n, c->stream);
  for (int lam = 0; lam < 2; ++lam) {
    int py = c->og[lam].Py;
    k_twiddles_n<<<ceil_div(py, 256), 256, 0, c->stream>>>(c->o64.twy[lam], py);
    if (c->o32.twy[lam]) launch_to_f32(c->o64.twy[lam], c->o32.twy[lam], py, c->stream);
  }
  return cudaGetLastError();
}

// Inverse X transform of the FP64 table copy for testing: out[ix][iy] = IFFT_x(Tx)/Px.
cudaError_t launch_debug_table(sgf_ctx* c, int lam, int kind, zd* out) {
  const Orient& o = c->og[lam];
  long n = (long)o.Px * o.Py;
  cudaMemcpyAsync(out, c->d_Tx[lam][kind], n * sizeof(zd), cudaMemcpyDeviceToDevice, c->stream);
  cudaError_t e = run_fft_x<double>(out, o, o.Py, 1, c->o64.tw, c->twlog, +1, c->stream);
  if (e != cudaSuccess) return e;
  k_scale<<<ceil_div(n, 256), 256, 0, c->stream>>>(out, n, 1.0 / o.Px);
  return cudaGetLastError();
}

// ============================================================== local kernel per cell offset
// phi[(o * nfit + t) * 2neq + s] for o = (dcx + 1) * n_dcy + (dcy - dcy_min): monopole / dipole
// shifted free-space kernel from source s of the orientation of sample t in the cell at offset
// (dcx, dcy) to sample t of the target cell (punctured at coincident points: m = 0 dropped).
__global__ void k_phi_off(GeoArgs g, int dcy_min, int n_dcy, const double* __restrict__ samp_rel,
                          const double* __restrict__ src_rel, const double* __restrict__ binw, zd* phi) {
  long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  long tot = (long)3 * n_dcy * g.nfit * 2 * g.neq;
  if (idx >= tot) return;
  int s2 = (int)(idx % (2 * g.neq));
  long rest = idx / (2 * g.neq);
  int t = (int)(rest % g.nfit);
  int o = (int)(rest / g.nfit);
  int dcx = o / n_dcy - 1, dcy = dcy_min + o % n_dcy;
  int lam = orient_of_sample(t, g.p);
  int s = s2 % g.neq;
  double X = samp_rel[2 * t] - (dcx * g.L + src_rel[(lam * g.neq + s) * 2]);
  double Y = samp_rel[2 * t + 1] - (dcy * g.L + src_rel[(lam * g.neq + s) * 2 + 1]);
  bool same = fabs(X) < 1e-12 * g.L && fabs(Y) < 1e-12 * g.L;
  bool mono = s2 < g.neq;
  GreenVal gv = green_j(g.k, g.j, g.h, same ? 0.0 : X, same ? 0.0 : Y, same, mono, binw);
  phi[idx] = mono ? gv.g : (lam == 0 ? -gv.gy : -gv.gx);
}

cudaError_t launch_phi_off(sgf_ctx* c, zd* d_phi, int dcy_min, int n_dcy, const double* d_samp_rel,
                           const double* d_src_rel) {
  GeoArgs g = geo_args(c);
  long tot = (long)3 * n_dcy * c->nfit * 2 * c->neq;
  k_phi_off<<<ceil_div(tot, 256), 256, 0, c->stream>>>(g, dcy_min, n_dcy, d_samp_rel, d_src_rel, c->d_binw, d_phi);
  return cudaGetLastError();
}

// ============================================================== near operator blocks
// Block per (q, r) pair: C_qr[i][l] = phase_r * ( exact (1 - S^f) dG_j/dnu w_l
//   + S^f (R_s K_s + dx K_r)  [only where S^f > 0]  -  sum_t I_q[i][t] sum_s Phi_off[t][s] P_r[s][l] )
// Derivative of the near-operator value (before the quasi-periodic phase and the folded local
// subtraction) with respect to the target's (dmode 1: f, 2: f') or the source's (3: f, 4: f') own
// position. Off the diagonal the value is (1 - S^f) dx K outside the singular band and
// dx K + S^f K_s (R_s - dx ln 4 sin^2(pi X/(2a))) inside it, K the kernel of the boundary condition
// and K_s its log coefficient; on the diagonal dx (f''/(4 pi (1 + f'^2)) + const).
__device__ inline zd near_dval(const GeoArgs& g, bool diag, long sidx, double X, double Y, double f1i, double si,
                               double f1l, double sl, double f2i, const double* kress, const double* binw) {
  const int dm = g.dmode;
  if (diag) {
    if (dm != 2) return zd(0, 0);
    double q = 1 + f1i * f1i;
    return zd(g.dx * (-f2i * 2 * f1i / (4 * SGF_PI * q * q)), 0);
  }
  const double sY = dm == 1 ? 1.0 : (dm == 3 ? -1.0 : 0.0);  // dY/dv
  const double k = g.k, rr = hypot(X, Y);
  GreenHess H = green_j_hess(k, g.j, g.h, X, Y, binw);
  zd kern, dkern;
  if (g.bc == 0) {
    kern = f1l * H.gx - H.gy;
    dkern = (dm == 1 || dm == 3) ? sY * (f1l * H.gxy - H.gyy) : (dm == 4 ? H.gx : zd(0, 0));
  } else {
    zd a = -f1i * H.gx + H.gy;
    kern = a * (sl / si);
    if (dm == 1 || dm == 3)
      dkern = (sY * sl / si) * (-f1i * H.gxy + H.gyy);
    else if (dm == 2)
      dkern = (-sl / si) * H.gx + (-f1i * sl / (si * si * si)) * a;
    else
      dkern = (f1l / (sl * si)) * a;
  }
  const double Sf = window_S(rr, g.gam, g.a_s);
  const double dSf = window_S_dx(rr, g.gam, g.a_s) * sY * Y / rr;
  if (Sf > 0 && sidx > -g.Ma && sidx < g.Ma) {
    const double q = k * j1(k * rr) / rr;
    const double dq = k * (k * j0(k * rr) / rr - 2 * j1(k * rr) / (rr * rr));  // d/dr
    double Ks, dKs;
    if (g.bc == 0) {
      const double b = Y - f1l * X;
      Ks = -q * b / (4 * SGF_PI);
      dKs = (dm == 1 || dm == 3) ? -(dq * sY * Y / rr * b + q * sY) / (4 * SGF_PI)
                                 : (dm == 4 ? q * X / (4 * SGF_PI) : 0.0);
    } else {
      const double b = -f1i * X + Y;
      Ks = q * b / (4 * SGF_PI) / si * sl;
      if (dm == 1 || dm == 3)
        dKs = (dq * sY * Y / rr * b + q * sY) / (4 * SGF_PI) * sl / si;
      else if (dm == 2)
        dKs = q / (4 * SGF_PI) * (-X / si + b * (-f1i / (si * si * si))) * sl;
      else
        dKs = q * b / (4 * SGF_PI) / si * (f1l / sl);
    }
    const double sn = sin(SGF_PI * X / (2 * g.a_s));
    const double w = kress[sidx + g.Ma - 1] - g.dx * log(4 * sn * sn);
    return g.dx * dkern + zd((dSf * Ks + Sf * dKs) * w, 0);
  }
  return (-dSf * g.dx) * kern + ((1.0 - Sf) * g.dx) * dkern;
}

// Target nodes read (f, f1, f2), source nodes (fs, f1s): the same arrays for the operator itself;
// a gradient moves the two roles separately (the diagonal belongs to the target).
__global__ void k_near(GeoArgs g, const int* __restrict__ cell_start, const int* __restrict__ node_idx,
                       const int* __restrict__ occ_cy, const double* __restrict__ x, const double* __restrict__ f,
                       const double* __restrict__ f1, const double* __restrict__ f2, const double* __restrict__ fs,
                       const double* __restrict__ f1s, const zd* __restrict__ phi,
                       int dcy_min, int n_dcy, const zd* __restrict__ Iplain, const zd* __restrict__ P,
                       const int* __restrict__ pq, const int* __restrict__ pr, const int* __restrict__ pw,
                       const long* __restrict__ poff, const int* __restrict__ pld, const int* __restrict__ pdcx,
                       const double* __restrict__ kress,
                       const double* __restrict__ binw, zd hk, zd* C, int lc) {
  extern __shared__ unsigned char smem_raw[];
  zd* Msh = reinterpret_cast<zd*>(smem_raw);  // [n_fit][lc]: one tile of source columns at a time
  const int b = blockIdx.x;
  const int q = pq[b], r = pr[b], wrap = pw[b];
  const long off = poff[b];
  const long ld = pld[b];
  const int qs = cell_start[q], nq = cell_start[q + 1] - qs;
  const int rs = cell_start[r], nr = cell_start[r + 1] - rs;
  const int dcx = pdcx[b];
  const int dcy = occ_cy[r] - occ_cy[q];
  const int o = (dcx + 1) * n_dcy + (dcy - dcy_min);
  const zd* ph_o = phi + (long)o * g.nfit * 2 * g.neq;
  const zd* Pr = P + (long)4 * g.neq * rs;
  const zd wph = expi(g.alpha * g.d * wrap);
  const double k = g.k;
  for (int l0 = 0; l0 < nr; l0 += lc) {
  const int ln = min(lc, nr - l0);
  // M[t][l] = sum_s Phi_off[t][s] P_r[lam(t)][s][l] for the tile's source columns l0 .. l0 + ln - 1
  __syncthreads();  // the previous tile's M has been used
  for (int idx = threadIdx.x; idx < g.nfit * ln; idx += blockDim.x) {
    int t = idx / ln, l = l0 + idx % ln;
    int lam = orient_of_sample(t, g.p);
    zd acc(0, 0);
    for (int s = 0; s < 2 * g.neq; ++s) acc += ph_o[t * 2 * g.neq + s] * Pr[(long)l * 4 * g.neq + lam * 2 * g.neq + s];
    Msh[idx] = acc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nq * ln; idx += blockDim.x) {
    int il = idx / ln, l = l0 + idx % ln;
    int i = node_idx[qs + il], ls = node_idx[rs + l];
    double xi = x[i], fi = f[i], f1i = f1[i], si = sqrt(1 + f1i * f1i);
    double xl = x[ls] + wrap * g.d, fl = fs[ls], f1l = f1s[ls], sl = sqrt(1 + f1l * f1l);
    double X = xi - xl, Y = fi - fl;
    double rr = hypot(X, Y);
    double Sf = window_S(rr, g.gam, g.a_s);
    zd val(0, 0);
    if (g.dmode != 0) {
      val = near_dval(g, i == ls && wrap == 0, (long)i - ((long)ls + (long)wrap * g.N), X, Y, f1i, si, f1l, sl, f2[i],
                      kress, binw);
    } else if (i == ls && wrap == 0) {
      double kr0 = f2[i] / (4 * SGF_PI * (1 + f1i * f1i));
      val = g.dx * (zd(kr0, 0) + (g.bc == 0 ? hk : -hk));
    } else {
      GreenVal gv = green_j(k, g.j, g.h, X, Y, false, false, binw);
      zd kern = g.bc == 0 ? (f1l * gv.gx - gv.gy) : ((-f1i * gv.gx + gv.gy) * (sl / si));
      val = ((1.0 - Sf) * g.dx) * kern;
      long sidx = (long)i - ((long)ls + (long)wrap * g.N);
      if (Sf > 0 && sidx > -g.Ma && sidx < g.Ma) {
        double j1r = k * j1(k * rr) / rr;
        double Ks = g.bc == 0 ? -j1r / (4 * SGF_PI) * (Y - f1l * X) : j1r / (4 * SGF_PI) * (-f1i * X + Y) / si * sl;
        double sn = sin(SGF_PI * X / (2 * g.a_s));
        double lg = log(4 * sn * sn);
        zd Kr = kern - (Ks * lg) * zd(1, 0);
        double rw = kress[sidx + g.Ma - 1];
        val += Sf * (zd(rw * Ks, 0) + g.dx * Kr);
      }
    }
    const zd* Ii = Iplain + (long)(qs + il) * g.nfit;
    zd sub(0, 0);
    for (int t = 0; t < g.nfit; ++t) sub += Ii[t] * Msh[t * ln + (l - l0)];
    C[off + (long)il * ld + l] = wph * (val - sub);
  }
  }
}

cudaError_t near_hk(sgf_ctx* c, zd* hk);

cudaError_t launch_near(sgf_ctx* c, const zd* d_phi, int dcy_min, int n_dcy, const zd* d_Iplain, const NearPairs& pp,
                        const double* d_kress) {
  return launch_near_geo(c, d_phi, dcy_min, n_dcy, d_Iplain, c->o64.P, pp, d_kress, c->d_f, c->d_f1, c->d_f2, c->d_f,
                         c->d_f1, c->d_C, 0);
}

cudaError_t launch_near_geo(sgf_ctx* c, const zd* d_phi, int dcy_min, int n_dcy, const zd* d_Iplain, const zd* P,
                            const NearPairs& pp, const double* d_kress, const double* ft, const double* f1t,
                            const double* f2t, const double* fs, const double* f1s, zd* C, int dmode) {
  GeoArgs g = geo_args(c);
  g.dmode = dmode;
  int maxnr = 0;
  for (int q = 0; q < c->n_occ; ++q) maxnr = std::max(maxnr, c->cell_start[q + 1] - c->cell_start[q]);
  // source columns per shared-memory tile of M (all of a cell's nodes when they fit)
  const int lc = std::max(1, std::min(maxnr, (int)((160 * 1024) / ((size_t)c->nfit * sizeof(zd)))));
  size_t sm = (size_t)c->nfit * lc * sizeof(zd);
  cudaFuncSetAttribute(k_near, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  zd hk(0, 0);
  cudaError_t e = near_hk(c, &hk);
  if (e != cudaSuccess) return e;
  k_near<<<pp.n, 256, sm, c->stream>>>(g, c->d_cell_start, c->d_node_idx, c->d_occ_cy, c->d_x, ft, f1t, f2t, fs, f1s,
                                       d_phi, dcy_min, n_dcy, d_Iplain, P, pp.q, pp.r, pp.wrap, pp.off, pp.ld, pp.dcx,
                                       d_kress, c->d_binw, hk, C, lc);
  return cudaGetLastError();
}

__global__ void k_hk(double k, int j, double h, const double* binw, zd* out) {
  zd acc(0, 0);
  for (int m = 1; m <= j; ++m) {
    zd h1 = hankel1(k * m * h);
    acc += (binw[m] * 0.25 * k) * zd(-h1.im, h1.re);
  }
  *out = acc;
}

cudaError_t near_hk(sgf_ctx* c, zd* hk) {
  k_hk<<<1, 1, 0, c->stream>>>(c->k, c->prm.j, c->prm.h, c->d_binw, c->d_msum);
  cudaMemcpyAsync(hk, c->d_msum, sizeof(zd), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  return cudaGetLastError();
}

// ============================================================== modes
// d_modes_n: per mode [alpha_n, beta_re, beta_im]; MT[i][n] target factors, MS[n][i] source factors.
__global__ void k_modes(GeoArgs g, int nm, const double* __restrict__ mn, const double* __restrict__ x,
                        const double* __restrict__ f, const double* __restrict__ f1, zd* MT, zd* MS) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  double s = sqrt(1 + f1[i] * f1[i]);
  for (int n = 0; n < nm; ++n) {
    double an = mn[3 * n];
    zd bn(mn[3 * n + 1], mn[3 * n + 2]);
    // i (alpha_n x + beta_n f)
    zd arg = zd(0, an * x[i]) + zd(0, 1) * (f[i] * bn);
    zd e = cexpz(arg), t = e;
    zd ibn = zd(0, 1) * bn;
    zd nf = zd(0, an * (-f1[i])) + ibn;  // Neumann factor (-i alpha_n f' + i beta_n), before 1/s
    if (g.bc == 1) t = e * (nf * (1.0 / s));
    zd ms = (s * g.dx) * cexpz(-arg);
    if (g.dmode == 1) {  // d/df: the exponents
      t = ibn * t;
      ms = (-1.0) * (ibn * ms);
    } else if (g.dmode == 2) {  // d/df': the Neumann normal factor and the arc-length weight
      t = g.bc == 1 ? e * (zd(0, -an / s) + (-f1[i] / (s * s * s)) * nf) : zd(0, 0);
      ms = (f1[i] / s * g.dx) * cexpz(-arg);
    }
    MT[(long)i * nm + n] = t;
    MS[(long)n * g.N + i] = ms;
  }
}

cudaError_t launch_modes_geo(sgf_ctx* c, const double* d_modes_n, const double* f, const double* f1, zd* MT, zd* MS,
                             int dmode) {
  if (c->nm == 0) return cudaSuccess;
  GeoArgs g = geo_args(c);
  g.dmode = dmode;
  k_modes<<<ceil_div(c->N, 128), 128, 0, c->stream>>>(g, c->nm, d_modes_n, c->d_x, f, f1, MT, MS);
  return cudaGetLastError();
}
cudaError_t launch_modes(sgf_ctx* c, const double* d_modes_n) {
  return launch_modes_geo(c, d_modes_n, c->d_f, c->d_f1, c->d_MT, c->d_MS, 0);
}

// ============================================================== right-hand side
__global__ void k_rhs(GeoArgs g, double beta, const double* x, const double* f, const double* f1, zd* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  zd u = expi(g.alpha * x[i] - beta * f[i]);
  const double s = sqrt(1 + f1[i] * f1[i]);
  zd v = g.bc == 0 ? -u : zd(0, (g.alpha * f1[i] + beta) / s) * u;
  if (g.dmode == 1) v = zd(0, -beta) * v;  // d/df of the phase
  if (g.dmode == 2)                         // d/df' (Neumann only)
    v = g.bc == 0 ? zd(0, 0) : zd(0, g.alpha / s - (g.alpha * f1[i] + beta) * f1[i] / (s * s * s)) * u;
  out[i] = v;
}
cudaError_t launch_rhs_geo(sgf_ctx* c, const double* f, const double* f1, zd* out, int dmode) {
  GeoArgs g = geo_args(c);
  g.dmode = dmode;
  k_rhs<<<ceil_div(c->N, 256), 256, 0, c->stream>>>(g, c->beta, c->d_x, f, f1, out);
  return cudaGetLastError();
}
cudaError_t launch_rhs(sgf_ctx* c, zd* out) { return launch_rhs_geo(c, c->d_f, c->d_f1, out, 0); }

// ============================================================== forward map
// Mode-sum partials (eq. D_M_deltax, source factors): block (n, chunk) of the grid tail sums
// MS[n][i] mu_i over one chunk of the nodes; FP64 for T = double, float-float for T = float.
template <typename T>
__device__ __forceinline__ void mode_partial(int n, int chunk, int MB, long N, const zd* __restrict__ mu,
                                             const zd* __restrict__ MS, const float4* __restrict__ MSff,
                                             zd* __restrict__ mpart, float4* __restrict__ mpart_ff) {
  __shared__ float4 redf[32];
  SGF_SHARED_ARRAY(zd, redd, 32);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const long len = (N + MB - 1) / MB, i0 = chunk * len, i1 = min(N, i0 + len);
  if (sizeof(T) == 4) {
    ff ar = {0.f, 0.f}, ai = {0.f, 0.f};
    for (long i = i0 + threadIdx.x; i < i1; i += blockDim.x) cff_mac(MSff[n * N + i], cff_from(mu[i]), ar, ai);
    for (int o = 16; o > 0; o >>= 1) {
      ar = ff_add(ar, {__shfl_down_sync(0xffffffffu, ar.hi, o), __shfl_down_sync(0xffffffffu, ar.lo, o)});
      ai = ff_add(ai, {__shfl_down_sync(0xffffffffu, ai.hi, o), __shfl_down_sync(0xffffffffu, ai.lo, o)});
    }
    if (lane == 0) redf[warp] = make_float4(ar.hi, ai.hi, ar.lo, ai.lo);
    __syncthreads();
    if (threadIdx.x == 0) {
      ff sr = {0.f, 0.f}, si = {0.f, 0.f};
      for (int w = 0; w < nw; ++w) {
        sr = ff_add(sr, {redf[w].x, redf[w].z});
        si = ff_add(si, {redf[w].y, redf[w].w});
      }
      mpart_ff[n * MB + chunk] = make_float4(sr.hi, si.hi, sr.lo, si.lo);
    }
  } else {
    zd acc(0, 0);
    for (long i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc += MS[n * N + i] * mu[i];
    acc = warp_sum(acc);
    if (lane == 0) redd[warp] = acc;
    __syncthreads();
    if (warp == 0) {
      zd v = lane < nw ? redd[lane] : zd(0, 0);
      v = warp_sum(v);
      if (lane == 0) mpart[n * MB + chunk] = v;
    }
  }
}

// EqSources + GlobalEqSMerge: block per occupied cell, one thread per output (orientation,
// monopole/dipole, source) of P_q mu_q (P stored [node][output]), scattered with the quasi-periodic
// twist into the X-major grids. The grid tail (nm * MB blocks) computes the mode-sum partials. For
// the mixed path the cell blocks also write the float-float copy of mu used by the near field.
// FP64: six blocks per SM (78 registers, no spills) so that the ~790 work items of the N = 16384
// workload run in one wave; FP32: five (96 registers: its 32 staged P values spill under six, and
// a one-block bound lets the compiler take 123).
template <typename T>
__global__ void __launch_bounds__(128, sizeof(T) == 8 ? 6 : 5) k_project(int n_occ, int neq, int nm, long N, const int* __restrict__ cell_start,
                          const int* __restrict__ node_idx, const zd* __restrict__ mu, const cplx<T>* __restrict__ P,
                          const int* __restrict__ src_gidx, const cplx<T>* __restrict__ src_tw,
                          cplx<T>* __restrict__ gH, long gH_stride, cplx<T>* __restrict__ gV, long gV_stride,
                          const zd* __restrict__ MS, const float4* __restrict__ MSff, zd* __restrict__ mpart,
                          float4* __restrict__ mpart_ff, float4* __restrict__ muff, int MB, int n_items,
                          const int* __restrict__ item_cell, const int* __restrict__ item_lo,
                          const int* __restrict__ item_hi) {
  extern __shared__ unsigned char smem_raw[];
  if ((int)blockIdx.x >= n_items) {
    const int t = blockIdx.x - n_items;
    mode_partial<T>(t / MB, t % MB, MB, N, mu, MS, MSff, mpart, mpart_ff);
    return;
  }
  // one block per chunk of at most 32 nodes of a cell: the scatter is additive, so chunks of one
  // cell add their partial densities independently
  cplx<T>* mus = reinterpret_cast<cplx<T>*>(smem_raw);
  const int q = item_cell[blockIdx.x];
  const int ncell = cell_start[q + 1] - cell_start[q];
  const int lo = item_lo[blockIdx.x], nq = item_hi[blockIdx.x] - lo;
  const int s0 = cell_start[q] + lo;
  if (sizeof(T) == 4 && 4 * neq <= (int)blockDim.x && nq <= 32) {
    // FP32 with one output per thread: the thread's column of P for the whole chunk, its grid index
    // and twist are loaded before the densities (which they do not depend on) arrive
    const int nout = 4 * neq, o = threadIdx.x;
    const cplx<T>* Pq = P + (long)nout * s0;
    cplx<T> pv[32];
    cplx<T> twv(0, 0);
    cplx<T>* dst = nullptr;
    if (o < nout) {
#pragma unroll
      for (int u = 0; u < 32; ++u)
        if (u < nq) pv[u] = Pq[(long)u * nout + o];
      const int lam = o / (2 * neq), sidx = o % (2 * neq), si = sidx % neq;
      const long idx = ((long)q * 2 + lam) * neq + si;
      twv = src_tw[idx];
      dst = (lam == 0 ? gH + (sidx < neq ? 0 : gH_stride) : gV + (sidx < neq ? 0 : gV_stride)) + src_gidx[idx];
    }
    for (int l = threadIdx.x; l < nq; l += blockDim.x) {
      const int nid = node_idx[s0 + l];
      const zd m = mu[nid];
      mus[l] = cplx<T>(m);
      if (muff) muff[nid] = cff_from(m);
    }
    __syncthreads();
    if (o < nout) {
      cplx<T> acc[4] = {cplx<T>(0, 0), cplx<T>(0, 0), cplx<T>(0, 0), cplx<T>(0, 0)};
#pragma unroll
      for (int u = 0; u < 32; ++u)
        if (u < nq) acc[u & 3] = fma_c(pv[u], mus[u], acc[u & 3]);
      const cplx<T> v = ((acc[0] + acc[1]) + (acc[2] + acc[3])) * twv;
      atomicAdd(&dst->re, v.re);
      atomicAdd(&dst->im, v.im);
    }
    return;
  }
  for (int l = threadIdx.x; l < nq; l += blockDim.x) {
    const int nid = node_idx[s0 + l];
    const zd m = mu[nid];
    mus[l] = cplx<T>(m);
    if (muff) muff[nid] = cff_from(m);
  }
  __syncthreads();
  const int nout = 4 * neq;
  const cplx<T>* Pq = P + (long)nout * s0;  // [node][output] rows of this chunk
  (void)ncell;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    // UN loads of P in flight per round (the whole chunk of <= 32 nodes in two rounds for FP32)
    constexpr int UN = sizeof(T) == 4 ? 16 : 8;
    cplx<T> acc[4] = {cplx<T>(0, 0), cplx<T>(0, 0), cplx<T>(0, 0), cplx<T>(0, 0)};
    for (int l0 = 0; l0 < nq; l0 += UN) {
      cplx<T> pv[UN];
#pragma unroll
      for (int u = 0; u < UN; ++u)
        if (l0 + u < nq) pv[u] = Pq[(long)(l0 + u) * nout + o];
#pragma unroll
      for (int u = 0; u < UN; ++u)
        if (l0 + u < nq) acc[u & 3] = fma_c(pv[u], mus[l0 + u], acc[u & 3]);
    }
    cplx<T> accs = (acc[0] + acc[1]) + (acc[2] + acc[3]);
    int lam = o / (2 * neq), s = o % (2 * neq);
    int si = s % neq;
    long gi = src_gidx[((long)q * 2 + lam) * neq + si];
    cplx<T> v = accs * src_tw[((long)q * 2 + lam) * neq + si];
    cplx<T>* base = lam == 0 ? gH + (s < neq ? 0 : gH_stride) : gV + (s < neq ? 0 : gV_stride);
    atomicAdd(&base[gi].re, v.re);
    atomicAdd(&base[gi].im, v.im);
  }
}

// Intersecting + EvalSingular (the block-sparse near operator C, local subtraction folded in) and
// the sigma/2 identity of AddOperators: out = C mu + sigma/2 mu. Block per work item (chunk of at
// most 32 target rows of a cell): the densities of the cell's local columns are staged in shared
// memory once (as float-float for the mixed path), each warp streams whole rows of the cell's near
// block. It needs nothing but mu, so it runs beside the projection and the FFT convolution; the
// far-field and mode terms are added afterwards by k_interp_far. T = double: FP64. T = float:
// float-float on the FP32 pipes, converted to FP64 at the store.
// Launch bounds: six 256-thread blocks per SM for the float-float path (40 registers), so that the
// ~800 work items of the N = 16384 workload run in one wave with 48 warps per SM in flight.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 4) k_near_rows(int mask, double half_sigma, const int* __restrict__ cell_start,
                            const int* __restrict__ node_idx, const int* __restrict__ cols,
                            const int* __restrict__ coloff, const long* __restrict__ cell_off,
                            const int* __restrict__ cell_W, const zd* __restrict__ C, const float4* __restrict__ Cff,
                            const int* __restrict__ item_cell, const int* __restrict__ item_lo,
                            const int* __restrict__ item_hi, const zd* __restrict__ mu, zd* __restrict__ out) {
  constexpr bool FF = sizeof(T) == 4;
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const int q = item_cell[blockIdx.x];
  const int rlo = item_lo[blockIdx.x];
  const int s0 = cell_start[q] + rlo, nq = item_hi[blockIdx.x] - rlo;
  const int W = cell_W[q];
  // shared layout: [W] densities (16 B each), then [nq] per-row results (16 B each)
  zd* mus = reinterpret_cast<zd*>(smem_raw);
  float4* musf = reinterpret_cast<float4*>(smem_raw);
  zd* resd = reinterpret_cast<zd*>(smem_raw) + W;
  float4* resf = reinterpret_cast<float4*>(smem_raw) + W;
  const int* cq = cols + coloff[q];
  if (mask & 2) {
    if (FF) {
      for (int cc = threadIdx.x; cc < W; cc += blockDim.x) musf[cc] = cff_from(mu[cq[cc]]);
    } else {
      for (int cc = threadIdx.x; cc < W; cc += blockDim.x) mus[cc] = mu[cq[cc]];
    }
  }
  __syncthreads();
  for (int il = warp; il < nq; il += nw) {
    if (FF) {
      dot2c a = {0.f, 0.f, 0.f, 0.f};
      if (mask & 2) {
        const float4* Cr = Cff + cell_off[q] + (long)(rlo + il) * W;
        dot2c b = {0.f, 0.f, 0.f, 0.f};
        for (int c0 = lane; c0 < W; c0 += 128) {  // four loads in flight per lane, two chains
          float4 v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (c0 + 32 * u < W) v[u] = Cr[c0 + 32 * u];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int cc = c0 + 32 * u;
            if (cc < W) dot2_mac(v[u], musf[cc], (u & 1) ? b : a);
          }
        }
        dot2_merge(a, b);
        for (int o = 16; o > 0; o >>= 1) {
          dot2c t = {__shfl_down_sync(0xffffffffu, a.sr, o), __shfl_down_sync(0xffffffffu, a.si, o),
                     __shfl_down_sync(0xffffffffu, a.er, o), __shfl_down_sync(0xffffffffu, a.ei, o)};
          dot2_merge(a, t);
        }
      }
      if (lane == 0) {
        ff vr = ff_add({a.sr, 0.f}, {a.er, 0.f}), vi = ff_add({a.si, 0.f}, {a.ei, 0.f});
        resf[il] = make_float4(vr.hi, vi.hi, vr.lo, vi.lo);
      }
    } else {
      zd acc(0, 0);
      if (mask & 2) {
        const zd* Cr = C + cell_off[q] + (long)(rlo + il) * W;
        zd acc1(0, 0), acc2(0, 0), acc3(0, 0);
        int cc = lane;
        for (; cc + 96 < W; cc += 128) {
          acc = fma_c(Cr[cc], mus[cc], acc);
          acc1 = fma_c(Cr[cc + 32], mus[cc + 32], acc1);
          acc2 = fma_c(Cr[cc + 64], mus[cc + 64], acc2);
          acc3 = fma_c(Cr[cc + 96], mus[cc + 96], acc3);
        }
        for (; cc < W; cc += 32) acc = fma_c(Cr[cc], mus[cc], acc);
        acc = warp_sum((acc + acc1) + (acc2 + acc3));
      }
      if (lane == 0) resd[il] = acc;
    }
  }
  __syncthreads();
  // thread per row: identity term, conversion, store
  for (int il = threadIdx.x; il < nq; il += blockDim.x) {
    const int i = node_idx[s0 + il];
    if (FF) {
      float4 r = resf[il];
      ff vr = {r.x, r.z}, vi = {r.y, r.w};
      if (mask & 8) {
        float4 m = cff_from(mu[i]);
        float hs = (float)half_sigma;  // +-1/2: exact scaling
        vr = ff_add(vr, {hs * m.x, hs * m.z});
        vi = ff_add(vi, {hs * m.y, hs * m.w});
      }
      out[i] = zd(ff_to_double(vr), ff_to_double(vi));
    } else {
      zd v = resd[il];
      if (mask & 8) v += half_sigma * mu[i];
      out[i] = v;
    }
  }
}

// Combine-lambda + NonIntersecting (PlaneWaveWeights folded into the reconstruction rows Ip) and
// EvalModes, added to the near-field result already in out. Block per work item: the cell's
// n_fit samples of the convolved grids are gathered once, each warp reduces rows of Ip against
// them (four threads per row, blockDim = 128), and one thread per row adds the far-field and mode
// terms to out[i]. T = float: FP32 far field, float-float mode sums; the final additions are FP64.
template <typename T>
__global__ void k_interp_far(int mask, int nfit, int nm, const int* __restrict__ cell_start,
                             const int* __restrict__ node_idx, const int* __restrict__ samp_gidx, int pH,
                             const cplx<T>* __restrict__ phiH, const cplx<T>* __restrict__ phiV,
                             const cplx<T>* __restrict__ Ip, const zd* __restrict__ MT,
                             const float4* __restrict__ MTff, const zd* __restrict__ mpart,
                             const float4* __restrict__ mpart_ff, int MB, const int* __restrict__ item_cell,
                             const int* __restrict__ item_lo, const int* __restrict__ item_hi,
                             zd* __restrict__ out) {
  constexpr bool FF = sizeof(T) == 4;
  SGF_SHARED_ARRAY(cplx<T>, ph, 64);
  SGF_SHARED_ARRAY(cplx<T>, far_s, 32);
  __shared__ float4 msf[8];
  SGF_SHARED_ARRAY(zd, msd, 8);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int q = item_cell[blockIdx.x];
  const int rlo = item_lo[blockIdx.x];
  const int s0 = cell_start[q] + rlo, nq = item_hi[blockIdx.x] - rlo;
  // loads that do not depend on the gathered samples go out first: this thread's share of its
  // row of Ip (four threads per row, every 4th sample; n_fit <= 64) and, for the first nq threads,
  // the row's current out value
  const int il = threadIdx.x / 4, part = threadIdx.x % 4;
  cplx<T> ir[16];
  if (il < nq && (mask & 1)) {
    const cplx<T>* Ir = Ip + (long)(s0 + il) * nfit;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (part + 4 * k < nfit) ir[k] = Ir[part + 4 * k];
  }
  int irow = 0;
  zd outv(0, 0);
  if ((int)threadIdx.x < nq) {
    irow = node_idx[s0 + threadIdx.x];
    outv = out[irow];
  }
  for (int t = threadIdx.x; t < nfit; t += blockDim.x) {
    long gi = samp_gidx[(long)q * nfit + t];
    ph[t] = t < 2 * (pH + 1) ? phiH[gi] : phiV[gi];
  }
  // mode sums from their chunk partials: warp w folds modes w, w + 4, ... (up to 8 modes, 4 warps)
  for (int n = warp; n < nm && (mask & 4); n += blockDim.x / 32) {
    if (FF) {
      ff sr = {0.f, 0.f}, si = {0.f, 0.f};
      for (int cch = lane; cch < MB; cch += 32) {
        float4 v = mpart_ff[n * MB + cch];
        sr = ff_add(sr, {v.x, v.z});
        si = ff_add(si, {v.y, v.w});
      }
      for (int o = 16; o > 0; o >>= 1) {
        sr = ff_add(sr, {__shfl_down_sync(0xffffffffu, sr.hi, o), __shfl_down_sync(0xffffffffu, sr.lo, o)});
        si = ff_add(si, {__shfl_down_sync(0xffffffffu, si.hi, o), __shfl_down_sync(0xffffffffu, si.lo, o)});
      }
      if (lane == 0) msf[n] = make_float4(sr.hi, si.hi, sr.lo, si.lo);
    } else {
      zd a(0, 0);
      for (int cch = lane; cch < MB; cch += 32) a += mpart[n * MB + cch];
      a = warp_sum(a);
      if (lane == 0) msd[n] = a;
    }
  }
  __syncthreads();
  {  // four threads per row (blockDim = 128 covers the 32 rows at once)
    cplx<T> far(0, 0);
    if (il < nq && (mask & 1)) {
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (part + 4 * k < nfit) far = fma_c(ir[k], ph[part + 4 * k], far);
    }
    for (int o = 2; o > 0; o >>= 1) {
      far.re += __shfl_down_sync(0xffffffffu, far.re, o);
      far.im += __shfl_down_sync(0xffffffffu, far.im, o);
    }
    if (part == 0 && il < nq) far_s[il] = far;
  }
  __syncthreads();
  if ((int)threadIdx.x < nq) {
    const int i = irow;
    zd v = outv + zd((double)far_s[threadIdx.x].re, (double)far_s[threadIdx.x].im);
    if (mask & 4) {
      if (FF) {
        ff vr = {0.f, 0.f}, vi = {0.f, 0.f};
        for (int n = 0; n < nm; ++n) cff_mac(MTff[(long)i * nm + n], msf[n], vr, vi);
        v += zd(ff_to_double(vr), ff_to_double(vi));
      } else {
        for (int n = 0; n < nm; ++n) v += MT[(long)i * nm + n] * msd[n];
      }
    }
    out[i] = v;
  }
}

// Y convolution launch: at most 15 FFT values per thread (radix-3 stages), at least 64 threads.
// The partial product K_m FFT(xi) stays in registers, with the twiddle table staged in shared
// memory next to the column, when both fit (FP64 columns up to 6144 points); otherwise it goes to
// the global scratch `accg` ([Px][Py]). Returns 0 (and launches nothing) when neither fits.
template <typename T, bool ADJ, int VPT, bool ACCG>
static int conv_regs() {
  static const int r = func_regs(ADJ ? (const void*)k_conv_y_adj<T, VPT, ACCG> : (const void*)k_conv_y<T, VPT, ACCG>);
  return r;
}

// 3: 8 values per thread, product in registers, twiddles in shared memory (the widest blocks; the
//    forward kernel also prefetches the spectra and the zeta column);
// 1: the same with 16 values per thread; 2: 16 values per thread, product in global scratch;
// 0: no variant fits one block.
template <typename T, bool ADJ>
static int conv_y_variant(const Orient& o) {
  // padded column, twiddle table (and the forward 8-value kernel's padded zeta column)
  const size_t col = (size_t)splen(o.Py) * sizeof(cplx<T>), twb = (size_t)o.Py * sizeof(cplx<T>);
  const int t8 = conv_threads(o.Py, 8, o.lb), t16 = conv_threads(o.Py, 16, o.lb);
  const size_t sm8 = col + twb + (ADJ ? 0 : col);
  if (t8 <= 1024 && sm8 <= 200 * 1024 && (long)conv_regs<T, ADJ, 8, false>() * t8 <= 65536) return 3;
  if (t16 > 1024) return 0;
  if (col + twb <= 200 * 1024 && (long)conv_regs<T, ADJ, 16, false>() * t16 <= 65536) return 1;
  if (col <= 200 * 1024 && (long)conv_regs<T, ADJ, 16, true>() * t16 <= 65536) return 2;
  return 0;
}

template <typename T, bool ADJ>
static bool conv_variant_fits(const Orient& o, int v) {
  const size_t col = (size_t)splen(o.Py) * sizeof(cplx<T>), twb = (size_t)o.Py * sizeof(cplx<T>);
  const int t8 = conv_threads(o.Py, 8, o.lb), t16 = conv_threads(o.Py, 16, o.lb);
  const size_t sm8 = col + twb + (ADJ ? 0 : col);
  switch (v) {
    case 3: return t8 <= 1024 && sm8 <= 200 * 1024 && (long)conv_regs<T, ADJ, 8, false>() * t8 <= 65536;
    case 1: return t16 <= 1024 && col + twb <= 200 * 1024 && (long)conv_regs<T, ADJ, 16, false>() * t16 <= 65536;
    case 2: return t16 <= 1024 && col <= 200 * 1024 && (long)conv_regs<T, ADJ, 16, true>() * t16 <= 65536;
    default: return false;
  }
}
template <typename T>
static bool variants_fit(const Orient& o, int conv_variant, int vpt) {
  if (conv_variant && !(conv_variant_fits<T, false>(o, conv_variant) && conv_variant_fits<T, true>(o, conv_variant)))
    return false;
  const int ty = fftx_ty(o.Px, o.nrow, sizeof(cplx<T>));
  if (vpt == 8) {
    const int t8 = fftx_threads(o.Px, ty, 8);
    if (t8 > 1024 || (long)fftx_regs<T, 8>() * t8 > 65536) return false;
  } else if (vpt == 16) {
    const int t16 = fftx_threads(o.Px, ty, 16);
    if (t16 > 1024 || (long)fftx_regs<T, 16>() * t16 > 65536) return false;
  } else if (vpt != 0) {
    return false;
  }
  return true;
}
bool debug_variants_fit(const Orient& o, int precision, int conv_variant, int fftx_vpt) {
  return precision == 64 ? variants_fit<double>(o, conv_variant, fftx_vpt) : variants_fit<float>(o, conv_variant, fftx_vpt);
}

int conv_y_variant_of(const Orient& o, int precision, bool adjoint) {
  if (adjoint) return precision == 64 ? conv_y_variant<double, true>(o) : conv_y_variant<float, true>(o);
  return precision == 64 ? conv_y_variant<double, false>(o) : conv_y_variant<float, false>(o);
}

// One launch of the Y convolution (ADJ: its adjoint) with the variant chosen by conv_y_variant.
template <typename T, bool ADJ, int VPT, bool ACCG>
static void conv_launch(cplx<T>* xi, cplx<T>* zeta, const cplx<T>* Km, const cplx<T>* Kd, const Orient& o,
                        const cplx<T>* twy, cplx<T>* accg, int threads, cudaStream_t s, int nset, long gstride,
                        long kstride) {
  // column (+ twiddle table) (+ the prefetched zeta column of the forward 8-value variant)
  const size_t col = (size_t)splen(o.Py) * sizeof(cplx<T>), twb = (size_t)o.Py * sizeof(cplx<T>);
  size_t sm = ACCG ? col : col + twb + (!ADJ && VPT <= 8 ? col : 0);
  const dim3 grid(o.Px, nset);
  if (ADJ) {
    cudaFuncSetAttribute(k_conv_y_adj<T, VPT, ACCG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_conv_y_adj<T, VPT, ACCG><<<grid, threads, sm, s>>>(xi, zeta, Km, Kd, o.Py, o.la, o.lb, o.nrow, twy, accg,
                                                          gstride, kstride);
  } else {
    cudaFuncSetAttribute(k_conv_y<T, VPT, ACCG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_conv_y<T, VPT, ACCG><<<grid, threads, sm, s>>>(xi, zeta, Km, Kd, o.Py, o.la, o.lb, o.nrow, twy, accg,
                                                      gstride, kstride);
  }
}

// nset column sets (densities) at once: grids gstride apart, spectra kstride apart (0: shared),
// the global-scratch variant's columns Px Py apart.
template <typename T, bool ADJ>
static cudaError_t conv_y_any(cplx<T>* xi, cplx<T>* zeta, const cplx<T>* Km, const cplx<T>* Kd, const Orient& o,
                              const cplx<T>* twy, cplx<T>* accg, cudaStream_t s, int nset = 1, long gstride = 0,
                              long kstride = 0) {
  switch (o.force_conv ? o.force_conv : conv_y_variant<T, ADJ>(o)) {
    case 3:
      conv_launch<T, ADJ, 8, false>(xi, zeta, Km, Kd, o, twy, nullptr, conv_threads(o.Py, 8, o.lb), s, nset, gstride,
                                    kstride);
      break;
    case 1:
      conv_launch<T, ADJ, 16, false>(xi, zeta, Km, Kd, o, twy, nullptr, conv_threads(o.Py, 16, o.lb), s, nset,
                                     gstride, kstride);
      break;
    case 2:
      if (!accg) return cudaErrorInvalidValue;
      conv_launch<T, ADJ, 16, true>(xi, zeta, Km, Kd, o, twy, accg, conv_threads(o.Py, 16, o.lb), s, nset, gstride,
                                    kstride);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t conv_y(cplx<T>* xi, const cplx<T>* zeta, const cplx<T>* Km, const cplx<T>* Kd, const Orient& o,
                          const cplx<T>* twy, cplx<T>* accg, cudaStream_t s) {
  return conv_y_any<T, false>(xi, const_cast<cplx<T>*>(zeta), Km, Kd, o, twy, accg, s);
}

template <typename T>
static cudaError_t conv_y_adj(cplx<T>* xi, cplx<T>* zeta, const cplx<T>* Km, const cplx<T>* Kd, const Orient& o,
                              const cplx<T>* twy, cplx<T>* accg, cudaStream_t s) {
  return conv_y_any<T, true>(xi, zeta, Km, Kd, o, twy, accg, s);
}

template <typename T>
static cudaError_t apply_t(sgf_ctx* c, OpData<T>& od, const zd* mu, zd* out) {
  cudaStream_t s = c->stream;
  const Orient& oH = c->og[0];
  const Orient& oV = c->og[1];
  long szH = (long)oH.Px * oH.nrow, szV = (long)oV.Px * oV.nrow;
  const double hs = c->bc == 0 ? 0.5 : -0.5;
  const size_t smn = (size_t)(c->maxW + 32) * sizeof(zd);
  cudaFuncSetAttribute(k_near_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smn);
  auto near_rows = [&](cudaStream_t st) {
    k_near_rows<T><<<c->n_nitems, 256, smn, st>>>(c->debug_mask, hs, c->d_cell_start, c->d_node_idx, c->d_cols,
                                                  c->d_coloff, c->d_cell_off, c->d_cell_W, c->d_C, c->d_Cff,
                                                  c->d_nitem_cell, c->d_nitem_lo, c->d_nitem_hi, mu, out);
  };
  // Three concurrent branches when not profiling: the near field (needs only mu) once the grids are
  // cleared, and after the projection the H and V convolutions; the far-field/mode kernel joins
  // them. (Forked before the clears, the near kernel's blocks fill every SM and hold back the
  // clears and the projection, which start the longer chain.)
  const bool branches = !c->profiling && c->side && c->side2;
  if (c->profiling) cudaEventRecord(c->ev[0], s);
  cudaMemsetAsync(od.grid[0], 0, 2 * szH * sizeof(cplx<T>), s);
  cudaMemsetAsync(od.grid[1], 0, 2 * szV * sizeof(cplx<T>), s);
  if (branches) {
    cudaEventRecord(c->ev_fork0, s);
    cudaStreamWaitEvent(c->side2, c->ev_fork0, 0);
    near_rows(c->side2);
    cudaEventRecord(c->ev_join2, c->side2);
  }
  k_project<T><<<c->n_items + c->nm * c->mode_chunks, 128, (size_t)32 * sizeof(cplx<T>), s>>>(
      c->n_occ, c->neq, c->nm, c->N, c->d_cell_start, c->d_node_idx, mu, od.P, c->d_src_gidx, od.src_tw, od.grid[0],
      szH, od.grid[1], szV, c->d_MS, c->d_MSff, c->d_mpart, c->d_mpart_ff, nullptr, c->mode_chunks, c->n_items,
      c->d_item_cell, c->d_item_lo, c->d_item_hi);
  if (c->profiling) cudaEventRecord(c->ev[1], s);
  cudaError_t e;
  if (!c->profiling && c->side) {
    // the two orientations are independent until the interpolation: V runs on the side stream
    cudaEventRecord(c->ev_fork, s);
    cudaStreamWaitEvent(c->side, c->ev_fork, 0);
    for (int lam = 0; lam < 2; ++lam) {
      const Orient& o = c->og[lam];
      cudaStream_t st = lam == 0 ? s : c->side;
      long sz = (long)o.Px * o.nrow;
      if ((e = run_fft_x<T>(od.grid[lam], o, o.nrow, 2, od.tw, c->twlog, -1, st)) != cudaSuccess) return e;
      e = conv_y<T>(od.grid[lam], od.grid[lam] + sz, od.Khat[lam][0], od.Khat[lam][1], o, od.twy[lam],
                    od.accg[lam], st);
      if (e != cudaSuccess) return e;
      if ((e = run_fft_x<T>(od.grid[lam], o, o.nrow, 1, od.tw, c->twlog, +1, st)) != cudaSuccess) return e;
    }
    cudaEventRecord(c->ev_join, c->side);
    cudaStreamWaitEvent(s, c->ev_join, 0);
  } else {
    for (int lam = 0; lam < 2; ++lam) {
      const Orient& o = c->og[lam];
      if ((e = run_fft_x<T>(od.grid[lam], o, o.nrow, 2, od.tw, c->twlog, -1, s)) != cudaSuccess) return e;
    }
    if (c->profiling) cudaEventRecord(c->ev[2], s);
    for (int lam = 0; lam < 2; ++lam) {
      const Orient& o = c->og[lam];
      long sz = (long)o.Px * o.nrow;
      e = conv_y<T>(od.grid[lam], od.grid[lam] + sz, od.Khat[lam][0], od.Khat[lam][1], o, od.twy[lam],
                    od.accg[lam], s);
      if (e != cudaSuccess) return e;
    }
    if (c->profiling) cudaEventRecord(c->ev[3], s);
    for (int lam = 0; lam < 2; ++lam) {
      const Orient& o = c->og[lam];
      if ((e = run_fft_x<T>(od.grid[lam], o, o.nrow, 1, od.tw, c->twlog, +1, s)) != cudaSuccess) return e;
    }
  }
  if (c->profiling) cudaEventRecord(c->ev[4], s);
  if (branches)
    cudaStreamWaitEvent(s, c->ev_join2, 0);
  else
    near_rows(s);
  if (c->profiling) cudaEventRecord(c->ev[5], s);
  k_interp_far<T><<<c->n_items, 128, 0, s>>>(c->debug_mask, c->nfit, c->nm, c->d_cell_start, c->d_node_idx,
                                             c->d_samp_gidx, c->prm.p, od.grid[0], od.grid[1], od.Ip, c->d_MT, c->d_MTff,
                                             c->d_mpart, c->d_mpart_ff, c->mode_chunks, c->d_item_cell, c->d_item_lo,
                                             c->d_item_hi, out);
  if (c->profiling) cudaEventRecord(c->ev[6], s);
  return cudaGetLastError();
}

cudaError_t launch_apply64(sgf_ctx* c, const zd* mu, zd* out) { return apply_t<double>(c, c->o64, mu, out); }
cudaError_t launch_apply32(sgf_ctx* c, const zd* mu, zd* out) { return apply_t<float>(c, c->o32, mu, out); }

// ============================================================== several densities at once
// The forward map on up to MC_MAX density columns in one pass over the operator data: the
// projection stages each chunk's P block in shared memory once for all columns, the near rows read
// each block-sparse row once for all columns, the reconstruction rows stay in registers across
// columns; the X passes and Y convolutions run every column's grids in one launch. Columns may
// belong to problems that differ only in the incidence angle (same surface, wavenumber and
// parameters): P, the reconstruction rows and the near operator are then shared, and the angle
// enters through per-column twists, phases, spectra and mode factors (MCol).

// Shared memory of k_near_multi: ncol staged density columns of W entries plus ncol results per row.
static size_t near_multi_smem(int maxW, int ncol, size_t esz) { return ((size_t)ncol * maxW + 32 * ncol) * esz; }

template <typename T>
__global__ void __launch_bounds__(128) k_project_multi(int neq, long N, const int* __restrict__ cell_start,
                                                       const int* __restrict__ node_idx, const cplx<T>* __restrict__ P,
                                                       const int* __restrict__ src_gidx, MCols<T> cols,
                                                       cplx<T>* __restrict__ gH, long gH_stride, cplx<T>* __restrict__ gV,
                                                       long gV_stride, zd* __restrict__ mpart, float4* __restrict__ mpart_ff,
                                                       long mp_col, int MB, int nm_max, int n_items,
                                                       const int* __restrict__ item_cell, const int* __restrict__ item_lo,
                                                       const int* __restrict__ item_hi) {
  extern __shared__ unsigned char smem_raw[];
  if ((int)blockIdx.x >= n_items) {  // mode partials: (column, mode, chunk)
    const int t = blockIdx.x - n_items;
    const int r = t / (nm_max * MB), rem = t % (nm_max * MB);
    const MCol<T>& cr = cols.c[r];
    if (rem / MB < cr.nm)
      mode_partial<T>(rem / MB, rem % MB, MB, N, cr.mu, cr.MS, cr.MSff, mpart + r * mp_col, mpart_ff + r * mp_col);
    return;
  }
  const int nout = 4 * neq;
  cplx<T>* Ps = reinterpret_cast<cplx<T>*>(smem_raw);  // [nq][nout] of this chunk
  cplx<T>* mus = Ps + 32 * nout;                       // [32] densities of one column
  const int q = item_cell[blockIdx.x];
  const int lo = item_lo[blockIdx.x], nq = item_hi[blockIdx.x] - lo;
  const int s0 = cell_start[q] + lo;
  for (int e = threadIdx.x; e < nq * nout; e += blockDim.x) Ps[e] = P[(long)nout * s0 + e];
  const int o = threadIdx.x;
  long idx = 0, goff = 0;
  int lam = 0;
  if (o < nout) {
    lam = o / (2 * neq);
    const int sidx = o % (2 * neq), si = sidx % neq;
    idx = ((long)q * 2 + lam) * neq + si;
    goff = (sidx < neq ? 0 : (lam == 0 ? gH_stride : gV_stride)) + src_gidx[idx];
  }
  for (int r = 0; r < cols.n; ++r) {
    __syncthreads();  // Ps staged; the previous column's densities consumed
    for (int l = threadIdx.x; l < nq; l += blockDim.x) mus[l] = cplx<T>(cols.c[r].mu[node_idx[s0 + l]]);
    __syncthreads();
    if (o < nout) {
      cplx<T> acc[4] = {cplx<T>(0, 0), cplx<T>(0, 0), cplx<T>(0, 0), cplx<T>(0, 0)};
      for (int u = 0; u < nq; ++u) acc[u & 3] = fma_c(Ps[u * nout + o], mus[u], acc[u & 3]);
      const cplx<T> v = ((acc[0] + acc[1]) + (acc[2] + acc[3])) * cols.c[r].src_tw[idx];
      cplx<T>* dst = (lam == 0 ? gH + r * 2 * gH_stride : gV + r * 2 * gV_stride) + goff;
      atomicAdd(&dst->re, v.re);
      atomicAdd(&dst->im, v.im);
    }
  }
}

// The block-sparse near rows plus the sigma/2 identity for ncol columns: each staged density of a
// wrapped source cell carries its column's quasi-periodic phase relative to the operator's
// (e^{i (alpha_col - alpha) d wrap}); each row of C is read once for all columns.
template <typename T, int NC>
__global__ void __launch_bounds__(256) k_near_multi(double half_sigma, double d, const int* __restrict__ cell_start,
                                                    const int* __restrict__ node_idx, const int* __restrict__ cols_idx,
                                                    const int* __restrict__ coloff, const signed char* __restrict__ colwrap,
                                                    const long* __restrict__ cell_off, const int* __restrict__ cell_W,
                                                    const zd* __restrict__ C, const float4* __restrict__ Cff,
                                                    const int* __restrict__ item_cell, const int* __restrict__ item_lo,
                                                    const int* __restrict__ item_hi, MCols<T> cols) {
  constexpr bool FF = sizeof(T) == 4;
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const int q = item_cell[blockIdx.x];
  const int rlo = item_lo[blockIdx.x];
  const int s0 = cell_start[q] + rlo, nq = item_hi[blockIdx.x] - rlo;
  const int W = cell_W[q], nc = cols.n;
  zd* mus = reinterpret_cast<zd*>(smem_raw);        // [nc][W] (FP64) or float4 pairs (float-float)
  float4* musf = reinterpret_cast<float4*>(smem_raw);
  zd* resd = mus + (long)nc * W;                    // [nq][nc]
  float4* resf = musf + (long)nc * W;
  const int* cq = cols_idx + coloff[q];
  const signed char* wq = colwrap + coloff[q];
  for (int e = threadIdx.x; e < nc * W; e += blockDim.x) {
    const int r = e / W, cc = e - r * W;
    zd m = cols.c[r].mu[cq[cc]];
    const int w = wq[cc];
    if (w != 0 && cols.c[r].dalpha != 0.0) m = m * expi(cols.c[r].dalpha * d * w);
    if (FF)
      musf[e] = cff_from(m);
    else
      mus[e] = m;
  }
  __syncthreads();
  for (int il = warp; il < nq; il += nw) {
    if (FF) {
      dot2c a[NC];
#pragma unroll
      for (int r = 0; r < NC; ++r) a[r] = {0.f, 0.f, 0.f, 0.f};
      const float4* Cr = Cff + cell_off[q] + (long)(rlo + il) * W;
      for (int cc = lane; cc < W; cc += 32) {
        const float4 v = Cr[cc];
#pragma unroll
        for (int r = 0; r < NC; ++r)
          if (r < nc) dot2_mac(v, musf[r * W + cc], a[r]);
      }
#pragma unroll
      for (int r = 0; r < NC; ++r) {
        if (r >= nc) break;
        for (int o2 = 16; o2 > 0; o2 >>= 1) {
          dot2c t = {__shfl_down_sync(0xffffffffu, a[r].sr, o2), __shfl_down_sync(0xffffffffu, a[r].si, o2),
                     __shfl_down_sync(0xffffffffu, a[r].er, o2), __shfl_down_sync(0xffffffffu, a[r].ei, o2)};
          dot2_merge(a[r], t);
        }
        if (lane == 0) {
          ff vr = ff_add({a[r].sr, 0.f}, {a[r].er, 0.f}), vi = ff_add({a[r].si, 0.f}, {a[r].ei, 0.f});
          resf[il * nc + r] = make_float4(vr.hi, vi.hi, vr.lo, vi.lo);
        }
      }
    } else {
      zd acc[NC];
#pragma unroll
      for (int r = 0; r < NC; ++r) acc[r] = zd(0, 0);
      const zd* Cr = C + cell_off[q] + (long)(rlo + il) * W;
      for (int cc = lane; cc < W; cc += 32) {
        const zd v = Cr[cc];
#pragma unroll
        for (int r = 0; r < NC; ++r)
          if (r < nc) acc[r] = fma_c(v, mus[r * W + cc], acc[r]);
      }
#pragma unroll
      for (int r = 0; r < NC; ++r) {
        if (r >= nc) break;
        const zd t = warp_sum(acc[r]);
        if (lane == 0) resd[il * nc + r] = t;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nq * nc; e += blockDim.x) {
    const int il = e / nc, r = e - il * nc;
    const int i = node_idx[s0 + il];
    const zd mi = cols.c[r].mu[i];
    zd v;
    if (FF) {
      const float4 rr = resf[e];
      ff vr = {rr.x, rr.z}, vi = {rr.y, rr.w};
      const float4 m = cff_from(mi);
      const float hs = (float)half_sigma;  // +-1/2: exact scaling
      vr = ff_add(vr, {hs * m.x, hs * m.z});
      vi = ff_add(vi, {hs * m.y, hs * m.w});
      v = zd(ff_to_double(vr), ff_to_double(vi));
    } else {
      v = resd[e] + half_sigma * mi;
    }
    cols.c[r].out[i] = v;
  }
}

// Combine-lambda + PlaneWaveWeights + NonIntersecting + EvalModes for ncol columns: the block's
// reconstruction rows are loaded once; each column gathers its cell samples, times the untwist
// e^{i (alpha_col - alpha) x_t} of sample t relative to the one folded into the rows, and adds its
// far field and its modes.
template <typename T>
__global__ void __launch_bounds__(128) k_interp_multi(int nfit, long N, const int* __restrict__ cell_start,
                                                      const int* __restrict__ node_idx, const int* __restrict__ samp_gidx,
                                                      int pH, const cplx<T>* __restrict__ gH, long gH_col,
                                                      const cplx<T>* __restrict__ gV, long gV_col,
                                                      const cplx<T>* __restrict__ Ip, const int* __restrict__ occ_cx,
                                                      double L, const double* __restrict__ samp_rel,
                                                      const zd* __restrict__ mpart, const float4* __restrict__ mpart_ff,
                                                      long mp_col, int MB, const int* __restrict__ item_cell,
                                                      const int* __restrict__ item_lo, const int* __restrict__ item_hi,
                                                      MCols<T> cols) {
  constexpr bool FF = sizeof(T) == 4;
  SGF_SHARED_ARRAY(cplx<T>, ph, 64);
  SGF_SHARED_ARRAY(cplx<T>, far_s, 32);
  __shared__ float4 msf[8];
  SGF_SHARED_ARRAY(zd, msd, 8);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  const int q = item_cell[blockIdx.x];
  const int rlo = item_lo[blockIdx.x];
  const int s0 = cell_start[q] + rlo, nq = item_hi[blockIdx.x] - rlo;
  const int il = threadIdx.x / 4, part = threadIdx.x % 4;
  cplx<T> ir[16];
  if (il < nq) {
    const cplx<T>* Ir = Ip + (long)(s0 + il) * nfit;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (part + 4 * k < nfit) ir[k] = Ir[part + 4 * k];
  }
  int irow = 0;
  if ((int)threadIdx.x < nq) irow = node_idx[s0 + threadIdx.x];
  const double cxl = occ_cx[q] * L;
  for (int r = 0; r < cols.n; ++r) {
    const MCol<T>& cr = cols.c[r];
    for (int t = threadIdx.x; t < nfit; t += blockDim.x) {
      const long gi = samp_gidx[(long)q * nfit + t];
      cplx<T> v = t < 2 * (pH + 1) ? gH[r * gH_col + gi] : gV[r * gV_col + gi];
      if (cr.dalpha != 0.0) v = v * cplx<T>(expi(cr.dalpha * (cxl + samp_rel[2 * t])));
      ph[t] = v;
    }
    // mode sums from their chunk partials: warp w folds modes w, w + 4, ... (up to 8 modes, 4 warps)
    for (int n = warp; n < cr.nm; n += blockDim.x / 32) {
      if (FF) {
        ff sr = {0.f, 0.f}, si = {0.f, 0.f};
        for (int cch = lane; cch < MB; cch += 32) {
          float4 v = mpart_ff[r * mp_col + n * MB + cch];
          sr = ff_add(sr, {v.x, v.z});
          si = ff_add(si, {v.y, v.w});
        }
        for (int o = 16; o > 0; o >>= 1) {
          sr = ff_add(sr, {__shfl_down_sync(0xffffffffu, sr.hi, o), __shfl_down_sync(0xffffffffu, sr.lo, o)});
          si = ff_add(si, {__shfl_down_sync(0xffffffffu, si.hi, o), __shfl_down_sync(0xffffffffu, si.lo, o)});
        }
        if (lane == 0) msf[n] = make_float4(sr.hi, si.hi, sr.lo, si.lo);
      } else {
        zd a(0, 0);
        for (int cch = lane; cch < MB; cch += 32) a += mpart[r * mp_col + n * MB + cch];
        a = warp_sum(a);
        if (lane == 0) msd[n] = a;
      }
    }
    __syncthreads();
    cplx<T> far(0, 0);
    if (il < nq) {
#pragma unroll
      for (int k = 0; k < 16; ++k)
        if (part + 4 * k < nfit) far = fma_c(ir[k], ph[part + 4 * k], far);
    }
    for (int o = 2; o > 0; o >>= 1) {
      far.re += __shfl_down_sync(0xffffffffu, far.re, o);
      far.im += __shfl_down_sync(0xffffffffu, far.im, o);
    }
    if (part == 0 && il < nq) far_s[il] = far;
    __syncthreads();
    if ((int)threadIdx.x < nq) {
      const int i = irow;
      zd v = cr.out[i] + zd((double)far_s[threadIdx.x].re, (double)far_s[threadIdx.x].im);
      if (FF) {
        ff vr = {0.f, 0.f}, vi = {0.f, 0.f};
        for (int n = 0; n < cr.nm; ++n) cff_mac(cr.MTff[(long)i * cr.nm + n], msf[n], vr, vi);
        v += zd(ff_to_double(vr), ff_to_double(vi));
      } else {
        for (int n = 0; n < cr.nm; ++n) v += cr.MT[(long)i * cr.nm + n] * msd[n];
      }
      cr.out[i] = v;
    }
    __syncthreads();  // ph, far_s and the mode sums are reused by the next column
  }
}

// Multi-column work space of one precision (allocated on first use): grids [col][xi, zeta][Px nrow]
// per orientation, the global-scratch convolution columns, mode partials [col][mode][chunk].
template <typename T>
cudaError_t multi_space(sgf_ctx* c, MultiSpace<T>& ms) {
  if (ms.ready) return cudaSuccess;
  cudaError_t e;
  for (int lam = 0; lam < 2; ++lam) {
    const Orient& o = c->og[lam];
    if ((e = cudaMalloc(&ms.grid[lam], (size_t)MC_MAX * 2 * o.Px * o.nrow * sizeof(cplx<T>))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&ms.accg[lam], (size_t)MC_MAX * o.Px * o.Py * sizeof(cplx<T>))) != cudaSuccess) return e;
  }
  const size_t mp = (size_t)MC_MAX * 8 * c->mode_chunks;
  if ((e = cudaMalloc(&ms.mpart, mp * sizeof(zd))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&ms.mpart_ff, mp * sizeof(float4))) != cudaSuccess) return e;
  ms.ready = true;
  return cudaSuccess;
}

template <typename T>
cudaError_t apply_multi_t(sgf_ctx* c, OpData<T>& od, MultiSpace<T>& ms, const MCols<T>& cols,
                          const cplx<T>* const Khat[2][2], long kstride, cudaStream_t s) {
  cudaError_t e = multi_space<T>(c, ms);
  if (e != cudaSuccess) return e;
  const int nc = cols.n;
  if (nc < 1 || nc > MC_MAX) return cudaErrorInvalidValue;
  int nm_max = 0;
  for (int r = 0; r < nc; ++r) nm_max = std::max(nm_max, cols.c[r].nm);
  const long mp_col = 8L * c->mode_chunks;
  long sz[2];
  for (int lam = 0; lam < 2; ++lam) {
    sz[lam] = (long)c->og[lam].Px * c->og[lam].nrow;
    cudaMemsetAsync(ms.grid[lam], 0, (size_t)nc * 2 * sz[lam] * sizeof(cplx<T>), s);
  }
  const int nout = 4 * c->neq;
  const size_t smp = ((size_t)32 * nout + 32) * sizeof(cplx<T>);
  cudaFuncSetAttribute(k_project_multi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
  k_project_multi<T><<<c->n_items + nc * nm_max * c->mode_chunks, 128, smp, s>>>(
      c->neq, c->N, c->d_cell_start, c->d_node_idx, od.P, c->d_src_gidx, cols, ms.grid[0], sz[0], ms.grid[1], sz[1],
      ms.mpart, ms.mpart_ff, mp_col, c->mode_chunks, nm_max, c->n_items, c->d_item_cell, c->d_item_lo,
      c->d_item_hi);
  for (int lam = 0; lam < 2; ++lam) {
    const Orient& o = c->og[lam];
    if ((e = run_fft_x<T>(ms.grid[lam], o, o.nrow, 2 * nc, od.tw, c->twlog, -1, s)) != cudaSuccess) return e;
    // kstride < 0: every column's spectra side by side, P_x P_y apart in each orientation
    const long ks = kstride < 0 ? (long)o.Px * o.Py : kstride;
    if ((e = conv_y_any<T, false>(ms.grid[lam], ms.grid[lam] + sz[lam], Khat[lam][0], Khat[lam][1], o, od.twy[lam],
                                  ms.accg[lam], s, nc, 2 * sz[lam], ks)) != cudaSuccess)
      return e;
    if ((e = run_fft_x<T>(ms.grid[lam], o, o.nrow, nc, od.tw, c->twlog, +1, s, 2 * sz[lam])) != cudaSuccess) return e;
  }
  const double hs = c->bc == 0 ? 0.5 : -0.5;
  const size_t smn = near_multi_smem(c->maxW, nc, sizeof(cplx<T>) == 8 ? sizeof(float4) : sizeof(zd));
  if (smn > 200 * 1024) return cudaErrorInvalidValue;
  cudaFuncSetAttribute(k_near_multi<T, MC_MAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smn);
  k_near_multi<T, MC_MAX><<<c->n_nitems, 256, smn, s>>>(hs, c->d, c->d_cell_start, c->d_node_idx, c->d_cols,
                                                         c->d_coloff, c->d_colwrap, c->d_cell_off, c->d_cell_W, c->d_C,
                                                         c->d_Cff, c->d_nitem_cell, c->d_nitem_lo, c->d_nitem_hi, cols);
  k_interp_multi<T><<<c->n_items, 128, 0, s>>>(c->nfit, c->N, c->d_cell_start, c->d_node_idx, c->d_samp_gidx, c->prm.p,
                                               ms.grid[0], 2 * sz[0], ms.grid[1], 2 * sz[1], od.Ip, c->d_occ_cx, c->L,
                                               c->keep.samp_rel, ms.mpart, ms.mpart_ff, mp_col, c->mode_chunks,
                                               c->d_item_cell, c->d_item_lo, c->d_item_hi, cols);
  return cudaGetLastError();
}

// nrhs densities of one operator (same alpha), MC_MAX columns per pass.
template <typename T>
static cudaError_t apply_nrhs_t(sgf_ctx* c, OpData<T>& od, MultiSpace<T>& ms, const zd* mu, zd* out, int nrhs) {
  const cplx<T>* K[2][2] = {{od.Khat[0][0], od.Khat[0][1]}, {od.Khat[1][0], od.Khat[1][1]}};
  // columns per pass: MC_MAX, or fewer when the staged densities of the longest near row would not
  // fit the shared memory
  const int nc_fit = (int)((200 * 1024) / (16 * ((size_t)c->maxW + 32)));
  const int chunk = std::max(1, std::min(MC_MAX, nc_fit));
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    MCols<T> cols;
    cols.n = std::min(chunk, nrhs - r0);
    for (int r = 0; r < cols.n; ++r) {
      MCol<T>& cr = cols.c[r];
      cr.mu = mu + (size_t)(r0 + r) * c->N;
      cr.out = out + (size_t)(r0 + r) * c->N;
      cr.src_tw = od.src_tw;
      cr.dalpha = 0.0;
      cr.MT = c->d_MT;
      cr.MS = c->d_MS;
      cr.MTff = c->d_MTff;
      cr.MSff = c->d_MSff;
      cr.nm = c->nm;
    }
    cudaError_t e = apply_multi_t<T>(c, od, ms, cols, K, 0, c->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t multi_space<double>(sgf_ctx*, MultiSpace<double>&);
template cudaError_t multi_space<float>(sgf_ctx*, MultiSpace<float>&);
template cudaError_t apply_multi_t<double>(sgf_ctx*, OpData<double>&, MultiSpace<double>&, const MCols<double>&,
                                           const cplx<double>* const[2][2], long, cudaStream_t);
template cudaError_t apply_multi_t<float>(sgf_ctx*, OpData<float>&, MultiSpace<float>&, const MCols<float>&,
                                          const cplx<float>* const[2][2], long, cudaStream_t);

cudaError_t launch_apply_nrhs64(sgf_ctx* c, const zd* mu, zd* out, int nrhs) {
  return apply_nrhs_t<double>(c, c->o64, c->ms64, mu, out, nrhs);
}
cudaError_t launch_apply_nrhs32(sgf_ctx* c, const zd* mu, zd* out, int nrhs) {
  return apply_nrhs_t<float>(c, c->o32, c->ms32, mu, out, nrhs);
}

// EqSources + GlobalEqSMerge + GlobalFFT alone, in FP64 on the context's stream: leaves the
// twisted phi^all of every grid point in o64.grid[lambda] (first array of each orientation) for
// evaluations at points other than the nodes.
cudaError_t launch_far_grids64(sgf_ctx* c, const zd* mu) {
  cudaStream_t s = c->stream;
  OpData<double>& od = c->o64;
  const Orient& oH = c->og[0];
  const Orient& oV = c->og[1];
  long szH = (long)oH.Px * oH.nrow, szV = (long)oV.Px * oV.nrow;
  cudaMemsetAsync(od.grid[0], 0, 2 * szH * sizeof(zd), s);
  cudaMemsetAsync(od.grid[1], 0, 2 * szV * sizeof(zd), s);
  k_project<double><<<c->n_items + c->nm * c->mode_chunks, 128, (size_t)32 * sizeof(zd), s>>>(
      c->n_occ, c->neq, c->nm, c->N, c->d_cell_start, c->d_node_idx, mu, od.P, c->d_src_gidx, od.src_tw, od.grid[0],
      szH, od.grid[1], szV, c->d_MS, c->d_MSff, c->d_mpart, c->d_mpart_ff, nullptr, c->mode_chunks, c->n_items,
      c->d_item_cell, c->d_item_lo, c->d_item_hi);
  cudaError_t e;
  for (int lam = 0; lam < 2; ++lam) {
    const Orient& o = c->og[lam];
    long sz = (long)o.Px * o.nrow;
    if ((e = run_fft_x<double>(od.grid[lam], o, o.nrow, 2, od.tw, c->twlog, -1, s)) != cudaSuccess) return e;
    e = conv_y<double>(od.grid[lam], od.grid[lam] + sz, od.Khat[lam][0], od.Khat[lam][1], o, od.twy[lam],
                       od.accg[lam], s);
    if (e != cudaSuccess) return e;
    if ((e = run_fft_x<double>(od.grid[lam], o, o.nrow, 1, od.tw, c->twlog, +1, s)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

// ============================================================== adjoint map
// The forward map is  out = hs mu + MT (MS mu) + C mu + Ip G(K (S P mu))  with P the per-cell
// projections, S the twisted scatter onto the grids, K the grid convolution, G the gather of the
// cell samples and Ip the (untwisted) reconstruction rows. Its conjugate transpose runs the same
// stages backwards: Ip^H and G^H (k_interp_adj), K^H (conjugate spectra, k_conv_y_adj), S^H and
// P^H (k_project_adj), with C^H stored as its own row-contiguous layout and the mode factors
// conjugate-transposed at build time.

// dst[c * R + r] = conj(src[r * Cc + c])
__global__ void k_conj_transpose(const zd* __restrict__ src, long R, long Cc, zd* __restrict__ dst) {
  long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= R * Cc) return;
  long r = t / Cc, cc = t % Cc;
  dst[cc * R + r] = conj(src[t]);
}
cudaError_t launch_conj_transpose(const zd* src, long R, long Cc, zd* dst, cudaStream_t s) {
  if (R * Cc == 0) return cudaSuccess;
  k_conj_transpose<<<ceil_div(R * Cc, 256), 256, 0, s>>>(src, R, Cc, dst);
  return cudaGetLastError();
}

// Block (q, r) of the near operator (n_q x n_r at src_off, leading dimension src_ld) conjugated
// and transposed into the rows of cell r of the adjoint layout (at dst_off, leading dimension dst_ld).
__global__ void k_near_transpose(const int* __restrict__ bq, const int* __restrict__ br,
                                 const long* __restrict__ src_off, const int* __restrict__ src_ld,
                                 const long* __restrict__ dst_off, const int* __restrict__ dst_ld,
                                 const int* __restrict__ cell_start, const zd* __restrict__ C, zd* __restrict__ CT) {
  const int b = blockIdx.x;
  const int q = bq[b], r = br[b];
  const int nq = cell_start[q + 1] - cell_start[q], nr = cell_start[r + 1] - cell_start[r];
  const zd* src = C + src_off[b];
  zd* dst = CT + dst_off[b];
  const int ls = src_ld[b], ld = dst_ld[b];
  for (int t = threadIdx.x; t < nq * nr; t += blockDim.x) {
    int i = t / nr, l = t % nr;
    dst[(long)l * ld + i] = conj(src[(long)i * ls + l]);
  }
}
cudaError_t launch_near_transpose(int nblk, const int* bq, const int* br, const long* src_off, const int* src_ld,
                                  const long* dst_off, const int* dst_ld, const int* cell_start, const zd* C, zd* CT,
                                  cudaStream_t s) {
  if (nblk == 0) return cudaSuccess;
  k_near_transpose<<<nblk, 256, 0, s>>>(bq, br, src_off, src_ld, dst_off, dst_ld, cell_start, C, CT);
  return cudaGetLastError();
}

// Ip^H and G^H: block per work item (chunk of at most 32 nodes of a cell), one thread per sample t:
// the sample's share sum_i conj(Ip[i][t]) v_i is added into the grid point it was gathered from.
// The tail blocks form the mode-sum partials sum_i conj(MT[i][n]) v_i; for the mixed path the
// item blocks also write the float-float copy of v used by the adjoint near field.
template <typename T>
__global__ void k_interp_adj(int mask, int nfit, long N, int pH, const int* __restrict__ cell_start,
                             const int* __restrict__ node_idx, const int* __restrict__ samp_gidx,
                             const cplx<T>* __restrict__ Ip, cplx<T>* __restrict__ gH, cplx<T>* __restrict__ gV,
                             const zd* __restrict__ MTh, const float4* __restrict__ MThff, zd* __restrict__ mpart,
                             float4* __restrict__ mpart_ff, float4* __restrict__ vff, int MB, int n_items,
                             const int* __restrict__ item_cell, const int* __restrict__ item_lo,
                             const int* __restrict__ item_hi, const zd* __restrict__ v) {
  SGF_SHARED_ARRAY(cplx<T>, vs, 32);
  if ((int)blockIdx.x >= n_items) {
    const int t = blockIdx.x - n_items;
    mode_partial<T>(t / MB, t % MB, MB, N, v, MTh, MThff, mpart, mpart_ff);
    return;
  }
  const int q = item_cell[blockIdx.x];
  const int lo = item_lo[blockIdx.x], nq = item_hi[blockIdx.x] - lo;
  const int s0 = cell_start[q] + lo;
  for (int l = threadIdx.x; l < nq; l += blockDim.x) {
    const int nid = node_idx[s0 + l];
    const zd m = v[nid];
    vs[l] = cplx<T>(m);
    if (vff) vff[nid] = cff_from(m);
  }
  __syncthreads();
  if (!(mask & 1)) return;
  for (int t = threadIdx.x; t < nfit; t += blockDim.x) {
    cplx<T> acc(0, 0);
    for (int l = 0; l < nq; ++l) acc += mulc(vs[l], Ip[(long)(s0 + l) * nfit + t]);
    long gi = samp_gidx[(long)q * nfit + t];
    cplx<T>* base = t < 2 * (pH + 1) ? gH : gV;
    atomicAdd(&base[gi].re, acc.re);
    atomicAdd(&base[gi].im, acc.im);
  }
}

// S^H and P^H, then C^H, the mode and identity terms: block per work item, rows are the nodes of
// the chunk. The adjoint source values g_o = conj(twist) * grid'(source o of the cell) are staged in
// shared memory with the densities of the cell's adjoint columns; each warp reduces a row's
// far (sum_o conj(P[i][o]) g_o) and near (C^H row) sums; one thread per row adds the identity and
// mode terms. T = float: FP32 far field, float-float near field and modes, as in the forward map.
template <typename T>
__global__ void k_project_adj(int mask, int neq, int nm, double half_sigma, const int* __restrict__ cell_start,
                              const int* __restrict__ node_idx, const cplx<T>* __restrict__ P,
                              const int* __restrict__ src_gidx, const cplx<T>* __restrict__ src_tw,
                              const cplx<T>* __restrict__ gH, long gH_stride, const cplx<T>* __restrict__ gV,
                              long gV_stride, const int* __restrict__ colsT, const int* __restrict__ coloffT,
                              const long* __restrict__ cell_offT, const int* __restrict__ cell_WT,
                              const zd* __restrict__ CT, const float4* __restrict__ CTff,
                              const float4* __restrict__ vff, const zd* __restrict__ MSh,
                              const float4* __restrict__ MShff, const zd* __restrict__ mpart,
                              const float4* __restrict__ mpart_ff, int MB, const int* __restrict__ item_cell,
                              const int* __restrict__ item_lo, const int* __restrict__ item_hi,
                              const zd* __restrict__ v, zd* __restrict__ out) {
  constexpr bool FF = sizeof(T) == 4;
  extern __shared__ unsigned char smem_raw[];
  __shared__ float4 msf[8];
  SGF_SHARED_ARRAY(zd, msd, 8);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const int q = item_cell[blockIdx.x];
  const int rlo = item_lo[blockIdx.x];
  const int s0 = cell_start[q] + rlo, nq = item_hi[blockIdx.x] - rlo;
  const int W = cell_WT[q];
  const int nout = 4 * neq;
  // shared layout: [W] densities, [32] per-row results, [nout] source values (16 B each)
  zd* vsd = reinterpret_cast<zd*>(smem_raw);
  float4* vsf = reinterpret_cast<float4*>(smem_raw);
  zd* resd = reinterpret_cast<zd*>(smem_raw) + W;
  float4* resf = reinterpret_cast<float4*>(smem_raw) + W;
  cplx<T>* g = reinterpret_cast<cplx<T>*>(reinterpret_cast<zd*>(smem_raw) + W + 32);
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    int lam = o / (2 * neq), sidx = o % (2 * neq), si = sidx % neq;
    long idx = ((long)q * 2 + lam) * neq + si;
    const cplx<T>* base = lam == 0 ? gH + (sidx < neq ? 0 : gH_stride) : gV + (sidx < neq ? 0 : gV_stride);
    g[o] = mulc(base[src_gidx[idx]], src_tw[idx]);
  }
  for (int n = warp; n < nm && (mask & 4); n += nw) {  // mode sums: warp w folds modes w, w + nw, ...
    if (FF) {
      ff sr = {0.f, 0.f}, si = {0.f, 0.f};
      for (int cch = lane; cch < MB; cch += 32) {
        float4 a = mpart_ff[n * MB + cch];
        sr = ff_add(sr, {a.x, a.z});
        si = ff_add(si, {a.y, a.w});
      }
      for (int o = 16; o > 0; o >>= 1) {
        sr = ff_add(sr, {__shfl_down_sync(0xffffffffu, sr.hi, o), __shfl_down_sync(0xffffffffu, sr.lo, o)});
        si = ff_add(si, {__shfl_down_sync(0xffffffffu, si.hi, o), __shfl_down_sync(0xffffffffu, si.lo, o)});
      }
      if (lane == 0) msf[n] = make_float4(sr.hi, si.hi, sr.lo, si.lo);
    } else {
      zd a(0, 0);
      for (int cch = lane; cch < MB; cch += 32) a += mpart[n * MB + cch];
      a = warp_sum(a);
      if (lane == 0) msd[n] = a;
    }
  }
  const int* cq = colsT + coloffT[q];
  if (FF) {
    for (int cc = threadIdx.x; cc < W; cc += blockDim.x) vsf[cc] = vff[cq[cc]];
  } else {
    for (int cc = threadIdx.x; cc < W; cc += blockDim.x) vsd[cc] = v[cq[cc]];
  }
  __syncthreads();
  for (int il = warp; il < nq; il += nw) {
    cplx<T> far(0, 0);
    if (mask & 1) {
      const cplx<T>* Pr = P + (long)(s0 + il) * nout;
      for (int o = lane; o < nout; o += 32) far += mulc(g[o], Pr[o]);
    }
    far = warp_sum(far);
    if (FF) {
      ff ar = {0.f, 0.f}, ai = {0.f, 0.f};
      if (mask & 2) {
        const float4* Cr = CTff + cell_offT[q] + (long)(rlo + il) * W;
        ff br = {0.f, 0.f}, bi = {0.f, 0.f};
        int cc = lane;
        for (; cc + 32 < W; cc += 64) {
          cff_mac(Cr[cc], vsf[cc], ar, ai);
          cff_mac(Cr[cc + 32], vsf[cc + 32], br, bi);
        }
        if (cc < W) cff_mac(Cr[cc], vsf[cc], ar, ai);
        ar = ff_add(ar, br);
        ai = ff_add(ai, bi);
        for (int o = 16; o > 0; o >>= 1) {
          ar = ff_add(ar, {__shfl_down_sync(0xffffffffu, ar.hi, o), __shfl_down_sync(0xffffffffu, ar.lo, o)});
          ai = ff_add(ai, {__shfl_down_sync(0xffffffffu, ai.hi, o), __shfl_down_sync(0xffffffffu, ai.lo, o)});
        }
      }
      if (lane == 0) {
        ar = ff_add(ar, {(float)far.re, 0.f});
        ai = ff_add(ai, {(float)far.im, 0.f});
        resf[il] = make_float4(ar.hi, ai.hi, ar.lo, ai.lo);
      }
    } else {
      zd acc(0, 0);
      if (mask & 2) {
        const zd* Cr = CT + cell_offT[q] + (long)(rlo + il) * W;
        zd acc1(0, 0), acc2(0, 0), acc3(0, 0);
        int cc = lane;
        for (; cc + 96 < W; cc += 128) {
          acc = fma_c(Cr[cc], vsd[cc], acc);
          acc1 = fma_c(Cr[cc + 32], vsd[cc + 32], acc1);
          acc2 = fma_c(Cr[cc + 64], vsd[cc + 64], acc2);
          acc3 = fma_c(Cr[cc + 96], vsd[cc + 96], acc3);
        }
        for (; cc < W; cc += 32) acc = fma_c(Cr[cc], vsd[cc], acc);
        acc = warp_sum((acc + acc1) + (acc2 + acc3));
      }
      if (lane == 0) resd[il] = acc + zd((double)far.re, (double)far.im);
    }
  }
  __syncthreads();
  for (int il = threadIdx.x; il < nq; il += blockDim.x) {
    const int i = node_idx[s0 + il];
    if (FF) {
      float4 r = resf[il];
      ff vr = {r.x, r.z}, vi = {r.y, r.w};
      if (mask & 8) {
        float4 m = vff[i];
        float hs = (float)half_sigma;
        vr = ff_add(vr, {hs * m.x, hs * m.z});
        vi = ff_add(vi, {hs * m.y, hs * m.w});
      }
      if (mask & 4)
        for (int n = 0; n < nm; ++n) cff_mac(MShff[(long)i * nm + n], msf[n], vr, vi);
      out[i] = zd(ff_to_double(vr), ff_to_double(vi));
    } else {
      zd a = resd[il];
      if (mask & 8) a += half_sigma * v[i];
      if (mask & 4)
        for (int n = 0; n < nm; ++n) a += MSh[(long)i * nm + n] * msd[n];
      out[i] = a;
    }
  }
}

template <typename T>
static cudaError_t apply_adj_t(sgf_ctx* c, OpData<T>& od, const zd* v, zd* out) {
  cudaStream_t s = c->stream;
  const Orient& oH = c->og[0];
  const Orient& oV = c->og[1];
  long szH = (long)oH.Px * oH.nrow, szV = (long)oV.Px * oV.nrow;
  cudaMemsetAsync(od.grid[0], 0, szH * sizeof(cplx<T>), s);
  cudaMemsetAsync(od.grid[1], 0, szV * sizeof(cplx<T>), s);
  k_interp_adj<T><<<c->n_items + c->nm * c->mode_chunks, 64, 0, s>>>(
      c->debug_mask, c->nfit, c->N, c->prm.p, c->d_cell_start, c->d_node_idx, c->d_samp_gidx, od.Ip, od.grid[0],
      od.grid[1], c->d_MTh, c->d_MThff, c->d_mpart, c->d_mpart_ff, sizeof(T) == 4 ? c->d_muff : nullptr,
      c->mode_chunks, c->n_items, c->d_item_cell, c->d_item_lo, c->d_item_hi, v);
  cudaError_t e;
  bool fork = c->side != nullptr;
  if (fork) {
    cudaEventRecord(c->ev_fork, s);
    cudaStreamWaitEvent(c->side, c->ev_fork, 0);
  }
  for (int lam = 0; lam < 2; ++lam) {
    const Orient& o = c->og[lam];
    cudaStream_t st = (fork && lam == 1) ? c->side : s;
    long sz = (long)o.Px * o.nrow;
    if ((e = run_fft_x<T>(od.grid[lam], o, o.nrow, 1, od.tw, c->twlog, -1, st)) != cudaSuccess) return e;
    e = conv_y_adj<T>(od.grid[lam], od.grid[lam] + sz, od.Khat[lam][0], od.Khat[lam][1], o, od.twy[lam],
                      od.accg[lam], st);
    if (e != cudaSuccess) return e;
    if ((e = run_fft_x<T>(od.grid[lam], o, o.nrow, 2, od.tw, c->twlog, +1, st)) != cudaSuccess) return e;
  }
  if (fork) {
    cudaEventRecord(c->ev_join, c->side);
    cudaStreamWaitEvent(s, c->ev_join, 0);
  }
  double hs = c->bc == 0 ? 0.5 : -0.5;
  size_t sm = (size_t)(c->maxWT + 32 + 4 * c->neq) * sizeof(zd);
  cudaFuncSetAttribute(k_project_adj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_project_adj<T><<<c->n_items, 256, sm, s>>>(
      c->debug_mask, c->neq, c->nm, hs, c->d_cell_start, c->d_node_idx, od.P, c->d_src_gidx, od.src_tw, od.grid[0],
      szH, od.grid[1], szV, c->d_colsT, c->d_coloffT, c->d_cell_offT, c->d_cell_WT, c->d_CT, c->d_CTff, c->d_muff,
      c->d_MSh, c->d_MShff, c->d_mpart, c->d_mpart_ff, c->mode_chunks, c->d_item_cell, c->d_item_lo, c->d_item_hi, v,
      out);
  return cudaGetLastError();
}

cudaError_t launch_apply_adj64(sgf_ctx* c, const zd* v, zd* out) { return apply_adj_t<double>(c, c->o64, v, out); }
cudaError_t launch_apply_adj32(sgf_ctx* c, const zd* v, zd* out) { return apply_adj_t<float>(c, c->o32, v, out); }

// ------------------------------------------------------------------ CUDA graph of the forward map
// Argument positions of mu / out in k_project and k_interp_near (kept in step with their signatures).
static const int kProjArgs = 24, kProjMu = 6;
static const int kNearArgs = 15, kNearMu = 13, kNearOut = 14;
static const int kFarArgs = 19, kFarOut = 18;

void destroy_graphs(sgf_ctx* c) {
  for (auto& gs : c->gs_nonear) {
    if (gs.exec) cudaGraphExecDestroy(gs.exec);
    if (gs.g) cudaGraphDestroy(gs.g);
    gs = GraphSlot();
  }
  for (auto& gs : c->gs) {
    if (gs.exec) cudaGraphExecDestroy(gs.exec);
    if (gs.g) cudaGraphDestroy(gs.g);
    gs = GraphSlot();
  }
}

// Captures one application (on an internal stream, from the context's staging buffers) and keeps
// the instantiated graph; returns the capture or instantiation error, in which case the context
// keeps launching the kernels directly.
cudaError_t build_apply_graph(sgf_ctx* c, int prec) { return build_apply_graph_mask(c, prec, 15, c->gs[prec == 64 ? 0 : 1]); }

// The same capture with the terms of `mask` only (sgf_debug_mask bits) into the given slot.
cudaError_t build_apply_graph_mask(sgf_ctx* c, int prec, int term_mask, GraphSlot& gs) {
  cudaStream_t orig = c->stream, cap = nullptr;
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  // the projection / convolution chain is the critical path: its nodes get the highest priority,
  // the near-field branch (side2) the lowest, so that it fills the SMs the chain leaves idle
  cudaError_t e = cudaStreamCreateWithPriority(&cap, cudaStreamNonBlocking, prio_hi);
  if (e != cudaSuccess) return e;
  const bool prof = c->profiling;
  const int mask = c->debug_mask;
  c->profiling = false;
  c->debug_mask = term_mask;
  c->stream = cap;
  cudaGraph_t g = nullptr;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t ea = prec == 64 ? launch_apply64(c, c->d_mu_tmp, c->d_out_tmp) : launch_apply32(c, c->d_mu_tmp, c->d_out_tmp);
    cudaError_t ee = cudaStreamEndCapture(cap, &g);
    e = ea != cudaSuccess ? ea : ee;
  }
  c->stream = orig;
  c->profiling = prof;
  c->debug_mask = mask;
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return e;
  }
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(g, nodes.data(), &nn);
  void* fp = prec == 64 ? (void*)k_project<double> : (void*)k_project<float>;
  void* fi = prec == 64 ? (void*)k_interp_far<double> : (void*)k_interp_far<float>;
  void* fn = prec == 64 ? (void*)k_near_rows<double> : (void*)k_near_rows<float>;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    cudaGraphNodeGetType(nd, &t);
    if (t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    cudaGraphKernelNodeGetParams(nd, &kp);
    if (kp.func == fp) { gs.n_proj = nd; gs.kp_proj = kp; }
    if (kp.func == fi) { gs.n_interp = nd; gs.kp_interp = kp; }
    if (kp.func == fn) { gs.n_near = nd; gs.kp_near = kp; }
  }
  if (!gs.n_proj || !gs.n_interp || !gs.n_near) {
    cudaGraphDestroy(g);
    gs = GraphSlot();
    return cudaErrorInvalidValue;
  }
  e = cudaGraphInstantiate(&gs.exec, g, cudaGraphInstantiateFlagUseNodePriority);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    gs = GraphSlot();
    return e;
  }
  gs.g = g;
  gs.ok = true;
  return cudaSuccess;
}

cudaError_t launch_apply_graph(sgf_ctx* c, int prec, const zd* mu, zd* out) {
  GraphSlot& gs = c->gs[prec == 64 ? 0 : 1];
  void* pa[kProjArgs];
  void* pb[kFarArgs];
  void* pc[kNearArgs];
  for (int i = 0; i < kProjArgs; ++i) pa[i] = gs.kp_proj.kernelParams[i];
  for (int i = 0; i < kFarArgs; ++i) pb[i] = gs.kp_interp.kernelParams[i];
  for (int i = 0; i < kNearArgs; ++i) pc[i] = gs.kp_near.kernelParams[i];
  pa[kProjMu] = (void*)&mu;
  pb[kFarOut] = (void*)&out;
  pc[kNearMu] = (void*)&mu;
  pc[kNearOut] = (void*)&out;
  cudaKernelNodeParams p1 = gs.kp_proj, p2 = gs.kp_interp, p3 = gs.kp_near;
  p1.kernelParams = pa;
  p1.extra = nullptr;
  p2.kernelParams = pb;
  p2.extra = nullptr;
  p3.kernelParams = pc;
  p3.extra = nullptr;
  cudaError_t e = cudaGraphExecKernelNodeSetParams(gs.exec, gs.n_proj, &p1);
  if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(gs.exec, gs.n_interp, &p2);
  if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(gs.exec, gs.n_near, &p3);
  if (e == cudaSuccess) e = cudaGraphLaunch(gs.exec, c->stream);
  return e;
}

// ============================================================== Rayleigh coefficients
// Block per mode: B_n = dx sum_i mu_i e^{-i(alpha_n x_i + beta_n f_i)} W_i (eq. rayexp with the
// Y > 0 spectral form of G~ and M^eta); mp[n] = [alpha_n, beta_re, beta_im, Q_re, Q_im, indicator].
__global__ void k_rayleigh(GeoArgs g, const double* __restrict__ mp, const double* __restrict__ x,
                           const double* __restrict__ f, const double* __restrict__ f1, const zd* __restrict__ mu,
                           zd* B) {
  SGF_SHARED_ARRAY(zd, red, 32);
  const int n = blockIdx.x;
  const double an = mp[6 * n];
  const zd bn(mp[6 * n + 1], mp[6 * n + 2]), Q(mp[6 * n + 3], mp[6 * n + 4]);
  const double ind = mp[6 * n + 5];
  zd acc(0, 0);
  for (int i = threadIdx.x; i < g.N; i += blockDim.x) {
    double s = sqrt(1 + f1[i] * f1[i]);
    zd e = cexpz(-(zd(0, an * x[i]) + zd(0, 1) * (f[i] * bn)));
    zd W = g.bc == 0 ? (bn - zd(an * f1[i], 0)) * Q * (0.5 / g.d) + zd(s * ind, 0)
                     : s * (zd(0, 0.5 / g.d) * Q + zd(ind, 0));
    acc += mu[i] * e * W;
  }
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  acc = warp_sum(acc);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    zd v = lane < nw ? red[lane] : zd(0, 0);
    v = warp_sum(v);
    if (lane == 0) B[n] = g.dx * v;
  }
}

__global__ void k_rayleigh_weights(GeoArgs g, const double* __restrict__ mp, const double* __restrict__ x,
                                   const double* __restrict__ f, const double* __restrict__ f1, zd* w) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.N) return;
  const double an = mp[0];
  const zd bn(mp[1], mp[2]), Q(mp[3], mp[4]);
  const double ind = mp[5];
  double s = sqrt(1 + f1[i] * f1[i]);
  zd e = cexpz(-(zd(0, an * x[i]) + zd(0, 1) * (f[i] * bn)));
  zd W = g.bc == 0 ? (bn - zd(an * f1[i], 0)) * Q * (0.5 / g.d) + zd(s * ind, 0)
                   : s * (zd(0, 0.5 / g.d) * Q + zd(ind, 0));
  if (g.dmode == 1) {  // d/df of the phase
    W = (zd(0, -1) * bn) * W;
  } else if (g.dmode == 2) {  // d/df' of the weight
    W = g.bc == 0 ? (-an * 0.5 / g.d) * Q + zd(f1[i] / s * ind, 0) : (f1[i] / s) * (zd(0, 0.5 / g.d) * Q + zd(ind, 0));
  }
  w[i] = g.dx * (e * W);
}
cudaError_t launch_rayleigh_weights(sgf_ctx* c, const double* d_mp, const double* f, const double* f1, zd* w,
                                    int dmode) {
  GeoArgs g = geo_args(c);
  g.dmode = dmode;
  k_rayleigh_weights<<<ceil_div(c->N, 256), 256, 0, c->stream>>>(g, d_mp, c->d_x, f, f1, w);
  return cudaGetLastError();
}

__global__ void k_offset(const double* __restrict__ src, double eps, long n, double* __restrict__ dst) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] + eps;
}
cudaError_t launch_offset(const double* src, double eps, long n, double* dst, cudaStream_t s) {
  k_offset<<<ceil_div(n, 256), 256, 0, s>>>(src, eps, n, dst);
  return cudaGetLastError();
}
__global__ void k_conj_vec(const zd* __restrict__ x, zd* __restrict__ y, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = conj(x[i]);
}
cudaError_t launch_conj(const zd* x, zd* y, long n, cudaStream_t s) {
  k_conj_vec<<<ceil_div(n, 256), 256, 0, s>>>(x, y, n);
  return cudaGetLastError();
}
__global__ void k_grad_acc(zd* __restrict__ g, double sc, const zd* __restrict__ a, const zd* __restrict__ u,
                           const zd* __restrict__ v, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) g[i] += sc * (a[i] * (u[i] - v[i]));
}
cudaError_t launch_grad_acc(zd* g, double s, const zd* a, const zd* u, const zd* v, long n, cudaStream_t st) {
  k_grad_acc<<<ceil_div(n, 256), 256, 0, st>>>(g, s, a, u, v, n);
  return cudaGetLastError();
}

cudaError_t launch_rayleigh_mp(sgf_ctx* c, const zd* mu, int nmodes, const double* d_mp, zd* d_B) {
  GeoArgs g = geo_args(c);
  k_rayleigh<<<nmodes, 256, 0, c->stream>>>(g, d_mp, c->d_x, c->d_f, c->d_f1, mu, d_B);
  return cudaGetLastError();
}

// ============================================================== Krylov helpers (FP64)
// partial[j][blk] = sum_{i in chunk blk} conj(V[j][i]) w[i]; then out[j] = sum_blk partial.
__global__ void k_dots_partial(const zd* __restrict__ V, long ldv, const zd* __restrict__ w, long n, zd* partial,
                               int nblk) {
  SGF_SHARED_ARRAY(zd, red, 32);
  const int j = blockIdx.y, blk = blockIdx.x;
  long chunk = (n + nblk - 1) / nblk;
  long i0 = blk * chunk, i1 = min(n, i0 + chunk);
  const zd* v = V + j * ldv;
  zd acc(0, 0);
  for (long i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc += mulc(w[i], v[i]);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  acc = warp_sum(acc);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    zd s = lane < nw ? red[lane] : zd(0, 0);
    s = warp_sum(s);
    if (lane == 0) partial[(long)j * nblk + blk] = s;
  }
}
__global__ void k_dots_final(const zd* partial, int nblk, int m, zd* out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  zd s(0, 0);
  for (int b = 0; b < nblk; ++b) s += partial[(long)j * nblk + b];
  out[j] = s;
}
cudaError_t launch_dots(const zd* V, int m, long ldv, const zd* w, long n, zd* partial, int nblk, zd* out,
                        cudaStream_t s) {
  dim3 g(nblk, m);
  k_dots_partial<<<g, 256, 0, s>>>(V, ldv, w, n, partial, nblk);
  k_dots_final<<<ceil_div(m, 128), 128, 0, s>>>(partial, nblk, m, out);
  return cudaGetLastError();
}
__global__ void k_axpby(zd* y, zd a, const zd* x, zd b, long n) {
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}
cudaError_t launch_axpby(zd* y, zd a, const zd* x, zd b, long n, cudaStream_t s) {
  k_axpby<<<ceil_div(n, 256), 256, 0, s>>>(y, a, x, b, n);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Arnoldi step in float-float
// The Gram-Schmidt projections of the FP64 Krylov vectors run on the FP32 pipes: each FP64 value is
// split into two floats with integer instructions only, and the products are accumulated with the
// compensated dot product (dot2_mac), about 48 significant bits. This GPU issues an FP64 warp
// instruction about once per 64 cycles per scheduler and an FP32 or integer one every cycle, so the
// four complex FP64 multiply-adds per element and basis vector of CGS2 would cost more than reading
// the vectors; this way the step moves at memory speed. Results are written back in FP64.

// x = hi + lo: hi keeps the top 24 significant bits of x (truncated), lo the remaining 29 rounded to
// 24, so hi + lo matches x to 2^-48 relative. |x| < 2^-126 gives 0 (the vectors are normalised,
// so this drops less than 1.2e-38); |x| >= 2^128, infinities and NaN give a NaN hi, so that a
// non-finite vector still yields a non-finite inner product.
__device__ __forceinline__ float2 split_d(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sg = hw & 0x80000000u;
  const int ex = (int)((hw >> 20) & 0x7ffu);  // biased FP64 exponent
  if (ex < 897) return make_float2(0.f, 0.f);
  if (ex > 1150) return make_float2(__int_as_float(0x7fc00000), 0.f);
  const float hi = __uint_as_float(sg | ((unsigned)(ex - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
  float lo = 0.f;
  if (ex >= 949) {  // 2^(ex - 1075), the weight of the remainder's last bit, is a normal float
    const float sc = __uint_as_float((unsigned)(ex - 948) << 23);
    lo = __uint_as_float(__float_as_uint(__fmul_rn(__uint2float_rn(lw & 0x1fffffffu), sc)) | sg);
  }
  return make_float2(hi, lo);
}
// complex double -> {re.hi, im.hi, re.lo, im.lo}; conj negates the imaginary parts
__device__ __forceinline__ float4 split_z(zd z, bool conj_ = false) {
  const float2 r = split_d(z.re), i = split_d(z.im);
  return conj_ ? make_float4(r.x, -i.x, r.y, -i.y) : make_float4(r.x, i.x, r.y, i.y);
}
__device__ __forceinline__ float4 pack_dot2(const dot2c& a) { return make_float4(a.sr, a.si, a.er, a.ei); }
__device__ __forceinline__ dot2c unpack_dot2(float4 v) { return dot2c{v.x, v.y, v.z, v.w}; }
// the warp's 32 partial sums folded into lane 0
__device__ __forceinline__ void warp_merge(dot2c& a) {
  for (int o = 16; o > 0; o >>= 1) {
    dot2c b{__shfl_down_sync(0xffffffffu, a.sr, o), __shfl_down_sync(0xffffffffu, a.si, o),
            __shfl_down_sync(0xffffffffu, a.er, o), __shfl_down_sync(0xffffffffu, a.ei, o)};
    dot2_merge(a, b);
  }
}
__device__ __forceinline__ zd dot2_value(const dot2c& a) {
  return zd((double)a.sr + (double)a.er, (double)a.si + (double)a.ei);
}

constexpr int KDOT_CHUNK = 256;  // elements of w per block of k_kdots
constexpr int KDOT_VECS = 8;     // basis vectors per block (one per warp)

// h[jj] = sum over i < n of conj(V[jj][i]) w[i], jj < m; Hc[jj] = h[jj] (add = 0) or += h[jj].
// Grid (chunks of 256 elements) x (groups of 8 basis vectors), warp q of a block takes vector
// 8 blockIdx.y + q, each lane 8 elements 32 apart; the V loads are issued before the block splits
// its chunk of w into shared memory, so that both latencies overlap. Each block writes its partial
// sums to part[jj][chunk]; the block that finishes its vector group last (ticket[group], reset by it
// for the next launch; the usual fence-and-counter pattern, no waiting) folds the group's partials.
// Block (bx, by) of a grid of gx chunks: the body shared by the one-problem and batched kernels.
// A chunk past the end of the vector (batched problems of different sizes) adds zeros.
__device__ __forceinline__ void kdots_body(const zd* __restrict__ V, int m, long ldv, const zd* __restrict__ w,
                                           long n, float4* part, zd* h, zd* Hc, int add, unsigned* ticket, int bx,
                                           int by, int gx) {
  __shared__ float4 ws[KDOT_CHUNK];
  __shared__ bool last;
  const long i0 = (long)bx * KDOT_CHUNK;
  const int lane = threadIdx.x & 31;
  const int jj = by * KDOT_VECS + (threadIdx.x >> 5);
  const int cnt = (int)max(0L, min((long)KDOT_CHUNK, n - i0));
  zd vr[KDOT_CHUNK / 32];
  if (jj < m) {
    const zd* v = V + (long)jj * ldv + i0;
#pragma unroll
    for (int k = 0; k < KDOT_CHUNK / 32; ++k) {
      const int t = lane + 32 * k;
      vr[k] = t < cnt ? v[t] : zd(0, 0);
    }
  }
  for (int t = threadIdx.x; t < KDOT_CHUNK; t += blockDim.x)
    ws[t] = t < cnt ? split_z(w[i0 + t]) : make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  if (jj < m) {
    dot2c acc{0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < KDOT_CHUNK / 32; ++k) dot2_mac(split_z(vr[k], true), ws[lane + 32 * k], acc);
    warp_merge(acc);
    if (lane == 0) part[(long)jj * gx + bx] = pack_dot2(acc);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&ticket[by], 1u) == (unsigned)gx - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (jj < m) {
    dot2c acc{0.f, 0.f, 0.f, 0.f};
    for (int b = lane; b < gx; b += 32) {
      const float4 pv = __ldcg(&part[(long)jj * gx + b]);
      dot2_merge(acc, unpack_dot2(pv));
    }
    warp_merge(acc);
    if (lane == 0) {
      const zd v = dot2_value(acc);
      h[jj] = v;
      if (Hc) Hc[jj] = add ? Hc[jj] + v : v;
    }
  }
  if (threadIdx.x == 0) ticket[by] = 0;
}
__global__ void __launch_bounds__(256) k_kdots(const zd* __restrict__ V, int m, long ldv, const zd* __restrict__ w,
                                               long n, float4* part, zd* h, zd* Hc, int add, unsigned* ticket) {
  kdots_body(V, m, ldv, w, n, part, h, Hc, add, ticket, blockIdx.x, blockIdx.y, gridDim.x);
}
// tickets: one counter per group of 8 basis vectors, zero before the first launch
int kdots_groups(int m) { return (int)ceil_div(m, KDOT_VECS); }
int kdots_chunks(long n) { return (int)ceil_div(n, (long)KDOT_CHUNK); }
cudaError_t launch_kdots(const zd* V, int m, long ldv, const zd* w, long n, float4* part, zd* h, zd* Hc, int add,
                         unsigned* ticket, cudaStream_t s) {
  const int nchunk = kdots_chunks(n);
  k_kdots<<<dim3(nchunk, kdots_groups(m)), 256, 0, s>>>(V, m, ldv, w, n, part, h, Hc, add, ticket);
  return cudaGetLastError();
}
int kupdate_blocks(long n) { return (int)ceil_div(n, 32L); }

// w[i] -= sum_jj V[jj][i] h[jj], jj < m. A block takes 32 consecutive elements (threadIdx.x) and
// splits the basis vectors among its 8 thread rows (threadIdx.y), four loads in flight per thread;
// the first four are issued before h (the previous kernel's output) is read and split into shared
// memory. The rows' sums are merged in shared memory and the FP64 result written once. With npart,
// the block also writes the compensated sum of |w_new[i]|^2 over its elements to npart[blockIdx.x]
// (the norm of the orthogonalised vector, for k_kscale).
__device__ __forceinline__ void kupdate_body(zd* w, const zd* __restrict__ V, int m, long ldv,
                                             const zd* __restrict__ h, long n, float4* npart, int bx) {
  __shared__ float4 hs[256];
  __shared__ float4 rows[8][33];
  const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 32 + tx;
  const long i = (long)bx * 32 + tx;
  zd pre[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int jj = ty + 8 * u;
    pre[u] = i < n && jj < m ? V[(long)jj * ldv + i] : zd(0, 0);
  }
  dot2c acc{0.f, 0.f, 0.f, 0.f};
  for (int j0 = 0; j0 < m; j0 += 256) {
    const int cnt = min(256, m - j0);
    __syncthreads();
    if (t < cnt) hs[t] = split_z(h[j0 + t]);
    __syncthreads();
    if (i >= n) continue;
    for (int jb = ty; jb < cnt; jb += 32) {
      zd v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int jj = jb + 8 * u;
        v[u] = j0 == 0 && jb == ty ? pre[u] : (jj < cnt ? V[(long)(j0 + jj) * ldv + i] : zd(0, 0));
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (jb + 8 * u < cnt) dot2_mac(split_z(v[u]), hs[jb + 8 * u], acc);
    }
  }
  rows[ty][tx] = pack_dot2(acc);
  __syncthreads();
  if (ty == 0) {
    dot2c a = unpack_dot2(rows[0][tx]);
#pragma unroll
    for (int r = 1; r < 8; ++r) dot2_merge(a, unpack_dot2(rows[r][tx]));
    zd wn(0, 0);
    if (i < n) {
      wn = w[i] - dot2_value(a);
      w[i] = wn;
    }
    if (npart) {
      dot2c q{0.f, 0.f, 0.f, 0.f};
      dot2_mac(split_z(wn, true), split_z(wn), q);
      warp_merge(q);
      if (tx == 0) npart[bx] = pack_dot2(q);
    }
  }
}
__global__ void __launch_bounds__(256) k_kupdate(zd* w, const zd* __restrict__ V, int m, long ldv,
                                                 const zd* __restrict__ h, long n, float4* npart) {
  kupdate_body(w, V, m, ldv, h, n, npart, blockIdx.x);
}
cudaError_t launch_kupdate(zd* w, const zd* V, int m, long ldv, const zd* h, long n, float4* npart, cudaStream_t s) {
  k_kupdate<<<kupdate_blocks(n), dim3(32, 8), 0, s>>>(w, V, m, ldv, h, n, npart);
  return cudaGetLastError();
}
// |w| from the norm partials of k_kupdate (each block folds them itself); w /= |w|, or w = 0 when
// |w| = 0 (breakdown); hsub = |w| (the subdiagonal entry h_{j+1,j}), written by block 0. A
// non-finite |w| is stored as it is and propagates into w.
__device__ __forceinline__ void kscale_body(zd* w, long n, const float4* __restrict__ npart, int nparts, zd* hsub,
                                            int bx) {
  __shared__ float4 red[8];
  __shared__ double sc;
  dot2c a{0.f, 0.f, 0.f, 0.f};
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) dot2_merge(a, unpack_dot2(npart[b]));
  warp_merge(a);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pack_dot2(a);
  __syncthreads();
  if (threadIdx.x == 0) {
    dot2c q = unpack_dot2(red[0]);
    for (int r = 1; r < (int)(blockDim.x >> 5); ++r) dot2_merge(q, unpack_dot2(red[r]));
    const double hn = sqrt(dot2_value(q).re);
    sc = hn > 0 ? 1.0 / hn : (hn == 0 ? 0.0 : hn);
    if (bx == 0) *hsub = zd(hn, 0);
  }
  __syncthreads();
  const long i = (long)bx * blockDim.x + threadIdx.x;
  if (i < n) w[i] = w[i] * sc;
}
__global__ void __launch_bounds__(256) k_kscale(zd* w, long n, const float4* __restrict__ npart, int nparts,
                                                zd* hsub) {
  kscale_body(w, n, npart, nparts, hsub, blockIdx.x);
}
cudaError_t launch_kscale(zd* w, long n, const float4* npart, int nparts, zd* hsub, cudaStream_t s) {
  k_kscale<<<ceil_div(n, 256L), 256, 0, s>>>(w, n, npart, nparts, hsub);
  return cudaGetLastError();
}

// The same Arnoldi step for a batch of problems in lockstep (step j of every problem at once):
// problem p = blockIdx.z (dots) or blockIdx.y (update, scale) reads its entry of the table; its
// basis [C | V] has mr recycled vectors in front, so the step projects w = V_{j+1} against
// m = mr + j + 1 vectors. The grids cover the largest problem; blocks past a smaller problem's end
// add zeros (dots, partial norms) or do nothing (scale).
__global__ void __launch_bounds__(256) k_bkdots(const KStep* __restrict__ tab, int j, int add) {
  const KStep a = tab[blockIdx.z];
  const int m = a.mr + j + 1;
  if ((int)blockIdx.y * KDOT_VECS >= m) return;  // this vector group is empty for this problem
  kdots_body(a.W, m, a.n, a.W + (long)m * a.n, a.n, a.part, a.h, a.H + (long)j * a.ldh, add, a.ticket, blockIdx.x,
             blockIdx.y, gridDim.x);
}
__global__ void __launch_bounds__(256) k_bkupdate(const KStep* __restrict__ tab, int j, int norm) {
  const KStep a = tab[blockIdx.y];
  const int m = a.mr + j + 1;
  kupdate_body(a.W + (long)m * a.n, a.W, m, a.n, a.h, a.n, norm ? a.npart : nullptr, blockIdx.x);
}
__global__ void __launch_bounds__(256) k_bkscale(const KStep* __restrict__ tab, int j, int nparts) {
  const KStep a = tab[blockIdx.y];
  if ((long)blockIdx.x * blockDim.x >= a.n) return;
  const int m = a.mr + j + 1;
  kscale_body(a.W + (long)m * a.n, a.n, a.npart, nparts, a.H + (long)j * a.ldh + m, blockIdx.x);
}
cudaError_t launch_batch_arnoldi_step(const KStep* d_tab, int nprob, int j, int mr_max, long n_max, cudaStream_t s) {
  const int m_max = mr_max + j + 1;
  const int nchunk = kdots_chunks(n_max), ntile = kupdate_blocks(n_max);
  for (int pass = 0; pass < 2; ++pass) {
    k_bkdots<<<dim3(nchunk, kdots_groups(m_max), nprob), 256, 0, s>>>(d_tab, j, pass);
    k_bkupdate<<<dim3(ntile, nprob), dim3(32, 8), 0, s>>>(d_tab, j, pass);
  }
  k_bkscale<<<dim3((unsigned)ceil_div(n_max, 256L), nprob), 256, 0, s>>>(d_tab, j, ntile);
  return cudaGetLastError();
}
