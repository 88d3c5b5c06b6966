// Scattered field off the surface (the remark after Algorithm 3 of Bruno & Maas): once the density
// solves the Nystrom system, Algorithm 3 run once with targets in place of nodes gives the field of
// eq. int_eq_dirichlet, discretised with the operator's trapezoid weights, anywhere in the cell
// box; above the box the same sum is evaluated in its Rayleigh form (the Y > 0 spectral series of
// G~, every shifted image lying below the target).
//
//   k_field_msum      completion-mode sums S_n = sum_l MS[n][l] mu_l (eq. D_M_deltax, source side)
//   k_field_cells     block per target cell: phi^ni = phi^all - phi^int on its n_fit boundary
//                     samples (gathered from the convolved grids, the local cells' equivalent
//                     sources subtracted with the free-space shifted kernel of their cell offset)
//                     and the Fourier-Bessel weights (eqs. psi_na_sum, combine_psi_pna, plwave_QR)
//   k_field_targets   warp per target: the weights at the target (eq. planewave), the exact sum
//                     over the nodes of the local cells with G_j (eq. final_correction_0; the target
//                     is off the surface, so no singular quadrature), the completion modes
//   k_field_ray_coef  block per mode: B'_n = dx sum_l w_ln e^{-i alpha_n x_l + i beta_n (y_R - f_l)} mu_l
//   k_field_ray_eval  warp per target above the box: sum_n B'_n e^{i alpha_n x + i beta_n (y - y_R)}
// Targets are reduced to the reference period, x = x_r + w d with x_r in [0, d), and the
// quasi-periodic factor e^{i alpha d w} is restored at the end. Everything runs in FP64.
#include <cmath>
#include <complex>

#include "sgf_internal.h"

namespace {

struct FieldArgs {
  double k, alpha, beta, d, dx, L, hmin, h;
  int j, bc, p, e, nfit, neq, nb, nfb, nm;
  int PxH, PxV;
  long nrowH, nrowV;
};

__global__ void k_field_msum(long N, const zd* __restrict__ MS, const zd* __restrict__ mu, zd* __restrict__ S) {
  SGF_SHARED_ARRAY(zd, red, 32);
  const int n = blockIdx.x;
  zd acc(0, 0);
  for (long i = threadIdx.x; i < N; i += blockDim.x) acc += MS[(long)n * N + i] * mu[i];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  acc = warp_sum(acc);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    zd v = lane < nw ? red[lane] : zd(0, 0);
    v = warp_sum(v);
    if (lane == 0) S[n] = v;
  }
}

// Dynamic shared memory: n_fit samples, then the 4 n_eq densities of the block in work.
__global__ void k_field_cells(FieldArgs a, const int* __restrict__ tc_cx, const int* __restrict__ tc_cy,
                              const int* __restrict__ tc_bstart, const int* __restrict__ blk_r,
                              const int* __restrict__ blk_wrap, const int* __restrict__ blk_o,
                              const int* __restrict__ cell_start, const int* __restrict__ node_idx,
                              const zd* __restrict__ mu, const zd* __restrict__ P, const zd* __restrict__ phi_off,
                              const double* __restrict__ samp_rel, const zd* __restrict__ pinv_fb,
                              const zd* __restrict__ gH, const zd* __restrict__ gV, zd* __restrict__ W) {
  extern __shared__ unsigned char smem_raw[];
  zd* ph = reinterpret_cast<zd*>(smem_raw);
  zd* xi = ph + a.nfit;
  const int q = blockIdx.x;
  const int cx = tc_cx[q], cy = tc_cy[q];
  // phi^all at the samples: the grids hold e^{-i alpha x} phi^all, x the unwrapped sample abscissa
  for (int t = threadIdx.x; t < a.nfit; t += blockDim.x) {
    const int lam = orient_of_sample(t, a.p);
    const int tt = lam == 0 ? t : t - 2 * (a.p + 1);
    const int b = tt / (a.p + 1), s = tt % (a.p + 1);
    long ixr, iy, nrow;
    int Px;
    if (lam == 0) {
      ixr = (long)cx * a.p + s; iy = cy + b; Px = a.PxH; nrow = a.nrowH;
    } else {
      ixr = cx + b; iy = (long)cy * a.p + s + a.e; Px = a.PxV; nrow = a.nrowV;
    }
    const long ixref = ((ixr % Px) + Px) % Px;
    const zd v = (lam == 0 ? gH : gV)[ixref * nrow + iy];
    ph[t] = v * expi(a.alpha * (cx * a.L + samp_rel[2 * t]));
  }
  __syncthreads();
  // phi^int: the equivalent sources of every local cell, with the phase of its period copy
  const int nsrc = 4 * a.neq;
  for (int bb = tc_bstart[q]; bb < tc_bstart[q + 1]; ++bb) {
    const int r = blk_r[bb], rs = cell_start[r], nr = cell_start[r + 1] - rs;
    const zd wph = expi(a.alpha * a.d * blk_wrap[bb]);
    for (int o = threadIdx.x; o < nsrc; o += blockDim.x) {
      zd acc(0, 0);
      for (int l = 0; l < nr; ++l) acc += P[(long)(rs + l) * nsrc + o] * mu[node_idx[rs + l]];
      xi[o] = acc * wph;
    }
    __syncthreads();
    const zd* po = phi_off + (long)blk_o[bb] * a.nfit * 2 * a.neq;
    for (int t = threadIdx.x; t < a.nfit; t += blockDim.x) {
      const int lam = orient_of_sample(t, a.p);
      zd acc(0, 0);
      for (int s2 = 0; s2 < 2 * a.neq; ++s2) acc += po[(long)t * 2 * a.neq + s2] * xi[lam * 2 * a.neq + s2];
      ph[t] -= acc;
    }
    __syncthreads();
  }
  for (int bi = threadIdx.x; bi < a.nb; bi += blockDim.x) {
    zd acc(0, 0);
    for (int t = 0; t < a.nfit; ++t) acc += pinv_fb[(long)bi * a.nfit + t] * ph[t];
    W[(long)q * a.nb + bi] = acc;
  }
}

__global__ void k_field_targets(FieldArgs a, long n_g, const double* __restrict__ t_xr, const double* __restrict__ t_y,
                                const double* __restrict__ t_w, const double* __restrict__ t_x0,
                                const int* __restrict__ t_cell, const long* __restrict__ t_out,
                                const int* __restrict__ tc_cx, const int* __restrict__ tc_cy,
                                const int* __restrict__ tc_cstart, const int* __restrict__ col_node,
                                const signed char* __restrict__ col_wrap, const double* __restrict__ x,
                                const double* __restrict__ f, const double* __restrict__ f1,
                                const zd* __restrict__ mu, const zd* __restrict__ W,
                                const double* __restrict__ modes_n, const zd* __restrict__ msum,
                                const double* __restrict__ binw, int total, zd* __restrict__ out,
                                int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const long wid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wid >= n_g) return;  // uniform across the warp
  const double xr = t_xr[wid], y = t_y[wid];
  const int q = t_cell[wid];
  const int cx = tc_cx[q], cy = tc_cy[q];
  zd acc(0, 0);
  {  // field of the non-local sources: the cell's Fourier-Bessel expansion about its centre
    const double X = xr - (cx + 0.5) * a.L, Y = y - (a.hmin + (cy + 0.5) * a.L);
    const double kr = a.k * hypot(X, Y), th = atan2(Y, X), krho0 = a.k * a.L / sqrt(2.0);
    for (int bi = lane; bi < a.nb; bi += 32) {
      const int n = bi - a.nfb;
      acc += (1.0 / fb_norm(n, krho0)) * (W[(long)q * a.nb + bi] * fb_Z(n, kr, th));
    }
  }
  for (int c = tc_cstart[q] + lane; c < tc_cstart[q + 1]; c += 32) {  // local nodes, exactly
    const int l = col_node[c];
    const int wr = col_wrap[c];
    const double X = xr - (x[l] + wr * a.d), Y = y - f[l];
    if (hypot(X, Y) < 1e-12 * a.L) {  // a target on a node: the kernel is singular there
      atomicOr(err, 1);
      continue;
    }
    const GreenVal gv = green_j(a.k, a.j, a.h, X, Y, false, a.bc == 1, binw);
    const zd kern = a.bc == 0 ? f1[l] * gv.gx - gv.gy : sqrt(1 + f1[l] * f1[l]) * gv.g;
    acc += (a.dx * kern) * (mu[l] * expi(a.alpha * a.d * wr));
  }
  for (int n = lane; n < a.nm; n += 32) {  // completion modes M^eta
    const double an = modes_n[3 * n];
    const zd bn(modes_n[3 * n + 1], modes_n[3 * n + 2]);
    acc += cexpz(zd(0, an * xr) + zd(0, 1) * (y * bn)) * msum[n];
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    zd v = acc * expi(a.alpha * a.d * t_w[wid]);
    if (total) v += expi(a.alpha * t_x0[wid] - a.beta * y);
    out[t_out[wid]] = v;
  }
}

// mp[6 n]: [alpha_n, Re beta_n, Im beta_n, Re Q_j, Im Q_j, n in U^eta]; the weights are those of the
// Rayleigh coefficients, the height shifted to y_R so that every factor is bounded by 1.
__global__ void k_field_ray_coef(FieldArgs a, long N, const double* __restrict__ mp, double yR,
                                 const double* __restrict__ x, const double* __restrict__ f,
                                 const double* __restrict__ f1, const zd* __restrict__ mu, zd* __restrict__ Bp) {
  SGF_SHARED_ARRAY(zd, red, 32);
  const int n = blockIdx.x;
  const double an = mp[6 * n];
  const zd bn(mp[6 * n + 1], mp[6 * n + 2]), Q(mp[6 * n + 3], mp[6 * n + 4]);
  const double ind = mp[6 * n + 5];
  zd acc(0, 0);
  for (long i = threadIdx.x; i < N; i += blockDim.x) {
    const double s = sqrt(1 + f1[i] * f1[i]);
    const zd e = cexpz(zd(0, -an * x[i]) + zd(0, 1) * ((yR - f[i]) * bn));
    const zd w = a.bc == 0 ? (bn - zd(an * f1[i], 0)) * Q * (0.5 / a.d) + zd(s * ind, 0)
                           : s * (zd(0, 0.5 / a.d) * Q + zd(ind, 0));
    acc += mu[i] * e * w;
  }
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  acc = warp_sum(acc);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    zd v = lane < nw ? red[lane] : zd(0, 0);
    v = warp_sum(v);
    if (lane == 0) Bp[n] = a.dx * v;
  }
}

// Each target sums only the modes its own height needs: |n - n_0| <= n_t with the same e^{-37}
// criterion as the call's range (n_c, set by the lowest target), applied to this target's gap.
__global__ void k_field_ray_eval(FieldArgs a, long n_r, int nmod, int n_c, double fmax, const double* __restrict__ mp,
                                 double yR, const zd* __restrict__ Bp, const double* __restrict__ t_xr,
                                 const double* __restrict__ t_y, const double* __restrict__ t_w,
                                 const double* __restrict__ t_x0, const long* __restrict__ t_out, int total,
                                 zd* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long wid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wid >= n_r) return;  // uniform across the warp
  const double xr = t_xr[wid], y = t_y[wid];
  const double nt = ceil((37.0 / (y - fmax) + a.k + SGF_PI / a.d) * a.d / (2 * SGF_PI)) + 1;
  const int n_t = nt < (double)n_c ? (int)nt : n_c;
  zd acc(0, 0);
  for (int n = n_c - n_t + lane; n <= n_c + n_t && n < nmod; n += 32) {
    const zd bn(mp[6 * n + 1], mp[6 * n + 2]);
    acc += Bp[n] * cexpz(zd(0, mp[6 * n] * xr) + zd(0, 1) * ((y - yR) * bn));
  }
  acc = warp_sum(acc);
  if (lane == 0) {
    zd v = acc * expi(a.alpha * a.d * t_w[wid]);
    if (total) v += expi(a.alpha * t_x0[wid] - a.beta * y);
    out[t_out[wid]] = v;
  }
}

// Device scratch of one call, released on every return path (after the stream has drained).
struct Scratch {
  cudaStream_t s = nullptr;
  std::vector<void*> p;
  ~Scratch() {
    if (s) cudaStreamSynchronize(s);
    for (void* q : p) cudaFree(q);
  }
  template <typename T>
  cudaError_t put(T** dst, const std::vector<T>& host) {
    *dst = nullptr;
    size_t n = std::max<size_t>(1, host.size());
    cudaError_t e = cudaMalloc((void**)dst, n * sizeof(T));
    if (e != cudaSuccess) return e;
    p.push_back(*dst);
    if (host.empty()) return cudaSuccess;
    return cudaMemcpyAsync(*dst, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, s);
  }
  template <typename T>
  cudaError_t alloc(T** dst, size_t n) {
    *dst = nullptr;
    cudaError_t e = cudaMalloc((void**)dst, std::max<size_t>(1, n) * sizeof(T));
    if (e == cudaSuccess) p.push_back(*dst);
    return e;
  }
};

}  // namespace

#define FCU(call)                                                                                     \
  do {                                                                                                \
    cudaError_t e__ = (call);                                                                         \
    if (e__ != cudaSuccess)                                                                           \
      return set_err(ctx, SGF_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e__)); \
  } while (0)

extern "C" sgf_status sgf_field(sgf_ctx* ctx, const void* mu_dev, long n_t, const double* xy, void* u_dev,
                                int total) {
  if (!ctx) return SGF_EINVAL;
  if (!ctx->built) return set_err(ctx, SGF_ESTATE, "operator not built");
  if (n_t < 0 || n_t > (1L << 30) || (total != 0 && total != 1))
    return set_err(ctx, SGF_EINVAL, "bad field arguments (n_targets %ld, total %d)", n_t, total);
  if (n_t == 0) return SGF_OK;
  if (!mu_dev || !xy || !u_dev) return set_err(ctx, SGF_EINVAL, "null pointer");
  sgf_ctx* c = ctx;
  FCU(cudaSetDevice(c->device));
  const sgf_params& P = c->prm;
  const double d = c->d, L = c->L, hmin = P.hmin, top = hmin + P.ny * L;
  const int nx = P.nx, ny = P.ny;

  // ---------------- classify: inside the cell box (Algorithm 3) or above it (Rayleigh form)
  std::vector<double> g_xr, g_y, g_w, g_x0, r_xr, r_y, r_w, r_x0;
  std::vector<long> g_out, r_out;
  std::vector<int> g_cid;
  for (long i = 0; i < n_t; ++i) {
    const double x = xy[2 * i], y = xy[2 * i + 1];
    if (!std::isfinite(x) || !std::isfinite(y)) return set_err(ctx, SGF_EINVAL, "target %ld is not finite", i);
    if (y < hmin) return set_err(ctx, SGF_EINVAL, "target %ld lies below the cell box (y < %g)", i, hmin);
    double w = std::floor(x / d);
    double xr = x - w * d;
    if (xr < 0) xr = 0;  // x / d rounded up to an integer: the target sits on the period boundary
    if (y >= top) {
      r_xr.push_back(xr); r_y.push_back(y); r_w.push_back(w); r_x0.push_back(x); r_out.push_back(i);
    } else {
      int cx = std::min((int)std::floor(xr / L), nx - 1);
      int cy = std::min((int)std::floor((y - hmin) / L), ny - 1);
      g_xr.push_back(xr); g_y.push_back(y); g_w.push_back(w); g_x0.push_back(x); g_out.push_back(i);
      g_cid.push_back(cy * nx + cx);
    }
  }
  Scratch S;
  S.s = c->stream;
  FieldArgs a;
  a.k = c->k; a.alpha = c->alpha; a.beta = c->beta; a.d = d; a.dx = c->dx; a.L = L; a.hmin = hmin; a.h = P.h;
  a.j = P.j; a.bc = c->bc; a.p = P.p; a.e = P.e; a.nfit = c->nfit; a.neq = c->neq; a.nb = c->nb; a.nfb = P.n_fb;
  a.nm = c->nm; a.PxH = c->og[0].Px; a.PxV = c->og[1].Px; a.nrowH = c->og[0].nrow; a.nrowV = c->og[1].nrow;
  zd* u = (zd*)u_dev;
  const zd* mu = (const zd*)mu_dev;
  int* d_err;
  FCU(S.alloc(&d_err, 1));
  FCU(cudaMemsetAsync(d_err, 0, sizeof(int), c->stream));

  const long n_g = (long)g_xr.size();
  if (n_g > 0) {
    // targets grouped by cell (counting sort on the cell id)
    const int ncell = nx * ny;
    std::vector<int> cnt(ncell + 1, 0);
    for (int id : g_cid) cnt[id + 1]++;
    for (int i = 0; i < ncell; ++i) cnt[i + 1] += cnt[i];
    std::vector<long> order(n_g);
    {
      std::vector<int> pos(cnt.begin(), cnt.end() - 1);
      for (long t = 0; t < n_g; ++t) order[pos[g_cid[t]]++] = t;
    }
    std::vector<int> cell_tc(ncell, -1), tc_cx, tc_cy;
    for (int id = 0; id < ncell; ++id)
      if (cnt[id + 1] > cnt[id]) {
        cell_tc[id] = (int)tc_cx.size();
        tc_cx.push_back(id % nx);
        tc_cy.push_back(id / nx);
      }
    const int n_tc = (int)tc_cx.size();
    std::vector<double> s_xr(n_g), s_y(n_g), s_w(n_g), s_x0(n_g);
    std::vector<long> s_out(n_g);
    std::vector<int> s_cell(n_g);
    for (long k = 0; k < n_g; ++k) {
      const long t = order[k];
      s_xr[k] = g_xr[t]; s_y[k] = g_y[t]; s_w[k] = g_w[t]; s_x0[k] = g_x0[t]; s_out[k] = g_out[t];
      s_cell[k] = cell_tc[g_cid[t]];
    }
    // local cells of every target cell (the same reach as the nodes' local sets) and their nodes
    std::vector<int> occ_id((size_t)ncell, -1);
    for (int q = 0; q < c->n_occ; ++q) occ_id[(size_t)c->occ_cy[q] * nx + c->occ_cx[q]] = q;
    // for each target row, the source rows whose local reach contains it (ascending)
    std::vector<std::vector<int>> src_rows(ny);
    for (int cyr = 0; cyr < ny; ++cyr)
      for (int cy : rows_of_Sj(cyr, P.j, P.h, L))
        if (cy >= 0 && cy < ny) src_rows[cy].push_back(cyr);
    std::vector<int> tc_bstart(n_tc + 1, 0), tc_cstart(n_tc + 1, 0), b_r, b_wrap, b_dcx, b_dcy, col_node;
    std::vector<signed char> col_wrap;
    int dmin = 1 << 30, dmax = -(1 << 30);
    for (int q = 0; q < n_tc; ++q) {
      tc_bstart[q] = (int)b_r.size();
      tc_cstart[q] = (int)col_node.size();
      for (int dcx = -1; dcx <= 1; ++dcx) {
        const int cxr = tc_cx[q] + dcx;
        const int ref = ((cxr % nx) + nx) % nx;
        const int wrap = (cxr - ref) / nx;
        for (int cyr : src_rows[tc_cy[q]]) {
          const int r = occ_id[(size_t)cyr * nx + ref];
          if (r < 0) continue;
          b_r.push_back(r); b_wrap.push_back(wrap); b_dcx.push_back(dcx); b_dcy.push_back(cyr - tc_cy[q]);
          dmin = std::min(dmin, cyr - tc_cy[q]);
          dmax = std::max(dmax, cyr - tc_cy[q]);
          const int l0 = c->cell_start[r], l1 = c->cell_start[r + 1];
          col_node.insert(col_node.end(), c->node_idx.begin() + l0, c->node_idx.begin() + l1);
          col_wrap.insert(col_wrap.end(), (size_t)(l1 - l0), (signed char)wrap);
        }
      }
    }
    tc_bstart[n_tc] = (int)b_r.size();
    tc_cstart[n_tc] = (int)col_node.size();
    const int nblk = (int)b_r.size();
    const int n_dcy = nblk > 0 ? dmax - dmin + 1 : 0;
    std::vector<int> b_o(nblk);
    for (int b = 0; b < nblk; ++b) b_o[b] = (b_dcx[b] + 1) * n_dcy + (b_dcy[b] - dmin);

    int *d_tc_cx, *d_tc_cy, *d_tc_bstart, *d_tc_cstart, *d_b_r, *d_b_wrap, *d_b_o, *d_col_node, *d_s_cell;
    signed char* d_col_wrap;
    double *d_s_xr, *d_s_y, *d_s_w, *d_s_x0;
    long* d_s_out;
    zd *d_phi = nullptr, *d_W, *d_msum;
    FCU(S.put(&d_tc_cx, tc_cx));
    FCU(S.put(&d_tc_cy, tc_cy));
    FCU(S.put(&d_tc_bstart, tc_bstart));
    FCU(S.put(&d_tc_cstart, tc_cstart));
    FCU(S.put(&d_b_r, b_r));
    FCU(S.put(&d_b_wrap, b_wrap));
    FCU(S.put(&d_b_o, b_o));
    FCU(S.put(&d_col_node, col_node));
    FCU(S.put(&d_col_wrap, col_wrap));
    FCU(S.put(&d_s_cell, s_cell));
    FCU(S.put(&d_s_xr, s_xr));
    FCU(S.put(&d_s_y, s_y));
    FCU(S.put(&d_s_w, s_w));
    FCU(S.put(&d_s_x0, s_x0));
    FCU(S.put(&d_s_out, s_out));
    FCU(S.alloc(&d_W, (size_t)n_tc * c->nb));
    FCU(S.alloc(&d_msum, std::max(1, c->nm)));
    if (nblk > 0) {
      FCU(S.alloc(&d_phi, (size_t)3 * n_dcy * c->nfit * 2 * c->neq));
      FCU(launch_phi_off(c, d_phi, dmin, n_dcy, c->keep.samp_rel, c->keep.src_rel));
    }
    FCU(launch_far_grids64(c, mu));
    if (c->nm > 0) {
      k_field_msum<<<c->nm, 256, 0, c->stream>>>(c->N, c->d_MS, mu, d_msum);
      FCU(cudaGetLastError());
    }
    const size_t smc = (size_t)(c->nfit + 4 * c->neq) * sizeof(zd);
    k_field_cells<<<n_tc, 128, smc, c->stream>>>(a, d_tc_cx, d_tc_cy, d_tc_bstart, d_b_r, d_b_wrap, d_b_o,
                                                 c->d_cell_start, c->d_node_idx, mu, c->o64.P, d_phi,
                                                 c->keep.samp_rel, c->keep.pinv_fb, c->o64.grid[0], c->o64.grid[1], d_W);
    FCU(cudaGetLastError());
    const long nblk_t = (n_g + 7) / 8;
    k_field_targets<<<(unsigned)nblk_t, 256, 0, c->stream>>>(
        a, n_g, d_s_xr, d_s_y, d_s_w, d_s_x0, d_s_cell, d_s_out, d_tc_cx, d_tc_cy, d_tc_cstart, d_col_node,
        d_col_wrap, c->d_x, c->d_f, c->d_f1, mu, d_W, c->keep.modes_n, d_msum, c->d_binw, total, u, d_err);
    FCU(cudaGetLastError());
  }

  const long n_r = (long)r_xr.size();
  if (n_r > 0) {
    // modes |n - n_0| <= n_c: beyond, every term is below e^{-37} of the field's scale at the lowest
    // such target (|beta_n| >= 2 pi |n - n_0| / d - pi / d - k)
    const double yR = *std::min_element(r_y.begin(), r_y.end());
    const double fmax = *std::max_element(c->hf.begin(), c->hf.end());
    const double gap = yR - fmax;
    if (!(gap > 0)) return set_err(ctx, SGF_EINVAL, "targets above the cell box must lie above the highest node");
    const double ncd = std::ceil((37.0 / gap + c->k + SGF_PI / d) * d / (2 * SGF_PI)) + 1;
    if (ncd > 100000)
      return set_err(ctx, SGF_EINVAL, "targets above the cell box too close to the highest node (gap %g)", gap);
    const int n_c = (int)ncd;
    const int n0 = (int)std::lround(-c->alpha * d / (2 * SGF_PI));
    const int nmod = 2 * n_c + 1;
    std::vector<double> mp(6 * (size_t)nmod);
    rayleigh_mode_params(c, n0 - n_c, nmod, mp.data());
    double *d_mp, *d_r_xr, *d_r_y, *d_r_w, *d_r_x0;
    long* d_r_out;
    zd* d_Bp;
    FCU(S.put(&d_mp, mp));
    FCU(S.put(&d_r_xr, r_xr));
    FCU(S.put(&d_r_y, r_y));
    FCU(S.put(&d_r_w, r_w));
    FCU(S.put(&d_r_x0, r_x0));
    FCU(S.put(&d_r_out, r_out));
    FCU(S.alloc(&d_Bp, nmod));
    k_field_ray_coef<<<nmod, 256, 0, c->stream>>>(a, c->N, d_mp, yR, c->d_x, c->d_f, c->d_f1, mu, d_Bp);
    FCU(cudaGetLastError());
    k_field_ray_eval<<<(unsigned)((n_r + 7) / 8), 256, 0, c->stream>>>(a, n_r, nmod, n_c, fmax, d_mp, yR, d_Bp, d_r_xr,
                                                                       d_r_y, d_r_w, d_r_x0, d_r_out, total, u);
    FCU(cudaGetLastError());
  }
  int herr = 0;
  FCU(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  FCU(cudaStreamSynchronize(c->stream));
  if (herr) return set_err(ctx, SGF_EINVAL, "a target coincides with a node of the surface");
  return SGF_OK;
}
