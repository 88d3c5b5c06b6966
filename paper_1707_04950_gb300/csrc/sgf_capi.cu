// Host side of the sgf library: the C ABI of include/sgf.h, parameter validation, the cell and
// index bookkeeping of Section 5.1 (binning, occupied cells, local sets L(q), grid indices of the
// equivalent sources and samples), the orchestration of Algorithm 2 and Algorithm 3, restarted
// GMRES with CGS2 Arnoldi (Algorithm 1), and Rayleigh extraction.
#include <chrono>
#include <complex>
#include <cmath>
#include <cstring>
#include <set>
#include <cstdlib>
#include <memory>

#include "sgf_internal.h"

typedef std::complex<double> cd;

sgf_status set_err(sgf_ctx* ctx, sgf_status st, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

template <typename T>
static sgf_status dalloc(sgf_ctx* ctx, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess)
    return set_err(ctx, SGF_ECUDA, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
  ctx->allocs.push_back((void*)*p);
  return SGF_OK;
}

#define TRY(x)                         \
  do {                                 \
    sgf_status st__ = (x);             \
    if (st__ != SGF_OK) return st__;   \
  } while (0)

#define CU(call)                                                                                      \
  do {                                                                                                \
    cudaError_t e__ = (call);                                                                         \
    if (e__ != cudaSuccess)                                                                           \
      return set_err(ctx, SGF_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e__)); \
  } while (0)

template <typename T>
static void free_multi(MultiSpace<T>& ms) {
  for (int l = 0; l < 2; ++l) {
    if (ms.grid[l]) cudaFree(ms.grid[l]);
    if (ms.accg[l]) cudaFree(ms.accg[l]);
  }
  if (ms.mpart) cudaFree(ms.mpart);
  if (ms.mpart_ff) cudaFree(ms.mpart_ff);
  ms = MultiSpace<T>();
}

static void free_all(sgf_ctx* ctx) {
  destroy_graphs(ctx);
  if (ctx->ms64.ready || ctx->ms32.ready) cudaStreamSynchronize(ctx->stream);
  free_multi(ctx->ms64);
  free_multi(ctx->ms32);
  for (void* p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
  ctx->o64 = OpData<double>();
  ctx->keep = BuildKeep();
  ctx->o32 = OpData<float>();
  ctx->built = false;
  ctx->d_Aex = nullptr;
  ctx->geom = ctx->exact_ready = ctx->op_exact = false;
}

static int ilog2_exact(long n) {
  int l = 0;
  while ((1L << l) < n) ++l;
  return ((1L << l) == n) ? l : -1;
}

extern "C" {

sgf_status sgf_create(sgf_ctx** out, int device, void* cuda_stream) {
  if (!out) return SGF_EINVAL;
  *out = nullptr;
  sgf_ctx* ctx = new sgf_ctx();
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    set_err(ctx, SGF_ECUDA, "cudaSetDevice(%d): %s", device, cudaGetErrorString(e));
    *out = ctx;
    return SGF_ECUDA;
  }
  for (int i = 0; i < 8; ++i) cudaEventCreate(&ctx->ev[i]);
  // side: V convolution chain (highest priority, critical path); side2: near field (lowest)
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess) ctx->side = nullptr;
  if (cudaStreamCreateWithPriority(&ctx->side2, cudaStreamNonBlocking, prio_lo) != cudaSuccess) ctx->side2 = nullptr;
  cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ctx->ev_fork0, cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ctx->ev_join2, cudaEventDisableTiming);
  *out = ctx;
  return SGF_OK;
}

void sgf_destroy(sgf_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_all(ctx);
  for (int i = 0; i < 8; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  for (cudaStream_t st : {ctx->side, ctx->side2})
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
  for (cudaEvent_t ev : {ctx->ev_fork, ctx->ev_join, ctx->ev_fork0, ctx->ev_join2})
    if (ev) cudaEventDestroy(ev);
  delete ctx;
}

const char* sgf_last_error(const sgf_ctx* ctx) { return ctx ? ctx->err : "null context"; }

sgf_status sgf_set_profile_fourier(sgf_ctx* ctx, double d, int M, const double* a, const double* b) {
  if (!ctx) return SGF_EINVAL;
  if (!(d > 0) || M < 0 || !a || !b) return set_err(ctx, SGF_EINVAL, "bad profile (d=%g, M=%d)", d, M);
  ctx->d = d;
  ctx->fa.assign(a, a + M + 1);
  ctx->fb.assign(b, b + M + 1);
  ctx->fb[0] = 0;
  ctx->have_profile = true;
  ctx->built = ctx->geom = ctx->exact_ready = ctx->op_exact = false;
  return SGF_OK;
}

sgf_status sgf_set_wave(sgf_ctx* ctx, double k, double theta, int bc) {
  if (!ctx) return SGF_EINVAL;
  if (!(k > 0) || !(fabs(theta) < 0.5 * SGF_PI) || (bc != 0 && bc != 1))
    return set_err(ctx, SGF_EINVAL, "bad wave (k=%g, theta=%g, bc=%d)", k, theta, bc);
  ctx->k = k;
  ctx->theta = theta;
  ctx->alpha = k * sin(theta);
  ctx->beta = k * cos(theta);
  ctx->bc = bc;
  ctx->have_wave = true;
  ctx->built = ctx->geom = ctx->exact_ready = ctx->op_exact = false;
  return SGF_OK;
}

sgf_status sgf_set_params(sgf_ctx* ctx, const sgf_params* p) {
  if (!ctx || !p) return SGF_EINVAL;
  ctx->prm = *p;
  ctx->have_params = true;
  ctx->built = ctx->geom = ctx->exact_ready = ctx->op_exact = false;
  return SGF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Relative layouts of one cell (lower-left corner at the origin), Section 5.1-5.2 readings:
// H sources (s dL, b L), V sources (b L, s dL), s = -e..p+e, b = 0,1; collocation points on the
// boundary of [-L, 2L]^2 at arc lengths (t + 1/2) 12L/n_coll; samples: H bottom, H top (s dL, b L),
// V left, V right (b L, s dL), s = 0..p.
static void layouts(sgf_ctx* c, std::vector<double>& src_rel, std::vector<double>& coll_rel,
                    std::vector<double>& samp_rel, std::vector<int>& src_off) {
  const int p = c->prm.p, e = c->prm.e, neq = c->neq;
  const double L = c->L, dL = L / p;
  src_rel.assign(2 * neq * 2, 0.0);
  src_off.assign(2 * neq * 2, 0);  // integer (o1, o2) offsets per orientation and source
  for (int lam = 0; lam < 2; ++lam) {
    int t = 0;
    for (int b = 0; b < 2; ++b)
      for (int s = -e; s <= p + e; ++s, ++t) {
        double* r = &src_rel[(lam * neq + t) * 2];
        int* o = &src_off[(lam * neq + t) * 2];
        if (lam == 0) {
          r[0] = s * dL; r[1] = b * L; o[0] = s; o[1] = b;
        } else {
          r[0] = b * L; r[1] = s * dL; o[0] = b; o[1] = s;
        }
      }
  }
  const int nc = c->prm.n_coll;
  coll_rel.assign(2 * nc, 0.0);
  for (int t = 0; t < nc; ++t) {
    double tt = (t + 0.5) * 12 * L / nc;
    int side = std::min((int)floor(tt / (3 * L)), 3);
    double u = tt - side * 3 * L;
    double X, Y;
    if (side == 0) { X = -L + u; Y = -L; }
    else if (side == 1) { X = 2 * L; Y = -L + u; }
    else if (side == 2) { X = 2 * L - u; Y = 2 * L; }
    else { X = -L; Y = 2 * L - u; }
    coll_rel[2 * t] = X;
    coll_rel[2 * t + 1] = Y;
  }
  samp_rel.assign(2 * c->nfit, 0.0);
  int t = 0;
  for (int b = 0; b < 2; ++b)
    for (int s = 0; s <= p; ++s, ++t) { samp_rel[2 * t] = s * dL; samp_rel[2 * t + 1] = b * L; }
  for (int b = 0; b < 2; ++b)
    for (int s = 0; s <= p; ++s, ++t) { samp_rel[2 * t] = b * L; samp_rel[2 * t + 1] = s * dL; }
}

// Rows c of cells meeting S^r - m h e_2 for some 0 <= m <= j (half-open cells, Section 5.3).
std::set<int> rows_of_Sj(int cy_r, int j, double h, double L) {
  std::set<int> rows;
  for (int m = 0; m <= j; ++m) {
    double sh = m * h / L;
    double lo = cy_r - 2 - sh, hi = cy_r + 2 - sh;
    for (int cc = (int)floor(lo) + 1; cc < (int)ceil(hi); ++cc)
      if (lo < cc && cc < hi) rows.insert(cc);
  }
  return rows;
}

// U^eta (eq. M_eta) restricted to |beta_n| <= k.
static std::vector<int> ueta_set(sgf_ctx* c) {
  std::vector<int> out;
  double k = c->k, d = c->d;
  int nlo = (int)floor((-sqrt(2.0) * k - c->alpha) * d / (2 * SGF_PI)) - 1;
  int nhi = (int)ceil((sqrt(2.0) * k - c->alpha) * d / (2 * SGF_PI)) + 1;
  for (int n = nlo; n <= nhi; ++n) {
    double an = c->alpha + 2 * SGF_PI * n / d;
    cd bn = beta_host(k, an);
    if (std::abs(Qj_host(bn, c->prm.h, c->prm.j)) < c->prm.eta && std::abs(bn) <= k) out.push_back(n);
  }
  return out;
}

void rayleigh_mode_params(sgf_ctx* c, int n_lo, int nmod, double* mp) {
  std::vector<int> ue = ueta_set(c);
  for (int t = 0; t < nmod; ++t) {
    int n = n_lo + t;
    double an = c->alpha + 2 * SGF_PI * n / c->d;
    cd bn = beta_host(c->k, an);
    cd Q = Qj_host(bn, c->prm.h, c->prm.j);
    bool in = std::find(ue.begin(), ue.end(), n) != ue.end();
    mp[6 * t] = an; mp[6 * t + 1] = bn.real(); mp[6 * t + 2] = bn.imag();
    mp[6 * t + 3] = Q.real(); mp[6 * t + 4] = Q.imag(); mp[6 * t + 5] = in ? 1.0 : 0.0;
  }
}

static sgf_status validate(sgf_ctx* ctx) {
  if (!ctx->have_profile || !ctx->have_wave || !ctx->have_params)
    return set_err(ctx, SGF_ESTATE, "profile, wave and params must be set before build");
  const sgf_params& p = ctx->prm;
  if (p.N < 8 || p.j < 0 || p.j > 24 || !(p.h > 0) || p.n_per < 1 || p.nx < 3 || p.ny < 1 || p.p < 1 || p.e < 0 ||
      p.n_coll < 8 || p.n_coll + 4 * (p.p + 1 + 2 * p.e) > 256 || p.n_fb < 0 || !(p.ls_reg >= 0) || p.Ma < 2 || !(p.c_win > 0 && p.c_win < 1) ||
      !(p.delta_min > 0) || !(p.spec_exp > 0))
    return set_err(ctx, SGF_EINVAL, "parameter out of range");
  if (p.precision != 64 && p.precision != 32) return set_err(ctx, SGF_EINVAL, "precision must be 64 or 32");
  if (p.N % p.nx != 0) return set_err(ctx, SGF_EINVAL, "N must be a multiple of nx");
  if (ilog2_exact((long)p.nx * p.p) < 0 || ilog2_exact(p.nx) < 0)
    return set_err(ctx, SGF_EINVAL, "nx and nx*p must be powers of two (cyclic FFT along X)");
  int nfit = 4 * (p.p + 1), nb = 2 * p.n_fb + 1;
  if (nb > 63 || nb > 2 * (p.p + 1) + 2 * (p.p - 1)) return set_err(ctx, SGF_EINVAL, "n_fb too large for the samples");
  if (2 * (p.p + 1 + 2 * p.e) * 2 > p.n_coll) return set_err(ctx, SGF_EINVAL, "n_coll below the number of unknowns");
  if (nfit > 64) return set_err(ctx, SGF_EINVAL, "p = %d gives %d cell samples (at most 64)", p.p, nfit);
  return SGF_OK;
}

// host wall clock in ms (build-stage timers)
static double wall_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

extern "C" sgf_status sgf_build_operator(sgf_ctx* ctx) {
  if (!ctx) return SGF_EINVAL;
  TRY(validate(ctx));
  const double t_build0 = wall_ms();
  CU(cudaSetDevice(ctx->device));
  free_all(ctx);
  sgf_ctx* c = ctx;
  const sgf_params& P = c->prm;
  c->N = P.N;
  c->dx = c->d / P.N;
  c->L = c->d / P.nx;
  c->a_s = P.Ma * c->dx;
  c->gam = 0.5 * c->a_s;
  c->neq = 2 * (P.p + 1 + 2 * P.e);
  c->nfit = 4 * (P.p + 1);
  c->nb = 2 * P.n_fb + 1;
  if (!(c->a_s < c->L)) return set_err(ctx, SGF_EWINDOW, "singular window a = %g must be below the cell side %g", c->a_s, c->L);
  for (int l = 0; l < 2; ++l) c->og[l].force_conv = c->og[l].force_vpt = 0;
  // grids
  Orient& H = c->og[0];
  Orient& V = c->og[1];
  H.Px = P.nx * P.p; H.logPx = ilog2_exact(H.Px); H.nrow = P.ny + 1; H.dxg = c->L / P.p; H.dyg = c->L;
  V.Px = P.nx; V.logPx = ilog2_exact(V.Px); V.nrow = P.ny * P.p + 1 + 2 * P.e; V.dxg = c->L; V.dyg = c->L / P.p;
  for (int l = 0; l < 2; ++l) {
    // smallest 2^a 3^b (b <= 2) holding the linear convolution of nrow rows
    long need = 2L * c->og[l].nrow - 1, best = 1L << 40;
    int ba = 0, bb = 0;
    for (int b = 0; b <= 2; ++b) {
      long p3 = b == 0 ? 1 : (b == 1 ? 3 : 9);
      int a = 0;
      while ((p3 << a) < need) ++a;
      if ((p3 << a) < best) { best = p3 << a; ba = a; bb = b; }
    }
    c->og[l].Py = (int)best;
    c->og[l].la = ba;
    c->og[l].lb = bb;
  }
  c->twlog = std::max(H.logPx, V.logPx);
  for (int l = 0; l < 2; ++l)
    if (!conv_y_variant_of(c->og[l], 64) || (c->prm.precision == 32 && !conv_y_variant_of(c->og[l], 32)) ||
        !conv_y_variant_of(c->og[l], 64, true) || (c->prm.precision == 32 && !conv_y_variant_of(c->og[l], 32, true)))
      return set_err(ctx, SGF_EINVAL, "Y transform of %d points (%d cell rows) exceeds one thread block",
                     c->og[l].Py, c->og[l].nrow);
  if (V.Py > 16384 || H.Py > 16384 || H.Px > 4096 || V.Px > 4096)
    return set_err(ctx, SGF_EINVAL, "FFT length above the shared-memory limit");
  // shifted poles must stay off the finest grid lag (0, -m h)
  for (int m = 1; m <= P.j; ++m) {
    double r = m * P.h / V.dyg;
    if (fabs(r - std::round(r)) < 1e-6)
      return set_err(ctx, SGF_EPOLE_ON_GRID, "shifted pole %d h lies on a grid lag", m);
  }
  {  // non-resonant cell: (kL/pi)^2 != m^2 + n^2, m, n >= 1
    double t = c->k * c->L / SGF_PI;
    t *= t;
    for (int m = 1; m * m < t + 1; ++m)
      for (int n = 1; m * m + n * n < t + 1; ++n)
        if (fabs(t - (m * m + n * n)) < 1e-3) return set_err(ctx, SGF_ERESONANT_CELL, "cell side resonant");
  }

  // ---------------- nodes and profile (device), copied back for the cell bookkeeping
  int M = (int)c->fa.size() - 1;
  TRY(dalloc(ctx, &c->d_coef, 2 * (M + 1)));
  CU(cudaMemcpyAsync(c->d_coef, c->fa.data(), (M + 1) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->d_coef + M + 1, c->fb.data(), (M + 1) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  TRY(dalloc(ctx, &c->d_x, c->N));
  TRY(dalloc(ctx, &c->d_f, c->N));
  TRY(dalloc(ctx, &c->d_f1, c->N));
  TRY(dalloc(ctx, &c->d_f2, c->N));
  CU(launch_profile(c));
  c->hx.resize(c->N); c->hf.resize(c->N); c->hf1.resize(c->N); c->hf2.resize(c->N);
  CU(cudaMemcpyAsync(c->hx.data(), c->d_x, c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(c->hf.data(), c->d_f, c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaMemcpyAsync(c->hf1.data(), c->d_f1, c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  double maxslope = 0;
  for (int i = 0; i < c->N; ++i) maxslope = std::max(maxslope, fabs(c->hf1[i]));
  // shifted poles (j > 0) must stay outside the singular window
  if (P.j > 0 && !(P.h > c->a_s * maxslope))
    return set_err(ctx, SGF_EWINDOW, "shift h = %g must exceed a max|f'| = %g", P.h, c->a_s * maxslope);

  // ---------------- binning (Remark cell_def: half-open cells)
  std::vector<int> ncx(c->N), ncy(c->N);
  for (int i = 0; i < c->N; ++i) {
    ncx[i] = (int)(((long)(i + 1) * P.nx + c->N - 1) / c->N) - 1;
    ncy[i] = (int)ceil((c->hf[i] - P.hmin) / c->L) - 1;
    if (ncy[i] < 0 || ncy[i] >= P.ny) return set_err(ctx, SGF_EINVAL, "node %d outside the cell box", i);
  }
  std::vector<int> occ_id((size_t)P.nx * P.ny, -1);
  std::vector<std::vector<int>> members;
  c->occ_cx.clear(); c->occ_cy.clear();
  // occupied cells ordered by (cy, cx)
  {
    std::vector<char> used((size_t)P.nx * P.ny, 0);
    for (int i = 0; i < c->N; ++i) used[(size_t)ncy[i] * P.nx + ncx[i]] = 1;
    for (int cy = 0; cy < P.ny; ++cy)
      for (int cx = 0; cx < P.nx; ++cx)
        if (used[(size_t)cy * P.nx + cx]) {
          occ_id[(size_t)cy * P.nx + cx] = (int)c->occ_cx.size();
          c->occ_cx.push_back(cx);
          c->occ_cy.push_back(cy);
        }
  }
  c->n_occ = (int)c->occ_cx.size();
  members.assign(c->n_occ, {});
  for (int i = 0; i < c->N; ++i) members[occ_id[(size_t)ncy[i] * P.nx + ncx[i]]].push_back(i);
  c->cell_start.assign(c->n_occ + 1, 0);
  c->node_idx.clear();
  std::vector<int> node_cell;
  int maxnq = 0;
  for (int q = 0; q < c->n_occ; ++q) {
    c->cell_start[q] = (int)c->node_idx.size();
    for (int i : members[q]) { c->node_idx.push_back(i); node_cell.push_back(q); }
    maxnq = std::max(maxnq, (int)members[q].size());
  }
  c->maxnq = maxnq;
  c->cell_start[c->n_occ] = c->N;
  {  // work items: chunks of at most 32 nodes of one cell (balances the per-cell kernels)
    std::vector<int> ic, il, ih;
    for (int q = 0; q < c->n_occ; ++q) {
      int nq = c->cell_start[q + 1] - c->cell_start[q];
      for (int lo = 0; lo < nq; lo += 32) {
        ic.push_back(q);
        il.push_back(lo);
        ih.push_back(std::min(nq, lo + 32));
      }
    }
    c->n_items = (int)ic.size();
    long covered = 0;
    for (size_t t = 0; t < ic.size(); ++t) covered += ih[t] - il[t];
    if (covered != c->N) return set_err(ctx, SGF_EINVAL, "internal: work items cover %ld of %d nodes", covered, c->N);
    TRY(dalloc(ctx, &c->d_item_cell, ic.size()));
    TRY(dalloc(ctx, &c->d_item_lo, il.size()));
    TRY(dalloc(ctx, &c->d_item_hi, ih.size()));
    CU(cudaMemcpy(c->d_item_cell, ic.data(), ic.size() * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->d_item_lo, il.data(), il.size() * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->d_item_hi, ih.data(), ih.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  TRY(dalloc(ctx, &c->d_cell_start, c->n_occ + 1));
  TRY(dalloc(ctx, &c->d_node_idx, c->N));
  TRY(dalloc(ctx, &c->d_node_cell, c->N));
  TRY(dalloc(ctx, &c->d_occ_cx, c->n_occ));
  TRY(dalloc(ctx, &c->d_occ_cy, c->n_occ));
  CU(cudaMemcpy(c->d_cell_start, c->cell_start.data(), (c->n_occ + 1) * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->d_node_idx, c->node_idx.data(), c->N * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->d_node_cell, node_cell.data(), c->N * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->d_occ_cx, c->occ_cx.data(), c->n_occ * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->d_occ_cy, c->occ_cy.data(), c->n_occ * sizeof(int), cudaMemcpyHostToDevice));

  // ---------------- layouts, grid indices and twists
  std::vector<double> src_rel, coll_rel, samp_rel;
  std::vector<int> src_off;
  layouts(c, src_rel, coll_rel, samp_rel, src_off);
  const int neq = c->neq, nfit = c->nfit;
  std::vector<int> src_gidx((size_t)c->n_occ * 2 * neq), samp_gidx((size_t)c->n_occ * nfit);
  std::vector<zd> src_tw((size_t)c->n_occ * 2 * neq);
  for (int q = 0; q < c->n_occ; ++q) {
    int cx = c->occ_cx[q], cy = c->occ_cy[q];
    for (int lam = 0; lam < 2; ++lam) {
      const Orient& o = c->og[lam];
      for (int s = 0; s < neq; ++s) {
        int o1 = src_off[(lam * neq + s) * 2], o2 = src_off[(lam * neq + s) * 2 + 1];
        long ixr, iy;
        if (lam == 0) { ixr = (long)cx * P.p + o1; iy = cy + o2; }
        else { ixr = cx + o1; iy = (long)cy * P.p + o2 + P.e; }
        long ixref = ((ixr % o.Px) + o.Px) % o.Px;
        src_gidx[((size_t)q * 2 + lam) * neq + s] = (int)(ixref * o.nrow + iy);
        double xs = ixr * o.dxg;
        src_tw[((size_t)q * 2 + lam) * neq + s] = zd(cos(-c->alpha * xs), sin(-c->alpha * xs));
      }
    }
    for (int t = 0; t < nfit; ++t) {
      int lam = t < 2 * (P.p + 1) ? 0 : 1;
      const Orient& o = c->og[lam];
      int tt = lam == 0 ? t : t - 2 * (P.p + 1);
      int b = tt / (P.p + 1), s = tt % (P.p + 1);
      long ixr, iy;
      if (lam == 0) { ixr = (long)cx * P.p + s; iy = cy + b; }
      else { ixr = cx + b; iy = (long)cy * P.p + s + P.e; }
      long ixref = ((ixr % o.Px) + o.Px) % o.Px;
      samp_gidx[(size_t)q * nfit + t] = (int)(ixref * o.nrow + iy);
    }
  }
  TRY(dalloc(ctx, &c->d_src_gidx, src_gidx.size()));
  TRY(dalloc(ctx, &c->d_samp_gidx, samp_gidx.size()));
  TRY(dalloc(ctx, &c->o64.src_tw, src_tw.size()));
  CU(cudaMemcpy(c->d_src_gidx, src_gidx.data(), src_gidx.size() * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->d_samp_gidx, samp_gidx.data(), samp_gidx.size() * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->o64.src_tw, src_tw.data(), src_tw.size() * sizeof(zd), cudaMemcpyHostToDevice));
  double *d_src_rel, *d_coll_rel, *d_samp_rel, *d_kress;
  TRY(dalloc(ctx, &d_src_rel, src_rel.size()));
  TRY(dalloc(ctx, &d_coll_rel, coll_rel.size()));
  TRY(dalloc(ctx, &d_samp_rel, samp_rel.size()));
  CU(cudaMemcpy(d_src_rel, src_rel.data(), src_rel.size() * sizeof(double), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(d_coll_rel, coll_rel.data(), coll_rel.size() * sizeof(double), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(d_samp_rel, samp_rel.data(), samp_rel.size() * sizeof(double), cudaMemcpyHostToDevice));
  // binomial weights and log-quadrature weights R_s, s = -(Ma-1)..(Ma-1)
  std::vector<double> binw(P.j + 1);
  for (int m = 0; m <= P.j; ++m) {
    double cb = 1;
    for (int i = 0; i < m; ++i) cb = cb * (P.j - i) / (i + 1);
    binw[m] = (m % 2 ? -1.0 : 1.0) * cb;
  }
  TRY(dalloc(ctx, &c->d_binw, binw.size()));
  CU(cudaMemcpy(c->d_binw, binw.data(), binw.size() * sizeof(double), cudaMemcpyHostToDevice));
  std::vector<double> kress(2 * P.Ma - 1);
  for (int s = -(P.Ma - 1); s <= P.Ma - 1; ++s) {
    double acc = 0;
    for (int m = 1; m < P.Ma; ++m) acc += cos(SGF_PI * m * s / P.Ma) / m;
    kress[s + P.Ma - 1] = -2 * c->dx * acc - c->dx / P.Ma * ((s & 1) ? -1.0 : 1.0);
  }
  TRY(dalloc(ctx, &d_kress, kress.size()));
  CU(cudaMemcpy(d_kress, kress.data(), kress.size() * sizeof(double), cudaMemcpyHostToDevice));

  // ---------------- least-squares operators (Algorithm 2, first step)
  CU(cudaStreamSynchronize(ctx->stream));
  const double t_ls0 = wall_ms();
  const int nc = P.n_coll;
  zd *d_Acoll, *d_Bfb, *d_pinv_eq, *d_pinv_fb, *d_qrs;
  const long lda = nc + 2 * neq;
  TRY(dalloc(ctx, &d_Acoll, (size_t)2 * lda * 2 * neq));
  TRY(dalloc(ctx, &d_Bfb, (size_t)nfit * c->nb));
  TRY(dalloc(ctx, &d_pinv_eq, (size_t)2 * 2 * neq * nc));
  TRY(dalloc(ctx, &d_pinv_fb, (size_t)c->nb * nfit));
  TRY(dalloc(ctx, &d_qrs, (size_t)(2 * neq) * (2 * neq) + 2 * neq + (size_t)lda * lda + 64));
  CU(launch_build_matrices(c, d_Acoll, d_Bfb, d_coll_rel, d_src_rel, d_samp_rel));
  for (int lam = 0; lam < 2; ++lam)
    CU(launch_qr_pinv(c, d_Acoll + (size_t)lam * lda * 2 * neq, nc, 2 * neq, true, P.ls_reg,
                      d_pinv_eq + (size_t)lam * 2 * neq * nc, d_qrs));
  CU(launch_qr_pinv(c, d_Bfb, nfit, c->nb, false, 0.0, d_pinv_fb, d_qrs));

  // ---------------- projection and reconstruction matrices
  TRY(dalloc(ctx, &c->o64.P, (size_t)4 * neq * c->N));
  CU(launch_build_P(c, d_pinv_eq, d_coll_rel));
  zd* d_Iplain;
  TRY(dalloc(ctx, &d_Iplain, (size_t)nfit * c->N));
  TRY(dalloc(ctx, &c->o64.Ip, (size_t)nfit * c->N));
  CU(launch_build_I(c, d_pinv_fb, d_Iplain, d_samp_rel));

  // ---------------- kernel tables and spectra
  CU(cudaStreamSynchronize(c->stream));
  const double t_tab0 = wall_ms();
  c->build_ms[2] = t_tab0 - t_ls0;
  TRY(dalloc(ctx, &c->o64.tw, (size_t)1 << c->twlog));
  bool mixed = P.precision == 32;
  if (mixed) TRY(dalloc(ctx, &c->o32.tw, (size_t)1 << c->twlog));
  for (int lam = 0; lam < 2; ++lam) {
    TRY(dalloc(ctx, &c->o64.twy[lam], c->og[lam].Py));
    if (mixed) TRY(dalloc(ctx, &c->o32.twy[lam], c->og[lam].Py));
  }
  CU(launch_twiddles(c));
  for (int lam = 0; lam < 2; ++lam) {
    long n = (long)c->og[lam].Px * c->og[lam].Py;
    for (int kd = 0; kd < 2; ++kd) {
      TRY(dalloc(ctx, &c->o64.Khat[lam][kd], n));
      TRY(dalloc(ctx, &c->d_Tx[lam][kd], n));
      if (mixed) TRY(dalloc(ctx, &c->o32.Khat[lam][kd], n));
    }
  }
  TRY(dalloc(ctx, &c->d_msum, 64));
  CU(launch_tables(c));
  CU(cudaStreamSynchronize(c->stream));
  const double t_near0 = wall_ms();
  c->build_ms[1] = t_near0 - t_tab0;

  // ---------------- local sets L(q) and the near-field block list
  // Values of cell q form one row-major n_q x W_q block (W_q = sum of n_r over its local cells, in
  // block order), so each target row is one contiguous stream.
  std::vector<int> pq, pr, pw, pdcx, pld, bcol;
  std::vector<long> poff, cell_off(c->n_occ + 1, 0);
  std::vector<int> blk_start(c->n_occ + 1, 0), cellW(c->n_occ, 0);
  std::vector<std::set<int>> rowsS(P.ny);
  for (int cy = 0; cy < P.ny; ++cy) rowsS[cy] = rows_of_Sj(cy, P.j, P.h, c->L);
  long off = 0;
  int dcy_min = 1 << 30, dcy_max = -(1 << 30);
  int maxW = 0;
  for (int q = 0; q < c->n_occ; ++q) {
    blk_start[q] = (int)pq.size();
    cell_off[q] = off;
    int cxq = c->occ_cx[q], cyq = c->occ_cy[q];
    int nq = c->cell_start[q + 1] - c->cell_start[q];
    int W = 0;
    for (int dcx = -1; dcx <= 1; ++dcx) {
      int cxr = cxq + dcx;
      int ref = ((cxr % P.nx) + P.nx) % P.nx;
      int wrap = (cxr - ref) / P.nx;
      for (int cyr = 0; cyr < P.ny; ++cyr) {
        int r = occ_id[(size_t)cyr * P.nx + ref];
        if (r < 0) continue;
        if (!rowsS[cyr].count(cyq)) continue;
        int nr = c->cell_start[r + 1] - c->cell_start[r];
        pq.push_back(q); pr.push_back(r); pw.push_back(wrap); pdcx.push_back(dcx);
        bcol.push_back(W);
        W += nr;
        dcy_min = std::min(dcy_min, cyr - cyq);
        dcy_max = std::max(dcy_max, cyr - cyq);
      }
    }
    for (int b = blk_start[q]; b < (int)pq.size(); ++b) {
      poff.push_back(off + bcol[b]);
      pld.push_back(W);
    }
    cellW[q] = W;
    maxW = std::max(maxW, W);
    off += (long)nq * W;
  }
  cell_off[c->n_occ] = off;
  blk_start[c->n_occ] = (int)pq.size();
  c->n_blk = (int)pq.size();
  c->nnz = off;
  c->maxW = maxW;
  {  // near-row work items (see sgf_ctx::n_nitems)
    std::vector<int> ic, il, ih;
    for (int q = 0; q < c->n_occ; ++q) {
      const int nq = c->cell_start[q + 1] - c->cell_start[q];
      const int rows = std::max(4, std::min(32, 4096 / std::max(1, cellW[q])));
      for (int lo = 0; lo < nq; lo += rows) {
        ic.push_back(q);
        il.push_back(lo);
        ih.push_back(std::min(nq, lo + rows));
      }
    }
    c->n_nitems = (int)ic.size();
    TRY(dalloc(ctx, &c->d_nitem_cell, ic.size()));
    TRY(dalloc(ctx, &c->d_nitem_lo, il.size()));
    TRY(dalloc(ctx, &c->d_nitem_hi, ih.size()));
    CU(cudaMemcpy(c->d_nitem_cell, ic.data(), ic.size() * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->d_nitem_lo, il.data(), il.size() * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->d_nitem_hi, ih.data(), ih.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  if ((size_t)maxW * sizeof(zd) > 200 * 1024)
    return set_err(ctx, SGF_EINVAL, "local set of %d nodes too large for the near-field kernel", maxW);
  int n_dcy = dcy_max - dcy_min + 1;
  NearPairs pp;
  pp.n = c->n_blk;
  TRY(dalloc(ctx, &pp.q, pp.n));
  TRY(dalloc(ctx, &pp.r, pp.n));
  TRY(dalloc(ctx, &pp.wrap, pp.n));
  TRY(dalloc(ctx, &pp.dcx, pp.n));
  TRY(dalloc(ctx, &pp.ld, pp.n));
  TRY(dalloc(ctx, &pp.off, pp.n));
  CU(cudaMemcpy(pp.q, pq.data(), pp.n * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(pp.r, pr.data(), pp.n * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(pp.wrap, pw.data(), pp.n * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(pp.dcx, pdcx.data(), pp.n * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(pp.ld, pld.data(), pp.n * sizeof(int), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(pp.off, poff.data(), pp.n * sizeof(long), cudaMemcpyHostToDevice));
  TRY(dalloc(ctx, &c->d_blk_start, c->n_occ + 1));
  CU(cudaMemcpy(c->d_blk_start, blk_start.data(), (c->n_occ + 1) * sizeof(int), cudaMemcpyHostToDevice));
  c->d_blk_r = pp.r;
  c->d_blk_off = pp.off;
  TRY(dalloc(ctx, &c->d_blk_col, pp.n));
  CU(cudaMemcpy(c->d_blk_col, bcol.data(), pp.n * sizeof(int), cudaMemcpyHostToDevice));
  TRY(dalloc(ctx, &c->d_cell_off, c->n_occ + 1));
  CU(cudaMemcpy(c->d_cell_off, cell_off.data(), (c->n_occ + 1) * sizeof(long), cudaMemcpyHostToDevice));
  TRY(dalloc(ctx, &c->d_cell_W, c->n_occ));
  CU(cudaMemcpy(c->d_cell_W, cellW.data(), c->n_occ * sizeof(int), cudaMemcpyHostToDevice));
  {  // node index of every local column of every cell (cells in order, columns in block order)
    std::vector<int> cols, coloff(c->n_occ + 1, 0);
    std::vector<signed char> colwrap;  // period copy (-1, 0, 1) of each column's source node
    for (int q = 0; q < c->n_occ; ++q) {
      coloff[q] = (int)cols.size();
      for (int b = blk_start[q]; b < blk_start[q + 1]; ++b) {
        int r = pr[b];
        for (int l = c->cell_start[r]; l < c->cell_start[r + 1]; ++l) {
          cols.push_back(c->node_idx[l]);
          colwrap.push_back((signed char)pw[b]);
        }
      }
    }
    coloff[c->n_occ] = (int)cols.size();
    TRY(dalloc(ctx, &c->d_colwrap, colwrap.size()));
    CU(cudaMemcpy(c->d_colwrap, colwrap.data(), colwrap.size(), cudaMemcpyHostToDevice));
    TRY(dalloc(ctx, &c->d_cols, cols.size()));
    TRY(dalloc(ctx, &c->d_coloff, c->n_occ + 1));
    CU(cudaMemcpy(c->d_cols, cols.data(), cols.size() * sizeof(int), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->d_coloff, coloff.data(), (c->n_occ + 1) * sizeof(int), cudaMemcpyHostToDevice));
  }
  TRY(dalloc(ctx, &c->d_C, c->nnz));
  zd* d_phi;
  TRY(dalloc(ctx, &d_phi, (size_t)3 * n_dcy * nfit * 2 * neq));
  CU(launch_phi_off(c, d_phi, dcy_min, n_dcy, d_samp_rel, d_src_rel));
  CU(launch_near(c, d_phi, dcy_min, n_dcy, d_Iplain, pp, d_kress));
  c->keep.coll_rel = d_coll_rel;
  c->keep.samp_rel = d_samp_rel;
  c->keep.src_rel = d_src_rel;
  c->keep.kress = d_kress;
  c->keep.pinv_eq = d_pinv_eq;
  c->keep.pinv_fb = d_pinv_fb;
  c->keep.phi = d_phi;
  c->keep.Iplain = d_Iplain;
  c->keep.dcy_min = dcy_min;
  c->keep.n_dcy = n_dcy;
  c->keep.pp = pp;

  CU(cudaStreamSynchronize(c->stream));
  c->build_ms[3] = wall_ms() - t_near0;

  // ---------------- adjoint near layout: the rows of cell r collect conj(C) of every block (q, r),
  // blocks in block order, so each adjoint row is again one contiguous stream
  {
    std::vector<std::vector<int>> byr(c->n_occ);
    for (int b = 0; b < c->n_blk; ++b) byr[pr[b]].push_back(b);
    std::vector<long> cell_offT(c->n_occ + 1, 0), dst_off(c->n_blk, 0);
    std::vector<int> cellWT(c->n_occ, 0), dst_ld(c->n_blk, 0), colsT, coloffT(c->n_occ + 1, 0);
    long offT = 0;
    int maxWT = 0;
    for (int r = 0; r < c->n_occ; ++r) {
      cell_offT[r] = offT;
      coloffT[r] = (int)colsT.size();
      int W = 0;
      for (int b : byr[r]) {
        dst_off[b] = offT + W;
        int q = pq[b];
        for (int l = c->cell_start[q]; l < c->cell_start[q + 1]; ++l) colsT.push_back(c->node_idx[l]);
        W += c->cell_start[q + 1] - c->cell_start[q];
      }
      for (int b : byr[r]) dst_ld[b] = W;
      cellWT[r] = W;
      maxWT = std::max(maxWT, W);
      offT += (long)(c->cell_start[r + 1] - c->cell_start[r]) * W;
    }
    cell_offT[c->n_occ] = offT;
    coloffT[c->n_occ] = (int)colsT.size();
    if (offT != c->nnz) return set_err(ctx, SGF_EINVAL, "adjoint near layout holds %ld of %ld entries", offT, c->nnz);
    c->maxWT = maxWT;
    c->adj_ok = (size_t)(maxWT + 32 + 4 * neq) * sizeof(zd) <= 200 * 1024;
    if (c->adj_ok) {
      long* d_dst_off;
      int* d_dst_ld;
      TRY(dalloc(ctx, &d_dst_off, c->n_blk));
      TRY(dalloc(ctx, &d_dst_ld, c->n_blk));
      CU(cudaMemcpy(d_dst_off, dst_off.data(), c->n_blk * sizeof(long), cudaMemcpyHostToDevice));
      CU(cudaMemcpy(d_dst_ld, dst_ld.data(), c->n_blk * sizeof(int), cudaMemcpyHostToDevice));
      c->keep.tr_off = d_dst_off;
      c->keep.tr_ld = d_dst_ld;
      TRY(dalloc(ctx, &c->d_cell_offT, c->n_occ + 1));
      TRY(dalloc(ctx, &c->d_cell_WT, c->n_occ));
      TRY(dalloc(ctx, &c->d_colsT, colsT.size()));
      TRY(dalloc(ctx, &c->d_coloffT, c->n_occ + 1));
      CU(cudaMemcpy(c->d_cell_offT, cell_offT.data(), (c->n_occ + 1) * sizeof(long), cudaMemcpyHostToDevice));
      CU(cudaMemcpy(c->d_cell_WT, cellWT.data(), c->n_occ * sizeof(int), cudaMemcpyHostToDevice));
      CU(cudaMemcpy(c->d_colsT, colsT.data(), colsT.size() * sizeof(int), cudaMemcpyHostToDevice));
      CU(cudaMemcpy(c->d_coloffT, coloffT.data(), (c->n_occ + 1) * sizeof(int), cudaMemcpyHostToDevice));
      TRY(dalloc(ctx, &c->d_CT, c->nnz));
      CU(launch_near_transpose(c->n_blk, pp.q, pp.r, pp.off, pp.ld, d_dst_off, d_dst_ld, c->d_cell_start, c->d_C,
                               c->d_CT, c->stream));
    }
  }

  // ---------------- modes
  std::vector<int> ue = ueta_set(c);
  c->nm = (int)ue.size();
  std::vector<double> mn(3 * std::max(1, c->nm));
  for (int t = 0; t < c->nm; ++t) {
    double an = c->alpha + 2 * SGF_PI * ue[t] / c->d;
    cd bn = beta_host(c->k, an);
    mn[3 * t] = an; mn[3 * t + 1] = bn.real(); mn[3 * t + 2] = bn.imag();
  }
  double* d_mn;
  TRY(dalloc(ctx, &d_mn, mn.size()));
  c->keep.modes_n = d_mn;
  CU(cudaMemcpy(d_mn, mn.data(), mn.size() * sizeof(double), cudaMemcpyHostToDevice));
  TRY(dalloc(ctx, &c->d_MT, (size_t)c->N * std::max(1, c->nm)));
  TRY(dalloc(ctx, &c->d_MS, (size_t)c->N * std::max(1, c->nm)));
  CU(launch_modes(c, d_mn));
  TRY(dalloc(ctx, &c->d_MTh, (size_t)c->N * std::max(1, c->nm)));
  TRY(dalloc(ctx, &c->d_MSh, (size_t)c->N * std::max(1, c->nm)));
  CU(launch_conj_transpose(c->d_MT, c->N, c->nm, c->d_MTh, c->stream));
  CU(launch_conj_transpose(c->d_MS, c->nm, c->N, c->d_MSh, c->stream));
  if (c->nm > 8) return set_err(ctx, SGF_EINVAL, "%d completion modes (at most 8 supported)", c->nm);
  TRY(dalloc(ctx, &c->d_mpart, (size_t)std::max(1, c->nm) * c->mode_chunks));
  TRY(dalloc(ctx, &c->d_mpart_ff, (size_t)std::max(1, c->nm) * c->mode_chunks));

  // ---------------- grids and FP32 copies
  for (int lam = 0; lam < 2; ++lam) {
    long sz = 2L * c->og[lam].Px * c->og[lam].nrow;
    TRY(dalloc(ctx, &c->o64.grid[lam], sz));
    if (conv_y_variant_of(c->og[lam], 64) == 2 || conv_y_variant_of(c->og[lam], 64, true) == 2)
      TRY(dalloc(ctx, &c->o64.accg[lam], (size_t)c->og[lam].Px * c->og[lam].Py));
    if (mixed) TRY(dalloc(ctx, &c->o32.grid[lam], sz));
    if (mixed && (conv_y_variant_of(c->og[lam], 32) == 2 || conv_y_variant_of(c->og[lam], 32, true) == 2))
      TRY(dalloc(ctx, &c->o32.accg[lam], (size_t)c->og[lam].Px * c->og[lam].Py));
  }
  if (mixed) {
    TRY(dalloc(ctx, &c->o32.P, (size_t)4 * neq * c->N));
    TRY(dalloc(ctx, &c->o32.Ip, (size_t)nfit * c->N));
    TRY(dalloc(ctx, &c->o32.src_tw, src_tw.size()));
    CU(launch_to_f32(c->o64.P, c->o32.P, (long)4 * neq * c->N, c->stream));
    CU(launch_to_f32(c->o64.Ip, c->o32.Ip, (long)nfit * c->N, c->stream));
    CU(launch_to_f32(c->o64.src_tw, c->o32.src_tw, (long)src_tw.size(), c->stream));
    TRY(dalloc(ctx, &c->d_Cff, c->nnz));
    TRY(dalloc(ctx, &c->d_muff, c->N));
    CU(launch_split_ff(c->d_C, c->d_Cff, c->nnz, c->stream));
    TRY(dalloc(ctx, &c->d_MTff, (size_t)c->N * std::max(1, c->nm)));
    TRY(dalloc(ctx, &c->d_MSff, (size_t)c->N * std::max(1, c->nm)));
    CU(launch_split_ff(c->d_MT, c->d_MTff, (long)c->N * c->nm, c->stream));
    CU(launch_split_ff(c->d_MS, c->d_MSff, (long)c->N * c->nm, c->stream));
    TRY(dalloc(ctx, &c->d_MThff, (size_t)c->N * std::max(1, c->nm)));
    TRY(dalloc(ctx, &c->d_MShff, (size_t)c->N * std::max(1, c->nm)));
    CU(launch_split_ff(c->d_MTh, c->d_MThff, (long)c->N * c->nm, c->stream));
    CU(launch_split_ff(c->d_MSh, c->d_MShff, (long)c->N * c->nm, c->stream));
    if (c->adj_ok) {
      TRY(dalloc(ctx, &c->d_CTff, c->nnz));
      CU(launch_split_ff(c->d_CT, c->d_CTff, c->nnz, c->stream));
    }
  }
  TRY(dalloc(ctx, &c->d_mu_tmp, (size_t)c->N * 2));
  TRY(dalloc(ctx, &c->d_out_tmp, (size_t)c->N * 2));
  CU(cudaStreamSynchronize(c->stream));
  CU(cudaGetLastError());

  // algorithmic bytes of one matvec (compulsory traffic; s bytes per complex of the far field)
  for (int prec = 0; prec < 2; ++prec) {
    double s = prec == 0 ? 16.0 : 8.0;
    double b = s * (4.0 * neq * c->N + (double)nfit * c->N) + 16.0 * c->nnz + 32.0 * c->N;
    for (int lam = 0; lam < 2; ++lam) {
      double Pk = (double)c->og[lam].Px * c->og[lam].Py, Mg = (double)c->og[lam].Px * c->og[lam].nrow;
      b += s * (2 * Pk + 2 * Mg + Mg);
    }
    if (prec == 0) c->bytes64 = b; else c->bytes32 = b;
  }
  c->launches_per_apply = 9;  // projection, 2 X passes, 2 Y convolutions, 2 inverse X passes, near rows, far rows
  c->built = true;
  // capture the forward map of each precision in use; on failure keep direct launches
  c->use_graphs = getenv("SGF_NO_GRAPH") == nullptr;
  if (c->use_graphs) {
    for (int prec : {64, 32}) {
      if (prec == 32 && !mixed) continue;
      cudaError_t ge = build_apply_graph(c, prec);
      if (ge != cudaSuccess) {
        c->use_graphs = false;
        snprintf(c->err, sizeof(c->err), "graph capture failed (%s); launching kernels directly",
                 cudaGetErrorString(ge));
        break;
      }
    }
  }
  CU(cudaStreamSynchronize(c->stream));
  c->build_ms[0] = wall_ms() - t_build0;
  return SGF_OK;
}

static sgf_status apply_prec(sgf_ctx* ctx, const zd* mu, zd* out, int prec);

static sgf_status apply_adj_prec(sgf_ctx* ctx, const zd* v, zd* out, int prec) {
  if (ctx->op_exact) {
    cudaError_t e = launch_exact_gemv(ctx, v, out, true);
    if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "exact adjoint apply: %s", cudaGetErrorString(e));
    return SGF_OK;
  }
  if (!ctx->adj_ok)
    return set_err(ctx, SGF_EINVAL, "adjoint near rows of %d columns exceed the shared-memory limit", ctx->maxWT);
  cudaError_t e = prec == 64 ? launch_apply_adj64(ctx, v, out) : launch_apply_adj32(ctx, v, out);
  if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "adjoint apply: %s", cudaGetErrorString(e));
  return SGF_OK;
}

static bool op_ready(const sgf_ctx* ctx) { return ctx->op_exact ? ctx->exact_ready : ctx->built; }

extern "C" sgf_status sgf_apply(sgf_ctx* ctx, const void* mu_dev, void* out_dev, int nrhs, int transpose_conj) {
  if (!ctx) return SGF_EINVAL;
  if (!op_ready(ctx)) return set_err(ctx, SGF_ESTATE, "operator not built");
  if (transpose_conj != 0 && transpose_conj != 1) return set_err(ctx, SGF_EINVAL, "transpose_conj must be 0 or 1");
  if (nrhs < 1 || !mu_dev || !out_dev) return set_err(ctx, SGF_EINVAL, "bad apply arguments");
  if (nrhs > 1 && !transpose_conj && !ctx->op_exact && !ctx->profiling && ctx->debug_mask == 15) {
    // several densities: one pass over the operator data per MC_MAX columns
    cudaError_t e = ctx->prm.precision == 64 ? launch_apply_nrhs64(ctx, (const zd*)mu_dev, (zd*)out_dev, nrhs)
                                             : launch_apply_nrhs32(ctx, (const zd*)mu_dev, (zd*)out_dev, nrhs);
    if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "multi-column apply: %s", cudaGetErrorString(e));
    return SGF_OK;
  }
  for (int r = 0; r < nrhs; ++r) {
    const zd* mu = (const zd*)mu_dev + (size_t)r * ctx->N;
    zd* out = (zd*)out_dev + (size_t)r * ctx->N;
    sgf_status st = transpose_conj ? apply_adj_prec(ctx, mu, out, ctx->prm.precision)
                                   : apply_prec(ctx, mu, out, ctx->prm.precision);
    if (st != SGF_OK) return st;
  }
  if (transpose_conj || ctx->op_exact) return SGF_OK;
  if (ctx->profiling) {
    cudaEventSynchronize(ctx->ev[6]);
    float ms;
    for (int i = 0; i < 6; ++i) {
      cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]);
      ctx->stage_ms[i] = ms;
    }
    cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[6]);
    ctx->stage_ms[6] = ms;
  }
  return SGF_OK;
}

static sgf_status apply_prec(sgf_ctx* ctx, const zd* mu, zd* out, int prec) {
  const GraphSlot& gs = ctx->gs[prec == 64 ? 0 : 1];
  cudaError_t e;
  if (ctx->op_exact) {
    e = launch_exact_gemv(ctx, mu, out, false);
    if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "exact apply: %s", cudaGetErrorString(e));
    return SGF_OK;
  }
  if (ctx->use_graphs && gs.ok && !ctx->profiling && ctx->debug_mask == 15)
    e = launch_apply_graph(ctx, prec, mu, out);
  else
    e = prec == 64 ? launch_apply64(ctx, mu, out) : launch_apply32(ctx, mu, out);
  if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "apply: %s", cudaGetErrorString(e));
  return SGF_OK;
}

extern "C" sgf_status sgf_apply_host(sgf_ctx* ctx, const void* mu_host, void* out_host, int nrhs) {
  if (!ctx) return SGF_EINVAL;
  if (!op_ready(ctx)) return set_err(ctx, SGF_ESTATE, "operator not built");
  size_t nb = (size_t)ctx->N * sizeof(zd);
  for (int r = 0; r < nrhs; ++r) {
    CU(cudaMemcpyAsync(ctx->d_mu_tmp, (const char*)mu_host + r * nb, nb, cudaMemcpyHostToDevice, ctx->stream));
    TRY(apply_prec(ctx, ctx->d_mu_tmp, ctx->d_out_tmp, ctx->prm.precision));
    CU(cudaMemcpyAsync((char*)out_host + r * nb, ctx->d_out_tmp, nb, cudaMemcpyDeviceToHost, ctx->stream));
  }
  CU(cudaStreamSynchronize(ctx->stream));
  return SGF_OK;
}

extern "C" sgf_status sgf_rhs(sgf_ctx* ctx, void* out_dev) {
  if (!ctx) return SGF_EINVAL;
  if (!ctx->built && !ctx->geom) return set_err(ctx, SGF_ESTATE, "operator not built");
  CU(launch_rhs(ctx, (zd*)out_dev));
  return SGF_OK;
}

// ------------------------------------------------------------------ GMRES (restarted, CGS2)
struct Krylov {
  zd *V = nullptr, *h = nullptr, *partial = nullptr, *r = nullptr;
  zd* H = nullptr;  // Hessenberg columns written by the device, [m][mrec + m + 1] column-major
  zd* Q = nullptr;  // (mrec + 1) x mrec: the recycled space's combination coefficients
  float4 *part = nullptr, *npart = nullptr;  // float-float partial sums of the Arnoldi kernels
  unsigned* ticket = nullptr;                 // completion counters of k_kdots (zero between launches)
  int m = 0, nblk = 32;
  int mrec = 0;  // vector slots in front of V for a recycled space C (C then V, contiguous)
};

// A Krylov space recycled from an earlier solve with the same operator, in the GCRO form of Parks,
// de Sturler, Mackey, Johnson and Maiti ("Recycling Krylov subspaces for sequences of linear
// systems", SIAM J. Sci. Comput. 28, 2006): C = A U with orthonormal columns (stored in the m slots
// just before the Krylov basis V) and U = Vold R^{-1}, from that solve's Arnoldi relation
// A V_m = V_{m+1} Hbar_m = (V_{m+1} Q_m) R. A later solve projects each cycle's residual onto the
// complement of range(C) (adding U C^H r to x) and orthogonalises every new Arnoldi vector against
// C together with its own basis; the coefficients against C, B = C^H A V_k, enter the solution as
// x -= U B y. The mixed path's refinement solves one correction system per step with the same
// operator; GMRES spends most of its first solve finding the few slow components of that
// operator, and the recycled space carries them into the later corrections.
struct Recycle {
  int m = 0;           // columns of C and U
  zd* Vold = nullptr;  // V_m of the solve it came from
  std::vector<cd> R;   // m x m upper triangle (column-major, leading dimension m)
};

// z = R^{-1} c for the recycled triangle
static void rec_solve(const Recycle& rc, const std::vector<cd>& c, std::vector<cd>& z) {
  const int m = rc.m;
  z.assign(m, cd(0));
  for (int i = m - 1; i >= 0; --i) {
    cd acc = c[i];
    for (int k = i + 1; k < m; ++k) acc -= rc.R[(size_t)k * m + i] * z[k];
    z[i] = acc / rc.R[(size_t)i * m + i];
  }
}

static sgf_status dot_host(sgf_ctx* ctx, Krylov& K, const zd* V, int m, const zd* w, std::vector<cd>& out) {
  CU(launch_dots(V, m, ctx->N, w, ctx->N, K.partial, K.nblk, K.h, ctx->stream));
  out.resize(m);
  CU(cudaMemcpyAsync(out.data(), K.h, m * sizeof(zd), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return SGF_OK;
}

// Solves A x = b from x = 0 with operator precision prec; returns applications in *its.
static sgf_status apply_op(sgf_ctx* ctx, const zd* x, zd* out, int prec, bool adj) {
  return adj ? apply_adj_prec(ctx, x, out, prec) : apply_prec(ctx, x, out, prec);
}

// Solves A x = b from x = 0 with operator precision prec; returns applications in *its. With
// true_check (outer and FP64 solves) a cycle whose Arnoldi estimate reaches tol is followed by the
// true residual b - A x: if that is still above tol another cycle runs. Without it (inner solves
// of the refinement) the estimate decides. Either way a cycle that reduces the true residual by
// less than 10% ends the solve (attainable accuracy reached, or restarted GMRES stagnating).
// rc: a recycled space of the same operator to deflate with; harvest: receives the space of this
// solve's last cycle (its C is written in front of K.V, where a later solve with rc reads it).
static sgf_status gmres(sgf_ctx* ctx, Krylov& K, int prec, bool adj, const zd* b, zd* x, double tol, int maxit,
                        int* its, double* relres, bool true_check = true, const Recycle* rc = nullptr,
                        Recycle* harvest = nullptr) {
  const long N = ctx->N;
  const int m = K.m;
  const int mr = rc ? rc->m : 0;
  const zd* Cb = K.V - (size_t)mr * N;  // [C | V]: the recycled space, then this solve's basis
  std::vector<cd> tmp;
  TRY(dot_host(ctx, K, b, 1, b, tmp));
  double bn = std::sqrt(tmp[0].real());
  CU(cudaMemsetAsync(x, 0, N * sizeof(zd), ctx->stream));
  if (!std::isfinite(bn)) return set_err(ctx, SGF_ENONFINITE, "non-finite right-hand side");
  if (bn == 0) { *relres = 0; return SGF_OK; }
  int total = 0;
  double res = bn;
  // x -= Vold z (z on the host)
  auto sub_vold = [&](const std::vector<cd>& z) -> sgf_status {
    CU(cudaMemcpyAsync(K.h, z.data(), z.size() * sizeof(zd), cudaMemcpyHostToDevice, ctx->stream));
    CU(launch_kupdate(x, rc->Vold, (int)z.size(), N, K.h, N, nullptr, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    return SGF_OK;
  };
  // The Arnoldi steps run on the device without host round trips: CGS2 projections and updates in
  // float-float arithmetic, the Hessenberg column, the norm and the normalisation. After each group
  // of steps the host reads the new Hessenberg columns, applies the Givens rotations to them (FP64,
  // on the host) and takes the residual estimates; steps taken after the estimate reached tol
  // within a group are counted as applications and otherwise discarded. A group holds the steps
  // that the last group's per-step reduction predicts to tol (at least 1, at most kCheck); a solve
  // that deflates with a recycled space starts with 2, as it converges within a few steps.
  constexpr int kCheck = 8;
  const long ldh = mr + m + 1;  // column: mr coefficients against C, then the Hessenberg column
  const int nparts = kupdate_blocks(N);
  std::vector<cd> Hh, g(m + 1), y(m), cs(m), sn(m), z;  // Hh grows with the columns in use
  double prev_true = 0;
  int cycles = 0, jdone = 0;
  while (total < maxit) {
    // r = b - A x
    TRY(apply_op(ctx, x, K.r, prec, adj));
    CU(launch_axpby(K.r, zd(1, 0), b, zd(-1, 0), N, ctx->stream));
    if (mr > 0) {
      // c = C^H r; r -= C c; x += U c = Vold R^{-1} c
      CU(launch_kdots(Cb, mr, N, K.r, N, K.part, K.h, nullptr, 0, K.ticket, ctx->stream));
      CU(launch_kupdate(K.r, Cb, mr, N, K.h, N, nullptr, ctx->stream));
      tmp.resize(mr);
      CU(cudaMemcpyAsync(tmp.data(), K.h, mr * sizeof(zd), cudaMemcpyDeviceToHost, ctx->stream));
      CU(cudaStreamSynchronize(ctx->stream));
      rec_solve(*rc, tmp, z);
      for (auto& v : z) v = -v;
      TRY(sub_vold(z));
    }
    TRY(dot_host(ctx, K, K.r, 1, K.r, tmp));
    double beta = std::sqrt(tmp[0].real());
    res = beta;
    if (beta / bn <= tol) break;
    if (cycles > 0 && beta > 0.9 * prev_true) break;  // under 10% progress over a whole cycle
    prev_true = beta;
    ++cycles;
    CU(cudaMemcpyAsync(K.V, K.r, N * sizeof(zd), cudaMemcpyDeviceToDevice, ctx->stream));
    CU(launch_axpby(K.V, zd(0, 0), K.V, zd(1.0 / beta, 0), N, ctx->stream));
    std::fill(g.begin(), g.end(), cd(0));
    g[0] = beta;
    int j = 0;
    jdone = 0;
    bool stop = false;
    int group = mr > 0 ? 2 : kCheck;
    while (!stop && j < m && total < maxit) {
      const int j0 = j, jend = std::min({m, j + group, j + (maxit - total)});
      const double res0 = res;  // the estimate before this group
      for (; j < jend; ++j) {
        zd* vj = K.V + (size_t)j * N;
        zd* w = K.V + (size_t)(j + 1) * N;
        zd* Hc = K.H + (size_t)j * ldh;
        TRY(apply_op(ctx, vj, w, prec, adj));
        ++total;
        for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt against [C | V_0..V_j], twice
          CU(launch_kdots(Cb, mr + j + 1, N, w, N, K.part, K.h, Hc, pass, K.ticket, ctx->stream));
          CU(launch_kupdate(w, Cb, mr + j + 1, N, K.h, N, pass == 1 ? K.npart : nullptr, ctx->stream));
        }
        CU(launch_kscale(w, N, K.npart, nparts, Hc + mr + j + 1, ctx->stream));
      }
      if (Hh.size() < (size_t)jend * ldh) Hh.resize((size_t)jend * ldh);
      CU(cudaMemcpy2DAsync(Hh.data() + (size_t)j0 * ldh, ldh * sizeof(zd), K.H + (size_t)j0 * ldh, ldh * sizeof(zd),
                           (mr + jend + 1) * sizeof(zd), jend - j0, cudaMemcpyDeviceToHost, ctx->stream));
      CU(cudaStreamSynchronize(ctx->stream));
      for (int jj = j0; jj < jend; ++jj) {
        cd* colB = Hh.data() + (size_t)jj * ldh;
        cd* col = colB + mr;
        for (int i = 0; i <= mr + jj + 1; ++i)
          if (!std::isfinite(colB[i].real()) || !std::isfinite(colB[i].imag()))
            return set_err(ctx, SGF_ENONFINITE, "non-finite Krylov vector");
        for (int i = 0; i < jj; ++i) {  // earlier rotations
          const cd a = col[i], bb = col[i + 1];
          col[i] = std::conj(cs[i]) * a + std::conj(sn[i]) * bb;
          col[i + 1] = -sn[i] * a + cs[i] * bb;
        }
        const double hn = col[jj + 1].real();
        const cd a = col[jj];
        const double den = std::sqrt(std::norm(a) + hn * hn);
        cs[jj] = den > 0 ? a / den : cd(1);
        sn[jj] = den > 0 ? cd(hn / den) : cd(0);
        col[jj] = den;
        col[jj + 1] = 0;
        g[jj + 1] = -sn[jj] * g[jj];
        g[jj] = std::conj(cs[jj]) * g[jj];
        jdone = jj + 1;
        res = std::abs(g[jj + 1]);
        if (getenv("SGF_VERBOSE"))
          fprintf(stderr, "gmres prec %d rec %d it %d j %d res %.3e\n", prec, mr, total - (jend - 1 - jj), jj,
                  res / bn);
        if (res / bn <= tol || hn == 0) {  // converged, or breakdown (the Krylov space is invariant)
          stop = true;
          break;
        }
      }
      // next group: the steps to tol at this group's geometric reduction per step
      const double rate = res0 > 0 && res > 0 ? std::pow(res / res0, 1.0 / (jend - j0)) : 1.0;
      group = kCheck;
      if (rate < 1.0) {
        const double need = std::ceil(std::log(tol * bn / res) / std::log(rate));
        if (need < kCheck) group = std::max(1, (int)need);
      }
    }
    // back-substitution with the rotated triangle R (columns 0..jdone-1, rows 0..jdone-1)
    for (int i = jdone - 1; i >= 0; --i) {
      cd sacc = g[i];
      for (int k2 = i + 1; k2 < jdone; ++k2) sacc -= Hh[(size_t)k2 * ldh + mr + i] * y[k2];
      y[i] = sacc / Hh[(size_t)i * ldh + mr + i];
    }
    std::vector<cd> ny(jdone);
    for (int i = 0; i < jdone; ++i) ny[i] = -y[i];
    if (jdone > 0) {
      CU(cudaMemcpyAsync(K.h, ny.data(), jdone * sizeof(zd), cudaMemcpyHostToDevice, ctx->stream));
      CU(launch_kupdate(x, K.V, jdone, N, K.h, N, nullptr, ctx->stream));
    }
    if (mr > 0 && jdone > 0) {
      // x -= U B y = Vold R^{-1} (B y)
      std::vector<cd> t(mr, cd(0));
      for (int k2 = 0; k2 < jdone; ++k2)
        for (int i = 0; i < mr; ++i) t[i] += Hh[(size_t)k2 * ldh + i] * y[k2];
      rec_solve(*rc, t, z);
      TRY(sub_vold(z));
    }
    CU(cudaStreamSynchronize(ctx->stream));
    if (!true_check && res / bn <= tol) break;
  }
  if (harvest && mr == 0 && jdone >= 4 && harvest->Vold) {
    // the last cycle's space: m_h <= K.mrec leading columns of its Arnoldi relation, whose QR is
    // given by the first m_h Givens rotations: R (rotated columns) and Q_m = G_1^H ... G_m^H [I; 0]
    const int mh = std::min(jdone, K.mrec);
    harvest->m = mh;
    harvest->R.assign((size_t)mh * mh, cd(0));
    for (int k2 = 0; k2 < mh; ++k2)
      for (int i = 0; i <= k2; ++i) harvest->R[(size_t)k2 * mh + i] = Hh[(size_t)k2 * ldh + i];
    std::vector<cd> q((size_t)(mh + 1) * mh, cd(0));
    for (int k2 = 0; k2 < mh; ++k2) {
      cd* qc = q.data() + (size_t)k2 * (mh + 1);
      qc[k2] = 1;
      for (int i = mh - 1; i >= 0; --i) {  // G_i^H on rows (i, i+1)
        const cd a = qc[i], bb = qc[i + 1];
        qc[i] = cs[i] * a - std::conj(sn[i]) * bb;
        qc[i + 1] = sn[i] * a + std::conj(cs[i]) * bb;
      }
      for (int i = 0; i <= mh; ++i) qc[i] = -qc[i];  // kupdate subtracts
    }
    zd* C = K.V - (size_t)mh * N;
    CU(cudaMemcpyAsync(K.Q, q.data(), q.size() * sizeof(zd), cudaMemcpyHostToDevice, ctx->stream));
    CU(cudaMemsetAsync(C, 0, (size_t)mh * N * sizeof(zd), ctx->stream));
    for (int k2 = 0; k2 < mh; ++k2)  // C_k = V_{m+1} Q[:, k]
      CU(launch_kupdate(C + (size_t)k2 * N, K.V, mh + 1, N, K.Q + (size_t)k2 * (mh + 1), N, nullptr, ctx->stream));
    CU(cudaMemcpyAsync(harvest->Vold, K.V, (size_t)mh * N * sizeof(zd), cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
  }
  // true residual
  TRY(apply_op(ctx, x, K.r, prec, adj));
  CU(launch_axpby(K.r, zd(1, 0), b, zd(-1, 0), N, ctx->stream));
  TRY(dot_host(ctx, K, K.r, 1, K.r, tmp));
  *relres = std::sqrt(tmp[0].real()) / bn;
  *its = total;
  return SGF_OK;
}

// GMRES on A x = b (adj: A^H x = b); b = nullptr takes the right-hand side of sgf_rhs.
static sgf_status solve_impl(sgf_ctx* ctx, const zd* b_in, bool adj, double tol, int maxit, void* x_dev, int* iters,
                             double* relres) {
  if (!ctx) return SGF_EINVAL;
  if (!op_ready(ctx)) return set_err(ctx, SGF_ESTATE, "operator not built");
  if (!(tol > 0) || maxit < 1 || !x_dev) return set_err(ctx, SGF_EINVAL, "bad solve arguments");
  if (adj && !ctx->op_exact && !ctx->adj_ok) return apply_adj_prec(ctx, nullptr, nullptr, 64);
  const long N = ctx->N;
  Krylov K;
  // restart length: up to 1000 Krylov vectors (unrestarted below that), within 2 GiB of basis
  K.m = (int)std::max(20L, std::min({1000L, (long)maxit, (2L << 30) / (16L * N) - 1}));
  std::vector<void*> mine;
  auto al = [&](zd** p, size_t n) -> sgf_status {
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(zd));
    if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
    mine.push_back(*p);
    return SGF_OK;
  };
  sgf_status st = SGF_OK;
  zd *b, *x, *dlt;
  auto alb = [&](void** p, size_t bytes) -> sgf_status {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
    mine.push_back(*p);
    return SGF_OK;
  };
  // the mixed path's refinement recycles up to 256 vectors of its first correction solve
  const bool mixed = !(ctx->prm.precision == 64 || ctx->op_exact);
  K.mrec = mixed && !getenv("SGF_NO_RECYCLE") ? std::min(K.m, 256) : 0;
  const long nchunk = kdots_chunks(N);
  const size_t nvec = (size_t)K.mrec + K.m + 1;  // [recycled C | Krylov basis V]
  zd* W = nullptr;
  Recycle rc;
  if ((st = al(&K.H, (size_t)(K.mrec + K.m + 1) * K.m)) || (st = al(&W, nvec * N)) ||
      (st = al(&K.h, (size_t)K.mrec + K.m + 2)) || (st = al(&K.partial, (size_t)(K.m + 2) * K.nblk)) ||
      (st = alb((void**)&K.part, (size_t)nchunk * nvec * sizeof(float4))) ||
      (st = alb((void**)&K.npart, (size_t)kupdate_blocks(N) * sizeof(float4))) ||
      (st = alb((void**)&K.ticket, (size_t)kdots_groups((int)nvec) * sizeof(unsigned))) ||
      (K.mrec > 0 && ((st = al(&K.Q, (size_t)(K.mrec + 1) * K.mrec)) || (st = al(&rc.Vold, (size_t)K.mrec * N)))) ||
      (st = al(&K.r, N)) ||
      (st = al(&b, N)) || (st = al(&x, N)) || (st = al(&dlt, N))) {
    for (void* p : mine) cudaFree(p);
    return st;
  }
  K.V = W + (size_t)K.mrec * N;
  cudaMemsetAsync(K.ticket, 0, (size_t)kdots_groups((int)nvec) * sizeof(unsigned), ctx->stream);
  int its = 0;
  double rr = 1;
  if (b_in)
    cudaMemcpyAsync(b, b_in, N * sizeof(zd), cudaMemcpyDeviceToDevice, ctx->stream);
  else
    launch_rhs(ctx, b);
  if (ctx->prm.precision == 64 || ctx->op_exact) {
    st = gmres(ctx, K, 64, adj, b, x, tol, maxit, &its, &rr);
  } else {
    // FP64 residual refinement around inner mixed-precision GMRES solves
    std::vector<cd> tmp;
    cudaMemsetAsync(x, 0, N * sizeof(zd), ctx->stream);
    cudaMemcpyAsync(K.r, b, N * sizeof(zd), cudaMemcpyDeviceToDevice, ctx->stream);
    st = dot_host(ctx, K, b, 1, b, tmp);
    double bn = std::sqrt(tmp[0].real());
    if (st == SGF_OK && !std::isfinite(bn)) st = set_err(ctx, SGF_ENONFINITE, "non-finite right-hand side");
    zd* r = nullptr;
    if (st == SGF_OK) st = al(&r, N);
    if (st == SGF_OK) cudaMemcpyAsync(r, b, N * sizeof(zd), cudaMemcpyDeviceToDevice, ctx->stream);
    if (st == SGF_OK && bn == 0) rr = 0;
    // Each step solves A_32 d = r to 1e-6 (Arnoldi estimate) and adds d. The step contracts the
    // FP64 residual by about |A_64 - A_32| |A_32^{-1}|; when a step gains less than a factor 10
    // (ill-conditioned systems), the remaining correction is solved with the FP64 operator to the
    // final tolerance instead.
    bool fp64_inner = false;
    double rr_prev = 1.0;
    for (int outer = 0; outer < 30 && st == SGF_OK && bn > 0; ++outer) {
      int it_in = 0;
      double rr_in = 1;
      double itol = fp64_inner ? std::min(0.5, tol / rr_prev) : 1e-6;
      // the first mixed correction solve leaves its Krylov space for the later ones
      const bool use_rc = !fp64_inner && rc.m > 0;
      st = gmres(ctx, K, fp64_inner ? 64 : 32, adj, r, dlt, itol, maxit - its > 0 ? maxit - its : 1, &it_in, &rr_in,
                 fp64_inner, use_rc ? &rc : nullptr, !fp64_inner && outer == 0 && K.mrec > 0 ? &rc : nullptr);
      if (st != SGF_OK) break;
      its += it_in;
      launch_axpby(x, zd(1, 0), dlt, zd(1, 0), N, ctx->stream);
      st = apply_op(ctx, x, r, 64, adj);
      ++its;
      if (st != SGF_OK) break;
      launch_axpby(r, zd(1, 0), b, zd(-1, 0), N, ctx->stream);
      st = dot_host(ctx, K, r, 1, r, tmp);
      rr = std::sqrt(tmp[0].real()) / bn;
      if (getenv("SGF_VERBOSE"))
        fprintf(stderr, "refinement %d inner %s (recycled %d) its %d outer rr %.3e\n", outer,
                fp64_inner ? "fp64" : "mixed", use_rc ? rc.m : 0, it_in, rr);
      if (rr <= tol || its >= maxit) break;
      if (fp64_inner && rr > 0.5 * rr_prev) break;  // the FP64 correction stagnated as well
      if (rr > 0.1 * rr_prev) fp64_inner = true;
      rr_prev = rr;
    }
  }
  if (st == SGF_OK) {
    cudaMemcpyAsync(x_dev, x, N * sizeof(zd), cudaMemcpyDeviceToDevice, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
  }
  for (void* p : mine) cudaFree(p);
  if (iters) *iters = its;
  if (relres) *relres = rr;
  if (st != SGF_OK) return st;
  if (!(rr <= tol)) return set_err(ctx, SGF_ENOCONV, "GMRES stopped at relative residual %g after %d applications", rr, its);
  return SGF_OK;
}

extern "C" sgf_status sgf_solve(sgf_ctx* ctx, double tol, int maxit, void* mu_dev, int* iters, double* relres) {
  return solve_impl(ctx, nullptr, false, tol, maxit, mu_dev, iters, relres);
}

extern "C" sgf_status sgf_solve_rhs(sgf_ctx* ctx, const void* rhs_dev, int transpose_conj, double tol, int maxit,
                                    void* x_dev, int* iters, double* relres) {
  if (!ctx) return SGF_EINVAL;
  if (!rhs_dev || (transpose_conj != 0 && transpose_conj != 1))
    return set_err(ctx, SGF_EINVAL, "bad solve arguments");
  return solve_impl(ctx, (const zd*)rhs_dev, transpose_conj == 1, tol, maxit, x_dev, iters, relres);
}

extern "C" sgf_status sgf_rayleigh(sgf_ctx* ctx, const void* mu_dev, int n_lo, int n_hi, double* B, double* eff,
                                   double* energy_err) {
  if (!ctx) return SGF_EINVAL;
  if (!ctx->built && !ctx->geom) return set_err(ctx, SGF_ESTATE, "operator not built");
  if (n_hi < n_lo || n_hi - n_lo > 100000) return set_err(ctx, SGF_EINVAL, "bad mode range");
  int nmod = n_hi - n_lo + 1;
  std::vector<double> mp(6 * nmod);
  rayleigh_mode_params(ctx, n_lo, nmod, mp.data());
  std::vector<cd> bns(nmod);
  for (int t = 0; t < nmod; ++t) bns[t] = cd(mp[6 * t + 1], mp[6 * t + 2]);
  double* d_mp;
  zd* d_B;
  CU(cudaMalloc(&d_mp, mp.size() * sizeof(double)));
  CU(cudaMalloc(&d_B, nmod * sizeof(zd)));
  cudaMemcpyAsync(d_mp, mp.data(), mp.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
  cudaError_t e = launch_rayleigh_mp(ctx, (const zd*)mu_dev, nmod, d_mp, d_B);
  std::vector<zd> hB(nmod);
  cudaMemcpyAsync(hB.data(), d_B, nmod * sizeof(zd), cudaMemcpyDeviceToHost, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(d_mp);
  cudaFree(d_B);
  if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "rayleigh: %s", cudaGetErrorString(e));
  double sum = 0;
  for (int t = 0; t < nmod; ++t) {
    if (B) { B[2 * t] = hB[t].re; B[2 * t + 1] = hB[t].im; }
    double an = ctx->alpha + 2 * SGF_PI * (n_lo + t) / ctx->d;
    bool prop = ctx->k * ctx->k - an * an > 0;
    double en = prop ? bns[t].real() / ctx->beta * abs2(hB[t]) : 0.0;
    if (eff) eff[t] = en;
    sum += en;
  }
  if (energy_err) *energy_err = 1.0 - sum;
  return SGF_OK;
}

extern "C" sgf_status sgf_info(const sgf_ctx* ctx, double* info) {
  if (!ctx || !info) return SGF_EINVAL;
  if (!ctx->built) return SGF_ESTATE;
  double v[24] = {(double)ctx->N, (double)ctx->n_occ, (double)ctx->nnz, (double)ctx->og[0].Px,
                  (double)ctx->og[0].nrow, (double)ctx->og[0].Py, (double)ctx->og[1].Px, (double)ctx->og[1].nrow,
                  (double)ctx->og[1].Py, (double)ctx->neq, (double)ctx->nfit, (double)ctx->nb,
                  (double)ctx->nm, ctx->bytes64, ctx->bytes32, (double)ctx->launches_per_apply,
                  ctx->use_graphs ? 1.0 : 0.0, (double)ctx->maxW, (double)ctx->maxnq, (double)ctx->twlog,
                  ctx->build_ms[0], ctx->build_ms[1], ctx->build_ms[2], ctx->build_ms[3]};
  memcpy(info, v, sizeof(v));
  return SGF_OK;
}

extern "C" sgf_status sgf_set_profiling(sgf_ctx* ctx, int on) {
  if (!ctx) return SGF_EINVAL;
  ctx->profiling = on != 0;
  return SGF_OK;
}

extern "C" sgf_status sgf_debug_mask(sgf_ctx* ctx, int mask) {
  if (!ctx || mask < 0 || mask > 15) return SGF_EINVAL;
  ctx->debug_mask = mask;
  return SGF_OK;
}

extern "C" sgf_status sgf_debug_force_variants(sgf_ctx* ctx, int conv_variant, int fftx_vpt) {
  if (!ctx) return SGF_EINVAL;
  if (!ctx->built) return set_err(ctx, SGF_ESTATE, "operator not built");
  if (conv_variant < 0 || conv_variant > 3 || (fftx_vpt != 0 && fftx_vpt != 8 && fftx_vpt != 16))
    return set_err(ctx, SGF_EINVAL, "conv_variant must be 0..3 and fftx_vpt 0, 8 or 16");
  sgf_ctx* c = ctx;
  const bool mixed = c->prm.precision == 32;
  for (int lam = 0; lam < 2; ++lam)
    for (int prec : {64, 32}) {
      if (prec == 32 && !mixed) continue;
      if (!debug_variants_fit(c->og[lam], prec, conv_variant, fftx_vpt))
        return set_err(ctx, SGF_EINVAL, "variant %d / %d values per thread does not fit orientation %d (FP%d)",
                       conv_variant, fftx_vpt, lam, prec);
    }
  CU(cudaSetDevice(c->device));
  CU(cudaStreamSynchronize(c->stream));
  if (conv_variant == 2)  // the global-scratch variant's partial products
    for (int lam = 0; lam < 2; ++lam) {
      size_t n = (size_t)c->og[lam].Px * c->og[lam].Py;
      if (!c->o64.accg[lam]) TRY(dalloc(ctx, &c->o64.accg[lam], n));
      if (mixed && !c->o32.accg[lam]) TRY(dalloc(ctx, &c->o32.accg[lam], n));
    }
  for (int lam = 0; lam < 2; ++lam) {
    c->og[lam].force_conv = conv_variant;
    c->og[lam].force_vpt = fftx_vpt;
  }
  // the captured forward maps hold the launch shapes: capture them again
  destroy_graphs(c);
  if (c->use_graphs)
    for (int prec : {64, 32}) {
      if (prec == 32 && !mixed) continue;
      cudaError_t ge = build_apply_graph(c, prec);
      if (ge != cudaSuccess) {
        c->use_graphs = false;
        destroy_graphs(c);
        break;
      }
    }
  CU(cudaStreamSynchronize(c->stream));
  return SGF_OK;
}

extern "C" sgf_status sgf_stage_times(const sgf_ctx* ctx, double* t) {
  if (!ctx || !t) return SGF_EINVAL;
  for (int i = 0; i < 8; ++i) t[i] = ctx->stage_ms[i];
  return SGF_OK;
}

extern "C" sgf_status sgf_debug_table(const sgf_ctx* ctx_, int lam, int kind, void* host_out) {
  sgf_ctx* ctx = const_cast<sgf_ctx*>(ctx_);
  if (!ctx || !host_out || lam < 0 || lam > 1 || kind < 0 || kind > 1) return SGF_EINVAL;
  if (!ctx->built) return set_err(ctx, SGF_ESTATE, "operator not built");
  long n = (long)ctx->og[lam].Px * ctx->og[lam].Py;
  zd* tmp;
  CU(cudaMalloc(&tmp, n * sizeof(zd)));
  cudaError_t e = launch_debug_table(ctx, lam, kind, tmp);
  cudaMemcpyAsync(host_out, tmp, n * sizeof(zd), cudaMemcpyDeviceToHost, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "debug table: %s", cudaGetErrorString(e));
  return SGF_OK;
}

// ------------------------------------------------------------------ gradient (discrete adjoint)
// Derivative of B_n (eq. rayexp) and e_n = beta_n/beta |B_n|^2 with respect to the profile's
// Fourier coefficients, through the adjoint of the accelerated system A(f) mu = b(f), B_n = w^T mu:
//   dB_n = (dw)^T mu + lam^T (db - dA mu),   A^T lam = w   (solved as A^H conj(lam) = conj(w)).
// Each factor of A is node-local: row i of the reconstruction rows, the right-hand side, the target
// mode factors and the target side of the near operator depend on node i alone; column l of the
// projection, the source mode factors, w and the source side of the near operator on node l alone;
// the kernel tables and the FFT convolution on no node. Moving ALL target positions by +-eps thus
// gives, row by row, the derivative of (A mu)_i with respect to node i's own position, and moving
// all source positions the derivative of (A^T lam)_l with respect to node l's. The node-local
// factors are rebuilt at the moved positions with the operator's own kernels and differenced
// centrally; the f'' dependence (the K_r diagonal) is analytic. Node sensitivities then go to the
// coefficients through f(x) = a_0 + sum a_m cos(2 pi m x/d) + b_m sin(2 pi m x/d).
static sgf_status gradient_impl(sgf_ctx* ctx, const void* mu_dev, int n_mode, double tol, int maxit, double* B,
                                double* e_n, double* grad_a, double* grad_b, int* adj_iters, bool analytic) {
  if (!ctx) return SGF_EINVAL;
  if (!ctx->built) return set_err(ctx, SGF_ESTATE, "operator not built");
  if (ctx->op_exact)
    return set_err(ctx, SGF_ESTATE, "the gradient differentiates the accelerated operator: select it first");
  if (!mu_dev || !grad_a || !grad_b || !(tol > 0) || maxit < 1) return set_err(ctx, SGF_EINVAL, "bad gradient arguments");
  if (!ctx->adj_ok || !ctx->keep.tr_off) return apply_adj_prec(ctx, nullptr, nullptr, 64);
  sgf_ctx* c = ctx;
  const long N = c->N;
  const int M = (int)c->fa.size() - 1;
  const int neq = c->neq, nfit = c->nfit;
  const size_t nmN = (size_t)N * std::max(1, c->nm);
  // mode parameters of n (as sgf_rayleigh)
  std::vector<int> ue = ueta_set(c);
  double an = c->alpha + 2 * SGF_PI * n_mode / c->d;
  cd bn = beta_host(c->k, an);
  cd Qn = Qj_host(bn, c->prm.h, c->prm.j);
  bool inU = std::find(ue.begin(), ue.end(), n_mode) != ue.end();
  double mp[6] = {an, bn.real(), bn.imag(), Qn.real(), Qn.imag(), inU ? 1.0 : 0.0};

  std::vector<void*> mine;
  auto al = [&](void** p, size_t bytes) -> sgf_status {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
    mine.push_back(*p);
    return SGF_OK;
  };
  double *d_mp, *fp, *f1p;
  zd *w, *wc, *wp, *lam, *lamc, *y, *bp, *g0, *g1, *Ip2, *Ipl2, *C2, *CT2, *MT2, *MS2, *MSh2, *P2, *dots, *part;
  sgf_status st = SGF_OK;
  const size_t zN = N * sizeof(zd);
  void** ptrs[] = {(void**)&w, (void**)&wc, (void**)&wp, (void**)&lam, (void**)&lamc, (void**)&y, (void**)&bp,
                   (void**)&g0, (void**)&g1};
  for (void** pp2 : ptrs)
    if (st == SGF_OK) st = al(pp2, zN);
  if (st == SGF_OK) st = al((void**)&d_mp, 6 * sizeof(double));
  if (st == SGF_OK) st = al((void**)&fp, N * sizeof(double));
  if (st == SGF_OK) st = al((void**)&f1p, N * sizeof(double));
  if (st == SGF_OK) st = al((void**)&Ip2, (size_t)nfit * N * sizeof(zd));
  if (st == SGF_OK) st = al((void**)&Ipl2, (size_t)nfit * N * sizeof(zd));
  if (st == SGF_OK) st = al((void**)&C2, (size_t)c->nnz * sizeof(zd));
  if (st == SGF_OK) st = al((void**)&CT2, (size_t)c->nnz * sizeof(zd));
  if (st == SGF_OK) st = al((void**)&MT2, nmN * sizeof(zd));
  if (st == SGF_OK) st = al((void**)&MS2, nmN * sizeof(zd));
  if (st == SGF_OK) st = al((void**)&MSh2, nmN * sizeof(zd));
  if (st == SGF_OK) st = al((void**)&P2, (size_t)4 * neq * N * sizeof(zd));
  if (st == SGF_OK) st = al((void**)&dots, 4 * sizeof(zd));
  if (st == SGF_OK) st = al((void**)&part, 64 * sizeof(zd));
  auto cleanup = [&]() {
    cudaStreamSynchronize(c->stream);
    for (void* p : mine) cudaFree(p);
  };
  if (st != SGF_OK) {
    cleanup();
    return st;
  }
  const int mask = c->debug_mask;
  c->debug_mask = 15;
  cudaError_t e = cudaSuccess;
  auto ck = [&](cudaError_t r) {
    if (e == cudaSuccess && r != cudaSuccess) e = r;
  };
  const zd* mu = (const zd*)mu_dev;
  ck(cudaMemcpyAsync(d_mp, mp, sizeof(mp), cudaMemcpyHostToDevice, c->stream));
  // B_n = sum_l w_l mu_l
  ck(launch_rayleigh_weights(c, d_mp, c->d_f, c->d_f1, w, 0));
  ck(launch_conj(w, wc, N, c->stream));
  ck(launch_dots(wc, 1, N, mu, N, part, 32, dots, c->stream));
  zd hB;
  ck(cudaMemcpyAsync(&hB, dots, sizeof(zd), cudaMemcpyDeviceToHost, c->stream));
  ck(cudaStreamSynchronize(c->stream));
  if (e != cudaSuccess) {
    c->debug_mask = mask;
    cleanup();
    return set_err(ctx, SGF_ECUDA, "gradient: %s", cudaGetErrorString(e));
  }
  // adjoint system A^H conj(lam) = conj(w)
  int its = 0;
  double rr = 1;
  st = solve_impl(c, wc, true, tol, maxit, y, &its, &rr);
  if (adj_iters) *adj_iters = its;
  if (st != SGF_OK) {
    c->debug_mask = mask;
    cleanup();
    return st;
  }
  ck(launch_conj(y, lam, N, c->stream));
  ck(cudaMemcpyAsync(lamc, y, zN, cudaMemcpyDeviceToDevice, c->stream));
  ck(cudaMemsetAsync(g0, 0, zN, c->stream));
  ck(cudaMemsetAsync(g1, 0, zN, c->stream));
  // node sensitivities of f (v = 0) and f' (v = 1): g_v = lam .* (db - dA_t mu) + mu .* (dw - dA_s^T lam)
  const BuildKeep& K = c->keep;
  // one evaluation of the target and source terms with the factors in the given buffers (derivative
  // factors, or the factors at moved positions), accumulated into g with weight sc
  auto terms = [&](zd* g, double sc, int dm_t, int dm_s, const double* ft, const double* f1t, const double* fs,
                   const double* f1s, int mask_apply) {
    ck(launch_build_I_geo(c, K.pinv_fb, Ipl2, K.samp_rel, ft, f1t, Ip2, dm_t));
    ck(launch_near_geo(c, K.phi, K.dcy_min, K.n_dcy, Ipl2, c->o64.P, K.pp, K.kress, ft, f1t, c->d_f2, c->d_f, c->d_f1,
                       C2, dm_t));
    ck(launch_modes_geo(c, K.modes_n, ft, f1t, MT2, MS2, dm_t));
    ck(launch_rhs_geo(c, ft, f1t, bp, dm_t));
    std::swap(c->o64.Ip, Ip2);
    std::swap(c->d_C, C2);
    std::swap(c->d_MT, MT2);
    c->debug_mask = mask_apply;
    ck(launch_apply64(c, mu, y));
    c->debug_mask = 15;
    std::swap(c->o64.Ip, Ip2);
    std::swap(c->d_C, C2);
    std::swap(c->d_MT, MT2);
    ck(launch_grad_acc(g, sc, lam, bp, y, N, c->stream));
    ck(launch_build_P_geo(c, K.pinv_eq, K.coll_rel, fs, f1s, P2, dm_s == 0 ? 0 : dm_s - 2));
    ck(launch_near_geo(c, K.phi, K.dcy_min, K.n_dcy, K.Iplain, P2, K.pp, K.kress, c->d_f, c->d_f1, c->d_f2, fs, f1s,
                       C2, dm_s));
    ck(launch_near_transpose(c->n_blk, K.pp.q, K.pp.r, K.pp.off, K.pp.ld, K.tr_off, K.tr_ld, c->d_cell_start, C2,
                             CT2, c->stream));
    ck(launch_modes_geo(c, K.modes_n, fs, f1s, MT2, MS2, dm_s == 0 ? 0 : dm_s - 2));
    ck(launch_conj_transpose(MS2, c->nm, N, MSh2, c->stream));
    ck(launch_rayleigh_weights(c, d_mp, fs, f1s, wp, dm_s == 0 ? 0 : dm_s - 2));
    std::swap(c->o64.P, P2);
    std::swap(c->d_CT, CT2);
    std::swap(c->d_MSh, MSh2);
    c->debug_mask = mask_apply;
    ck(launch_apply_adj64(c, lamc, y));
    c->debug_mask = 15;
    std::swap(c->o64.P, P2);
    std::swap(c->d_CT, CT2);
    std::swap(c->d_MSh, MSh2);
    ck(launch_conj(y, y, N, c->stream));
    ck(launch_grad_acc(g, sc, mu, wp, y, N, c->stream));
  };
  for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
    zd* g = v == 0 ? g0 : g1;
    if (analytic) {
      // derivative factors at the nodes' positions; the applications leave out the sigma/2 identity,
      // which does not depend on the nodes
      terms(g, 1.0, v + 1, v + 3, c->d_f, c->d_f1, c->d_f, c->d_f1, 7);
      continue;
    }
    double vmax = 1.0;
    for (long i = 0; i < N; ++i) vmax = std::max(vmax, std::fabs(v == 0 ? c->hf[i] : c->hf1[i]));
    const double eps = 1e-6 * vmax;
    for (int sgn = 1; sgn >= -1 && e == cudaSuccess; sgn -= 2) {
      ck(launch_offset(c->d_f, v == 0 ? sgn * eps : 0.0, N, fp, c->stream));
      ck(launch_offset(c->d_f1, v == 1 ? sgn * eps : 0.0, N, f1p, c->stream));
      terms(g, sgn / (2 * eps), 0, 0, fp, f1p, fp, f1p, 15);
    }
  }
  std::vector<zd> h0(N), h1(N), hl(N), hm(N);
  ck(cudaMemcpyAsync(h0.data(), g0, zN, cudaMemcpyDeviceToHost, c->stream));
  ck(cudaMemcpyAsync(h1.data(), g1, zN, cudaMemcpyDeviceToHost, c->stream));
  ck(cudaMemcpyAsync(hl.data(), lam, zN, cudaMemcpyDeviceToHost, c->stream));
  ck(cudaMemcpyAsync(hm.data(), mu, zN, cudaMemcpyDeviceToHost, c->stream));
  ck(cudaStreamSynchronize(c->stream));
  c->debug_mask = mask;
  cleanup();
  if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "gradient: %s", cudaGetErrorString(e));
  // f'' (K_r diagonal, dx f''/(4 pi (1 + f'^2))): analytic; chain rule to the coefficients
  std::vector<cd> g2(N);
  for (long i = 0; i < N; ++i) {
    cd li(hl[i].re, hl[i].im), mi(hm[i].re, hm[i].im);
    g2[i] = -li * mi * (c->dx / (4 * SGF_PI * (1 + c->hf1[i] * c->hf1[i])));
  }
  std::vector<cd> dBa(M + 1, cd(0)), dBb(M + 1, cd(0));
  for (int m = 0; m <= M; ++m) {
    double km = 2 * SGF_PI * m / c->d;
    cd sa(0), sb(0);
    for (long i = 0; i < N; ++i) {
      double cs = std::cos(km * c->hx[i]), sn = std::sin(km * c->hx[i]);
      cd a0(h0[i].re, h0[i].im), a1(h1[i].re, h1[i].im);
      sa += a0 * cs - a1 * (km * sn) - g2[i] * (km * km * cs);
      sb += a0 * sn + a1 * (km * cs) - g2[i] * (km * km * sn);
    }
    dBa[m] = sa;
    dBb[m] = m == 0 ? cd(0) : sb;
  }
  cd Bn(hB.re, hB.im);
  bool prop = c->k * c->k - an * an > 0;
  double pref = prop ? bn.real() / c->beta : 0.0;
  if (B) {
    B[0] = Bn.real();
    B[1] = Bn.imag();
  }
  if (e_n) *e_n = pref * std::norm(Bn);
  for (int m = 0; m <= M; ++m) {
    grad_a[m] = pref * 2 * std::real(std::conj(Bn) * dBa[m]);
    grad_b[m] = pref * 2 * std::real(std::conj(Bn) * dBb[m]);
  }
  return SGF_OK;
}

// ------------------------------------------------------------------ parameters and cell-size tuning
extern "C" sgf_status sgf_get_params(const sgf_ctx* ctx, sgf_params* out) {
  if (!ctx || !out) return SGF_EINVAL;
  if (!ctx->have_params) return SGF_ESTATE;
  *out = ctx->prm;
  return SGF_OK;
}

// Cell-size autotuner. For each candidate cell count nx the quantities tied to the cell side
// L = d/nx are re-derived as for the workloads: box bottom hmin = min f - L/2 and rows
// ny = floor((max f - hmin)/L) + 1, singular window a = floor(0.75 L/dx) dx, shift
// h = (round(h0/dg) + 1/(j+1)) dg with dg = L/p and h0 the shift currently set. Every candidate
// that builds is timed over `reps` applications (CUDA events around the context's own launch
// path), and the context is left built with the fastest.
// Timing (and, with eps_tol > 0, accuracy) of each cell-count candidate; see sgf_autotune_cells
// and sgf_autotune in sgf.h.
static sgf_status autotune_impl(sgf_ctx* ctx, const int* nx_list, int n, int reps, double eps_tol, int* best_nx,
                                double* ms, double* eps_out) {
  if (!ctx) return SGF_EINVAL;
  if (!nx_list || n < 1 || reps < 1) return set_err(ctx, SGF_EINVAL, "bad autotune arguments");
  if (!ctx->have_profile || !ctx->have_wave || !ctx->have_params)
    return set_err(ctx, SGF_ESTATE, "profile, wave and params must be set before tuning");
  const sgf_params base = ctx->prm;
  const int N = base.N;
  const double d = ctx->d, dx = d / N;
  // profile at the nodes x_l = l d / N, l = 1..N
  double fmin = 1e300, fmax = -1e300, slope = 0;
  for (int l = 1; l <= N; ++l) {
    double x = l * dx, f = ctx->fa[0], f1 = 0;
    for (size_t m = 1; m < ctx->fa.size(); ++m) {
      double w = 2 * SGF_PI * m / d, t = w * x;
      f += ctx->fa[m] * std::cos(t) + ctx->fb[m] * std::sin(t);
      f1 += w * (-ctx->fa[m] * std::sin(t) + ctx->fb[m] * std::cos(t));
    }
    fmin = std::min(fmin, f);
    fmax = std::max(fmax, f);
    slope = std::max(slope, std::fabs(f1));
  }
  // the quantities tied to L are re-derived per candidate; with shifts (j > 0) h follows the
  // parameter rule of sgf_suggest_params: at least the shift set, clear of the singular window
  // (h >= 1.2 a max|f'|, Section 5.1), moved off the grid lags of the finest spacing L/p
  auto candidate = [&](int nx) {
    sgf_params P = base;
    const double L = d / nx;
    P.nx = nx;
    P.hmin = fmin - 0.5 * L;
    P.ny = (int)std::floor((fmax - P.hmin) / L) + 1;
    P.Ma = (int)std::floor(0.75 * L / dx + 1e-9);
    const double dg = L / base.p, a_s = P.Ma * dx;
    double h0 = base.h;
    if (base.j > 0) h0 = std::max(h0, 1.2 * a_s * slope);
    P.h = (std::round(h0 / dg) + 1.0 / (std::max(base.j, 1) + 1)) * dg;
    if (base.j > 0 && !(P.h > a_s * slope)) P.h += dg;
    return P;
  };
  double best = 1e300, best_eps = 1e300;
  int bnx = -1, enx = -1;  // fastest eligible candidate; most accurate one (fallback)
  zd* xsol = nullptr;
  if (eps_tol > 0 && cudaMalloc(&xsol, (size_t)N * sizeof(zd)) != cudaSuccess)
    return set_err(ctx, SGF_ECUDA, "autotune: allocation of the solution buffer failed");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return set_err(ctx, SGF_ECUDA, "autotune: event creation failed");
  }
  sgf_status fail = SGF_OK;
  for (int i = 0; i < n && fail == SGF_OK; ++i) {
    if (ms) ms[i] = -(double)SGF_EINVAL;
    if (nx_list[i] < 1 || N % nx_list[i] != 0) continue;
    ctx->prm = candidate(nx_list[i]);
    sgf_status st = sgf_build_operator(ctx);
    if (st != SGF_OK) {
      if (ms) ms[i] = -(double)st;
      continue;
    }
    float t = 0;
    if (cudaMemsetAsync(ctx->d_mu_tmp, 0, (size_t)N * sizeof(zd), ctx->stream) != cudaSuccess) fail = SGF_ECUDA;
    for (int w = 0; w < 3 && fail == SGF_OK; ++w) fail = apply_prec(ctx, ctx->d_mu_tmp, ctx->d_out_tmp, ctx->prm.precision);
    if (fail == SGF_OK && cudaEventRecord(e0, ctx->stream) != cudaSuccess) fail = SGF_ECUDA;
    for (int r = 0; r < reps && fail == SGF_OK; ++r)
      fail = apply_prec(ctx, ctx->d_mu_tmp, ctx->d_out_tmp, ctx->prm.precision);
    if (fail == SGF_OK && (cudaEventRecord(e1, ctx->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                           cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
      fail = SGF_ECUDA;
    if (fail != SGF_OK) break;
    double per = t / reps;
    if (ms) ms[i] = per;
    bool eligible = true;
    if (eps_tol > 0) {
      // the energy balance of the solution (eq. energy_error): the accuracy the candidate reaches
      int its = 0;
      double rr = 0, eps = 1e300;
      sgf_status ss = solve_impl(ctx, nullptr, false, 1e-12, 4000, xsol, &its, &rr);
      if (ss == SGF_OK || ss == SGF_ENOCONV) {
        const double k = ctx->k, d = ctx->d, al = ctx->alpha;
        const int nlo = (int)std::ceil((-k - al) * d / (2 * SGF_PI)), nhi = (int)std::floor((k - al) * d / (2 * SGF_PI));
        if (sgf_rayleigh(ctx, xsol, nlo, nhi, nullptr, nullptr, &eps) != SGF_OK) eps = 1e300;
      }
      if (eps_out) eps_out[i] = eps;
      eligible = std::fabs(eps) < eps_tol;
      if (std::fabs(eps) < best_eps) {
        best_eps = std::fabs(eps);
        enx = nx_list[i];
      }
    }
    if (eligible && per < best) {
      best = per;
      bnx = nx_list[i];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (xsol) cudaFree(xsol);
  if (fail != SGF_OK) {
    ctx->prm = base;
    ctx->built = false;
    return fail == SGF_ECUDA ? set_err(ctx, SGF_ECUDA, "autotune: timing a candidate failed") : fail;
  }
  if (bnx < 0 && enx >= 0) {  // built, but none reached eps_tol: keep the most accurate
    if (best_nx) *best_nx = enx;
    ctx->prm = candidate(enx);
    TRY(sgf_build_operator(ctx));
    return set_err(ctx, SGF_ENOCONV, "no candidate reaches the energy error %g (best %g with %d cell columns)",
                   eps_tol, best_eps, enx);
  }
  if (bnx < 0) {
    ctx->prm = base;
    ctx->built = false;
    return set_err(ctx, SGF_EINVAL, "no candidate cell count builds for this problem");
  }
  if (best_nx) *best_nx = bnx;
  ctx->prm = candidate(bnx);
  return sgf_build_operator(ctx);
}

extern "C" sgf_status sgf_autotune_cells(sgf_ctx* ctx, const int* nx_list, int n, int reps, int* best_nx, double* ms) {
  return autotune_impl(ctx, nx_list, n, reps, 0.0, best_nx, ms, nullptr);
}

extern "C" sgf_status sgf_autotune(sgf_ctx* ctx, const int* nx_list, int n, int reps, double eps_tol, int* best_nx,
                                   double* ms, double* eps) {
  if (!(eps_tol > 0)) return set_err(ctx, SGF_EINVAL, "sgf_autotune needs an energy-error tolerance eps_tol > 0");
  return autotune_impl(ctx, nx_list, n, reps, eps_tol, best_nx, ms, eps);
}

extern "C" sgf_status sgf_gradient(sgf_ctx* ctx, const void* mu_dev, int n_mode, double tol, int maxit, double* B,
                                   double* e_n, double* grad_a, double* grad_b, int* adj_iters) {
  return gradient_impl(ctx, mu_dev, n_mode, tol, maxit, B, e_n, grad_a, grad_b, adj_iters, true);
}

extern "C" sgf_status sgf_gradient_fd(sgf_ctx* ctx, const void* mu_dev, int n_mode, double tol, int maxit, double* B,
                                      double* e_n, double* grad_a, double* grad_b, int* adj_iters) {
  return gradient_impl(ctx, mu_dev, n_mode, tol, maxit, B, e_n, grad_a, grad_b, adj_iters, false);
}

// ------------------------------------------------------------------------------------------
// The unaccelerated operator as a dense matrix (Section 4). Without an accelerated build it sets up
// the nodes, the log-quadrature weights and the completion modes itself (no cells are needed).
extern "C" sgf_status sgf_build_exact(sgf_ctx* ctx) {
  if (!ctx) return SGF_EINVAL;
  if (!ctx->have_profile || !ctx->have_wave || !ctx->have_params)
    return set_err(ctx, SGF_ESTATE, "profile, wave and params must be set before build");
  const sgf_params& P = ctx->prm;
  if (P.N < 8 || P.N > 32768 || P.j < 0 || P.j > 24 || !(P.h > 0) || P.n_per < 1 || P.Ma < 2 || 2 * P.Ma >= P.N ||
      !(P.c_win > 0 && P.c_win < 1) || !(P.delta_min > 0) || !(P.spec_exp > 0))
    return set_err(ctx, SGF_EINVAL, "parameter out of range for the dense operator (8 <= N <= 32768, 2 <= Ma < N/2)");
  CU(cudaSetDevice(ctx->device));
  sgf_ctx* c = ctx;
  if (!c->built && !c->geom) {
    free_all(ctx);
    c->N = P.N;
    c->dx = c->d / P.N;
    c->a_s = P.Ma * c->dx;
    c->gam = 0.5 * c->a_s;
    int M = (int)c->fa.size() - 1;
    TRY(dalloc(ctx, &c->d_coef, 2 * (M + 1)));
    CU(cudaMemcpyAsync(c->d_coef, c->fa.data(), (M + 1) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CU(cudaMemcpyAsync(c->d_coef + M + 1, c->fb.data(), (M + 1) * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    TRY(dalloc(ctx, &c->d_x, c->N));
    TRY(dalloc(ctx, &c->d_f, c->N));
    TRY(dalloc(ctx, &c->d_f1, c->N));
    TRY(dalloc(ctx, &c->d_f2, c->N));
    CU(launch_profile(c));
    c->hx.resize(c->N); c->hf.resize(c->N); c->hf1.resize(c->N); c->hf2.resize(c->N);
    CU(cudaMemcpyAsync(c->hx.data(), c->d_x, c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(c->hf.data(), c->d_f, c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaMemcpyAsync(c->hf1.data(), c->d_f1, c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    double maxslope = 0;
    for (int i = 0; i < c->N; ++i) maxslope = std::max(maxslope, fabs(c->hf1[i]));
    if (P.j > 0 && !(P.h > c->a_s * maxslope))
      return set_err(ctx, SGF_EWINDOW, "shift h = %g must exceed a max|f'| = %g", P.h, c->a_s * maxslope);
    std::vector<double> binw(P.j + 1);
    for (int m = 0; m <= P.j; ++m) {
      double cb = 1;
      for (int i = 0; i < m; ++i) cb = cb * (P.j - i) / (i + 1);
      binw[m] = (m % 2 ? -1.0 : 1.0) * cb;
    }
    TRY(dalloc(ctx, &c->d_binw, binw.size()));
    CU(cudaMemcpy(c->d_binw, binw.data(), binw.size() * sizeof(double), cudaMemcpyHostToDevice));
    std::vector<double> kress(2 * P.Ma - 1);
    for (int s = -(P.Ma - 1); s <= P.Ma - 1; ++s) {
      double acc = 0;
      for (int m = 1; m < P.Ma; ++m) acc += cos(SGF_PI * m * s / P.Ma) / m;
      kress[s + P.Ma - 1] = -2 * c->dx * acc - c->dx / P.Ma * ((s & 1) ? -1.0 : 1.0);
    }
    TRY(dalloc(ctx, &c->keep.kress, kress.size()));
    CU(cudaMemcpy(c->keep.kress, kress.data(), kress.size() * sizeof(double), cudaMemcpyHostToDevice));
    std::vector<int> ue = ueta_set(c);
    c->nm = (int)ue.size();
    std::vector<double> mn(3 * std::max(1, c->nm));
    for (int t = 0; t < c->nm; ++t) {
      double an = c->alpha + 2 * SGF_PI * ue[t] / c->d;
      cd bn = beta_host(c->k, an);
      mn[3 * t] = an; mn[3 * t + 1] = bn.real(); mn[3 * t + 2] = bn.imag();
    }
    TRY(dalloc(ctx, &c->keep.modes_n, mn.size()));
    CU(cudaMemcpy(c->keep.modes_n, mn.data(), mn.size() * sizeof(double), cudaMemcpyHostToDevice));
    TRY(dalloc(ctx, &c->d_MT, (size_t)c->N * std::max(1, c->nm)));
    TRY(dalloc(ctx, &c->d_MS, (size_t)c->N * std::max(1, c->nm)));
    CU(launch_modes(c, c->keep.modes_n));
    TRY(dalloc(ctx, &c->d_msum, 64));
    TRY(dalloc(ctx, &c->d_mu_tmp, (size_t)c->N * 2));
    TRY(dalloc(ctx, &c->d_out_tmp, (size_t)c->N * 2));
    c->geom = true;
  }
  if (!c->d_Aex) TRY(dalloc(ctx, &c->d_Aex, (size_t)c->N * c->N));
  zd hk(0, 0);
  CU(near_hk(c, &hk));
  CU(launch_exact_entries(c, hk));
  CU(cudaStreamSynchronize(c->stream));
  c->exact_ready = true;
  return SGF_OK;
}

extern "C" sgf_status sgf_select_operator(sgf_ctx* ctx, int exact) {
  if (!ctx) return SGF_EINVAL;
  if (exact != 0 && exact != 1) return set_err(ctx, SGF_EINVAL, "operator selector must be 0 or 1");
  if (exact && !ctx->exact_ready) return set_err(ctx, SGF_ESTATE, "dense operator not built");
  ctx->op_exact = exact == 1;
  return SGF_OK;
}

extern "C" sgf_status sgf_exact_matrix(const sgf_ctx* ctx_, void* A_dev) {
  sgf_ctx* ctx = const_cast<sgf_ctx*>(ctx_);
  if (!ctx || !A_dev) return SGF_EINVAL;
  if (!ctx->exact_ready) return set_err(ctx, SGF_ESTATE, "dense operator not built");
  CU(cudaMemcpyAsync(A_dev, ctx->d_Aex, (size_t)ctx->N * ctx->N * sizeof(zd), cudaMemcpyDeviceToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return SGF_OK;
}
