// Internal state of an sgf context and the kernel launchers shared by the two translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string>
#include <complex>
#include <cmath>
#include <set>
#include <vector>
#include <algorithm>

#include "../../include/sgf.h"
#include "sgf_common.cuh"

// Geometry of one equivalent-source grid Pi_lambda^per (Section 5.4): X cyclic with Px points,
// nrow rows in Y; FFT length Py >= 2 nrow - 1 in Y (linear convolution).
struct Orient {
  int Px, logPx, nrow, Py, la, lb;  // Py = 2^la 3^lb >= 2 nrow - 1
  double dxg, dyg;
  // testing hook (sgf_debug_force_variants): 0 = chosen per launch, else the forced Y-convolution
  // variant (1 registers/16 values, 2 global scratch, 3 8 values) and X-pass values per thread
  int force_conv = 0, force_vpt = 0;
};

// Device operator data of one precision (T = double or float).
template <typename T>
struct OpData {
  cplx<T>* P = nullptr;        // per cell [2 orientations][2 neq][n_q] projection matrices
  cplx<T>* Ip = nullptr;       // per node [n_fit] reconstruction rows times the untwist e^{i alpha x_t}
  cplx<T>* src_tw = nullptr;   // [n_occ][2][neq] twist e^{-i alpha x_src} of the scatter
  cplx<T>* Khat[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [lam][mono, dip] spectra / (Px Py)
  cplx<T>* grid[2] = {nullptr, nullptr};                          // [lam]: xi then zeta, Px*nrow each
  cplx<T>* tw = nullptr;       // FFT twiddles e^{-2 pi i k / 2^twlog}, full circle (X passes)
  cplx<T>* twy[2] = {nullptr, nullptr};  // [lam] full-circle twiddles of length Py (Y passes)
  cplx<T>* accg[2] = {nullptr, nullptr};  // [lam] Y-convolution scratch [Px][Py] (FP64, long columns)
};

// Per-column data of the multi-column forward map: the column's density and output, and what
// depends on its problem's incidence angle (the scatter twist, alpha relative to the operator's, the
// completion-mode factors). Passed by value (MC_MAX columns per launch).
constexpr int MC_MAX = 8;
template <typename T>
struct MCol {
  const zd* mu = nullptr;
  zd* out = nullptr;
  const cplx<T>* src_tw = nullptr;
  double dalpha = 0.0;
  const zd* MT = nullptr;
  const zd* MS = nullptr;
  const float4* MTff = nullptr;
  const float4* MSff = nullptr;
  int nm = 0;
};
template <typename T>
struct MCols {
  MCol<T> c[MC_MAX];
  int n = 0;
};
template <typename T>
struct MultiSpace {
  cplx<T>* grid[2] = {nullptr, nullptr};
  cplx<T>* accg[2] = {nullptr, nullptr};
  zd* mpart = nullptr;
  float4* mpart_ff = nullptr;
  bool ready = false;
};

// One captured forward map: the kernel nodes that take mu/out are updated before each launch.
struct GraphSlot {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t n_proj = nullptr, n_interp = nullptr, n_near = nullptr;
  cudaKernelNodeParams kp_proj{}, kp_interp{}, kp_near{};
  bool ok = false;
};

struct NearPairs {  // device arrays of the (q, r) block list
  int n = 0;
  int *q = nullptr, *r = nullptr, *wrap = nullptr, *dcx = nullptr, *ld = nullptr;
  long* off = nullptr;
};

// Build-time operands kept after sgf_build_operator so that the node-dependent factors (P, I, the
// near operator, mode factors) can be rebuilt at moved node positions by sgf_gradient.
struct BuildKeep {
  double *coll_rel = nullptr, *samp_rel = nullptr, *src_rel = nullptr, *kress = nullptr, *modes_n = nullptr;
  zd *pinv_eq = nullptr, *pinv_fb = nullptr, *phi = nullptr, *Iplain = nullptr;
  long* tr_off = nullptr;  // adjoint near layout: destination offset and leading dimension per block
  int* tr_ld = nullptr;
  int dcy_min = 0, n_dcy = 0;
  NearPairs pp;
};

struct sgf_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  char err[2048] = {0};
  // problem definition
  double d = 0;
  std::vector<double> fa, fb;
  double k = 0, theta = 0, alpha = 0, beta = 0;
  int bc = 0;
  sgf_params prm{};
  bool have_profile = false, have_wave = false, have_params = false, built = false;
  // derived sizes
  int N = 0, neq = 0, nfit = 0, nb = 0, n_occ = 0, nm = 0;
  double dx = 0, L = 0, a_s = 0, gam = 0;
  Orient og[2];
  int twlog = 0;
  // host geometry
  std::vector<double> hx, hf, hf1, hf2;
  std::vector<int> cell_start;  // [n_occ + 1] into node_idx
  std::vector<int> node_idx;    // nodes in cell order
  std::vector<int> occ_cx, occ_cy;
  // device geometry and index tables
  double *d_x = nullptr, *d_f = nullptr, *d_f1 = nullptr, *d_f2 = nullptr, *d_coef = nullptr;
  int *d_cell_start = nullptr, *d_node_idx = nullptr, *d_node_cell = nullptr;
  int *d_occ_cx = nullptr, *d_occ_cy = nullptr;
  int* d_src_gidx = nullptr;   // [n_occ][2][neq]
  int* d_samp_gidx = nullptr;  // [n_occ][n_fit]
  double* d_binw = nullptr;    // (-1)^m C(j,m)
  // near field: blocks (q, r) of dense n_q x n_r values
  int n_blk = 0;
  long nnz = 0;
  int* d_blk_start = nullptr;  // [n_occ + 1] into block list
  int* d_blk_r = nullptr;      // occupied index of the source cell
  long* d_blk_off = nullptr;   // value offset of the block's first entry
  int* d_blk_col = nullptr;    // column offset of the block within its cell's rows
  long* d_cell_off = nullptr;  // [n_occ + 1] value offset of each cell's n_q x W_q rows
  int* d_cell_W = nullptr;     // [n_occ] row length W_q
  int* d_cols = nullptr;       // node index of each local column, cells in order
  int* d_coloff = nullptr;     // [n_occ + 1] offsets into d_cols
  signed char* d_colwrap = nullptr;  // period copy (-1, 0, 1) of each local column (its block's wrap)
  int maxW = 0;
  // adjoint near field: rows of each cell r hold conj(C) of the blocks (q, r), W^T_r columns
  zd* d_CT = nullptr;
  float4* d_CTff = nullptr;
  long* d_cell_offT = nullptr;
  int *d_cell_WT = nullptr, *d_colsT = nullptr, *d_coloffT = nullptr;
  int maxWT = 0;
  bool adj_ok = false;
  zd* d_blk_ph = nullptr;      // quasi-periodic phase of the source cell copy
  zd* d_C = nullptr;
  float4* d_Cff = nullptr;      // near operator as float-float pairs (mixed path)
  float4* d_muff = nullptr;     // [N] float-float copy of the density (mixed path)
  // modes
  zd *d_MT = nullptr, *d_MS = nullptr, *d_msum = nullptr;
  float4 *d_MTff = nullptr, *d_MSff = nullptr;  // float-float mode factors (mixed path)
  zd *d_MTh = nullptr, *d_MSh = nullptr;        // adjoint mode factors: MTh[n][i], MSh[i][n]
  float4 *d_MThff = nullptr, *d_MShff = nullptr;
  zd* d_mpart = nullptr;        // [nm][mode_chunks] FP64 mode-sum partials
  float4* d_mpart_ff = nullptr; // [nm][mode_chunks] float-float partials
  int mode_chunks = 64;
  // work items of the forward map: chunks of at most 32 nodes of one cell
  int n_items = 0;
  int *d_item_cell = nullptr, *d_item_lo = nullptr, *d_item_hi = nullptr;
  // work items of the near rows: chunks of one cell's rows holding about 4096 near entries
  // (4 to 32 rows), so that cells with long rows are spread over more blocks
  int n_nitems = 0;
  int *d_nitem_cell = nullptr, *d_nitem_lo = nullptr, *d_nitem_hi = nullptr;
  // precision-specific operator data
  OpData<double> o64;
  OpData<float> o32;
  MultiSpace<double> ms64;  // multi-column forward map work space (allocated on first use)
  MultiSpace<float> ms32;
  // FP64 kernel-table copies before the Y transform (testing)
  zd* d_Tx[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  // workspace
  zd *d_mu_tmp = nullptr, *d_out_tmp = nullptr;
  std::vector<void*> allocs;
  // profiling
  bool profiling = false;
  GraphSlot gs[2];  // [0] FP64, [1] mixed
  GraphSlot gs_nonear[2];  // the same without the near operator (angle-sharing batches), on demand
  bool use_graphs = true;
  int maxnq = 0;
  int debug_mask = 15;
  cudaEvent_t ev[8] = {nullptr};
  cudaStream_t side = nullptr;   // second stream for the V orientation of the forward map
  cudaStream_t side2 = nullptr;  // third stream for the near field of the forward map
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork0 = nullptr, ev_join2 = nullptr;
  double stage_ms[8] = {0};
  // wall times of the last sgf_build_operator (ms): total, kernel tables and spectra (A1), least
  // squares + projection/reconstruction factors, near operator (local sets, blocks, values)
  double build_ms[4] = {0};
  int launches_per_apply = 0;
  double bytes64 = 0, bytes32 = 0;
  BuildKeep keep;
  // the unaccelerated operator as a dense row-major N x N matrix (sgf_build_exact); geom: the nodes,
  // weights and mode factors exist without the accelerated build
  zd* d_Aex = nullptr;
  bool geom = false, exact_ready = false, op_exact = false;
};

sgf_status set_err(sgf_ctx* ctx, sgf_status st, const char* fmt, ...);
// host helpers shared by the entry points (sgf_capi.cu)
// cell rows cy_q whose cells lie within the local reach S_j of source row cy_r (the local sets L(q))
std::set<int> rows_of_Sj(int cy_r, int j, double h, double L);
// per mode n_lo .. n_lo + nmod - 1: [alpha_n, Re beta_n, Im beta_n, Re Q_j, Im Q_j, n in U^eta]
void rayleigh_mode_params(sgf_ctx* c, int n_lo, int nmod, double* mp);

// ---------------------------------------------------------------- launchers (sgf_kernels.cu)
struct BuildArgs;
cudaError_t launch_profile(sgf_ctx* c);
cudaError_t launch_build_matrices(sgf_ctx* c, zd* d_Acoll, zd* d_Bfb, const double* d_coll_rel,
                                  const double* d_src_rel, const double* d_samp_rel);
cudaError_t launch_qr_pinv(sgf_ctx* c, zd* A, int m_out, int n, bool augment, double reg, zd* pinv, zd* scratch);
cudaError_t launch_build_P(sgf_ctx* c, const zd* pinv_eq, const double* d_coll_rel);
cudaError_t launch_build_I(sgf_ctx* c, const zd* pinv_fb, zd* d_Iplain, const double* d_samp_rel);
cudaError_t launch_tables(sgf_ctx* c);
cudaError_t launch_phi_off(sgf_ctx* c, zd* d_phi, int dcy_min, int n_dcy, const double* d_samp_rel,
                           const double* d_src_rel);
cudaError_t launch_near(sgf_ctx* c, const zd* d_phi, int dcy_min, int n_dcy, const zd* d_Iplain, const NearPairs& pp,
                        const double* d_kress);
cudaError_t launch_modes(sgf_ctx* c, const double* d_modes_n);
cudaError_t launch_to_f32(const zd* src, zf* dst, long n, cudaStream_t s);
cudaError_t launch_split_ff(const zd* src, float4* dst, long n, cudaStream_t s);
cudaError_t launch_rhs(sgf_ctx* c, zd* out);
// The same builders at given node positions and into given buffers (gradient). dmode 0 builds the
// factors; 1 / 2 their derivatives with respect to each node's own f / f' (for the near operator
// 1 / 2 move the target node, 3 / 4 the source node).
cudaError_t launch_build_P_geo(sgf_ctx* c, const zd* pinv_eq, const double* d_coll_rel, const double* f,
                              const double* f1, zd* P, int dmode);
cudaError_t launch_build_I_geo(sgf_ctx* c, const zd* pinv_fb, zd* d_Iplain, const double* d_samp_rel, const double* f,
                              const double* f1, zd* Ip, int dmode);
cudaError_t launch_near_geo(sgf_ctx* c, const zd* d_phi, int dcy_min, int n_dcy, const zd* d_Iplain, const zd* P,
                            const NearPairs& pp, const double* d_kress, const double* ft, const double* f1t,
                            const double* f2t, const double* fs, const double* f1s, zd* C, int dmode);
cudaError_t launch_modes_geo(sgf_ctx* c, const double* d_modes_n, const double* f, const double* f1, zd* MT, zd* MS,
                             int dmode);
cudaError_t launch_rhs_geo(sgf_ctx* c, const double* f, const double* f1, zd* out, int dmode);
// w[i] = weight of mu_i in B_n (mp: the 6 mode parameters of sgf_rayleigh) at node positions f, f1
cudaError_t launch_rayleigh_weights(sgf_ctx* c, const double* d_mp, const double* f, const double* f1, zd* w,
                                    int dmode);
// gradient helpers: dst = src + eps; y = conj(x); g += s * a .* (u - v)
cudaError_t launch_offset(const double* src, double eps, long n, double* dst, cudaStream_t s);
cudaError_t launch_conj(const zd* x, zd* y, long n, cudaStream_t s);
cudaError_t launch_grad_acc(zd* g, double s, const zd* a, const zd* u, const zd* v, long n, cudaStream_t st);
cudaError_t launch_apply64(sgf_ctx* c, const zd* mu, zd* out);
cudaError_t launch_apply32(sgf_ctx* c, const zd* mu, zd* out);
// the multi-column forward map of the operator in c (its P, near operator and reconstruction rows)
// on the columns `cols`, with column r's spectra at Khat + r kstride; the work space is allocated by
// multi_space (before any stream capture)
template <typename T>
cudaError_t multi_space(sgf_ctx* c, MultiSpace<T>& ms);
template <typename T>
cudaError_t apply_multi_t(sgf_ctx* c, OpData<T>& od, MultiSpace<T>& ms, const MCols<T>& cols,
                          const cplx<T>* const Khat[2][2], long kstride, cudaStream_t s);
// nrhs densities (columns N apart) in passes of up to MC_MAX columns
cudaError_t launch_apply_nrhs64(sgf_ctx* c, const zd* mu, zd* out, int nrhs);
cudaError_t launch_apply_nrhs32(sgf_ctx* c, const zd* mu, zd* out, int nrhs);
cudaError_t launch_far_grids64(sgf_ctx* c, const zd* mu);
// the dense unaccelerated operator (sgf_exact.cu): entries of d_Aex; y = A x or A^H x
cudaError_t launch_exact_entries(sgf_ctx* c, zd hk);
cudaError_t launch_exact_gemv(sgf_ctx* c, const zd* x, zd* y, bool adjoint);
// sum_{m=1..j} (-1)^m C(j,m) (ik/4) H1(k m h): the shifted images' part of the K_r diagonal
cudaError_t near_hk(sgf_ctx* c, zd* hk);  // phi^all on the grids only (field evaluation)
cudaError_t launch_apply_adj64(sgf_ctx* c, const zd* v, zd* out);
cudaError_t launch_apply_adj32(sgf_ctx* c, const zd* v, zd* out);
cudaError_t launch_conj_transpose(const zd* src, long R, long Cc, zd* dst, cudaStream_t s);
cudaError_t launch_near_transpose(int nblk, const int* bq, const int* br, const long* src_off, const int* src_ld,
                                  const long* dst_off, const int* dst_ld, const int* cell_start, const zd* C, zd* CT,
                                  cudaStream_t s);
cudaError_t build_apply_graph(sgf_ctx* c, int prec);
cudaError_t build_apply_graph_mask(sgf_ctx* c, int prec, int term_mask, GraphSlot& gs);
cudaError_t launch_apply_graph(sgf_ctx* c, int prec, const zd* mu, zd* out);
void destroy_graphs(sgf_ctx* c);
cudaError_t launch_rayleigh_mp(sgf_ctx* c, const zd* mu, int nmodes, const double* d_mp, zd* d_B);
cudaError_t launch_twiddles(sgf_ctx* c);
// which Y-convolution kernel serves this orientation: 1 registers, 2 global scratch, 0 none fits
int conv_y_variant_of(const Orient& o, int precision, bool adjoint = false);
// whether the forced variants fit the launch limits (threads, shared memory, registers) of this
// orientation in this precision, forward and adjoint (0 = not forced)
bool debug_variants_fit(const Orient& o, int precision, int conv_variant, int fftx_vpt);
cudaError_t launch_debug_table(sgf_ctx* c, int lam, int kind, zd* out);
// Krylov helpers
cudaError_t launch_dots(const zd* V, int m, long ldv, const zd* w, long n, zd* partial, int nblk, zd* out,
                        cudaStream_t s);
cudaError_t launch_axpby(zd* y, zd a, const zd* x, zd b, long n, cudaStream_t s);  // y = a x + b y
// Arnoldi step in float-float arithmetic on FP64 vectors: h = V^H w over m basis vectors (part: at
// least kdots_chunks(n) * m float4 partials; Hc, when given, stores or accumulates h; ticket: at least
// kdots_groups(m) counters, zero on entry and on return); w -= V h (with npart, kupdate_blocks(n)
// float4 partials of |w|^2 are written too); w /= |w| with hsub = |w|.
cudaError_t launch_kdots(const zd* V, int m, long ldv, const zd* w, long n, float4* part, zd* h, zd* Hc, int add,
                         unsigned* ticket, cudaStream_t s);
int kdots_groups(int m);
int kdots_chunks(long n);  // blocks of k_kdots along a vector of n elements
// One problem's state for the batched Arnoldi step: basis [C | V] (mr recycled vectors, then the
// Krylov vectors, n apart), Hessenberg storage (column j at H + j ldh: mr coefficients against C,
// then the column), coefficient scratch h, float-float partials (part: kdots_chunks(n_max) per basis
// vector; npart: kupdate_blocks(n_max)), k_kdots tickets (kdots_groups(mr + m + 1), zero).
struct KStep {
  zd* W;
  zd* H;
  zd* h;
  float4* part;
  float4* npart;
  unsigned* ticket;
  long n, ldh;
  int mr, pad_;
};
// Step j of every problem of the table (device array of nprob entries): CGS2 against
// [C | V_0..V_j], the norm and the normalisation of V_{j+1}; n_max the largest n, mr_max the
// largest mr.
cudaError_t launch_batch_arnoldi_step(const KStep* d_tab, int nprob, int j, int mr_max, long n_max, cudaStream_t s);

cudaError_t launch_kupdate(zd* w, const zd* V, int m, long ldv, const zd* h, long n, float4* npart, cudaStream_t s);
cudaError_t launch_kscale(zd* w, long n, const float4* npart, int nparts, zd* hsub, cudaStream_t s);
int kupdate_blocks(long n);

// Host mode helpers shared by the Rayleigh entry points, the mode completion and the gradient.
// beta_n = sqrt(k^2 - alpha_n^2) with the branch i sqrt(alpha_n^2 - k^2) for evanescent modes
// (Section 2, eq. alpha_beta_def).
inline std::complex<double> beta_host(double k, double an) {
  double q = k * k - an * an;
  return q >= 0 ? std::complex<double>(std::sqrt(q), 0) : std::complex<double>(0, std::sqrt(-q));
}
// Q_j = (1 - e^{i beta h})^j / beta; for |beta h| < 1 in the form (-2i)^j e^{i j beta h/2}
// sin^{j-1}(beta h/2) (h/2) sinc(beta h/2) that is exact at beta = 0 (eq. betan_taylor). Beyond, the
// quotient is well conditioned, while the rewrite's factors (growing like sinh(|beta| h/2) for
// evanescent modes) would overflow before the decaying e^{i j beta h/2} cancels them.
inline std::complex<double> Qj_host(std::complex<double> beta, double h, int j) {
  typedef std::complex<double> c;
  if (j == 0) return 1.0 / beta;
  if (std::abs(beta * h) >= 1.0) {
    c q = 1.0 - std::exp(c(0, 1) * (beta * h)), acc = 1.0;
    for (int m = 0; m < j; ++m) acc *= q;
    return acc / beta;
  }
  c half = 0.5 * h * beta;
  c sn = std::sin(half);
  c sinc = std::abs(half) < 1e-3 ? 1.0 - half * half / 6.0 + std::pow(half, 4) / 120.0 : std::sin(half) / half;
  c acc = 0.5 * h * sinc;
  for (int m = 1; m < j; ++m) acc *= sn;
  return std::pow(c(0, -2), j) * std::exp(c(0, 1) * (double)j * half) * acc;
}
