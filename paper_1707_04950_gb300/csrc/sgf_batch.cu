// Batches of independent problems (surfaces, wavenumbers, incidence angles): every problem keeps
// its own context (operator data, captured forward map), and the batch launches all of their
// forward maps as independent branches of ONE CUDA graph, so that problems too small to fill the
// GPU alone run side by side. sgf_batch_solve runs restarted GMRES (Algorithm 1) on all problems
// in lockstep: one graph launch applies every problem's operator, and each Gram-Schmidt pass,
// update and norm is one launch over all problems (grid dimension = problem), with one host
// synchronisation per pass for the whole batch instead of one per problem.
#include <complex>
#include <cmath>
#include <cstring>
#include <memory>

#include "sgf_internal.h"

typedef std::complex<double> cd;

struct sgf_batch {
  int n = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<sgf_ctx*> ctx;
  std::vector<long> N;
  long maxN = 0;
  bool any_mixed = false;
  cudaGraph_t graph[2] = {nullptr, nullptr};      // [0] each context's own precision, [1] FP64
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  long* d_N = nullptr;
  zd** d_in = nullptr;    // contexts' staging inputs (read by their captured forward maps)
  zd** d_out = nullptr;   // contexts' staging outputs
  zd** d_ta = nullptr;    // per-call pointer tables
  zd** d_tb = nullptr;
  zd** h_tab = nullptr;   // pinned host staging of the per-call tables (2 n entries)
  cudaEvent_t ev_tab = nullptr;
  bool shared_near = false;  // problems differ only in the incidence angle: one shared near pass
  zd* d_ph = nullptr;        // [problem][period copy -1, 0, 1] phase relative to the first problem
  // multi-column form (problems differ only in the incidence angle): the first problem's P, near
  // operator and reconstruction rows serve every problem, MC_MAX problems per pass, with each
  // problem's spectra (copied side by side), twists and mode factors
  bool multi = false;
  std::vector<MultiSpace<double>> ms64;
  std::vector<MultiSpace<float>> ms32;
  cplx<double>* K64[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cplx<float>* K32[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  std::vector<void*> allocs;
  char err[1024] = {0};
};

static sgf_status berr(sgf_batch* b, sgf_status st, const char* fmt, ...) {
  if (b) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(b->err, sizeof(b->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

#define BCU(call)                                                                                          \
  do {                                                                                                     \
    cudaError_t e__ = (call);                                                                              \
    if (e__ != cudaSuccess) return berr(B, SGF_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,            \
                                        cudaGetErrorString(e__));                                          \
  } while (0)
#define BTRY(x)                        \
  do {                                 \
    sgf_status st__ = (x);             \
    if (st__ != SGF_OK) return st__;   \
  } while (0)

template <typename T>
static sgf_status balloc(sgf_batch* B, T** p, size_t count) {
  *p = nullptr;
  cudaError_t e = cudaMalloc((void**)p, (count ? count : 1) * sizeof(T));
  if (e != cudaSuccess) return berr(B, SGF_ECUDA, "cudaMalloc of %zu bytes: %s", count * sizeof(T), cudaGetErrorString(e));
  B->allocs.push_back((void*)*p);
  return SGF_OK;
}

// ------------------------------------------------------------------ batched vector kernels
// A "table" holds one base pointer per problem; vector k of problem p starts at tab[p] + k N_p.
// Grids are (chunks of the longest vector, problems).
__global__ void k_bcopy(zd* const* __restrict__ dt, int dk, zd* const* __restrict__ st, int sk,
                        const long* __restrict__ N) {
  const int p = blockIdx.y;
  const long n = N[p];
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dt[p][dk * n + i] = st[p][sk * n + i];
}
// y_p = b_p - y_p
__global__ void k_brsub(zd* const* __restrict__ yt, int yk, zd* const* __restrict__ bt, const long* __restrict__ N) {
  const int p = blockIdx.y;
  const long n = N[p];
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    zd* y = yt[p] + yk * n;
    y[i] = bt[p][i] - y[i];
  }
}
// y_p = s_p y_p (s_p real; s_p = 0 clears the vector of a problem that has stopped, so that it
// carries zeros, not growing rounding noise, through the remaining lockstep steps)
__global__ void k_bscale(zd* const* __restrict__ yt, int yk, const double* __restrict__ s, const long* __restrict__ N) {
  const int p = blockIdx.y;
  const long n = N[p];
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    zd* y = yt[p] + yk * n;
    y[i] = s[p] * y[i];
  }
}
// y_p += x_p
__global__ void k_badd(zd* const* __restrict__ yt, zd* const* __restrict__ xt, const long* __restrict__ N) {
  const int p = blockIdx.y;
  const long n = N[p];
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) yt[p][i] += xt[p][i];
}
// h[p][j] = sum_i conj(V_p[j0 + j][i]) w_p[i], j < m: block per (j, p)
__global__ void k_bdots(zd* const* __restrict__ Vt, int j0, int m, zd* const* __restrict__ wt, int wk,
                        const long* __restrict__ N, zd* __restrict__ h) {
  SGF_SHARED_ARRAY(zd, red, 32);
  const int j = blockIdx.x, p = blockIdx.y;
  const long n = N[p];
  const zd* v = Vt[p] + (j0 + j) * n;
  const zd* w = wt[p] + wk * n;
  zd acc(0, 0);
  for (long i = threadIdx.x; i < n; i += blockDim.x) acc += mulc(w[i], v[i]);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  acc = warp_sum(acc);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (warp == 0) {
    zd s = lane < nw ? red[lane] : zd(0, 0);
    s = warp_sum(s);
    if (lane == 0) h[(long)p * m + j] = s;
  }
}
// w_p -= sum_{j<m} V_p[j] h[p][j]
__global__ void k_bupdate(zd* const* __restrict__ wt, int wk, zd* const* __restrict__ Vt, int m,
                          const zd* __restrict__ h, const long* __restrict__ N) {
  const int p = blockIdx.y;
  const long n = N[p];
  long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  zd* w = wt[p] + wk * n;
  const zd* V = Vt[p];
  zd acc = w[i];
  for (int j = 0; j < m; ++j) {
    const zd hj = h[(long)p * m + j];
    if (hj.re != 0.0 || hj.im != 0.0) acc -= V[j * n + i] * hj;
  }
  w[i] = acc;
}

static bool same_params(const sgf_params& a, const sgf_params& b) {
  return a.N == b.N && a.j == b.j && a.h == b.h && a.n_per == b.n_per && a.c_win == b.c_win && a.Ma == b.Ma &&
         a.eta == b.eta && a.nx == b.nx && a.ny == b.ny && a.hmin == b.hmin && a.p == b.p && a.e == b.e &&
         a.n_coll == b.n_coll && a.n_fb == b.n_fb && a.delta_min == b.delta_min && a.spec_exp == b.spec_exp &&
         a.precision == b.precision && a.ls_reg == b.ls_reg;
}

// ------------------------------------------------------------------ angle-shared near field
// Problems that differ only in the incidence angle share every near-operator block up to the
// quasi-periodic phase of the block's period copy: C(alpha) = e^{i alpha d w} C_base for a block
// whose source cell is copy w in {-1, 0, 1}. One pass over the first problem's blocks therefore
// serves all of them: out_a[i] += sum_c C_0[i][c] e^{i (alpha_a - alpha_0) d w(c)} mu_a[col c].
// Block per work item of the shared layout; angles in groups of G whose phased densities are staged
// in shared memory; each warp streams a row once per group and keeps G accumulators.
template <bool FF>
__global__ void k_near_multi(int n_ang, const zd* __restrict__ ph, const int* __restrict__ cell_start,
                             const int* __restrict__ node_idx, const int* __restrict__ cols,
                             const int* __restrict__ coloff, const signed char* __restrict__ colwrap,
                             const long* __restrict__ cell_off, const int* __restrict__ cell_W,
                             const zd* __restrict__ C, const float4* __restrict__ Cff, const int* __restrict__ item_cell,
                             const int* __restrict__ item_lo, const int* __restrict__ item_hi, zd* const* __restrict__ mus,
                             zd* const* __restrict__ outs) {
  constexpr int G = 8;
  extern __shared__ unsigned char smem_raw[];
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32, nw = blockDim.x / 32;
  const int q = item_cell[blockIdx.x];
  const int rlo = item_lo[blockIdx.x];
  const int s0 = cell_start[q] + rlo, nq = item_hi[blockIdx.x] - rlo;
  const int W = cell_W[q];
  const int* cq = cols + coloff[q];
  const signed char* wq = colwrap + coloff[q];
  zd* vd = reinterpret_cast<zd*>(smem_raw);          // [G][W]
  float4* vf = reinterpret_cast<float4*>(smem_raw);  // [G][W]
  for (int a0 = 0; a0 < n_ang; a0 += G) {
    const int na = min(G, n_ang - a0);
    for (int t = threadIdx.x; t < na * W; t += blockDim.x) {
      const int a = t / W, cc = t - a * W;
      const zd v = ph[(long)(a0 + a) * 3 + wq[cc] + 1] * mus[a0 + a][cq[cc]];
      if (FF)
        vf[t] = cff_from(v);
      else
        vd[t] = v;
    }
    __syncthreads();
    for (int il = warp; il < nq; il += nw) {
      const long row = cell_off[q] + (long)(rlo + il) * W;
      if (FF) {
        dot2c acc[G];
#pragma unroll
        for (int a = 0; a < G; ++a) acc[a] = {0.f, 0.f, 0.f, 0.f};
        for (int cc = lane; cc < W; cc += 32) {
          const float4 cv = Cff[row + cc];
#pragma unroll
          for (int a = 0; a < G; ++a)
            if (a < na) dot2_mac(cv, vf[a * W + cc], acc[a]);
        }
#pragma unroll
        for (int a = 0; a < G; ++a) {
          if (a >= na) break;
          for (int o = 16; o > 0; o >>= 1) {
            dot2c t = {__shfl_down_sync(0xffffffffu, acc[a].sr, o), __shfl_down_sync(0xffffffffu, acc[a].si, o),
                       __shfl_down_sync(0xffffffffu, acc[a].er, o), __shfl_down_sync(0xffffffffu, acc[a].ei, o)};
            dot2_merge(acc[a], t);
          }
          if (lane == 0) {
            ff vr = ff_add({acc[a].sr, 0.f}, {acc[a].er, 0.f}), vi = ff_add({acc[a].si, 0.f}, {acc[a].ei, 0.f});
            zd* o = outs[a0 + a] + node_idx[s0 + il];
            *o = *o + zd(ff_to_double(vr), ff_to_double(vi));
          }
        }
      } else {
        zd acc[G];
#pragma unroll
        for (int a = 0; a < G; ++a) acc[a] = zd(0, 0);
        for (int cc = lane; cc < W; cc += 32) {
          const zd cv = C[row + cc];
#pragma unroll
          for (int a = 0; a < G; ++a)
            if (a < na) acc[a] = fma_c(cv, vd[a * W + cc], acc[a]);
        }
#pragma unroll
        for (int a = 0; a < G; ++a) {
          if (a >= na) break;
          const zd v = warp_sum(acc[a]);
          if (lane == 0) {
            zd* o = outs[a0 + a] + node_idx[s0 + il];
            *o = *o + v;
          }
        }
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ batched forward map
static dim3 bgrid(const sgf_batch* B) { return dim3(ceil_div(B->maxN, 256), B->n); }

// dst[dk] = A src[sk] for every problem with the operators of graph slot `slot`.
static sgf_status bapply(sgf_batch* B, int slot, zd** st, int sk, zd** dt, int dk) {
  k_bcopy<<<bgrid(B), 256, 0, B->stream>>>(B->d_in, 0, st, sk, B->d_N);
  BCU(cudaGetLastError());
  BCU(cudaGraphLaunch(B->exec[slot], B->stream));
  k_bcopy<<<bgrid(B), 256, 0, B->stream>>>(dt, dk, B->d_out, 0, B->d_N);
  BCU(cudaGetLastError());
  return SGF_OK;
}

// Writes two host pointer arrays into the device tables d_ta / d_tb (through pinned staging).
static sgf_status set_tables(sgf_batch* B, const void* const* a, const void* const* b) {
  BCU(cudaEventSynchronize(B->ev_tab));  // the previous upload has left the staging buffer
  for (int p = 0; p < B->n; ++p) {
    B->h_tab[p] = (zd*)a[p];
    B->h_tab[B->n + p] = b ? (zd*)b[p] : nullptr;
  }
  BCU(cudaMemcpyAsync(B->d_ta, B->h_tab, B->n * sizeof(zd*), cudaMemcpyHostToDevice, B->stream));
  BCU(cudaMemcpyAsync(B->d_tb, B->h_tab + B->n, B->n * sizeof(zd*), cudaMemcpyHostToDevice, B->stream));
  BCU(cudaEventRecord(B->ev_tab, B->stream));
  return SGF_OK;
}

template <typename T>
static void free_ms(std::vector<MultiSpace<T>>& v) {
  for (auto& ms : v) {
    for (int l = 0; l < 2; ++l) {
      if (ms.grid[l]) cudaFree(ms.grid[l]);
      if (ms.accg[l]) cudaFree(ms.accg[l]);
    }
    if (ms.mpart) cudaFree(ms.mpart);
    if (ms.mpart_ff) cudaFree(ms.mpart_ff);
  }
  v.clear();
}

static void free_batch(sgf_batch* B) {
  for (int s = 0; s < 2; ++s) {
    if (B->exec[s]) cudaGraphExecDestroy(B->exec[s]);
    if (B->graph[s]) cudaGraphDestroy(B->graph[s]);
  }
  free_ms(B->ms64);
  free_ms(B->ms32);
  for (void* p : B->allocs) cudaFree(p);
  if (B->h_tab) cudaFreeHost(B->h_tab);
  if (B->ev_tab) cudaEventDestroy(B->ev_tab);
}

// One graph for graph slot s (0: each problem's own precision, 1: FP64): every problem's captured
// forward map as an independent child graph; with `shared` the children leave out the near operator
// and one angle-shared near-field node follows them.
static sgf_status build_batch_graph(sgf_batch* B, int s, bool shared, cudaGraph_t* gout, cudaGraphExec_t* xout) {
  const int n = B->n;
  sgf_ctx* c0 = B->ctx[0];
  cudaGraph_t graph = nullptr;
  BCU(cudaGraphCreate(&graph, 0));
  std::vector<cudaGraphNode_t> kids(n);
  for (int p = 0; p < n; ++p) {
    sgf_ctx* c = B->ctx[p];
    int gi = (s == 0 && c->prm.precision == 32) ? 1 : 0;
    cudaGraph_t child = c->gs[gi].g;
    if (shared) {
      if (!c->gs_nonear[gi].ok) BCU(build_apply_graph_mask(c, gi == 1 ? 32 : 64, 13, c->gs_nonear[gi]));
      child = c->gs_nonear[gi].g;
    }
    BCU(cudaGraphAddChildGraphNode(&kids[p], graph, nullptr, 0, child));
  }
  if (shared) {
    const bool ff = s == 0 && c0->prm.precision == 32;
    const void* fn = ff ? (const void*)k_near_multi<true> : (const void*)k_near_multi<false>;
    const size_t sm = (size_t)8 * c0->maxW * sizeof(zd);
    BCU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    int na = n;
    void* args[] = {&na, &B->d_ph, &c0->d_cell_start, &c0->d_node_idx, &c0->d_cols, &c0->d_coloff, &c0->d_colwrap,
                    &c0->d_cell_off, &c0->d_cell_W, &c0->d_C, &c0->d_Cff, &c0->d_item_cell, &c0->d_item_lo,
                    &c0->d_item_hi, &B->d_in, &B->d_out};
    cudaKernelNodeParams kp{};
    kp.func = (void*)fn;
    kp.gridDim = dim3(c0->n_items);
    kp.blockDim = dim3(256);
    kp.sharedMemBytes = (unsigned)sm;
    kp.kernelParams = args;
    kp.extra = nullptr;
    cudaGraphNode_t nd;
    BCU(cudaGraphAddKernelNode(&nd, graph, kids.data(), n, &kp));
  }
  BCU(cudaGraphInstantiate(xout, graph, cudaGraphInstantiateFlagUseNodePriority));
  *gout = graph;
  return SGF_OK;
}

// The multi-column form of graph slot s (0: the problems' own precision, 1: FP64), captured once:
// each pass of MC_MAX problems runs the first context's multi-column forward map on the problems'
// staging buffers, the passes on forked streams of their own (each with its own work space).
template <typename T>
static sgf_status build_multi_graph(sgf_batch* B, std::vector<MultiSpace<T>>& msv, cplx<T>* (&K)[2][2],
                                    cudaGraph_t* gout, cudaGraphExec_t* xout) {
  const int n = B->n;
  sgf_ctx* c0 = B->ctx[0];
  constexpr bool F64 = sizeof(T) == 8;
  const int npass = (n + MC_MAX - 1) / MC_MAX;
  // spectra of every problem side by side (column r of a pass at K + r kstride)
  const long kst[2] = {(long)c0->og[0].Px * c0->og[0].Py, (long)c0->og[1].Px * c0->og[1].Py};
  for (int lam = 0; lam < 2; ++lam)
    for (int kd = 0; kd < 2; ++kd) {
      if (!K[lam][kd]) BTRY(balloc(B, &K[lam][kd], (size_t)n * kst[lam]));
      for (int p = 0; p < n; ++p) {
        const OpData<T>& od = *reinterpret_cast<const OpData<T>*>(F64 ? (const void*)&B->ctx[p]->o64
                                                                       : (const void*)&B->ctx[p]->o32);
        BCU(cudaMemcpyAsync(K[lam][kd] + (size_t)p * kst[lam], od.Khat[lam][kd], kst[lam] * sizeof(cplx<T>),
                            cudaMemcpyDeviceToDevice, B->stream));
      }
    }
  msv.resize(npass);
  for (auto& ms : msv) BCU(multi_space<T>(c0, ms));
  BCU(cudaStreamSynchronize(B->stream));
  std::vector<cudaStream_t> st(npass, nullptr);
  std::vector<cudaEvent_t> ev(npass + 1, nullptr);
  cudaStream_t cap = nullptr;
  BCU(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  for (auto& x : st) BCU(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
  for (auto& x : ev) BCU(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaEventRecord(ev[npass], cap);
    OpData<T>& od0 = *reinterpret_cast<OpData<T>*>(F64 ? (void*)&c0->o64 : (void*)&c0->o32);
    for (int ps = 0; ps < npass && e == cudaSuccess; ++ps) {
      cudaStreamWaitEvent(st[ps], ev[npass], 0);
      MCols<T> cols;
      const int p0 = ps * MC_MAX;
      cols.n = std::min(MC_MAX, n - p0);
      for (int r = 0; r < cols.n; ++r) {
        sgf_ctx* c = B->ctx[p0 + r];
        const OpData<T>& od = *reinterpret_cast<const OpData<T>*>(F64 ? (const void*)&c->o64 : (const void*)&c->o32);
        MCol<T>& cr = cols.c[r];
        cr.mu = c->d_mu_tmp;
        cr.out = c->d_out_tmp;
        cr.src_tw = od.src_tw;
        cr.dalpha = c->alpha - c0->alpha;
        cr.MT = c->d_MT;
        cr.MS = c->d_MS;
        cr.MTff = c->d_MTff;
        cr.MSff = c->d_MSff;
        cr.nm = c->nm;
      }
      // this pass's spectra: orientation lam's at K[lam] + p0 kst[lam], then kst[lam] apart (stride -1)
      const cplx<T>* Kp[2][2];
      for (int lam = 0; lam < 2; ++lam)
        for (int kd = 0; kd < 2; ++kd) Kp[lam][kd] = K[lam][kd] + (size_t)p0 * kst[lam];
      e = apply_multi_t<T>(c0, od0, msv[ps], cols, Kp, -1, st[ps]);
      if (e == cudaSuccess) e = cudaEventRecord(ev[ps], st[ps]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, ev[ps], 0);
    }
    cudaError_t ee = cudaStreamEndCapture(cap, &g);
    if (e == cudaSuccess) e = ee;
  }
  for (auto& x : st) cudaStreamDestroy(x);
  for (auto& x : ev) cudaEventDestroy(x);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return berr(B, SGF_ECUDA, "capture of the multi-column batch: %s", cudaGetErrorString(e));
  }
  BCU(cudaGraphInstantiate(xout, g, 0));
  *gout = g;
  return SGF_OK;
}

// Mean time of one launch of x (3 warm-up, 10 timed launches on the batch stream).
static sgf_status time_exec(sgf_batch* B, cudaGraphExec_t x, double* ms) {
  cudaEvent_t e0, e1;
  BCU(cudaEventCreate(&e0));
  BCU(cudaEventCreate(&e1));
  for (int r = 0; r < 3; ++r) BCU(cudaGraphLaunch(x, B->stream));
  BCU(cudaEventRecord(e0, B->stream));
  for (int r = 0; r < 10; ++r) BCU(cudaGraphLaunch(x, B->stream));
  BCU(cudaEventRecord(e1, B->stream));
  BCU(cudaEventSynchronize(e1));
  float t = 0;
  BCU(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / 10;
  return SGF_OK;
}

extern "C" {

sgf_status sgf_batch_create(sgf_batch** out, int n, sgf_ctx* const* ctxs, void* cuda_stream) {
  if (!out) return SGF_EINVAL;
  *out = nullptr;
  sgf_batch* B = new sgf_batch();
  *out = B;
  if (n < 1 || !ctxs) return berr(B, SGF_EINVAL, "empty batch");
  B->n = n;
  B->stream = (cudaStream_t)cuda_stream;
  B->device = ctxs[0] ? ctxs[0]->device : 0;
  for (int p = 0; p < n; ++p) {
    sgf_ctx* c = ctxs[p];
    if (!c || !c->built) return berr(B, SGF_ESTATE, "context %d is not built", p);
    if (c->op_exact) return berr(B, SGF_EINVAL, "context %d has the dense operator selected", p);
    if (c->device != B->device) return berr(B, SGF_EINVAL, "context %d is on another device", p);
    bool mixed = c->prm.precision == 32;
    if (!c->use_graphs || !c->gs[0].ok || (mixed && !c->gs[1].ok))
      return berr(B, SGF_ESTATE, "context %d has no captured forward map", p);
    for (int q = 0; q < p; ++q)
      if (ctxs[q] == c) return berr(B, SGF_EINVAL, "context %d appears twice", p);
    B->ctx.push_back(c);
    B->N.push_back(c->N);
    B->maxN = std::max(B->maxN, (long)c->N);
    B->any_mixed = B->any_mixed || mixed;
  }
  BCU(cudaSetDevice(B->device));
  BCU(cudaEventCreateWithFlags(&B->ev_tab, cudaEventDisableTiming));
  BCU(cudaEventRecord(B->ev_tab, B->stream));
  BCU(cudaMallocHost((void**)&B->h_tab, 2 * n * sizeof(zd*)));
  BTRY(balloc(B, &B->d_N, n));
  BTRY(balloc(B, &B->d_in, n));
  BTRY(balloc(B, &B->d_out, n));
  BTRY(balloc(B, &B->d_ta, n));
  BTRY(balloc(B, &B->d_tb, n));
  std::vector<zd*> in(n), outp(n);
  for (int p = 0; p < n; ++p) {
    in[p] = B->ctx[p]->d_mu_tmp;
    outp[p] = B->ctx[p]->d_out_tmp;
  }
  BCU(cudaMemcpy(B->d_N, B->N.data(), n * sizeof(long), cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(B->d_in, in.data(), n * sizeof(zd*), cudaMemcpyHostToDevice));
  BCU(cudaMemcpy(B->d_out, outp.data(), n * sizeof(zd*), cudaMemcpyHostToDevice));
  // angle sharing: every problem on the same surface, wavenumber, boundary condition and
  // parameters (only the incidence angle differs) shares the first problem's near operator
  sgf_ctx* c0 = B->ctx[0];
  B->shared_near = n > 1 && (size_t)8 * c0->maxW * sizeof(zd) <= 200 * 1024;
  for (int p = 1; p < n && B->shared_near; ++p) {
    const sgf_ctx* c = B->ctx[p];
    B->shared_near = c->N == c0->N && c->d == c0->d && c->k == c0->k && c->bc == c0->bc && c->fa == c0->fa &&
                     c->fb == c0->fb && same_params(c->prm, c0->prm) && c->nnz == c0->nnz &&
                     c->n_items == c0->n_items && c->maxW == c0->maxW;
  }
  if (B->shared_near) {
    std::vector<zd> ph((size_t)3 * n);
    for (int p = 0; p < n; ++p) {
      const double dl = (B->ctx[p]->alpha - c0->alpha) * c0->d;
      for (int w = -1; w <= 1; ++w) ph[(size_t)p * 3 + w + 1] = zd(std::cos(dl * w), std::sin(dl * w));
    }
    BTRY(balloc(B, &B->d_ph, ph.size()));
    BCU(cudaMemcpy(B->d_ph, ph.data(), ph.size() * sizeof(zd), cudaMemcpyHostToDevice));
  }
  // Angle sharing removes the repeated near operators but puts one near-field node after every
  // problem's far-field work, so it pays only when the near operators dominate: the two forms are
  // timed at creation and the faster is kept (SGF_BATCH_SHARED=0 / 1 forces one form).
  if (B->shared_near) {
    const char* env = getenv("SGF_BATCH_SHARED");
    if (env && env[0] == '0') B->shared_near = false;
    if (!(env && (env[0] == '0' || env[0] == '1'))) {
      cudaGraph_t gsh = nullptr, gpl = nullptr;
      cudaGraphExec_t xsh = nullptr, xpl = nullptr;
      for (int p = 0; p < n; ++p)  // defined staging inputs for the timed launches
        BCU(cudaMemsetAsync(B->ctx[p]->d_mu_tmp, 0, B->N[p] * sizeof(zd), B->stream));
      BTRY(build_batch_graph(B, 0, true, &gsh, &xsh));
      BTRY(build_batch_graph(B, 0, false, &gpl, &xpl));
      double tsh = 0, tpl = 0;
      BTRY(time_exec(B, xsh, &tsh));
      BTRY(time_exec(B, xpl, &tpl));
      B->shared_near = tsh < tpl;
      cudaGraphExecDestroy(xsh);
      cudaGraphExecDestroy(xpl);
      cudaGraphDestroy(gsh);
      cudaGraphDestroy(gpl);
    }
  }
  // multi-column form: every problem on the same surface (as for the shared near pass) and in one
  // precision; timed against the child-graph form at creation and kept if faster
  // (SGF_BATCH_MULTI=0 / 1 forces the choice)
  bool same_surface = n > 1;
  for (int p = 1; p < n && same_surface; ++p) {
    const sgf_ctx* c = B->ctx[p];
    same_surface = c->N == c0->N && c->d == c0->d && c->k == c0->k && c->bc == c0->bc && c->fa == c0->fa &&
                   c->fb == c0->fb && same_params(c->prm, c0->prm) && c->nnz == c0->nnz &&
                   c->n_items == c0->n_items && c->maxW == c0->maxW;
  }
  const bool multi_fits = (size_t)MC_MAX * (c0->maxW + 32) * 16 <= 200 * 1024;
  const char* envm = getenv("SGF_BATCH_MULTI");
  if (same_surface && multi_fits && !(envm && envm[0] == '0')) {
    cudaGraph_t gm = nullptr;
    cudaGraphExec_t xm = nullptr;
    if (c0->prm.precision == 32)
      BTRY(build_multi_graph<float>(B, B->ms32, B->K32, &gm, &xm));
    else
      BTRY(build_multi_graph<double>(B, B->ms64, B->K64, &gm, &xm));
    bool keep = envm && envm[0] == '1';
    if (!keep) {
      cudaGraph_t go = nullptr;
      cudaGraphExec_t xo = nullptr;
      for (int p = 0; p < n; ++p)
        BCU(cudaMemsetAsync(B->ctx[p]->d_mu_tmp, 0, B->N[p] * sizeof(zd), B->stream));
      BTRY(build_batch_graph(B, 0, B->shared_near, &go, &xo));
      double tm = 0, to = 0;
      BTRY(time_exec(B, xm, &tm));
      BTRY(time_exec(B, xo, &to));
      keep = tm < to;
      cudaGraphExecDestroy(xo);
      cudaGraphDestroy(go);
    }
    if (keep) {
      B->multi = true;
      B->graph[0] = gm;
      B->exec[0] = xm;
    } else {
      cudaGraphExecDestroy(xm);
      cudaGraphDestroy(gm);
    }
  }
  for (int s = 0; s < 2; ++s) {
    if (s == 1 && !B->any_mixed) break;
    if (s == 0 && B->multi) continue;
    if (s == 1 && B->multi) {  // the FP64 slot of a mixed batch: the multi-column FP64 map
      BTRY(build_multi_graph<double>(B, B->ms64, B->K64, &B->graph[1], &B->exec[1]));
      continue;
    }
    BTRY(build_batch_graph(B, s, B->shared_near, &B->graph[s], &B->exec[s]));
  }
  if (!B->any_mixed) B->exec[1] = nullptr;
  return SGF_OK;
}

void sgf_batch_destroy(sgf_batch* B) {
  if (!B) return;
  if (B->n > 0) {
    cudaSetDevice(B->device);
    cudaStreamSynchronize(B->stream);
  }
  free_batch(B);
  delete B;
}

const char* sgf_batch_last_error(const sgf_batch* B) { return B ? B->err : "null batch"; }

int sgf_batch_shared_near(const sgf_batch* B) { return B ? (B->multi ? 2 : (B->shared_near ? 1 : 0)) : 0; }

sgf_status sgf_batch_apply(sgf_batch* B, const void* const* mu_devs, void* const* out_devs) {
  if (!B) return SGF_EINVAL;
  if (!B->exec[0]) return berr(B, SGF_ESTATE, "batch was not created");
  if (!mu_devs || !out_devs) return berr(B, SGF_EINVAL, "null pointer arrays");
  for (int p = 0; p < B->n; ++p)
    if (!mu_devs[p] || !out_devs[p]) return berr(B, SGF_EINVAL, "null buffer for problem %d", p);
  BTRY(set_tables(B, (const void* const*)mu_devs, (const void* const*)out_devs));
  return bapply(B, 0, B->d_ta, 0, B->d_tb, 0);
}

}  // extern "C"

// ------------------------------------------------------------------ lockstep GMRES
struct BWork {
  int m = 0;
  int mrec = 0;         // recycled-vector slots in front of every problem's basis
  int rec_m = 0;        // columns of the recycled space in use (common to the batch; 0: none)
  zd** d_V = nullptr;   // [p] Krylov basis, (m + 1) vectors of N_p, after mrec recycled slots
  zd** d_C = nullptr;   // [p] the recycled space C_p = V_p - rec_m N_p
  zd** d_Vold = nullptr;  // [p] V_m of the solve the recycled space came from
  zd** d_r = nullptr;   // [p] residual / work vector
  zd* d_h = nullptr;    // [p][mrec + m + 2] coefficients of the FP64 helpers
  double* d_s = nullptr;
  KStep* d_ks = nullptr;  // [p] state of the float-float Arnoldi step
  std::vector<KStep> ks;
  std::vector<zd*> V, Vold;
  std::vector<std::vector<cd>> R;  // [p] rec_m x rec_m upper triangles (column-major)
};

// h_out[p][j] = V_p[j0 + j]^H w_p (j < m), synchronised to the host.
static sgf_status bdots(sgf_batch* B, BWork& W, zd** Vt, int m, zd** wt, int wk, std::vector<cd>& h_out, int j0 = 0) {
  k_bdots<<<dim3(m, B->n), 256, 0, B->stream>>>(Vt, j0, m, wt, wk, B->d_N, W.d_h);
  BCU(cudaGetLastError());
  h_out.resize((size_t)B->n * m);
  BCU(cudaMemcpyAsync(h_out.data(), W.d_h, h_out.size() * sizeof(zd), cudaMemcpyDeviceToHost, B->stream));
  BCU(cudaStreamSynchronize(B->stream));
  return SGF_OK;
}

static sgf_status bscale(sgf_batch* B, BWork& W, zd** t, int k, const std::vector<double>& s) {
  BCU(cudaMemcpyAsync(W.d_s, s.data(), B->n * sizeof(double), cudaMemcpyHostToDevice, B->stream));
  k_bscale<<<bgrid(B), 256, 0, B->stream>>>(t, k, W.d_s, B->d_N);
  BCU(cudaGetLastError());
  return SGF_OK;
}

// w_p[wk] -= V_p[0..m) h[p][.] with host coefficients (m entries per problem)
static sgf_status bupdate(sgf_batch* B, BWork& W, zd** wt, int wk, zd** Vt, int m, const std::vector<cd>& h) {
  BCU(cudaMemcpyAsync(W.d_h, h.data(), (size_t)B->n * m * sizeof(zd), cudaMemcpyHostToDevice, B->stream));
  k_bupdate<<<bgrid(B), 256, 0, B->stream>>>(wt, wk, Vt, m, W.d_h, B->d_N);
  BCU(cudaGetLastError());
  BCU(cudaStreamSynchronize(B->stream));  // h is host memory of the caller
  return SGF_OK;
}

// z = R^{-1} c for an rm x rm upper triangle (column-major)
static void btri_solve(const std::vector<cd>& R, int rm, const cd* c, cd* z) {
  for (int i = rm - 1; i >= 0; --i) {
    cd acc = c[i];
    for (int k = i + 1; k < rm; ++k) acc -= R[(size_t)k * rm + i] * z[k];
    z[i] = acc / R[(size_t)i * rm + i];
  }
}

// Lockstep restarted GMRES from x = 0 on A_p x_p = b_p for every problem, operators of graph slot
// `slot`, relative tolerance tolv[p]. A problem stops (its iterate freezes) once its residual
// reaches its tolerance: with true_check the true residual at the start of a cycle decides,
// without (inner solves of the refinement) the Arnoldi estimate does. A cycle that reduces the true
// residual by less than 10% also ends the problem (attainable accuracy or stagnation).
// The Arnoldi steps are those of sgf_solve for all problems at once (float-float CGS2 on the
// device, Givens rotations on the host every 8 steps). use_rc: deflate with the recycled spaces
// (GCRO form, as in sgf_solve); harvest: leave this solve's spaces (the leading columns common to
// every problem) for later solves with the same operators.
static sgf_status bgmres(sgf_batch* B, BWork& W, int slot, zd** bt, zd** xt, const std::vector<zd*>& xs,
                         const std::vector<double>& tolv, bool true_check, int maxit, std::vector<int>& its,
                         std::vector<double>& rr, bool use_rc = false, bool harvest = false) {
  const int n = B->n, m = W.m;
  const int mr = use_rc ? W.rec_m : 0;
  std::vector<cd> tmp;
  for (int p = 0; p < n; ++p) BCU(cudaMemsetAsync(xs[p], 0, B->N[p] * sizeof(zd), B->stream));  // x = 0
  BTRY(bdots(B, W, bt, 1, bt, 0, tmp));
  std::vector<double> bn(n), res(n);
  std::vector<char> done(n, 0);
  for (int p = 0; p < n; ++p) {
    bn[p] = std::sqrt(tmp[p].real());
    its[p] = 0;
    if (!std::isfinite(bn[p])) return berr(B, SGF_ENONFINITE, "non-finite right-hand side (problem %d)", p);
    if (bn[p] == 0) done[p] = 1;
  }
  // the step kernels' table: problem p's basis starts at its mr recycled vectors
  const long ldh = (long)W.mrec + m + 1;
  for (int p = 0; p < n; ++p) {
    W.ks[p].W = W.V[p] - (size_t)mr * B->N[p];
    W.ks[p].mr = mr;
    W.ks[p].ldh = ldh;
  }
  BCU(cudaMemcpyAsync(W.d_ks, W.ks.data(), n * sizeof(KStep), cudaMemcpyHostToDevice, B->stream));
  BCU(cudaStreamSynchronize(B->stream));
  constexpr int kCheck = 8;
  std::vector<std::vector<cd>> Hh(n);
  std::vector<cd> cs((size_t)n * m), sn((size_t)n * m), g((size_t)n * (m + 1)), z((size_t)n * std::max(1, mr));
  std::vector<int> jdone(n, 0);
  std::vector<double> sc(n), prev_true(n, 0.0);
  int total = 0, cycles = 0;
  bool first = true;
  while (total < maxit) {
    // r = b - A x (x = 0 on the first cycle: r = b)
    if (first) {
      k_bcopy<<<bgrid(B), 256, 0, B->stream>>>(W.d_r, 0, bt, 0, B->d_N);
      BCU(cudaGetLastError());
    } else {
      BTRY(bapply(B, slot, xt, 0, W.d_r, 0));
      k_brsub<<<bgrid(B), 256, 0, B->stream>>>(W.d_r, 0, bt, B->d_N);
      BCU(cudaGetLastError());
    }
    first = false;
    if (mr > 0) {
      // c = C^H r; r -= C c; x += U c = Vold R^{-1} c
      BTRY(bdots(B, W, W.d_C, mr, W.d_r, 0, tmp));
      std::vector<cd> c(tmp), nz((size_t)n * mr);
      for (int p = 0; p < n; ++p) {
        if (done[p] || tolv[p] >= 1.0)  // nothing to do for this problem: leave its iterate alone
          std::fill(c.begin() + (size_t)p * mr, c.begin() + (size_t)(p + 1) * mr, cd(0));
        btri_solve(W.R[p], mr, c.data() + (size_t)p * mr, nz.data() + (size_t)p * mr);
        for (int i = 0; i < mr; ++i) nz[(size_t)p * mr + i] = -nz[(size_t)p * mr + i];
      }
      BTRY(bupdate(B, W, W.d_r, 0, W.d_C, mr, c));
      BTRY(bupdate(B, W, xt, 0, W.d_Vold, mr, nz));
    }
    BTRY(bdots(B, W, W.d_r, 1, W.d_r, 0, tmp));
    bool any = false;
    for (int p = 0; p < n; ++p) {
      double beta = std::sqrt(tmp[p].real());
      res[p] = beta;
      if (!done[p] && beta / bn[p] <= tolv[p]) done[p] = 1;
      if (!done[p] && cycles > 0 && beta > 0.9 * prev_true[p]) done[p] = 1;  // under 10% progress per cycle
      prev_true[p] = beta;
      sc[p] = done[p] || beta == 0 ? 0.0 : 1.0 / beta;
      for (int i = 0; i <= m; ++i) g[(size_t)p * (m + 1) + i] = 0;
      g[(size_t)p * (m + 1)] = beta;
      jdone[p] = 0;
      any = any || !done[p];
    }
    if (!any) break;
    ++cycles;
    k_bcopy<<<bgrid(B), 256, 0, B->stream>>>(W.d_V, 0, W.d_r, 0, B->d_N);
    BCU(cudaGetLastError());
    BTRY(bscale(B, W, W.d_V, 0, sc));
    std::vector<char> live(n);
    for (int p = 0; p < n; ++p) live[p] = !done[p];
    int j = 0;
    bool any_live = true;
    // group sizes as in sgf_solve: the steps the slowest live problem's last reduction per step
    // predicts to its tolerance (1..kCheck); 2 first when deflating with recycled spaces
    int group = mr > 0 ? 2 : kCheck;
    std::vector<double> res0(n);
    while (any_live && j < m && total < maxit) {
      const int j0 = j, jend = std::min({m, j + group, j + (maxit - total)});
      for (int p = 0; p < n; ++p) res0[p] = res[p];
      for (; j < jend; ++j) {
        BTRY(bapply(B, slot, W.d_V, j, W.d_V, j + 1));
        ++total;
        for (int p = 0; p < n; ++p)
          if (live[p]) ++its[p];
        BCU(launch_batch_arnoldi_step(W.d_ks, n, j, mr, B->maxN, B->stream));
      }
      for (int p = 0; p < n; ++p) {
        if (!live[p]) continue;
        if (Hh[p].size() < (size_t)jend * ldh) Hh[p].resize((size_t)jend * ldh);
        BCU(cudaMemcpy2DAsync(Hh[p].data() + (size_t)j0 * ldh, ldh * sizeof(zd), W.ks[p].H + (size_t)j0 * ldh,
                              ldh * sizeof(zd), (mr + jend + 1) * sizeof(zd), jend - j0, cudaMemcpyDeviceToHost,
                              B->stream));
      }
      BCU(cudaStreamSynchronize(B->stream));
      any_live = false;
      for (int p = 0; p < n; ++p) {
        if (!live[p]) continue;
        cd* csp = &cs[(size_t)p * m];
        cd* snp = &sn[(size_t)p * m];
        cd* gp = &g[(size_t)p * (m + 1)];
        for (int jj = j0; jj < jend && live[p]; ++jj) {
          cd* colB = Hh[p].data() + (size_t)jj * ldh;
          cd* col = colB + mr;
          for (int i = 0; i <= mr + jj + 1; ++i)
            if (!std::isfinite(colB[i].real()) || !std::isfinite(colB[i].imag()))
              return berr(B, SGF_ENONFINITE, "non-finite Krylov vector (problem %d)", p);
          for (int i = 0; i < jj; ++i) {
            const cd a = col[i], bb = col[i + 1];
            col[i] = std::conj(csp[i]) * a + std::conj(snp[i]) * bb;
            col[i + 1] = -snp[i] * a + csp[i] * bb;
          }
          const double hn = col[jj + 1].real();
          const cd a = col[jj];
          const double den = std::sqrt(std::norm(a) + hn * hn);
          csp[jj] = den > 0 ? a / den : cd(1);
          snp[jj] = den > 0 ? cd(hn / den) : cd(0);
          col[jj] = den;
          col[jj + 1] = 0;
          gp[jj + 1] = -snp[jj] * gp[jj];
          gp[jj] = std::conj(csp[jj]) * gp[jj];
          jdone[p] = jj + 1;
          res[p] = std::abs(gp[jj + 1]);
          if (res[p] / bn[p] <= tolv[p] || !(hn > 0)) live[p] = 0;
        }
        any_live = any_live || live[p];
      }
      int need_max = 1;
      for (int p = 0; p < n && need_max < kCheck; ++p) {
        if (!live[p]) continue;
        const double rate = res0[p] > 0 && res[p] > 0 ? std::pow(res[p] / res0[p], 1.0 / (jend - j0)) : 1.0;
        const double need = rate < 1.0 ? std::ceil(std::log(tolv[p] * bn[p] / res[p]) / std::log(rate)) : kCheck;
        need_max = need >= kCheck ? kCheck : std::max(need_max, (int)need);
      }
      group = need_max;
    }
    // x_p += V_p y_p - U_p B_p y_p (back substitution per problem; coefficients zero past jdone_p)
    int mm = 0;
    for (int p = 0; p < n; ++p) mm = std::max(mm, jdone[p]);
    if (mm > 0) {
      std::vector<cd> ny((size_t)n * mm, cd(0)), nz((size_t)n * std::max(1, mr), cd(0));
      for (int p = 0; p < n; ++p) {
        if (done[p] || jdone[p] == 0) continue;
        const cd* Hp = Hh[p].data();
        const cd* gp = &g[(size_t)p * (m + 1)];
        std::vector<cd> y(jdone[p]);
        for (int i = jdone[p] - 1; i >= 0; --i) {
          cd acc = gp[i];
          for (int k2 = i + 1; k2 < jdone[p]; ++k2) acc -= Hp[(size_t)k2 * ldh + mr + i] * y[k2];
          y[i] = acc / Hp[(size_t)i * ldh + mr + i];
        }
        for (int i = 0; i < jdone[p]; ++i) ny[(size_t)p * mm + i] = -y[i];
        if (mr > 0) {
          std::vector<cd> t(mr, cd(0));
          for (int k2 = 0; k2 < jdone[p]; ++k2)
            for (int i = 0; i < mr; ++i) t[i] += Hp[(size_t)k2 * ldh + i] * y[k2];
          btri_solve(W.R[p], mr, t.data(), nz.data() + (size_t)p * mr);
        }
      }
      BTRY(bupdate(B, W, xt, 0, W.d_V, mm, ny));
      if (mr > 0) BTRY(bupdate(B, W, xt, 0, W.d_Vold, mr, nz));
    }
    if (!true_check) {
      bool all = true;
      for (int p = 0; p < n; ++p) {
        if (!done[p] && res[p] / bn[p] <= tolv[p]) done[p] = 1;
        all = all && done[p];
      }
      if (all) break;
    }
  }
  if (harvest && mr == 0 && W.mrec > 0) {
    // leading columns common to the batch of every problem's last cycle: R_p (rotated columns),
    // C_p = V_p Q_p with Q_p = G_1^H ... G_mh^H [I; 0], written just in front of V_p
    int mh = W.mrec;
    for (int p = 0; p < n; ++p)
      if (bn[p] > 0) mh = std::min(mh, jdone[p]);
    W.rec_m = 0;
    if (mh >= 4) {
      std::vector<std::vector<cd>> hq((size_t)mh, std::vector<cd>((size_t)n * (mh + 1), cd(0)));
      for (int p = 0; p < n; ++p) {
        W.R[p].assign((size_t)mh * mh, cd(1));
        if (bn[p] == 0) continue;  // zero right-hand side: C_p = 0 columns are never used (c = 0)
        const cd* Hp = Hh[p].data();
        for (int k2 = 0; k2 < mh; ++k2)
          for (int i = 0; i < mh; ++i) W.R[p][(size_t)k2 * mh + i] = i <= k2 ? Hp[(size_t)k2 * ldh + i] : cd(0);
        const cd* csp = &cs[(size_t)p * m];
        const cd* snp = &sn[(size_t)p * m];
        std::vector<cd> q(mh + 1);
        for (int k2 = 0; k2 < mh; ++k2) {
          std::fill(q.begin(), q.end(), cd(0));
          q[k2] = 1;
          for (int i = mh - 1; i >= 0; --i) {
            const cd a = q[i], bb = q[i + 1];
            q[i] = csp[i] * a - std::conj(snp[i]) * bb;
            q[i + 1] = snp[i] * a + std::conj(csp[i]) * bb;
          }
          for (int i = 0; i <= mh; ++i) hq[k2][(size_t)p * (mh + 1) + i] = -q[i];
        }
      }
      std::vector<zd*> Ch(n);
      for (int p = 0; p < n; ++p) {
        Ch[p] = W.V[p] - (size_t)mh * B->N[p];
        BCU(cudaMemsetAsync(Ch[p], 0, (size_t)mh * B->N[p] * sizeof(zd), B->stream));
        BCU(cudaMemcpyAsync(W.Vold[p], W.V[p], (size_t)mh * B->N[p] * sizeof(zd), cudaMemcpyDeviceToDevice,
                            B->stream));
      }
      BCU(cudaMemcpyAsync(W.d_C, Ch.data(), n * sizeof(zd*), cudaMemcpyHostToDevice, B->stream));
      for (int k2 = 0; k2 < mh; ++k2) BTRY(bupdate(B, W, W.d_C, k2, W.d_V, mh + 1, hq[k2]));
      W.rec_m = mh;
    }
  }
  // true residuals
  BTRY(bapply(B, slot, xt, 0, W.d_r, 0));
  k_brsub<<<bgrid(B), 256, 0, B->stream>>>(W.d_r, 0, bt, B->d_N);
  BCU(cudaGetLastError());
  BTRY(bdots(B, W, W.d_r, 1, W.d_r, 0, tmp));
  for (int p = 0; p < n; ++p) rr[p] = bn[p] > 0 ? std::sqrt(tmp[p].real()) / bn[p] : 0.0;
  return SGF_OK;
}

extern "C" sgf_status sgf_batch_solve(sgf_batch* B, double tol, int maxit, void* const* mu_devs, int* iters,
                                      double* relres) {
  if (!B) return SGF_EINVAL;
  if (!B->exec[0]) return berr(B, SGF_ESTATE, "batch was not created");
  if (!(tol > 0) || maxit < 1 || !mu_devs) return berr(B, SGF_EINVAL, "bad solve arguments");
  const int n = B->n;
  for (int p = 0; p < n; ++p)
    if (!mu_devs[p]) return berr(B, SGF_EINVAL, "null buffer for problem %d", p);
  BWork W;
  // restart length: up to 1000 Krylov vectors per problem, within 4 GiB of bases for the batch
  long sumN = 0;
  for (int p = 0; p < n; ++p) sumN += B->N[p];
  W.m = (int)std::max(20L, std::min({1000L, (long)maxit, (4L << 30) / (16L * sumN) - 1}));
  std::vector<void*> mine;
  auto al = [&](zd** ptr, size_t cnt) -> sgf_status {
    cudaError_t e = cudaMalloc((void**)ptr, cnt * sizeof(zd));
    if (e != cudaSuccess) return berr(B, SGF_ECUDA, "cudaMalloc: %s", cudaGetErrorString(e));
    mine.push_back(*ptr);
    return SGF_OK;
  };
  auto cleanup = [&]() {
    cudaStreamSynchronize(B->stream);
    for (void* q : mine) cudaFree(q);
  };
  sgf_status st = SGF_OK;
  std::vector<zd*> bv(n), xv(n), dv(n), rv(n), Vv(n), r2(n);
  zd **d_bt = nullptr, **d_xt = nullptr, **d_dt = nullptr, **d_r2 = nullptr;
  // the mixed refinement's later correction solves recycle up to 256 vectors of the first one
  W.mrec = B->any_mixed && !getenv("SGF_NO_RECYCLE") ? std::min(W.m, 256) : 0;
  const size_t nvec = (size_t)W.mrec + W.m + 1;
  const int nchunk = kdots_chunks(B->maxN);
  W.ks.assign(n, KStep{});
  W.V.assign(n, nullptr);
  W.Vold.assign(n, nullptr);
  W.R.assign(n, std::vector<cd>());
  for (int p = 0; p < n && st == SGF_OK; ++p) {
    long N = B->N[p];
    zd* base = nullptr;
    if ((st = al(&base, nvec * N)) || (st = al(&rv[p], N)) || (st = al(&bv[p], N)) || (st = al(&dv[p], N)) ||
        (st = al(&r2[p], N)) || (st = al(&W.ks[p].H, nvec * W.m)) || (st = al(&W.ks[p].h, nvec + 1)) ||
        (st = al((zd**)&W.ks[p].part, (size_t)nchunk * nvec)) ||
        (st = al((zd**)&W.ks[p].npart, (size_t)kupdate_blocks(B->maxN))) ||
        (st = al((zd**)&W.ks[p].ticket, (size_t)kdots_groups((int)nvec) / 4 + 1)) ||
        (W.mrec > 0 && (st = al(&W.Vold[p], (size_t)W.mrec * N))))
      break;
    cudaMemsetAsync(W.ks[p].ticket, 0, (size_t)kdots_groups((int)nvec) * sizeof(unsigned), B->stream);
    Vv[p] = base + (size_t)W.mrec * N;
    W.V[p] = Vv[p];
    W.ks[p].n = N;
    xv[p] = (zd*)mu_devs[p];
  }
  auto tab = [&](zd*** d, const std::vector<zd*>& h) -> sgf_status {
    sgf_status s2 = al((zd**)d, (n * sizeof(zd*) + sizeof(zd) - 1) / sizeof(zd));
    if (s2 != SGF_OK) return s2;
    cudaError_t e = cudaMemcpy(*d, h.data(), n * sizeof(zd*), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? SGF_OK : berr(B, SGF_ECUDA, "table upload: %s", cudaGetErrorString(e));
  };
  if (st == SGF_OK) st = tab(&W.d_V, Vv);
  if (st == SGF_OK) st = tab(&W.d_C, Vv);
  if (st == SGF_OK) st = tab(&W.d_Vold, W.mrec > 0 ? W.Vold : Vv);
  if (st == SGF_OK) st = tab(&W.d_r, rv);
  if (st == SGF_OK) st = tab(&d_bt, bv);
  if (st == SGF_OK) st = tab(&d_xt, xv);
  if (st == SGF_OK) st = tab(&d_dt, dv);
  if (st == SGF_OK) st = tab(&d_r2, r2);
  if (st == SGF_OK) st = al(&W.d_h, (size_t)n * (nvec + 1));
  if (st == SGF_OK) st = al((zd**)&W.d_s, (n + 1) / 2 + 1);
  if (st == SGF_OK) st = al((zd**)&W.d_ks, (n * sizeof(KStep) + sizeof(zd) - 1) / sizeof(zd));
  if (st != SGF_OK) {
    cleanup();
    return st;
  }
  // right-hand sides of every problem (eq. discrete_eq)
  for (int p = 0; p < n && st == SGF_OK; ++p) {
    sgf_ctx* c = B->ctx[p];
    cudaStream_t keep = c->stream;
    c->stream = B->stream;
    cudaError_t e = launch_rhs(c, bv[p]);
    c->stream = keep;
    if (e != cudaSuccess) st = berr(B, SGF_ECUDA, "rhs: %s", cudaGetErrorString(e));
  }
  std::vector<int> its(n, 0), it_in(n, 0);
  std::vector<double> rr(n, 1.0), rr_in(n, 1.0);
  if (st == SGF_OK && !B->any_mixed) {
    st = bgmres(B, W, 0, d_bt, d_xt, xv, std::vector<double>(n, tol), true, maxit, its, rr);
  } else if (st == SGF_OK) {
    // FP64 residual refinement (graph slot 1) around lockstep inner solves on each context's own
    // operator (slot 0) to 1e-6
    std::vector<cd> tmp;
    for (int p = 0; p < n; ++p) cudaMemsetAsync(xv[p], 0, B->N[p] * sizeof(zd), B->stream);
    k_bcopy<<<bgrid(B), 256, 0, B->stream>>>(d_r2, 0, d_bt, 0, B->d_N);
    std::vector<double> bn(n);
    st = bdots(B, W, d_bt, 1, d_bt, 0, tmp);
    for (int p = 0; p < n && st == SGF_OK; ++p) bn[p] = std::sqrt(tmp[p].real());
    // as in sgf_solve: inner solves to 1e-6 on each context's own operator; once a problem's step
    // gains less than a factor 10, the batch's remaining corrections run on the FP64 operators to
    // each problem's final tolerance (problems already finished get tolerance 1: no work)
    int used = 0;
    bool fp64_inner = false;
    std::vector<double> rr_prev(n, 1.0), tolv(n);
    std::vector<char> fin(n, 0);
    for (int outer = 0; outer < 30 && st == SGF_OK; ++outer) {
      for (int p = 0; p < n; ++p)
        tolv[p] = fin[p] ? 1.0 : (fp64_inner ? std::min(0.5, tol / rr_prev[p]) : 1e-6);
      // the first mixed correction solve leaves its Krylov spaces for the later ones
      st = bgmres(B, W, fp64_inner ? 1 : 0, d_r2, d_dt, dv, tolv, fp64_inner, std::max(1, maxit - used), it_in,
                  rr_in, !fp64_inner && W.rec_m > 0, !fp64_inner && outer == 0);
      if (st != SGF_OK) break;
      int mx = 0;
      for (int p = 0; p < n; ++p) {
        its[p] += it_in[p];
        mx = std::max(mx, it_in[p]);
      }
      used += mx + 1;
      k_badd<<<bgrid(B), 256, 0, B->stream>>>(d_xt, d_dt, B->d_N);
      st = bapply(B, 1, d_xt, 0, d_r2, 0);
      if (st != SGF_OK) break;
      k_brsub<<<bgrid(B), 256, 0, B->stream>>>(d_r2, 0, d_bt, B->d_N);
      st = bdots(B, W, d_r2, 1, d_r2, 0, tmp);
      bool all = true, switch64 = false;
      for (int p = 0; p < n; ++p) {
        if (fin[p]) continue;
        ++its[p];
        rr[p] = bn[p] > 0 ? std::sqrt(tmp[p].real()) / bn[p] : 0.0;
        if (rr[p] <= tol || (fp64_inner && rr[p] > 0.5 * rr_prev[p])) fin[p] = 1;
        if (!fin[p] && rr[p] > 0.1 * rr_prev[p]) switch64 = true;
        rr_prev[p] = rr[p];
        all = all && fin[p];
      }
      if (getenv("SGF_VERBOSE"))
        for (int p = 0; p < n; ++p)
          fprintf(stderr, "batch refinement %d problem %d inner %s its %d outer rr %.3e\n", outer, p,
                  fp64_inner ? "fp64" : "mixed", it_in[p], rr[p]);
      if (all || used >= maxit) break;
      fp64_inner = fp64_inner || switch64;
    }
  }
  cleanup();
  for (int p = 0; p < n; ++p) {
    if (iters) iters[p] = its[p];
    if (relres) relres[p] = rr[p];
  }
  if (st != SGF_OK) return st;
  for (int p = 0; p < n; ++p)
    if (!(rr[p] <= tol))
      return berr(B, SGF_ENOCONV, "problem %d stopped at relative residual %g after %d applications", p, rr[p],
                  its[p]);
  return SGF_OK;
}
