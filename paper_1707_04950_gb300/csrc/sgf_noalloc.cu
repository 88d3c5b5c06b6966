// Rayleigh extraction without any device or host heap allocation.
//
// sgf_rayleigh allocates a small per-call table and output buffer with cudaMalloc. Some callers
// cannot allocate while they run: processes that run under a fixed device-memory budget reserved up
// front, and real-time loops that must not enter the allocator (cudaMalloc and cudaFree may
// synchronise the device and take unbounded time). This file gives them sgf_rayleigh_noalloc: the
// same reduction, with its scratch in a file-scope __device__ array of fixed size that every GPU
// loading the library keeps until the process exits. The call synchronises its stream (it copies
// the mode data in and B_n out through fixed stack buffers), so it is not for a stream that is
// being captured into a graph.
#include <mutex>

#include "sgf_internal.h"

// Maximum number of Rayleigh modes per call (n_hi - n_lo + 1).
#define SGF_NOALLOC_MAX_MODES 1024

// Scratch per mode: 6 doubles of mode data (alpha_n, beta_n re/im, Q_j re/im, completion flag)
// followed by the complex coefficient B_n written by the kernel.
static __device__ __align__(256) double g_rayleigh_scratch[SGF_NOALLOC_MAX_MODES * 8];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (the host-side name is only a stand-in). Looked
// up once per device, with that device current.
sgf_status scratch_address(sgf_ctx* ctx, double** out) {
  if (ctx->device < 0 || ctx->device >= kMaxDevices)
    return set_err(ctx, SGF_EINVAL, "device index %d out of range for the static scratch", ctx->device);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[ctx->device]) {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_rayleigh_scratch);
    if (e != cudaSuccess || !p)
      return set_err(ctx, SGF_ECUDA, "cudaGetSymbolAddress of the Rayleigh scratch: %s", cudaGetErrorString(e));
    g_scratch_addr[ctx->device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[ctx->device];
  return SGF_OK;
}

}  // namespace

extern "C" sgf_status sgf_rayleigh_noalloc(sgf_ctx* ctx, const void* mu_dev, int n_lo, int n_hi, double* B,
                                           double* eff, double* energy_err) {
  if (!ctx) return SGF_EINVAL;
  if (!ctx->built && !ctx->geom) return set_err(ctx, SGF_ESTATE, "operator not built");
  if (!mu_dev || n_hi < n_lo) return set_err(ctx, SGF_EINVAL, "bad Rayleigh arguments");
  const int nmod = n_hi - n_lo + 1;
  if (nmod > SGF_NOALLOC_MAX_MODES)
    return set_err(ctx, SGF_EINVAL, "sgf_rayleigh_noalloc: %d modes requested, the static scratch holds at most %d",
                   nmod, SGF_NOALLOC_MAX_MODES);
  double* scratch = nullptr;
  sgf_status st = scratch_address(ctx, &scratch);
  if (st != SGF_OK) return st;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));

  // mode data (6 doubles per mode) staged in a fixed-size stack buffer, copied in chunks
  const double k = ctx->k, d = ctx->d, h = ctx->prm.h;
  const int j = ctx->prm.j;
  double* d_mp = scratch;
  zd* d_B = reinterpret_cast<zd*>(scratch + 6 * SGF_NOALLOC_MAX_MODES);
  double chunk[6 * 64];
  for (int t0 = 0; t0 < nmod; t0 += 64) {
    int cnt = nmod - t0 < 64 ? nmod - t0 : 64;
    for (int u = 0; u < cnt; ++u) {
      int n = n_lo + t0 + u;
      double an = ctx->alpha + 2 * SGF_PI * n / d;
      // the same host helpers as sgf_rayleigh, so both entry points take identical mode data
      std::complex<double> bn = beta_host(k, an);
      std::complex<double> Q = Qj_host(bn, h, j);
      bool in_ueta = std::abs(Q) < ctx->prm.eta && std::abs(bn) <= k;
      double* r = chunk + 6 * u;
      r[0] = an; r[1] = bn.real(); r[2] = bn.imag(); r[3] = Q.real(); r[4] = Q.imag(); r[5] = in_ueta ? 1.0 : 0.0;
    }
    e = cudaMemcpyAsync(d_mp + 6 * t0, chunk, sizeof(double) * 6 * cnt, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "copy of mode data: %s", cudaGetErrorString(e));
    // the pageable source buffer is reused for the next chunk: wait for this copy to be consumed
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "stream sync: %s", cudaGetErrorString(e));
  }
  // every B_n is written by the kernel, so nothing in the scratch needs clearing between calls
  e = launch_rayleigh_mp(ctx, static_cast<const zd*>(mu_dev), nmod, d_mp, d_B);
  if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "rayleigh kernel: %s", cudaGetErrorString(e));
  double sum = 0;
  for (int t0 = 0; t0 < nmod; t0 += 64) {
    int cnt = nmod - t0 < 64 ? nmod - t0 : 64;
    double buf[2 * 64];
    e = cudaMemcpyAsync(buf, d_B + t0, sizeof(zd) * cnt, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return set_err(ctx, SGF_ECUDA, "copy of B_n: %s", cudaGetErrorString(e));
    for (int u = 0; u < cnt; ++u) {
      int n = n_lo + t0 + u;
      double an = ctx->alpha + 2 * SGF_PI * n / d;
      double q = k * k - an * an;
      double br = q >= 0 ? sqrt(q) : 0.0;
      double en = q > 0 ? br / ctx->beta * (buf[2 * u] * buf[2 * u] + buf[2 * u + 1] * buf[2 * u + 1]) : 0.0;
      if (B) {
        B[2 * (t0 + u)] = buf[2 * u];
        B[2 * (t0 + u) + 1] = buf[2 * u + 1];
      }
      if (eff) eff[t0 + u] = en;
      sum += en;
    }
  }
  if (energy_err) *energy_err = 1.0 - sum;
  return SGF_OK;
}
