// The unaccelerated Nystrom operator (Section 4: eqs. discrete_eq, D_deltax) as a dense N x N
// matrix in HBM, for small problems, crossover studies and as an independent check of the
// accelerated operator:
//
//   A = sigma/2 I + D~_sing + D~_reg + D_M
//   D~_reg  (eqs. D_ns, G_jq_s): dx K[ grad G~ - sum_{p=-1..1} e^{-i alpha p d} S^f_p grad G_j(X + p d, Y) ]
//           with G~ = G~_j^qper by the hybrid evaluation: the shifted spectral series (eq.
//           shifted_quasi_per_rayleigh, Wood-safe form of eq. betan_taylor) where
//           delta = min_m |Y + m h| >= delta_min, the windowed lattice sum (eq. Gq_limit) otherwise
//   D~_sing (eq. local_mat): (r_s K_s + dx K_r) S^f on the band |i - l| < M_a (quasi-periodic wrap)
//   D_M     (eq. D_M_deltax): MT MS
// K is the kernel of the boundary condition applied to a gradient: f'_l G_X - G_Y (Dirichlet double
// layer) or (-f'_i G_X + G_Y) s_l / s_i (Neumann, target-normal derivative of the single layer).
//
//   k_exact_entries  warp per entry: lanes share the spectral terms or the lattice periods of G~,
//                    lanes 0-2 the windowed p = -1, 0, 1 subtraction, lane 3 the singular band,
//                    lane 4 the modes and the identity
//   k_exact_gemv     y = A x, warp per row (each row one contiguous 16 N-byte stream); four FP64 FMAs
//                    per 16-byte entry put it above GB300's FP64 ridge (1.25 TFLOP/s against
//                    ~6.7 TB/s): it is bound by the FP64 pipes, not by HBM
//   k_exact_gemv_adj y = A^H x, a thread per column over a chunk of rows (coalesced across the
//                    warp), chunks combined with atomics
#include "sgf_internal.h"

namespace {

struct ExactArgs {
  double k, alpha, d, dx, h, a_s, gam, A, cwin, delta_min, spec_exp, hs;
  int N, j, bc, Ma, nm;
};

__device__ inline zd kernel_bc(const ExactArgs& a, zd gx, zd gy, double f1t, double st, double f1s, double ss) {
  return a.bc == 0 ? f1s * gx - gy : (-f1t * gx + gy) * (ss / st);
}

// This lane's share of grad G~_j^qper at (X, Y) (the warp sums the shares); punct drops the
// (p = 0, m = 0) term at coincident points.
__device__ inline void gtilde_grad_share(const ExactArgs& a, int lane, double X, double Y, bool punct,
                                         const double* binw, zd& gx, zd& gy) {
  gx = zd(0, 0);
  gy = zd(0, 0);
  const double dl = row_delta(Y, a.j, a.h);
  if (dl >= a.delta_min) {
    const double T = sqrt(a.k * a.k + (a.spec_exp / dl) * (a.spec_exp / dl));
    const long n_hi = (long)ceil((T - a.alpha) * a.d / (2 * SGF_PI));
    const long n_lo = (long)floor((-T - a.alpha) * a.d / (2 * SGF_PI));
    for (long n = n_lo + lane; n <= n_hi; n += 32) {
      zd c, cy;
      double an;
      spec_coef(a.k, a.alpha, a.d, a.j, a.h, Y, (int)n, binw, c, cy, an);
      const zd e = expi(an * X);
      gx += zd(0, an) * (c * e);
      gy += cy * e;
    }
  } else {
    const double q = floor((X + 0.5 * a.d) / a.d);  // X = X_r + q d, X_r in [-d/2, d/2)
    const double Xr = X - q * a.d;
    const int P = (int)ceil(a.A / a.d) + 1;
    for (int p = -P + lane; p <= P; p += 32) {
      const double xp = Xr + p * a.d;
      const double S = window_S(xp, a.cwin * a.A, a.A);
      if (S <= 0) continue;
      const GreenVal gv = green_j(a.k, a.j, a.h, xp, Y, punct && p == 0, false, binw);
      const zd ph = expi(-a.alpha * p * a.d);
      gx += (S * ph) * gv.gx;
      gy += (S * ph) * gv.gy;
    }
    const zd qph = expi(a.alpha * q * a.d);
    gx = gx * qph;
    gy = gy * qph;
  }
}

__global__ void k_exact_entries(ExactArgs a, long row0, long nrows, const double* __restrict__ x,
                                const double* __restrict__ f, const double* __restrict__ f1,
                                const double* __restrict__ f2, const double* __restrict__ binw,
                                const double* __restrict__ kress, const zd* __restrict__ MT,
                                const zd* __restrict__ MS, zd hk, zd* __restrict__ A) {
  const int lane = threadIdx.x & 31;
  const long wid = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (wid >= nrows * a.N) return;  // uniform across the warp
  const long i = row0 + wid / a.N, l = wid % a.N;
  const bool diag = i == l;
  const double xi = x[i], fi = f[i], f1i = f1[i], si = sqrt(1 + f1i * f1i);
  const double xl = x[l], fl = f[l], f1l = f1[l], sl = sqrt(1 + f1l * f1l);
  const double X = xi - xl, Y = fi - fl;
  zd gx, gy;
  gtilde_grad_share(a, lane, X, Y, diag, binw, gx, gy);
  zd v = a.dx * kernel_bc(a, gx, gy, f1i, si, f1l, sl);
  if (lane < 3) {  // the windowed near part of the period copies p = -1, 0, 1
    const int p = lane - 1;
    const double Xp = X + p * a.d;
    const double Sf = window_S(hypot(Xp, Y), a.gam, a.a_s);
    if (Sf > 0) {
      const GreenVal gv = green_j(a.k, a.j, a.h, Xp, Y, diag && p == 0, false, binw);
      v -= (a.dx * Sf) * (expi(-a.alpha * p * a.d) * kernel_bc(a, gv.gx, gv.gy, f1i, si, f1l, sl));
    }
  } else if (lane == 3) {  // the singular band: source l in its period copy w with |i - (l + w N)| < M_a
    for (int w = -1; w <= 1; ++w) {
      const long s = i - (l + (long)w * a.N);
      if (s <= -a.Ma || s >= a.Ma) continue;
      const double xw = xl + w * a.d;
      const double Xs = xi - xw, rr = hypot(Xs, Y);
      const double Sf = window_S(rr, a.gam, a.a_s);
      zd val;
      if (s == 0) {
        val = (a.dx * Sf) * (zd(f2[i] / (4 * SGF_PI * (1 + f1i * f1i)), 0) + (a.bc == 0 ? hk : -hk));
      } else {
        const GreenVal gv = green_j(a.k, a.j, a.h, Xs, Y, false, false, binw);
        const zd kern = kernel_bc(a, gv.gx, gv.gy, f1i, si, f1l, sl);
        const double j1r = a.k * j1(a.k * rr) / rr;
        const double Ks = a.bc == 0 ? -j1r / (4 * SGF_PI) * (Y - f1l * Xs) : j1r / (4 * SGF_PI) * (-f1i * Xs + Y) / si * sl;
        const double sn = sin(SGF_PI * Xs / (2 * a.a_s));
        const zd Kr = kern - zd(Ks * log(4 * sn * sn), 0);
        val = Sf * (zd(kress[s + a.Ma - 1] * Ks, 0) + a.dx * Kr);
      }
      v += val * expi(a.alpha * a.d * w);
    }
  } else if (lane == 4) {  // completion modes and the identity
    for (int n = 0; n < a.nm; ++n) v += MT[i * a.nm + n] * MS[(long)n * a.N + l];
    if (diag) v += zd(a.hs, 0);
  }
  v = warp_sum(v);
  if (lane == 0) A[i * a.N + l] = v;
}

constexpr int GEMV_U = 4;

__global__ void k_exact_gemv(long N, const zd* __restrict__ A, const zd* __restrict__ x, zd* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const long row = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= N) return;  // uniform across the warp
  const zd* Ar = A + row * N;
  zd acc[GEMV_U];
#pragma unroll
  for (int u = 0; u < GEMV_U; ++u) acc[u] = zd(0, 0);
  for (long c0 = lane; c0 < N; c0 += 32 * GEMV_U) {
    zd av[GEMV_U], xv[GEMV_U];
#pragma unroll
    for (int u = 0; u < GEMV_U; ++u) {
      const long c = c0 + 32 * u;
      if (c < N) {
        av[u] = Ar[c];
        xv[u] = x[c];
      } else {
        av[u] = zd(0, 0);
        xv[u] = zd(0, 0);
      }
    }
#pragma unroll
    for (int u = 0; u < GEMV_U; ++u) acc[u] = fma_c(av[u], xv[u], acc[u]);
  }
  zd s = (acc[0] + acc[1]) + (acc[2] + acc[3]);
  s = warp_sum(s);
  if (lane == 0) y[row] = s;
}

__global__ void k_exact_gemv_adj(long N, long rows_per, const zd* __restrict__ A, const zd* __restrict__ x,
                                 zd* __restrict__ y) {
  const long col = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= N) return;
  const long r0 = (long)blockIdx.y * rows_per, r1 = min(N, r0 + rows_per);
  zd acc(0, 0);
  for (long r = r0; r < r1; ++r) {  // acc += conj(A[r][col]) x[r]
    const zd av = A[r * N + col], xv = x[r];
    acc.re = fma(av.re, xv.re, fma(av.im, xv.im, acc.re));
    acc.im = fma(av.re, xv.im, fma(-av.im, xv.re, acc.im));
  }
  atomicAdd(&y[col].re, acc.re);
  atomicAdd(&y[col].im, acc.im);
}

}  // namespace

cudaError_t launch_exact_entries(sgf_ctx* c, zd hk) {
  ExactArgs a;
  a.k = c->k; a.alpha = c->alpha; a.d = c->d; a.dx = c->dx; a.h = c->prm.h; a.a_s = c->a_s; a.gam = c->gam;
  a.A = c->prm.n_per * c->d; a.cwin = c->prm.c_win; a.delta_min = c->prm.delta_min; a.spec_exp = c->prm.spec_exp;
  a.hs = c->bc == 0 ? 0.5 : -0.5;
  a.N = c->N; a.j = c->prm.j; a.bc = c->bc; a.Ma = c->prm.Ma; a.nm = c->nm;
  // row chunks of at most 2^24 entries (one warp each) per launch
  const long N = c->N;
  const long chunk = std::max(1L, (1L << 24) / N);
  for (long r0 = 0; r0 < N; r0 += chunk) {
    const long nr = std::min(chunk, N - r0);
    const long warps = nr * N;
    k_exact_entries<<<(unsigned)((warps + 7) / 8), 256, 0, c->stream>>>(a, r0, nr, c->d_x, c->d_f, c->d_f1, c->d_f2,
                                                                        c->d_binw, c->keep.kress, c->d_MT, c->d_MS, hk,
                                                                        c->d_Aex);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_exact_gemv(sgf_ctx* c, const zd* x, zd* y, bool adjoint) {
  const long N = c->N;
  if (!adjoint) {
    k_exact_gemv<<<(unsigned)((N + 7) / 8), 256, 0, c->stream>>>(N, c->d_Aex, x, y);
    return cudaGetLastError();
  }
  cudaError_t e = cudaMemsetAsync(y, 0, N * sizeof(zd), c->stream);
  if (e != cudaSuccess) return e;
  const long colb = (N + 255) / 256;
  // about 8 blocks per SM in total
  const long chunks = std::max(1L, std::min(N, (long)(152 * 8) / std::max(1L, colb)));
  const long rows_per = (N + chunks - 1) / chunks;
  k_exact_gemv_adj<<<dim3((unsigned)colb, (unsigned)chunks), 256, 0, c->stream>>>(N, rows_per, c->d_Aex, x, y);
  return cudaGetLastError();
}
