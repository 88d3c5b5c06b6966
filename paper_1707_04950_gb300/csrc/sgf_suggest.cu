// Numerical parameters from a problem's geometry and a target accuracy (host only; no GPU work).
//
// The paper fixes its parameters per table and describes how they should move (Section 6.1,
// "Computing costs"): the shift h/lambda between 1/3 and 1, larger for deeper gratings so that the
// first shifted source stays clear of the surface; more periods n_per in the spatial lattice sum as
// h/lambda grows; an accelerator cell of about a wavelength. These rules are applied here, with the
// library's own constraints (cyclic X transform of n_x p points, h > a max|f'|, shifted poles off the
// grid lags, non-resonant cells) and a direct convergence test for n_per: the windowed lattice sum
// of G_j (eq. Gq_limit) at points next to the shifted images is evaluated with A = n_per d doubled
// until it stops changing at the target accuracy.
#include <cmath>
#include <complex>

#include "sgf_internal.h"

namespace {

typedef std::complex<double> cdh;

// Free-space shifted Green function G_j = sum_m (-1)^m C(j,m) (i/4) H0(k r_m) (eq.
// shifted_green_space), value only, from the C library's Bessel functions of integer order.
cdh green_j_host(double k, int j, double h, double X, double Y) {
  cdh acc(0, 0);
  double cb = 1;
  for (int m = 0; m <= j; ++m) {
    if (m > 0) cb = cb * (j - m + 1) / m;
    const double r = std::hypot(X, Y + m * h);
    const double kr = k * r;
    const cdh h0(j0(kr), y0(kr));
    acc += ((m & 1) ? -cb : cb) * cdh(0, 0.25) * h0;
  }
  return acc;
}

// The windowed lattice sum sum_p e^{-i alpha p d} S_{cA,A}(X + p d) G_j(X + p d, Y) (eq. Gq_limit).
cdh lattice_sum(double k, double alpha, double d, int j, double h, double X, double Y, double A, double c) {
  cdh acc(0, 0);
  const int P = (int)std::ceil(A / d) + 1;
  for (int p = -P; p <= P; ++p) {
    const double xp = X + p * d;
    const double S = window_S(xp, c * A, A);
    if (S <= 0) continue;
    acc += S * std::exp(cdh(0, -alpha * p * d)) * green_j_host(k, j, h, xp, Y);
  }
  return acc;
}

}  // namespace

extern "C" sgf_status sgf_suggest_params(double d, int M, const double* a, const double* b, double k, double theta,
                                         int bc, double tol, int precision, sgf_params* out) {
  if (!(d > 0) || M < 0 || !a || !b || !(k > 0) || !(std::fabs(theta) < 0.5 * SGF_PI) || (bc != 0 && bc != 1) ||
      !(tol >= 1e-14 && tol <= 1e-2) || (precision != 32 && precision != 64) || !out)
    return SGF_EINVAL;
  const double lam = 2 * SGF_PI / k, alpha = k * std::sin(theta);
  // profile: range, steepest slope, arc length
  const int S = 8192;
  double fmin = 1e300, fmax = -1e300, slope = 0, arc = 0;
  for (int s = 0; s < S; ++s) {
    const double x = d * s / S;
    double f = a[0], f1 = 0;
    for (int m = 1; m <= M; ++m) {
      const double w = 2 * SGF_PI * m / d;
      f += a[m] * std::cos(w * x) + b[m] * std::sin(w * x);
      f1 += w * (-a[m] * std::sin(w * x) + b[m] * std::cos(w * x));
    }
    fmin = std::min(fmin, f);
    fmax = std::max(fmax, f);
    slope = std::max(slope, std::fabs(f1));
    arc += std::sqrt(1 + f1 * f1) * d / S;
  }
  const double H = fmax - fmin;
  sgf_params P{};
  // cells: side L <= 0.45 lambda (the Fourier-Bessel reconstruction of 25 functions is accurate to
  // ~1e-8 up to k L / sqrt(2) = 2), n_x a power of two, the cell not resonant
  int nx = 4;
  while (d / nx > 0.45 * lam) nx *= 2;
  for (;;) {
    const double t = std::pow(k * (d / nx) / SGF_PI, 2);
    bool res = false;
    for (int m = 1; m * m < t + 1; ++m)
      for (int n = 1; m * m + n * n < t + 1; ++n) res = res || std::fabs(t - (m * m + n * n)) < 1e-2;
    if (!res) break;
    nx *= 2;
  }
  const double L = d / nx;
  // nodes: points per wavelength of arc length growing with the digits asked for (measured with the
  // exact system: 6 per digit reaches the target energy balance on shallow and Wood sinusoids, 3 per
  // digit stays 1-2 orders short), a multiple of n_x
  const double ppw = std::max(16.0, 6.0 * std::log10(1.0 / tol));
  int N = (int)std::ceil(ppw * arc / lam);
  N = std::max(N, 2 * nx);
  N = ((N + nx - 1) / nx) * nx;
  P.N = N;
  P.nx = nx;
  P.hmin = fmin - 0.5 * L;
  P.ny = (int)std::floor((fmax - P.hmin) / L) + 1;
  const double dx = d / N;
  // the widest singular window inside a cell (a < L): the log quadrature gains with the window
  P.Ma = std::max(2, (int)std::floor(0.95 * L / dx + 1e-9));
  const double a_s = P.Ma * dx;
  // shifts: j = 8 near a Wood anomaly (some |beta_n| below k / 10), none otherwise
  double bmin = 1e300;
  for (int n = (int)std::floor((-2 * k - alpha) * d / (2 * SGF_PI)); n <= (int)std::ceil((2 * k - alpha) * d / (2 * SGF_PI)); ++n) {
    const double an = alpha + 2 * SGF_PI * n / d;
    bmin = std::min(bmin, std::sqrt(std::fabs(k * k - an * an)));
  }
  P.j = bmin < 0.1 * k ? 8 : 0;
  // h/lambda from 1/3 (shallow) up to 1 (deep), clear of the singular window, off the grid lags
  P.p = 8;
  P.e = 1;
  double h = std::min(1.0, std::max(1.0 / 3.0, 1.0 / 3.0 + 0.06 * H / lam)) * lam;
  h = std::max(h, 1.2 * a_s * slope);
  const double dg = L / P.p;
  const int jj = std::max(P.j, 1);
  P.h = (std::round(h / dg) + 1.0 / (jj + 1)) * dg;
  if (!(P.h > a_s * slope)) P.h += dg;
  P.c_win = 0.5;
  P.delta_min = d / 64.0;
  P.spec_exp = 40.0;
  P.eta = 1e-3;
  P.n_coll = 200;
  P.n_fb = 12;
  P.precision = precision;
  P.ls_reg = k * L < 1.0 ? 1e-6 : 1e-9;
  // n_per: double A until the windowed sums next to the shifted images agree to tol / 10
  const int jl = P.j;
  const double Ys[2] = {jl > 0 ? -P.h + 0.5 * P.delta_min : 0.5 * P.delta_min, 0.25 * P.delta_min};
  const double Xs[2] = {0.23 * d, 0.41 * d};
  // the largest n_per tried is 16384 (its check sums 32768 periods)
  bool converged = false;
  int n_per = 8;
  for (; n_per <= 16384; n_per *= 2) {
    double worst = 0;
    for (double Y : Ys)
      for (double X : Xs) {
        const cdh s1 = lattice_sum(k, alpha, d, jl, P.h, X, Y, n_per * d, P.c_win);
        const cdh s2 = lattice_sum(k, alpha, d, jl, P.h, X, Y, 2.0 * n_per * d, P.c_win);
        worst = std::max(worst, std::abs(s2 - s1) / std::max(1e-300, std::abs(s2)));
      }
    if (worst < 0.1 * tol) {
      converged = true;
      break;
    }
  }
  P.n_per = std::min(n_per, 16384);
  *out = P;
  // the record is filled either way; SGF_ENOCONV says the lattice-sum check did not reach tol / 10
  return converged ? SGF_OK : SGF_ENOCONV;
}
