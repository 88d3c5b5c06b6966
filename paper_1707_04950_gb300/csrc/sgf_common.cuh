// Shared device helpers of the sgf library: complex arithmetic, free-space and shifted Green
// functions (Bruno & Maas, eqs. free_space, shifted_green_function), the smooth windows of
// eq. S_def, and launch/error helpers.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define SGF_PI 3.14159265358979323846

template <typename T>
struct cplx {
  T re, im;
  __host__ __device__ cplx() : re(0), im(0) {}
  __host__ __device__ cplx(T r, T i = 0) : re(r), im(i) {}
  template <typename U>
  __host__ __device__ explicit cplx(const cplx<U>& o) : re((T)o.re), im((T)o.im) {}
};

template <typename T>
__host__ __device__ inline cplx<T> operator+(cplx<T> a, cplx<T> b) { return cplx<T>(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ inline cplx<T> operator-(cplx<T> a, cplx<T> b) { return cplx<T>(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ inline cplx<T> operator-(cplx<T> a) { return cplx<T>(-a.re, -a.im); }
template <typename T>
__host__ __device__ inline cplx<T> operator*(cplx<T> a, cplx<T> b) {
  return cplx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__host__ __device__ inline cplx<T> operator*(T s, cplx<T> a) { return cplx<T>(s * a.re, s * a.im); }
template <typename T>
__host__ __device__ inline cplx<T> operator*(cplx<T> a, T s) { return cplx<T>(s * a.re, s * a.im); }
template <typename T>
__host__ __device__ inline cplx<T>& operator+=(cplx<T>& a, cplx<T> b) { a.re += b.re; a.im += b.im; return a; }
template <typename T>
__host__ __device__ inline cplx<T>& operator-=(cplx<T>& a, cplx<T> b) { a.re -= b.re; a.im -= b.im; return a; }
template <typename T>
__host__ __device__ inline cplx<T> conj(cplx<T> a) { return cplx<T>(a.re, -a.im); }
template <typename T>
__host__ __device__ inline T abs2(cplx<T> a) { return a.re * a.re + a.im * a.im; }
// a * conj(b)
template <typename T>
__host__ __device__ inline cplx<T> mulc(cplx<T> a, cplx<T> b) {
  return cplx<T>(a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im);
}
template <typename T>
__device__ inline cplx<T> fma_c(cplx<T> a, cplx<T> b, cplx<T> c) {  // a*b + c
  return cplx<T>(fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im)));
}

// sum over the 32 lanes of a warp (lane 0 holds the result)
template <typename T>
__device__ inline T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ inline cplx<T> warp_sum(cplx<T> v) {
  v.re = warp_sum(v.re);
  v.im = warp_sum(v.im);
  return v;
}

// Shared-memory array of n elements of a complex type without running its constructor (every
// element is written before it is read; shared variables cannot be dynamically initialised).
#define SGF_SHARED_ARRAY(T, name, n)                                \
  __shared__ __align__(16) unsigned char name##_raw[(n) * sizeof(T)]; \
  T* name = reinterpret_cast<T*>(name##_raw)

typedef cplx<double> zd;
typedef cplx<float> zf;

__host__ __device__ inline zd cdiv(zd a, zd b) {
  double s = b.re * b.re + b.im * b.im;
  return zd((a.re * b.re + a.im * b.im) / s, (a.im * b.re - a.re * b.im) / s);
}

// e^{i t}
__device__ inline zd expi(double t) {
  double s, c;
  sincos(t, &s, &c);
  return zd(c, s);
}
// e^{z} for complex z
__device__ inline zd cexpz(zd z) {
  double m = exp(z.re), s, c;
  sincos(z.im, &s, &c);
  return zd(m * c, m * s);
}
// sin(z), complex
__device__ inline zd csin(zd z) {
  double s, c;
  sincos(z.re, &s, &c);
  return zd(s * cosh(z.im), c * sinh(z.im));
}
// sin(z)/z with the series 1 - z^2/6 + z^4/120 for |z| < 1e-3
__device__ inline zd csinc(zd z) {
  double a2 = z.re * z.re + z.im * z.im;
  if (a2 < 1e-6) {
    zd z2 = z * z;
    return zd(1.0, 0.0) - (1.0 / 6.0) * z2 + (1.0 / 120.0) * (z2 * z2);
  }
  return cdiv(csin(z), z);
}

__device__ inline int orient_of_sample(int t, int p) { return t < 2 * (p + 1) ? 0 : 1; }

// J_n(x) e^{i n th} for any integer n (J_{-n} = (-1)^n J_n): the Fourier-Bessel functions of the
// cell reconstruction, normalised by fb_norm(n, k rho_0) = (k rho_0 / 2)^|n| / |n|!
__device__ inline zd fb_Z(int n, double kr, double th) {
  int an = n < 0 ? -n : n;
  // J_n(0) = delta_{n0}; evaluated explicitly (a node can sit exactly at a cell centre)
  double J = kr > 0 ? jn(an, kr) : (an == 0 ? 1.0 : 0.0);
  if (n < 0 && (an & 1)) J = -J;
  zd e = expi(n * th);
  return J * e;
}
__device__ inline double fb_norm(int n, double krho0) {
  int an = n < 0 ? -n : n;
  double v = 1.0;
  for (int i = 1; i <= an; ++i) v *= (krho0 / 2.0) / i;
  return v;
}

// H0^(1)(x), H1^(1)(x) for real x > 0 from the CUDA Bessel functions of the first and second kind.
__device__ inline zd hankel0(double x) { return zd(j0(x), y0(x)); }
__device__ inline zd hankel1(double x) { return zd(j1(x), y1(x)); }

// Free-space G = (i/4) H0(k r) and its gradient (dG/dX, dG/dY) = (i/4)(-k H1(k r)) (X, Y)/r.
struct GreenVal {
  zd g, gx, gy;
};
__device__ inline void green0_add(double k, double X, double Y, double w, bool want_val, GreenVal& acc) {
  double r = hypot(X, Y);
  double kr = k * r;
  if (want_val) {
    zd h0 = hankel0(kr);
    acc.g += zd(-0.25 * w * h0.im, 0.25 * w * h0.re);
  }
  zd h1 = hankel1(kr);
  // (i/4)(-k) h1 / r = (-k/(4r)) * (i h1) = (-k/(4r)) * (-h1.im, h1.re)
  double c = -0.25 * k * w / r;
  zd ih1(-h1.im, h1.re);
  acc.gx += (c * X) * ih1;
  acc.gy += (c * Y) * ih1;
}

// Shifted G_j = sum_{m=0..j} (-1)^m C(j,m) G(X, Y + m h) and gradient; skip_m0 drops the m = 0
// term (the self term of the punctured Green function at coincident points).
__device__ inline GreenVal green_j(double k, int j, double h, double X, double Y, bool skip_m0,
                                   bool want_val, const double* binw) {
  GreenVal acc;
  acc.g = zd(0, 0);
  acc.gx = zd(0, 0);
  acc.gy = zd(0, 0);
  for (int m = skip_m0 ? 1 : 0; m <= j; ++m) green0_add(k, X, Y + m * h, binw[m], want_val, acc);
  return acc;
}

// min_m |Y + m h|: the distance of a lag row to the shifted images
__device__ inline double row_delta(double Y, int j, double h) {
  double dl = fabs(Y);
  for (int m = 1; m <= j; ++m) dl = fmin(dl, fabs(Y + m * h));
  return dl;
}

// (1 - e^{i beta h})^j / beta = (-2i)^j e^{i j beta h/2} sin^{j-1}(beta h/2) (h/2) sinc(beta h/2)
__device__ inline zd Qj_dev(zd beta, double h, int j) {
  if (j == 0) return cdiv(zd(1, 0), beta);
  zd half = (0.5 * h) * beta;
  zd sn = csin(half);
  zd acc = (0.5 * h) * csinc(half);
  for (int m = 1; m < j; ++m) acc = acc * sn;
  zd mi2(1, 0);
  for (int m = 0; m < j; ++m) mi2 = mi2 * zd(0, -2);
  zd ij = cexpz(zd(0, (double)j) * half);
  return mi2 * ij * acc;
}

// c_n(Y) and cy_n(Y) of the shifted spectral series (eq. shifted_quasi_per_rayleigh), with the
// exact beta -> 0 rewrite of eq. betan_taylor where |beta| (|Y| + j h) < 1.
__device__ inline void spec_coef(double k, double alpha, double d, int j, double h, double Y, int n,
                                 const double* binw, zd& c, zd& cy, double& an) {
  an = alpha + 2.0 * SGF_PI * n / d;
  double q = k * k - an * an;
  bool real_b = q >= 0;
  double bm = sqrt(fabs(q));
  zd beta = real_b ? zd(bm, 0) : zd(0, bm);
  zd S0(0, 0), S1(0, 0);
  for (int m = 0; m <= j; ++m) {
    double t = Y + m * h, at = fabs(t);
    zd em = real_b ? expi(bm * at) : zd(exp(-bm * at), 0);
    S0 += binw[m] * em;
    S1 += (t > 0 ? binw[m] : (t < 0 ? -binw[m] : 0.0)) * em;
  }
  cy = (-0.5 / d) * S1;
  if (j >= 1 && bm * (fabs(Y) + j * h) < 1.0) {
    zd acc = cexpz(zd(0, 1) * (Y * beta)) * Qj_dev(beta, h, j);
    for (int m = 0; m <= j; ++m) {
      double t = Y + m * h;
      if (t < 0) acc -= zd(0, 2.0 * binw[m] * t) * csinc(t * beta);
    }
    c = zd(0, 0.5 / d) * acc;
  } else {
    c = zd(0, 0.5 / d) * cdiv(S0, beta);
  }
}

// G_j with its gradient and the Y-derivatives of the gradient (G_xy, G_yy), for the analytic node
// derivatives of the gradient computation. Per source: G = (i/4) H0(kr), G_x = c X, G_y = c Y with
// c(r) = -(ik/4) H1(kr)/r and c'(r) = -(ik/4)(k H0(kr)/r - 2 H1(kr)/r^2) (H0' = -H1,
// H1'(z) = H0(z) - H1(z)/z), so G_xy = c' X Y/r and G_yy = c + c' Y^2/r.
struct GreenHess {
  zd g, gx, gy, gxy, gyy;
};
__device__ inline void green0_hess_add(double k, double X, double Y, double w, GreenHess& a) {
  double r = hypot(X, Y), kr = k * r;
  zd h0 = hankel0(kr), h1 = hankel1(kr);
  zd ih0(-h0.im, h0.re), ih1(-h1.im, h1.re);
  zd c = (-0.25 * k / r) * ih1;
  zd dc = (-0.25 * k) * ((k / r) * ih0 - (2.0 / (r * r)) * ih1);
  a.g += (0.25 * w) * ih0;
  a.gx += (w * X) * c;
  a.gy += (w * Y) * c;
  a.gxy += (w * X * Y / r) * dc;
  a.gyy += w * (c + (Y * Y / r) * dc);
}
__device__ inline GreenHess green_j_hess(double k, int j, double h, double X, double Y, const double* binw) {
  GreenHess a;
  a.g = a.gx = a.gy = a.gxy = a.gyy = zd(0, 0);
  for (int m = 0; m <= j; ++m) green0_hess_add(k, X, Y + m * h, binw[m], a);
  return a;
}

// S_{gamma,a}(x) of eq. S_def.
__host__ __device__ inline double window_S(double x, double gamma, double a) {
  x = fabs(x);
  if (x <= gamma) return 1.0;
  if (x >= a) return 0.0;
  double u = (x - gamma) / (a - gamma);
  return exp(2.0 * exp(-1.0 / u) / (u - 1.0));
}

// dS_{gamma,a}/dx for x >= 0: with u = (x - gamma)/(a - gamma) and S = exp(2 e^{-1/u}/(u - 1)),
// dS/dx = S 2 e^{-1/u} ((u - 1)/u^2 - 1)/(u - 1)^2 / (a - gamma) on (gamma, a), 0 elsewhere.
__host__ __device__ inline double window_S_dx(double x, double gamma, double a) {
  x = fabs(x);
  if (x <= gamma || x >= a) return 0.0;
  double u = (x - gamma) / (a - gamma);
  double e = exp(-1.0 / u);
  double S = exp(2.0 * e / (u - 1.0));
  return S * 2.0 * e * ((u - 1.0) / (u * u) - 1.0) / ((u - 1.0) * (u - 1.0)) / (a - gamma);
}

// ---------------------------------------------------------------- float-float arithmetic
// A value hi + lo held in two FP32 numbers (|lo| <= ulp(hi)/2): about 48 significant bits, computed
// on the FP32 pipes with error-free transformations (two-sum, fma-based two-product). The explicit
// round-to-nearest intrinsics keep the compiler from contracting or reassociating the steps.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s = __fadd_rn(a.hi, b.hi);
  float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_quick_two_sum(s, e);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_quick_two_sum(p, e);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_from_double(double x) {
  float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
// complex float-float packed as float4 {re.hi, im.hi, re.lo, im.lo}
__device__ __forceinline__ float4 cff_from(zd z) {
  ff r = ff_from_double(z.re), i = ff_from_double(z.im);
  return make_float4(r.hi, i.hi, r.lo, i.lo);
}
// acc_re + i acc_im += c * m
__device__ __forceinline__ void cff_mac(float4 c, float4 m, ff& acc_re, ff& acc_im) {
  ff cr = {c.x, c.z}, ci = {c.y, c.w}, mr = {m.x, m.z}, mi = {m.y, m.w};
  acc_re = ff_add(acc_re, ff_mul(cr, mr));
  acc_re = ff_add(acc_re, ff_neg(ff_mul(ci, mi)));
  acc_im = ff_add(acc_im, ff_mul(cr, mi));
  acc_im = ff_add(acc_im, ff_mul(ci, mr));
}

// Compensated complex dot product of float-float operands (the Dot2 scheme of Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005)): the hi*hi products are
// split exactly (fma residual), summed with TwoSum into an FP32 running sum whose rounding errors,
// the product residuals and the hi*lo cross terms collect in a separate FP32 error sum. The result
// is as accurate as a float-float evaluation for these sums at about two thirds of the instructions.
struct dot2c {
  float sr, si, er, ei;
};
__device__ __forceinline__ void two_sum_into(float& s, float& e, float p) {
  float t = __fadd_rn(s, p);
  float bp = __fsub_rn(t, s);
  e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp)));
  s = t;
}
// a += c * m; float4 = {re.hi, im.hi, re.lo, im.lo}
__device__ __forceinline__ void dot2_mac(float4 c, float4 m, dot2c& a) {
  float p1 = __fmul_rn(c.x, m.x), q1 = __fmaf_rn(c.x, m.x, -p1);
  float p2 = __fmul_rn(-c.y, m.y), q2 = __fmaf_rn(-c.y, m.y, -p2);
  float p3 = __fmul_rn(c.x, m.y), q3 = __fmaf_rn(c.x, m.y, -p3);
  float p4 = __fmul_rn(c.y, m.x), q4 = __fmaf_rn(c.y, m.x, -p4);
  float xr = __fmaf_rn(c.x, m.z, __fmaf_rn(c.z, m.x, __fmaf_rn(-c.y, m.w, -__fmul_rn(c.w, m.y))));
  float xi = __fmaf_rn(c.x, m.w, __fmaf_rn(c.z, m.y, __fmaf_rn(c.y, m.z, __fmul_rn(c.w, m.x))));
  two_sum_into(a.sr, a.er, p1);
  two_sum_into(a.sr, a.er, p2);
  two_sum_into(a.si, a.ei, p3);
  two_sum_into(a.si, a.ei, p4);
  a.er = __fadd_rn(a.er, __fadd_rn(__fadd_rn(q1, q2), xr));
  a.ei = __fadd_rn(a.ei, __fadd_rn(__fadd_rn(q3, q4), xi));
}
// b folded into a (two partial dot products of one row)
__device__ __forceinline__ void dot2_merge(dot2c& a, const dot2c& b) {
  two_sum_into(a.sr, a.er, b.sr);
  two_sum_into(a.si, a.ei, b.si);
  a.er = __fadd_rn(a.er, b.er);
  a.ei = __fadd_rn(a.ei, b.ei);
}

#define SGF_CUDA_CHECK(call)                                                  \
  do {                                                                            \
    cudaError_t err__ = (call);                                                   \
    if (err__ != cudaSuccess) {                                                   \
      return set_err(ctx, SGF_ECUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call,   \
                     cudaGetErrorString(err__));                                  \
    }                                                                             \
  } while (0)

static inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }
