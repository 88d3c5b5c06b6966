// Shared-memory Stockham FFT used by the global convolution of the accelerated operator
// (Bruno & Maas, eq. large_convolution_per_grid: cyclic in X after the quasi-periodic twist,
// linear in Y with zero padding).
#pragma once
#include "sgf_common.cuh"

// Shared-memory address of element e of a transform buffer: one element of padding after every 16
// keeps the stride-R stores of the first Stockham stages (and the stride-ty tiles of the X passes)
// off a single bank group. splen(n) elements hold a padded buffer of n.
__host__ __device__ __forceinline__ int spad(int e) { return e + (e >> 4); }
__host__ __device__ __forceinline__ int splen(int n) { return n + (n >> 4) + 1; }

// v * e^{dir i t} for t with cos t = c, sin t = sn (dir = -1: the forward DFT's twiddle)
template <typename T>
__device__ __forceinline__ cplx<T> rot(cplx<T> v, T c, T sn, int dir) {
  return dir < 0 ? cplx<T>(v.re * c + v.im * sn, v.im * c - v.re * sn)
                 : cplx<T>(v.re * c - v.im * sn, v.im * c + v.re * sn);
}

template <typename T, int R>
__device__ __forceinline__ void dft_reg(cplx<T>* a, int dir);

// Radix-9 and radix-16 DFTs as 3 x 3 and 4 x 4 (Cooley-Tukey with m = 3 or 4: element n = m n1 + n2;
// length-m transforms over n1 for each n2, the twiddles w^{n2 k1} of the full length, length-m
// transforms over n2; output k1 + m k2, in natural order).
template <typename T>
__device__ __forceinline__ void dft9_reg(cplx<T>* a, int dir) {
  // cos and sin of 2 pi m / 9 for m = 1, 2, 4
  const T c1 = (T)0.76604444311897803520, s1 = (T)0.64278760968653932632;
  const T c2 = (T)0.17364817766693034885, s2 = (T)0.98480775301220805936;
  const T c4 = (T)-0.93969262078590838405, s4 = (T)0.34202014332566873304;
  cplx<T> b[3][3];
#pragma unroll
  for (int n2 = 0; n2 < 3; ++n2) {
    b[n2][0] = a[n2];
    b[n2][1] = a[n2 + 3];
    b[n2][2] = a[n2 + 6];
    dft_reg<T, 3>(b[n2], dir);
  }
  b[1][1] = rot(b[1][1], c1, s1, dir);
  b[1][2] = rot(b[1][2], c2, s2, dir);
  b[2][1] = rot(b[2][1], c2, s2, dir);
  b[2][2] = rot(b[2][2], c4, s4, dir);
#pragma unroll
  for (int k1 = 0; k1 < 3; ++k1) {
    cplx<T> t[3] = {b[0][k1], b[1][k1], b[2][k1]};
    dft_reg<T, 3>(t, dir);
    a[k1] = t[0];
    a[k1 + 3] = t[1];
    a[k1 + 6] = t[2];
  }
}
template <typename T>
__device__ __forceinline__ void dft16_reg(cplx<T>* a, int dir) {
  // cos and sin of 2 pi m / 16 for m = 1, 2, 3 (m = 4, 6, 9 follow by symmetry)
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;
  const T h = (T)0.70710678118654752440;
  cplx<T> b[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < 4; ++n1) b[n2][n1] = a[4 * n1 + n2];
    dft_reg<T, 4>(b[n2], dir);
  }
  // w^{n2 k1}, w = e^{dir 2 pi i / 16}
  b[1][1] = rot(b[1][1], c1, s1, dir);
  b[1][2] = rot(b[1][2], h, h, dir);
  b[1][3] = rot(b[1][3], s1, c1, dir);
  b[2][1] = rot(b[2][1], h, h, dir);
  b[2][2] = rot(b[2][2], (T)0, (T)1, dir);
  b[2][3] = rot(b[2][3], -h, h, dir);
  b[3][1] = rot(b[3][1], s1, c1, dir);
  b[3][2] = rot(b[3][2], -h, h, dir);
  b[3][3] = rot(b[3][3], -c1, -s1, dir);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cplx<T> t[4] = {b[0][k1], b[1][k1], b[2][k1], b[3][k1]};
    dft_reg<T, 4>(t, dir);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) a[k1 + 4 * k2] = t[k2];
  }
}

// Radix-R DFT in registers, R in {2, 3, 4, 8, 9, 16}; dir = -1 forward, +1 inverse.
template <typename T, int R>
__device__ __forceinline__ void dft_reg(cplx<T>* a, int dir) {
  if (R == 9) {
    dft9_reg<T>(a, dir);
  } else if (R == 16) {
    dft16_reg<T>(a, dir);
  } else if (R == 3) {
    const T h = (T)0.86602540378443864676;  // sqrt(3)/2
    cplx<T> t1 = a[1] + a[2], df = a[1] - a[2];
    cplx<T> t2 = a[0] - (T)0.5 * t1;
    cplx<T> m = dir < 0 ? cplx<T>(h * df.im, -h * df.re) : cplx<T>(-h * df.im, h * df.re);
    a[0] = a[0] + t1;
    a[1] = t2 + m;
    a[2] = t2 - m;
  } else if (R == 2) {
    cplx<T> t = a[0];
    a[0] = t + a[1];
    a[1] = t - a[1];
  } else if (R == 4) {
    // w4 = -i (forward) / +i (inverse)
    cplx<T> v0 = a[0] + a[2], v2 = a[0] - a[2], v1 = a[1] + a[3], d = a[1] - a[3];
    cplx<T> v3 = dir < 0 ? cplx<T>(d.im, -d.re) : cplx<T>(-d.im, d.re);
    a[0] = v0 + v1;
    a[2] = v0 - v1;
    a[1] = v2 + v3;
    a[3] = v2 - v3;
  } else {
    const T h = (T)0.70710678118654752440;
    cplx<T> u[8];
    for (int r = 0; r < 4; ++r) {
      u[r] = a[r] + a[r + 4];
      u[r + 4] = a[r] - a[r + 4];
    }
    // u5 *= w, u6 *= w^2, u7 *= w^3 with w = e^{-+ 2 pi i/8}
    cplx<T> t5 = u[5], t6 = u[6], t7 = u[7];
    if (dir < 0) {
      u[5] = cplx<T>(h * (t5.re + t5.im), h * (t5.im - t5.re));
      u[6] = cplx<T>(t6.im, -t6.re);
      u[7] = cplx<T>(h * (t7.im - t7.re), -h * (t7.re + t7.im));
    } else {
      u[5] = cplx<T>(h * (t5.re - t5.im), h * (t5.im + t5.re));
      u[6] = cplx<T>(-t6.im, t6.re);
      u[7] = cplx<T>(-h * (t7.re + t7.im), h * (t7.re - t7.im));
    }
    for (int g = 0; g < 2; ++g) {
      cplx<T>* c = u + 4 * g;
      cplx<T> v0 = c[0] + c[2], v2 = c[0] - c[2], v1 = c[1] + c[3], d = c[1] - c[3];
      cplx<T> v3 = dir < 0 ? cplx<T>(d.im, -d.re) : cplx<T>(-d.im, d.re);
      a[g] = v0 + v1;
      a[g + 4] = v0 - v1;
      a[g + 2] = v2 + v3;
      a[g + 6] = v2 - v3;
    }
  }
}

// Butterflies per thread of a radix-R stage when a thread may hold VPT values (at least one). A
// block has at least n / VPT threads (n / 15 and n / 6 when n has a factor 3, for VPT = 16 and 8),
// so that items * threads covers the n / R butterflies: radix 9 takes two per thread when VPT = 16.
template <int VPT, int R>
struct StageItems {
  static constexpr int value = R == 9 ? (VPT + R - 1) / R : (VPT / R > 0 ? VPT / R : 1);
};

// One Stockham radix-R stage (self-sorting, in place through registers) over `batch` sequences;
// each thread takes up to U butterflies (every item of the stage is loaded before any store).
// Index of butterfly idx of a stage: sequence b, position j in it, and j = jq Ns + k. Ns = 2^ns2 3^ns3;
// shifts and masks replace the divisions wherever the sizes are powers of two (all batched
// transforms and every radix-8/4/2 stage), and the single factor 3 divides by a constant.
__device__ __forceinline__ void stage_index(int idx, int nR, int lognR, int batch, int ns2, int ns3, int Ns, int& b,
                                            int& j, int& jq, int& k) {
  if (batch == 1) {
    b = 0;
    j = idx;
  } else if (lognR >= 0) {
    b = idx >> lognR;
    j = idx & (nR - 1);
  } else {
    b = idx / nR;
    j = idx - b * nR;
  }
  if (ns3 == 0) {
    jq = j >> ns2;
    k = j & ((1 << ns2) - 1);
  } else if (ns3 == 1) {
    jq = (int)((unsigned)(j >> ns2) / 3u);
    k = j - jq * Ns;
  } else {
    jq = j / Ns;
    k = j - jq * Ns;
  }
}

// One Stockham radix-R stage (self-sorting, in place through registers) over `batch` sequences;
// each thread takes up to U butterflies (every item of the stage is loaded before any store).
// Ns = 2^ns2 3^ns3 is the length already transformed; lognR = log2(n/R) when that is an integer.
template <typename T, int R, int U>
__device__ __forceinline__ void stockham_stage(cplx<T>* s, int n, int lognR, int ns2, int ns3, int es, int batch,
                                               int bs, const cplx<T>* __restrict__ tw, int twlen, int dir) {
  const int nR = lognR >= 0 ? (1 << lognR) : n / R;
  const int Ns = (1 << ns2) * (ns3 == 0 ? 1 : (ns3 == 1 ? 3 : 9));
  const int tot = batch * nR;
  const int tstep = twlen / (Ns * R);  // table stride of e^{-2 pi i / (Ns R)} in a table of twlen
  cplx<T> a[U][R];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int idx = u * blockDim.x + threadIdx.x;
    if (idx < tot) {
      int b, j, jq, k;
      stage_index(idx, nR, lognR, batch, ns2, ns3, Ns, b, j, jq, k);
#pragma unroll
      for (int r = 0; r < R; ++r) a[u][r] = s[spad(b * bs + (j + r * nR) * es)];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cplx<T> w = tw[r * k * tstep];
          if (dir > 0) w.im = -w.im;
          a[u][r] = a[u][r] * w;
        }
      }
      dft_reg<T, R>(a[u], dir);
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int idx = u * blockDim.x + threadIdx.x;
    if (idx < tot) {
      int b, j, jq, k;
      stage_index(idx, nR, lognR, batch, ns2, ns3, Ns, b, j, jq, k);
      const int od = jq * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[spad(b * bs + (od + r * Ns) * es)] = a[u][r];
    }
  }
  __syncthreads();
}

// In-place FFT of `batch` sequences of length n = 2^la 3^lb held in shared memory; element i of
// sequence b sits at s[b*bs + i*es]. Self-sorting Stockham stages of radix 16 and 8 (then 4 or 2),
// then radix 9 (then 3). tw[k] = e^{-2 pi i k / twlen} over the full circle, n dividing twlen. dir = -1 forward,
// +1 inverse (unnormalised). All threads of the block must call it. Each stage exchanges through
// registers in place, so every thread holds all of its items at once: with VPT = 16 the caller
// must keep batch * n <= 16 * blockDim.x (<= 15 * blockDim.x when lb > 0); with VPT = 8,
// batch * n <= 8 * blockDim.x (<= 6 * blockDim.x when lb > 0).
// R16: radix-16 stages allowed (the 16-value kernels and the X passes; in the 8-value Y
// convolution its sixteen values would raise the register count past what 768-thread blocks hold).
template <typename T, int VPT = 16, bool R16 = (VPT >= 16)>
__device__ void smem_fftn(cplx<T>* s, int n, int la, int lb, int es, int batch, int bs,
                          const cplx<T>* __restrict__ tw, int twlen, int dir) {
  int ns2 = 0, ns3 = 0, rem = la;
  // log2(n / R) for the power-of-two lengths (lb = 0), -1 otherwise
  auto lognR = [&](int logR) { return lb == 0 ? la - logR : -1; };
  // fewest stages: ceil(la / 4) radix-16/8 stages for 2^la (radix 16 where radix 8 would need one
  // more stage), one radix-9 stage per 3^2 (radix 8 then 4 or 2, and radix 3, without R16)
  const int nst = (la + 3) / 4;
  for (int n16 = R16 ? la - 3 * nst : 0; n16 > 0; --n16) {
    stockham_stage<T, 16, StageItems<VPT, 16>::value>(s, n, lognR(4), ns2, ns3, es, batch, bs, tw, twlen, dir);
    ns2 += 4;
    rem -= 4;
  }
  while (rem >= 3) {
    stockham_stage<T, 8, StageItems<VPT, 8>::value>(s, n, lognR(3), ns2, ns3, es, batch, bs, tw, twlen, dir);
    ns2 += 3;
    rem -= 3;
  }
  if (rem == 2) {
    stockham_stage<T, 4, StageItems<VPT, 4>::value>(s, n, lognR(2), ns2, ns3, es, batch, bs, tw, twlen, dir);
    ns2 += 2;
  }
  if (rem == 1) {
    stockham_stage<T, 2, StageItems<VPT, 2>::value>(s, n, lognR(1), ns2, ns3, es, batch, bs, tw, twlen, dir);
    ns2 += 1;
  }
  // radix 9 only where a thread already holds 15 values (the 8-value kernels keep radix 3)
  for (int t = 0; VPT >= 16 && t + 1 < lb; t += 2) {
    stockham_stage<T, 9, StageItems<VPT, 9>::value>(s, n, -1, ns2, ns3, es, batch, bs, tw, twlen, dir);
    ns3 += 2;
  }
  while (ns3 < lb) {
    stockham_stage<T, 3, StageItems<VPT, 3>::value>(s, n, -1, ns2, ns3, es, batch, bs, tw, twlen, dir);
    ns3 += 1;
  }
  if (n == 1) __syncthreads();
}

// Power-of-two length 2^logn with a full-circle table of length 2^twlog.
template <typename T, int VPT = 16>
__device__ void smem_fft(cplx<T>* s, int logn, int es, int batch, int bs, const cplx<T>* __restrict__ tw,
                         int twlog, int dir) {
  smem_fftn<T, VPT, true>(s, 1 << logn, logn, 0, es, batch, bs, tw, 1 << twlog, dir);
}

// FFT along X (the strided dimension) of arrays laid out g[ix * nrow + iy], ix < Px = 2^logPx,
// iy < nrow; block b transforms rows iy in [b*ty, b*ty + ty). blockIdx.y selects the array
// (arrays are nrow*Px apart).
template <typename T, int VPT>
__global__ void k_fft_x(cplx<T>* __restrict__ g, int logPx, int nrow, int ty, long arr_stride,
                        const cplx<T>* __restrict__ tw, int twlog, int dir) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* s = reinterpret_cast<cplx<T>*>(smem_raw);
  const int Px = 1 << logPx;
  cplx<T>* tws = s + splen(Px * ty);  // twiddles of this length, staged once per block
  cplx<T>* a = g + blockIdx.y * arr_stride;
  const int iy0 = blockIdx.x * ty;
  const int tot = Px * ty;  // <= VPT * blockDim.x (launch rule), as is Px
  // every global load of the thread (tile element s[ix * ty + t] = s[idx], and twiddles) is
  // issued before any shared-memory store, so their latencies overlap
  constexpr int C = VPT < 8 ? VPT : 8;  // values staged per round (bounds the registers)
#pragma unroll
  for (int base = 0; base < VPT; base += C) {
    cplx<T> v[C], tv[C];
#pragma unroll
    for (int r = 0; r < C; ++r) {
      const int idx = threadIdx.x + (base + r) * blockDim.x;
      v[r] = cplx<T>(0, 0);
      if (idx < tot) {
        const int iy = iy0 + idx % ty;
        if (iy < nrow) v[r] = a[(long)(idx / ty) * nrow + iy];
      }
      if (idx < Px) tv[r] = tw[idx << (twlog - logPx)];
    }
#pragma unroll
    for (int r = 0; r < C; ++r) {
      const int idx = threadIdx.x + (base + r) * blockDim.x;
      if (idx < tot) s[spad(idx)] = v[r];
      if (idx < Px) tws[idx] = tv[r];
    }
  }
  __syncthreads();
  smem_fft<T, VPT>(s, logPx, ty, ty, 1, tws, logPx, dir);
  for (int idx = threadIdx.x; idx < Px * ty; idx += blockDim.x) {
    int t = idx % ty, ix = idx / ty;
    int iy = iy0 + t;
    if (iy < nrow) a[(long)ix * nrow + iy] = s[spad(ix * ty + t)];
  }
}

// FFT along Y (contiguous) of rows g[kx * Py + ...], Py = 2^la 3^lb, in place, one block per kx;
// twy: full-circle table of length Py.
template <typename T>
__global__ void __launch_bounds__(1024) k_fft_y_full(cplx<T>* __restrict__ g, int Py, int la, int lb, const cplx<T>* __restrict__ twy,
                             int dir) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* s = reinterpret_cast<cplx<T>*>(smem_raw);
  cplx<T>* a = g + (long)blockIdx.x * Py;
  for (int i = threadIdx.x; i < Py; i += blockDim.x) s[spad(i)] = a[i];
  __syncthreads();
  smem_fftn<T>(s, Py, la, lb, 1, 1, 0, twy, Py, dir);
  for (int i = threadIdx.x; i < Py; i += blockDim.x) a[i] = s[spad(i)];
}

// Y-direction convolution of one X-frequency column (one block per kx):
//   phi^(kx) = IFFT_y( Km^(kx) . FFT_y(xi^(kx)) + Kd^(kx) . FFT_y(zeta^(kx)) )
// xi, zeta hold nrow rows (zero padded to Py here); the first nrow outputs overwrite xi.
// K* hold the Py-point spectra per kx, already scaled by 1/(Px Py).
// Asynchronous global -> shared copy of one element (8 or 16 bytes; cp.async, sm_80 and later) and
// the wait for all of this thread's outstanding copies.
template <typename T>
__device__ __forceinline__ void cp_async_elem(cplx<T>* dst_smem, const cplx<T>* src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  if (sizeof(cplx<T>) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// MAXR values per thread (the FFT stages' and the registers' share of the column). ACCG: the
// partial product K_m FFT(xi) waits in a global scratch column (when shared memory cannot hold a
// twiddle table next to the column and registers cannot hold the product next to the FFT's own
// values); otherwise it stays in registers and the twiddles are staged in shared memory. With
// MAXR = 8 (PF) every global read is issued up front: the spectra K_m, K_d go to registers and the
// zeta column to a second shared buffer by asynchronous copies, both in flight during the first
// transform.
// blockIdx.y selects a column set (several densities at once): its grids are gstride apart, its
// spectra kstride apart (0: shared), its scratch columns Px Py apart.
template <typename T, int MAXR, bool ACCG>
__global__ void k_conv_y(cplx<T>* __restrict__ xi, const cplx<T>* __restrict__ zeta,
                         const cplx<T>* __restrict__ Km, const cplx<T>* __restrict__ Kd, int Py, int la, int lb,
                         int nrow, const cplx<T>* __restrict__ twy, cplx<T>* __restrict__ accg, long gstride,
                         long kstride) {
  constexpr bool PF = !ACCG && MAXR <= 8;
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* s = reinterpret_cast<cplx<T>*>(smem_raw);
  const long kx = blockIdx.x;
  cplx<T> acc[ACCG ? 1 : MAXR];
  cplx<T> pkm[PF ? MAXR : 1], pkd[PF ? MAXR : 1];
  const long cs = blockIdx.y;
  cplx<T>* col = xi + cs * gstride + kx * nrow;
  const cplx<T>* colz = zeta + cs * gstride + kx * nrow;
  const cplx<T>* km = Km + cs * kstride + kx * Py;
  const cplx<T>* kd = Kd + cs * kstride + kx * Py;
  cplx<T>* ag = ACCG ? accg + (cs * gridDim.x + kx) * Py : nullptr;
  cplx<T>* s2 = s + splen(Py) + Py;  // PF: the zeta column (after the twiddle table)
  if (PF) {
    for (int i = threadIdx.x; i < Py; i += blockDim.x) {
      if (i < nrow)
        cp_async_elem(s2 + spad(i), colz + i);
      else
        s2[spad(i)] = cplx<T>(0, 0);
    }
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      int i = threadIdx.x + r * blockDim.x;
      if (i < Py) {
        pkm[PF ? r : 0] = km[i];
        pkd[PF ? r : 0] = kd[i];
      }
    }
  }
  const cplx<T>* twf = twy;
  if (ACCG) {
    for (int i = threadIdx.x; i < Py; i += blockDim.x) s[spad(i)] = (i < nrow) ? col[i] : cplx<T>(0, 0);
  } else {
    // column and twiddle loads all issued before the shared-memory stores (Py <= MAXR * blockDim.x)
    cplx<T>* tws = s + splen(Py);
    constexpr int C = MAXR < 8 ? MAXR : 8;  // values staged per round (bounds the registers)
#pragma unroll
    for (int base = 0; base < MAXR; base += C) {
      cplx<T> v[C], tv[C];
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const int i = threadIdx.x + (base + r) * blockDim.x;
        if (i < Py) {
          v[r] = i < nrow ? col[i] : cplx<T>(0, 0);
          tv[r] = twy[i];
        }
      }
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const int i = threadIdx.x + (base + r) * blockDim.x;
        if (i < Py) {
          s[spad(i)] = v[r];
          tws[i] = tv[r];
        }
      }
    }
    twf = tws;
  }
  __syncthreads();
  smem_fftn<T, MAXR>(s, Py, la, lb, 1, 1, 0, twf, Py, -1);
  if (ACCG) {
    for (int i = threadIdx.x; i < Py; i += blockDim.x) ag[i] = s[spad(i)] * km[i];
  } else {
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      int i = threadIdx.x + r * blockDim.x;
      if (i < Py) acc[ACCG ? 0 : r] = s[spad(i)] * (PF ? pkm[PF ? r : 0] : km[i]);
    }
  }
  cplx<T>* sz = s;
  if (PF) {
    cp_async_commit_wait_all();
    sz = s2;
  } else {
    __syncthreads();
    for (int i = threadIdx.x; i < Py; i += blockDim.x) s[spad(i)] = (i < nrow) ? colz[i] : cplx<T>(0, 0);
  }
  __syncthreads();
  smem_fftn<T, MAXR>(sz, Py, la, lb, 1, 1, 0, twf, Py, -1);
  if (ACCG) {
    for (int i = threadIdx.x; i < Py; i += blockDim.x) sz[spad(i)] = sz[spad(i)] * kd[i] + ag[i];
  } else {
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      int i = threadIdx.x + r * blockDim.x;
      if (i < Py) sz[spad(i)] = sz[spad(i)] * (PF ? pkd[PF ? r : 0] : kd[i]) + acc[ACCG ? 0 : r];
    }
  }
  __syncthreads();
  smem_fftn<T, MAXR>(sz, Py, la, lb, 1, 1, 0, twf, Py, +1);
  for (int i = threadIdx.x; i < nrow; i += blockDim.x) col[i] = sz[spad(i)];
}

// Adjoint of k_conv_y (one block per kx). The forward column map is xi, zeta -> restrict(IFFT(Km
// FFT(pad xi) + Kd FFT(pad zeta))), with the inverse transform unnormalised and 1/(Px Py) inside K*;
// its adjoint takes phi (in xi, nrow rows) to
//   xi   <- restrict(IFFT(conj(Km) . FFT(pad phi))),   zeta <- restrict(IFFT(conj(Kd) . FFT(pad phi)))
// (the adjoint of zero padding is restriction and the adjoint of the unnormalised inverse DFT is
// the forward DFT). FFT(pad phi) waits in registers, or in the global scratch column accg when
// ACCG, between the two inverse transforms.
template <typename T, int MAXR, bool ACCG>
__global__ void k_conv_y_adj(cplx<T>* __restrict__ xi, cplx<T>* __restrict__ zeta,
                             const cplx<T>* __restrict__ Km, const cplx<T>* __restrict__ Kd, int Py, int la, int lb,
                             int nrow, const cplx<T>* __restrict__ twy, cplx<T>* __restrict__ accg, long gstride,
                             long kstride) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* s = reinterpret_cast<cplx<T>*>(smem_raw);
  const long kx = blockIdx.x;
  cplx<T> acc[ACCG ? 1 : MAXR];
  const cplx<T>* twf = twy;
  if (!ACCG) {
    cplx<T>* tws = s + splen(Py);
    for (int i = threadIdx.x; i < Py; i += blockDim.x) tws[i] = twy[i];
    twf = tws;
  }
  const long cs = blockIdx.y;
  cplx<T>* col = xi + cs * gstride + kx * nrow;
  cplx<T>* colz = zeta + cs * gstride + kx * nrow;
  const cplx<T>* km = Km + cs * kstride + kx * Py;
  const cplx<T>* kd = Kd + cs * kstride + kx * Py;
  cplx<T>* ag = ACCG ? accg + (cs * gridDim.x + kx) * Py : nullptr;
  for (int i = threadIdx.x; i < Py; i += blockDim.x) s[spad(i)] = (i < nrow) ? col[i] : cplx<T>(0, 0);
  __syncthreads();
  smem_fftn<T, MAXR>(s, Py, la, lb, 1, 1, 0, twf, Py, -1);
  if (ACCG) {
    for (int i = threadIdx.x; i < Py; i += blockDim.x) {
      cplx<T> v = s[spad(i)];
      ag[i] = v;
      s[spad(i)] = mulc(v, km[i]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      int i = threadIdx.x + r * blockDim.x;
      if (i < Py) {
        acc[ACCG ? 0 : r] = s[spad(i)];
        s[spad(i)] = mulc(acc[ACCG ? 0 : r], km[i]);
      }
    }
  }
  __syncthreads();
  smem_fftn<T, MAXR>(s, Py, la, lb, 1, 1, 0, twf, Py, +1);
  for (int i = threadIdx.x; i < nrow; i += blockDim.x) col[i] = s[spad(i)];
  __syncthreads();
  if (ACCG) {
    for (int i = threadIdx.x; i < Py; i += blockDim.x) s[spad(i)] = mulc(ag[i], kd[i]);
  } else {
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      int i = threadIdx.x + r * blockDim.x;
      if (i < Py) s[spad(i)] = mulc(acc[ACCG ? 0 : r], kd[i]);
    }
  }
  __syncthreads();
  smem_fftn<T, MAXR>(s, Py, la, lb, 1, 1, 0, twf, Py, +1);
  for (int i = threadIdx.x; i < nrow; i += blockDim.x) colz[i] = s[spad(i)];
}
