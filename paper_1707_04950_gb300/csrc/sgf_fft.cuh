// Shared-memory radix-2 FFT used by the global convolution of the accelerated operator
// (Bruno & Maas, eq. large_convolution_per_grid: cyclic in X after the quasi-periodic twist,
// linear in Y with zero padding).
#pragma once
#include "sgf_common.cuh"

// In-place radix-2 decimation-in-time FFT of `batch` sequences of length n = 2^logn held in shared
// memory; element i of sequence b sits at s[b*bs + i*es]. tw[k] = e^{-2 pi i k / 2^twlog},
// k < 2^(twlog-1). dir = -1 forward (e^{-2 pi i}), +1 inverse (unnormalised). Must be called by all
// threads of the block; ends with __syncthreads().
template <typename T>
__device__ void smem_fft(cplx<T>* s, int logn, int es, int batch, int bs, const cplx<T>* __restrict__ tw,
                         int twlog, int dir) {
  const int n = 1 << logn;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < batch * n; idx += nt) {
    int b = idx >> logn, i = idx & (n - 1);
    int r = (int)(__brev((unsigned)i) >> (32 - logn));
    if (r > i) {
      cplx<T> t = s[b * bs + i * es];
      s[b * bs + i * es] = s[b * bs + r * es];
      s[b * bs + r * es] = t;
    }
  }
  __syncthreads();
  const int halfn = n >> 1;
  for (int st = 1; st <= logn; ++st) {
    const int half = 1 << (st - 1);
    for (int idx = tid; idx < batch * halfn; idx += nt) {
      int b = idx / halfn, kk = idx - b * halfn;
      int j = kk & (half - 1);
      int i0 = ((kk >> (st - 1)) << st) + j;
      int i1 = i0 + half;
      cplx<T> w = tw[j << (twlog - st)];
      if (dir > 0) w.im = -w.im;
      cplx<T> a = s[b * bs + i0 * es];
      cplx<T> c = s[b * bs + i1 * es] * w;
      s[b * bs + i0 * es] = a + c;
      s[b * bs + i1 * es] = a - c;
    }
    __syncthreads();
  }
}

// FFT along X (the strided dimension) of arrays laid out g[ix * nrow + iy], ix < Px = 2^logPx,
// iy < nrow; block b transforms rows iy in [b*ty, b*ty + ty). blockIdx.y selects the array
// (arrays are nrow*Px apart).
template <typename T>
__global__ void k_fft_x(cplx<T>* __restrict__ g, int logPx, int nrow, int ty, long arr_stride,
                        const cplx<T>* __restrict__ tw, int twlog, int dir) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* s = reinterpret_cast<cplx<T>*>(smem_raw);
  const int Px = 1 << logPx;
  cplx<T>* a = g + blockIdx.y * arr_stride;
  const int iy0 = blockIdx.x * ty;
  for (int idx = threadIdx.x; idx < Px * ty; idx += blockDim.x) {
    int t = idx % ty, ix = idx / ty;
    int iy = iy0 + t;
    s[ix * ty + t] = (iy < nrow) ? a[(long)ix * nrow + iy] : cplx<T>(0, 0);
  }
  __syncthreads();
  smem_fft<T>(s, logPx, ty, ty, 1, tw, twlog, dir);
  for (int idx = threadIdx.x; idx < Px * ty; idx += blockDim.x) {
    int t = idx % ty, ix = idx / ty;
    int iy = iy0 + t;
    if (iy < nrow) a[(long)ix * nrow + iy] = s[ix * ty + t];
  }
}

// Forward FFT along Y (contiguous) of rows g[kx * Py + ...], in place, one block per kx.
template <typename T>
__global__ void k_fft_y_full(cplx<T>* __restrict__ g, int logPy, const cplx<T>* __restrict__ tw, int twlog,
                             int dir) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* s = reinterpret_cast<cplx<T>*>(smem_raw);
  const int Py = 1 << logPy;
  cplx<T>* a = g + (long)blockIdx.x * Py;
  for (int i = threadIdx.x; i < Py; i += blockDim.x) s[i] = a[i];
  __syncthreads();
  smem_fft<T>(s, logPy, 1, 1, 0, tw, twlog, dir);
  for (int i = threadIdx.x; i < Py; i += blockDim.x) a[i] = s[i];
}

// Y-direction convolution of one X-frequency column (one block per kx):
//   phi^(kx) = IFFT_y( Km^(kx) . FFT_y(xi^(kx)) + Kd^(kx) . FFT_y(zeta^(kx)) )
// xi, zeta hold nrow rows (zero padded to Py here); the first nrow outputs overwrite xi.
// K* hold the Py-point spectra per kx, already scaled by 1/(Px Py).
template <typename T, int MAXR>
__global__ void k_conv_y(cplx<T>* __restrict__ xi, const cplx<T>* __restrict__ zeta,
                         const cplx<T>* __restrict__ Km, const cplx<T>* __restrict__ Kd, int logPy, int nrow,
                         const cplx<T>* __restrict__ tw, int twlog) {
  extern __shared__ unsigned char smem_raw[];
  cplx<T>* s = reinterpret_cast<cplx<T>*>(smem_raw);
  const int Py = 1 << logPy;
  const long kx = blockIdx.x;
  cplx<T> acc[MAXR];
  cplx<T>* col = xi + kx * nrow;
  const cplx<T>* colz = zeta + kx * nrow;
  const cplx<T>* km = Km + kx * Py;
  const cplx<T>* kd = Kd + kx * Py;
  for (int i = threadIdx.x; i < Py; i += blockDim.x) s[i] = (i < nrow) ? col[i] : cplx<T>(0, 0);
  __syncthreads();
  smem_fft<T>(s, logPy, 1, 1, 0, tw, twlog, -1);
#pragma unroll
  for (int r = 0; r < MAXR; ++r) {
    int i = threadIdx.x + r * blockDim.x;
    if (i < Py) acc[r] = s[i] * km[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < Py; i += blockDim.x) s[i] = (i < nrow) ? colz[i] : cplx<T>(0, 0);
  __syncthreads();
  smem_fft<T>(s, logPy, 1, 1, 0, tw, twlog, -1);
#pragma unroll
  for (int r = 0; r < MAXR; ++r) {
    int i = threadIdx.x + r * blockDim.x;
    if (i < Py) s[i] = s[i] * kd[i] + acc[r];
  }
  __syncthreads();
  smem_fft<T>(s, logPy, 1, 1, 0, tw, twlog, +1);
  for (int i = threadIdx.x; i < nrow; i += blockDim.x) col[i] = s[i];
}
