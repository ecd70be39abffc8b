// Shared-memory Stockham FFT used by the 2-D lattice convolution
// (device/kernels.cu) and the 3-D one (device/apply3.cu).
#pragma once
#include "cplx.cuh"

namespace lsd {

// In-place radix-4 (plus one radix-2 stage when log2 N is odd) Stockham
// autosort transform of one length-N sequence held in shared memory, run by
// G = N / 8 threads of the block (thread t): 2 radix-4 butterflies or 4
// radix-2 butterflies per thread and stage.  Every stage reads all inputs to
// registers, synchronises the block, then writes, so one buffer suffices.
// tw[m * tws] = exp(-2 pi i m / N) (tws > 1: a sub-length transform on a
// longer table); the inverse uses conjugate twiddles (no scaling).  Threads
// with active == false only take part in the block barriers (every thread of
// the block must call with the same N).
template <typename T>
__device__ void fft_smem(T* x, int N, int logN, bool inv, const T* __restrict__ tw, int t, int tws = 1,
                         bool active = true) {
  const int G = N / 8;
  int Ns = 1;
  if (logN & 1) {
    T a[8];
    if (active) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = t + c * G;
        a[2 * c] = x[j];
        a[2 * c + 1] = x[j + N / 2];
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = t + c * G;
        x[2 * j] = cadd(a[2 * c], a[2 * c + 1]);
        x[2 * j + 1] = csub(a[2 * c], a[2 * c + 1]);
      }
    }
    __syncthreads();
    Ns = 2;
  }
  for (; Ns < N; Ns *= 4) {
    T v[2][4];
    const int tstep = N / (4 * Ns) * tws;
    if (active) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int j = t + c * G;
        const int k = j & (Ns - 1);
#pragma unroll
        for (int r = 0; r < 4; ++r) v[c][r] = x[j + r * (N / 4)];
        if (Ns > 1) {
#pragma unroll
          for (int r = 1; r < 4; ++r) {
            T w = tw[r * k * tstep];
            if (inv) w = cconj(w);
            v[c][r] = cmul(v[c][r], w);
          }
        }
        const T s02 = cadd(v[c][0], v[c][2]), d02 = csub(v[c][0], v[c][2]);
        const T s13 = cadd(v[c][1], v[c][3]), d13 = csub(v[c][1], v[c][3]);
        const T rot = inv ? cmul_i(d13) : cmul_mi(d13);   // (-i or +i) (v1 - v3)
        v[c][0] = cadd(s02, s13);
        v[c][2] = csub(s02, s13);
        v[c][1] = cadd(d02, rot);
        v[c][3] = csub(d02, rot);
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int j = t + c * G;
        const int k = j & (Ns - 1);
        const int base = (j - k) * 4 + k;
#pragma unroll
        for (int r = 0; r < 4; ++r) x[base + r * Ns] = v[c][r];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ radix-16 Stockham transform
// Length N = 256, 512, 1024 or 2048 held in shared memory in a padded layout
// (element i at fpad(i) = i + i / 16, so that a thread's 16 consecutive
// outputs of the first pass do not fall on one bank), run by G = N / 16
// threads (thread t): two radix-16 passes with the 16 values of a butterfly in
// registers (a 16-point DFT as 4 x 4), then one pass of radix N / 256 (2, 4 or
// 8) that writes back where it read.  Five block barriers for N > 256, against
// ten for the radix-4 transform of N = 1024.  Same table and conventions as
// fft_smem (tw[m * tws] = exp(-2 pi i m / N), inverse unscaled); the caller
// synchronises before reading the result.
__device__ __forceinline__ int fpad(int i) { return i + (i >> 4); }

namespace fft16_detail {

template <typename T>
__device__ __forceinline__ void dft2(T& a, T& b) {
  const T s = cadd(a, b);
  b = csub(a, b);
  a = s;
}

// natural order in and out; forward uses exp(-2 pi i / 4) = -i
template <typename T, bool INV>
__device__ __forceinline__ void dft4(T& a0, T& a1, T& a2, T& a3) {
  const T s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
  const T rot = INV ? cmul_i(d13) : cmul_mi(d13);
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, rot);
  a3 = csub(d02, rot);
}

// exp(-+2 pi i m / 16) for the m = n2 k1 of the 4 x 4 split (0 <= n2, k1 < 4)
template <typename T, bool INV>
__device__ __forceinline__ T w16(T v, int m) {
  using R = decltype(v.x);
  const R c = R(0.92387953251128675613), sn = R(0.38268343236508977173), h = R(0.70710678118654752440);
  R re, im;                                     // forward value of exp(-2 pi i m / 16)
  switch (m) {
    case 1: re = c; im = -sn; break;
    case 2: re = h; im = -h; break;
    case 3: re = sn; im = -c; break;
    case 4: re = 0; im = -1; break;
    case 6: re = -h; im = -h; break;
    default: re = -c; im = sn; break;        // m = 9
  }
  if (INV) im = -im;
  return mk(v.x * re - v.y * im, v.x * im + v.y * re);
}

// 16-point DFT, natural order in and out: n = 4 n1 + n2, k = k1 + 4 k2
template <typename T, bool INV>
__device__ __forceinline__ void dft16(T (&v)[16]) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<T, INV>(v[n2], v[4 + n2], v[8 + n2], v[12 + n2]);   // over n1 -> k1
#pragma unroll
  for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) v[4 * k1 + n2] = w16<T, INV>(v[4 * k1 + n2], n2 * k1);
  // a[n2][k1] sits at v[4 k1 + n2]; the DFT over n2 gives X[k1 + 4 k2]
  T o[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    T b0 = v[4 * k1], b1 = v[4 * k1 + 1], b2 = v[4 * k1 + 2], b3 = v[4 * k1 + 3];
    dft4<T, INV>(b0, b1, b2, b3);
    o[k1] = b0;
    o[k1 + 4] = b1;
    o[k1 + 8] = b2;
    o[k1 + 12] = b3;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = o[i];
}

// 8-point DFT, natural order: n = 2 n1 + n2, k = k1 + 4 k2
template <typename T, bool INV>
__device__ __forceinline__ void dft8(T (&v)[8]) {
  using R = decltype(v[0].x);
  const R h = R(0.70710678118654752440);
  dft4<T, INV>(v[0], v[2], v[4], v[6]);        // n2 = 0: k1 at v[2 k1]
  dft4<T, INV>(v[1], v[3], v[5], v[7]);        // n2 = 1: k1 at v[2 k1 + 1]
  // twiddles exp(-+2 pi i k1 / 8) on the n2 = 1 values
  const R sg = INV ? R(1) : R(-1);
  v[3] = mk(h * (v[3].x - sg * v[3].y), h * (v[3].y + sg * v[3].x));
  v[5] = INV ? cmul_i(v[5]) : cmul_mi(v[5]);
  v[7] = mk(h * (-v[7].x - sg * v[7].y), h * (-v[7].y + sg * v[7].x));
  T o[8];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    T a = v[2 * k1], b = v[2 * k1 + 1];
    dft2(a, b);
    o[k1] = a;
    o[k1 + 4] = b;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = o[i];
}

template <typename T, bool INV>
__device__ __forceinline__ T twiddle(const T* __restrict__ tw, int idx) {
  const T w = tw[idx];
  return INV ? cconj(w) : w;
}

// the last pass, radix RAD = N / 256 with Ns = 256: butterfly j < 256 reads and
// writes x[j + 256 q]; thread t takes j = t + m G (m < 16 / RAD)
template <typename T, bool INV, int RAD>
__device__ __forceinline__ void last_pass(T* x, int G, const T* __restrict__ tw, int tws, int t) {
#pragma unroll
  for (int m = 0; m < 16 / RAD; ++m) {
    const int j = t + m * G;
    T v[RAD];
#pragma unroll
    for (int q = 0; q < RAD; ++q) v[q] = x[fpad(j + 256 * q)];
#pragma unroll
    for (int q = 1; q < RAD; ++q) v[q] = cmul(v[q], twiddle<T, INV>(tw, q * j * tws));
    if constexpr (RAD == 2) {
      dft2(v[0], v[1]);
    } else if constexpr (RAD == 4) {
      dft4<T, INV>(v[0], v[1], v[2], v[3]);
    } else {
      dft8<T, INV>(v);
    }
#pragma unroll
    for (int q = 0; q < RAD; ++q) x[fpad(j + 256 * q)] = v[q];
  }
}

template <typename T, bool INV>
__device__ void fft16_run(T* x, int N, const T* __restrict__ tw, int t, int tws, bool active) {
  const int G = N >> 4;
  T v[16];
  // pass 1: radix 16, Ns = 1 (no twiddles): y[16 j + q] = DFT16 of x[j + G q]
  if (active) {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = x[fpad(t + G * q)];
    dft16<T, INV>(v);
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int q = 0; q < 16; ++q) x[fpad(16 * t + q)] = v[q];
  }
  __syncthreads();
  // pass 2: radix 16, Ns = 16: twiddles exp(-+2 pi i q k / 256), k = j mod 16
  const int k = t & 15;
  if (active) {
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = x[fpad(t + G * q)];
    const int step = k * (N >> 8) * tws;
#pragma unroll
    for (int q = 1; q < 16; ++q) v[q] = cmul(v[q], twiddle<T, INV>(tw, q * step));
    dft16<T, INV>(v);
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int q = 0; q < 16; ++q) x[fpad(16 * (t - k) + k + 16 * q)] = v[q];
  }
  if (N == 256) return;
  __syncthreads();
  // pass 3: radix N / 256, in place
  if (active) {
    if (N == 512) last_pass<T, INV, 2>(x, G, tw, tws, t);
    else if (N == 1024) last_pass<T, INV, 4>(x, G, tw, tws, t);
    else last_pass<T, INV, 8>(x, G, tw, tws, t);
  }
}

}  // namespace fft16_detail

// Every thread of the block calls with the same N (256 .. 2048, a power of two);
// threads with active == false only take part in the barriers.  x holds
// fpad(N - 1) + 1 elements.
template <typename T>
__device__ __forceinline__ void fft16_smem(T* x, int N, bool inv, const T* __restrict__ tw, int t, int tws = 1,
                                           bool active = true) {
  if (inv) fft16_detail::fft16_run<T, true>(x, N, tw, t, tws, active);
  else fft16_detail::fft16_run<T, false>(x, N, tw, t, tws, active);
}

// elements of a padded transform buffer of length N
__host__ __device__ constexpr int fft16_len(int N) { return N + N / 16; }

}  // namespace lsd
