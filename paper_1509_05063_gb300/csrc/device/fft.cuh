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

}  // namespace lsd
