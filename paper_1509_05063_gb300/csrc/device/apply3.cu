// sm_103a kernels of the 3-D apply (Section 5: the Section 3.2 accelerator on
// cube cells, with a 3-D lattice FFT, plus the stored adjacent part).  One
// template per arithmetic precision: T = double2 (complex128) or float2
// (complex64 inner path of mixed precision).
//
//   k3_project    sigma_c = P_c u_c                      (two-face equivalent sources)
//   k3_fill       sigma -> monopole / dipole values on the x1-face planes of the lattice
//   k3_fft_axis   batched line FFTs along one axis of the M^3 lattice, over the
//                 box of lines that can be nonzero (forward) or are read (inverse)
//   k3_conv_a     the a-axis stage: forward lines of both arrays, V^ = S_m^ G^ + S_d^ D^,
//                 inverse line, in one pass (k3_spectral when M > 1024)
//   k3_gather, k3_gemm (FP64) or k3_gemm_df (double-float, complex64 apply), k3_reduce
//                 gamma_c = B^+ V_c - sum_o (B^+ T_o) sigma_{c+o}   (27 neighbours; one GEMM over cells)
//   k3_near       out_q = u_q + kappa^2 (sum_l W_ql u_l + Phi_q . gamma_c): FP64 from a CSR in
//                 three-multiplication form, complex64 from dense per-cell blocks over the
//                 27 neighbour cells' nodes plus a CSR remainder
// The complex64 apply runs the projection, the adjacent part and the
// evaluation in complex64, the lattice convolution in FP64 and the local
// coefficients in double-float (ApplyData3::lattice64 says why).
#include <algorithm>
#include <cstdint>

#include "cplx.cuh"
#include "fft.cuh"
#include "kernels.cuh"

namespace lsd {
namespace {

constexpr int kT3 = 256;

// sigma_c = P_c u_c: block = occupied cell, 1024 threads = output rows
// i < n_es (a pass of up to 1024 rows at a time) x S = 1024 / rows segments
// of the cell's nodes (node j in segment j mod S); the cell's inputs staged in
// shared memory 1024 at a time, P_c read [node][i] (consecutive threads,
// consecutive entries), the S partial sums added in segment order.  FP64:
// also writes the staged input (c, c + d, d - c) of the adjacent part for the
// cell's nodes.
constexpr int kTP = 1024;
template <typename T>
__global__ void __launch_bounds__(kTP) k3_project(ApplyData3<T> d, const T* __restrict__ u) {
  __shared__ T us[kTP];
  __shared__ T ps[kTP];
  const int k = blockIdx.x, t = threadIdx.x;
  const int64_t s0 = d.occ_start[k];
  const int nc = int(d.occ_start[k + 1] - s0);
  const T* P = d.P + d.P_off[k];
  const int ni = d.n_es < kTP ? d.n_es : kTP, S = kTP / ni;
  const int il = t % ni, sg = t / ni;
  for (int i0 = 0; i0 < d.n_es; i0 += ni) {
    const int i = i0 + il;
    T acc = czero(T());
    for (int j0 = 0; j0 < nc; j0 += kTP) {
      const int nj = nc - j0 < kTP ? nc - j0 : kTP;
      __syncthreads();
      if (t < nj) {
        const T v = u[s0 + j0 + t];
        us[t] = v;
        if constexpr (sizeof(T) == 16)
          if (i0 == 0) {                 // the staged input of the FP64 adjacent part
            double* w = d.u3 + 3 * (s0 + j0 + t);
            w[0] = v.x;
            w[1] = v.x + v.y;
            w[2] = v.y - v.x;
          }
      }
      __syncthreads();
      if (sg < S && i < d.n_es)
        for (int j = sg; j < nj; j += S) acc = cfma(P[int64_t(j0 + j) * d.n_es + i], us[j], acc);
    }
    ps[t] = acc;
    __syncthreads();
    if (t < ni && i < d.n_es) {
      T v = ps[t];
      for (int q = 1; q < S; ++q) v = cadd(v, ps[q * ni + t]);
      d.sigma[int64_t(k) * d.n_es + i] = v;
    }
    __syncthreads();
  }
}

// lattice sources: element (a, b, c) of the M^3 arrays ([a][b][c], c fastest)
// gathers, in a fixed order, the equivalent sources of every occupied cell
// that has this lattice point on one of its two x1-faces (up to 2 x 2 x 2
// cells share a point); zero elsewhere
template <typename T>
__global__ void __launch_bounds__(kT3) k3_fill(ApplyData3<T> d) {
  const int64_t MM = int64_t(d.M) * d.M, total = MM * d.M;
  const int Ne = d.Ne, L = d.L, nl = L * Ne, nf = (Ne + 1) * (Ne + 1);
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int a = int(e / MM), b = int((e / d.M) % d.M), c = int(e % d.M);
    T sm = czero(T()), sd = czero(T());
    if (a <= nl && b <= nl && c <= nl && a % Ne == 0) {
      const int fa = a / Ne;
      for (int da = 0; da < 2; ++da) {                 // face x1 = H of cell fa - 1, face x1 = 0 of cell fa
        const int ci = fa - 1 + da;
        if (ci < 0 || ci >= L) continue;
        const int face = 1 - da;
        for (int db = 0; db < 2; ++db) {
          const int cj = b / Ne - db;
          if (cj < 0 || cj >= L || (db == 1 && b % Ne != 0)) continue;
          for (int dc = 0; dc < 2; ++dc) {
            const int ck = c / Ne - dc;
            if (ck < 0 || ck >= L || (dc == 1 && c % Ne != 0)) continue;
            const int occ = d.occ_of_cell[(ck * L + cj) * L + ci];
            if (occ < 0) continue;
            const int lb = b - cj * Ne, lc = c - ck * Ne;
            const T* sg = d.sigma + int64_t(occ) * d.n_es;
            const int idx = face * nf + lb * (Ne + 1) + lc;
            sm = cadd(sm, sg[idx]);
            sd = cadd(sd, sg[2 * nf + idx]);
          }
        }
      }
    }
    d.Sm[e] = sm;
    d.Sd[e] = sd;
  }
}

// line transforms along one axis of an M^3 array ([a][b][c], c fastest) over
// a box of lines: line j = o n_in + i (o < n_out, i < n_in) has outer
// coordinate o ostep and inner coordinate i, where (outer, inner) is (a, b)
// for the c axis (axis 2), (a, c) for the b axis (1) and (b, c) for the a
// axis (0).  A block takes LPB = blockDim.x / (M / 8) consecutive lines of the
// box, M / 8 threads per line, lines padded to M + 1 in shared memory (LPB is
// chosen per launch so that the lines spread over every SM: in FP64 a line
// transform costs an SM's pipe about 700 cycles); loads and stores
// run along c (within a line for axis 2, across consecutive lines otherwise),
// so that they coalesce.  Lines outside the box are not touched: the lattice
// convolution skips the lines it knows to be zero on input or unread later.
struct LineBox {
  int axis, n_out, ostep, n_in;
};

// address of element e of line lj of the box (lines fewer than 2^31)
__device__ __forceinline__ int64_t line_addr(const LineBox& bx, int logM, int lj, int e) {
  const int64_t o = int64_t(lj / bx.n_in) * bx.ostep, i = lj % bx.n_in;
  if (bx.axis == 2) return (o << (2 * logM)) + (i << logM) + e;
  if (bx.axis == 1) return (o << (2 * logM)) + (int64_t(e) << logM) + i;
  return (o << logM) + i + (int64_t(e) << (2 * logM));
}

// Every thread moves exactly M / G = 8 elements of the block's lines
// (LPB lines x M elements over LPB G threads); the eight loads of a thread are
// issued together before any is used.
constexpr int kLineEl = 8;

template <typename T>
__global__ void __launch_bounds__(kT3) k3_fft_axis(T* __restrict__ X0, T* __restrict__ X1, int M, int logM,
                                                  const T* __restrict__ tw, bool inv, LineBox bx) {
  T* __restrict__ X = blockIdx.y == 0 ? X0 : X1;     // the same pass over one or two arrays
  extern __shared__ __align__(16) unsigned char raw3[];
  T* s = reinterpret_cast<T*>(raw3);
  const int G = M / 8, nt = blockDim.x, LPB = nt / G, lg = __ffs(LPB) - 1, t = threadIdx.x;
  const int l0 = blockIdx.x * LPB, nl = bx.n_out * bx.n_in;
  auto je = [&](int idx, int& j, int& e) {
    if (bx.axis == 2) { j = idx >> logM; e = idx & (M - 1); }
    else { j = idx & (LPB - 1); e = idx >> lg; }
  };
  T v[kLineEl];
#pragma unroll
  for (int q = 0; q < kLineEl; ++q) {
    int j, e;
    je(t + q * nt, j, e);
    v[q] = l0 + j < nl ? X[line_addr(bx, logM, l0 + j, e)] : czero(T());
  }
#pragma unroll
  for (int q = 0; q < kLineEl; ++q) {
    int j, e;
    je(t + q * nt, j, e);
    s[j * (M + 1) + e] = v[q];
  }
  __syncthreads();
  fft_smem<T>(s + (t / G) * (M + 1), M, logM, inv, tw, t % G);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kLineEl; ++q) {
    int j, e;
    je(t + q * nt, j, e);
    if (l0 + j < nl) X[line_addr(bx, logM, l0 + j, e)] = s[j * (M + 1) + e];
  }
}

// the a-axis stage of the lattice convolution in one pass over the (b, c)
// lines: forward transforms of a monopole and a dipole line, V^ = S_m^ G^ +
// S_d^ D^, inverse transform, V written back into Sm for a <= a_max only (the
// later stages read no more).  H = blockDim.x / (M / 4) line pairs per block:
// shared slots [0, H) hold monopole lines, [H, 2H) dipole lines.
template <typename T>
__global__ void __launch_bounds__(kT3) k3_conv_a(T* __restrict__ Sm, const T* __restrict__ Sd,
                                                const T* __restrict__ Gs, const T* __restrict__ Ds, int M,
                                                int logM, const T* __restrict__ tw, int a_max) {
  extern __shared__ __align__(16) unsigned char raw3[];
  T* s = reinterpret_cast<T*>(raw3);
  const int G = M / 8, nt = blockDim.x, LPB = nt / G, H = LPB / 2, lg = __ffs(LPB) - 1, t = threadIdx.x;
  const int64_t l0 = int64_t(blockIdx.x) * H;
  T v[kLineEl];
#pragma unroll
  for (int q = 0; q < kLineEl; ++q) {
    const int idx = t + q * nt, j = idx & (LPB - 1), e = idx >> lg;
    v[q] = (j < H ? Sm : Sd)[l0 + (j % H) + (int64_t(e) << (2 * logM))];
  }
#pragma unroll
  for (int q = 0; q < kLineEl; ++q) {
    const int idx = t + q * nt, j = idx & (LPB - 1), e = idx >> lg;
    s[j * (M + 1) + e] = v[q];
  }
  __syncthreads();
  fft_smem<T>(s + (t / G) * (M + 1), M, logM, false, tw, t % G);
  __syncthreads();
  // H M = nt kLineEl / 2 products: four per thread, the spectra loaded together
  T gs[kLineEl / 2], ds[kLineEl / 2];
#pragma unroll
  for (int q = 0; q < kLineEl / 2; ++q) {
    const int idx = t + q * nt, j = idx % H, e = idx / H;
    const int64_t ad = l0 + j + (int64_t(e) << (2 * logM));
    gs[q] = Gs[ad];
    ds[q] = Ds[ad];
  }
#pragma unroll
  for (int q = 0; q < kLineEl / 2; ++q) {
    const int idx = t + q * nt, j = idx % H, e = idx / H;
    T* w = s + j * (M + 1) + e;
    *w = cfma(w[H * (M + 1)], ds[q], cmul(*w, gs[q]));
  }
  __syncthreads();
  fft_smem<T>(s + (t / G) * (M + 1), M, logM, true, tw, t % G, 1, t / G < H);
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kLineEl / 2; ++q) {
    const int idx = t + q * nt, j = idx % H, e = idx / H;
    if (e <= a_max) Sm[l0 + j + (int64_t(e) << (2 * logM))] = s[j * (M + 1) + e];
  }
}

template <typename T>
__global__ void __launch_bounds__(kT3) k3_spectral(T* __restrict__ Sm, const T* __restrict__ Sd,
                                                  const T* __restrict__ Gs, const T* __restrict__ Ds, int64_t n) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    Sm[e] = cfma(Sd[e], Ds[e], cmul(Sm[e], Gs[e]));
}

// The local coefficients of every cell as one GEMM, gamma (cells x nb) =
// X (cells x K) LA (K x nb), K = (N_eq + 1)^3 + 27 n_es, with X_c = [V at the
// closed cell's lattice points; sigma of the 27 neighbours, offset
// (oi + 1) 9 + (oj + 1) 3 + (ok + 1), zero where there is none].
// k3_gather writes X; k3_gemm multiplies tiles of kGC cells x kGN outputs over
// one of S slices of K (enough blocks to fill the GPU); k3_reduce adds the S
// partial products in slice order.
template <typename T>
__global__ void __launch_bounds__(kT3) k3_gather(ApplyData3<T> d, bool df) {
  const int k = blockIdx.x, t = threadIdx.x, L = d.L, Ne = d.Ne, n1 = Ne + 1;
  const int cell = d.occ_cells[k], ci = cell % L, cj = (cell / L) % L, ck = cell / (L * L);
  const int64_t MM = int64_t(d.M) * d.M;
  const int K = d.n_loc + 27 * d.n_es;
  // FP64 GEMM: X as is; double-float GEMM (FP64 data only): the forms
  // (c, c + d, d - c) of each entry split into FP32 hi + lo, 6 floats
  auto put = [&](int p, T v) {
    if constexpr (sizeof(T) == 16) {
      if (df) {
        const double f[3] = {v.x, v.x + v.y, v.y - v.x};
        float* w = d.X6 + 6 * (int64_t(k) * K + p);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const float hi = float(f[q]);
          w[2 * q] = hi;
          w[2 * q + 1] = float(f[q] - double(hi));
        }
        return;
      }
    }
    d.X[int64_t(k) * K + p] = v;
  };
  for (int p = t; p < d.n_loc; p += kT3) {
    const int la = p / (n1 * n1), lb = (p / n1) % n1, lc = p % n1;
    put(p, d.Sm[int64_t(ci * Ne + la) * MM + int64_t(cj * Ne + lb) * d.M + (ck * Ne + lc)]);
  }
  for (int p = t; p < 27 * d.n_es; p += kT3) {
    const int o = p / d.n_es, l = p % d.n_es;
    const int ni = ci + o / 9 - 1, nj = cj + (o / 3) % 3 - 1, nk = ck + o % 3 - 1;
    T v = czero(T());
    if (ni >= 0 && ni < L && nj >= 0 && nj < L && nk >= 0 && nk < L) {
      const int occ = d.occ_of_cell[(nk * L + nj) * L + ni];
      if (occ >= 0) v = d.sigma[int64_t(occ) * d.n_es + l];
    }
    put(d.n_loc + p, v);
  }
}

constexpr int kGC = 32, kGN = 32, kGK = 16;   // GEMM tile: cells x outputs x K step

// K entries of each of the S slices: whole K steps; S of them cover K
__host__ __device__ inline int slice_len(int K, int S) { return ((K + S - 1) / S + kGK - 1) / kGK * kGK; }

// block (cell tile, output tile, slice s): thread (tc, tn) accumulates cells
// tc, tc + 16 against outputs tn, tn + 16 over its slice of K.  Complex
// products take three real multiplications (Gauss's form): with a + ib an
// entry of LA and c + id one of X, staged as (a, b, a + b) and (c, c + d,
// d - c), P += (a + b) c, Q += b (c + d), S += a (d - c) and the product is
// (P - Q) + i (P + S).  On GB300's FP64 pipe that is 3 FMAs instead of 4.
template <typename R>
struct G3 {
  R a, b, s;
};
template <typename T>
__global__ void __launch_bounds__(kT3) k3_gemm(ApplyData3<T> d, int S) {
  using R = decltype(T().x);
  __shared__ G3<R> xs[kGK][kGC + 1];
  __shared__ G3<R> as[kGK][kGN];
  const int K = d.n_loc + 27 * d.n_es;
  const int c0 = blockIdx.x * kGC, n0 = blockIdx.y * kGN, sl = blockIdx.z;
  const int kper = slice_len(K, S), kb = sl * kper, ke = kb + kper < K ? kb + kper : K;
  const int t = threadIdx.x, tc = t / 16, tn = t % 16;
  R P[2][2], Q[2][2], U[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) P[a][b] = Q[a][b] = U[a][b] = R(0);
  for (int k0 = kb; k0 < ke; k0 += kGK) {
    __syncthreads();
    for (int i = t; i < kGK * kGC; i += kT3) {        // X tile: consecutive threads along K
      const int kk = i % kGK, cc = i / kGK, c = c0 + cc, kg = k0 + kk;
      const T v = (c < d.nocc && kg < ke) ? d.X[int64_t(c) * K + kg] : czero(T());
      xs[kk][cc] = G3<R>{v.x, v.x + v.y, v.y - v.x};
    }
    for (int i = t; i < kGK * kGN; i += kT3) {        // LA tile: consecutive threads along the outputs
      const int kk = i / kGN, nn = i % kGN, n = n0 + nn, kg = k0 + kk;
      const T v = (n < d.nb && kg < ke) ? d.LA[int64_t(kg) * d.nb + n] : czero(T());
      as[kk][nn] = G3<R>{v.x, v.y, v.x + v.y};
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      const G3<R> x[2] = {xs[kk][tc], xs[kk][tc + 16]};
      const G3<R> l[2] = {as[kk][tn], as[kk][tn + 16]};
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          P[a][b] = fma(l[b].s, x[a].a, P[a][b]);     // (a + b) c
          Q[a][b] = fma(l[b].b, x[a].b, Q[a][b]);     // b (c + d)
          U[a][b] = fma(l[b].a, x[a].s, U[a][b]);     // a (d - c)
        }
    }
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int c = c0 + tc + 16 * a, n = n0 + tn + 16 * b;
      if (c < d.nocc && n < d.nb) d.part[(int64_t(sl) * d.nocc + c) * d.nb + n] = mk(P[a][b] - Q[a][b], P[a][b] + U[a][b]);
    }
}

// The same GEMM for the complex64 apply in double-float arithmetic on the
// FP32 pipe (GB300 issues 64 FP32 operations per FP64 FMA).  The local step
// subtracts large, nearly equal terms, so its sums need about FP64 accuracy:
// each complex product takes Gauss's three real products of the forms above,
// every form split into FP32 hi + lo, and each real sum is a compensated dot
// product (Ogita, Rump and Oishi's Dot2): the leading product ah xh goes into
// the running sum through an error-free TwoSum, and its exact rounding error
// (one FMA), the cross terms ah xl + al xh and the TwoSum error collect in a
// second FP32 word.  Twelve FP32 operations per real product; the result is
// as accurate as a sum computed in twice the FP32 precision.  The rounded
// operations (__fmul_rn, __fadd_rn) keep the compiler from fusing them.
struct DF6 {
  float h[3], l[3];   // forms (0, 1, 2), hi and lo
};

__device__ __forceinline__ void dot2_step(float ah, float al, float xh, float xl, float& s, float& c) {
  const float ph = __fmul_rn(ah, xh);
  const float pe = fmaf(ah, xh, -ph);                   // exact: ah xh = ph + pe
  c = __fadd_rn(c, pe);
  c = fmaf(ah, xl, c);
  c = fmaf(al, xh, c);
  const float sn = __fadd_rn(s, ph);                    // TwoSum(s, ph) = sn + e
  const float bp = __fsub_rn(sn, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bp)), __fsub_rn(ph, bp));
  s = sn;
  c = __fadd_rn(c, e);
}

__global__ void __launch_bounds__(kT3) k3_gemm_df(ApplyData3<double2> d, int S) {
  __shared__ DF6 xs[kGK][kGC + 1];
  __shared__ DF6 as[kGK][kGN];
  const int K = d.n_loc + 27 * d.n_es;
  const int c0 = blockIdx.x * kGC, n0 = blockIdx.y * kGN, sl = blockIdx.z;
  const int kper = slice_len(K, S), kb = sl * kper, ke = kb + kper < K ? kb + kper : K;
  const int t = threadIdx.x, tc = t / 16, tn = t % 16;
  float hs[2][2][3], hc[2][2][3];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int f = 0; f < 3; ++f) hs[a][b][f] = hc[a][b][f] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += kGK) {
    __syncthreads();
    for (int i = t; i < kGK * kGC; i += kT3) {        // X tile, already in the split forms
      const int kk = i % kGK, cc = i / kGK, c = c0 + cc, kg = k0 + kk;
      DF6 w;
      if (c < d.nocc && kg < ke) {
        const float* src = d.X6 + 6 * (int64_t(c) * K + kg);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          w.h[q] = src[2 * q];
          w.l[q] = src[2 * q + 1];
        }
      } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) w.h[q] = w.l[q] = 0.f;
      }
      xs[kk][cc] = w;
    }
    for (int i = t; i < kGK * kGN; i += kT3) {        // LA tile, already in the split forms
      const int kk = i / kGN, nn = i % kGN, n = n0 + nn, kg = k0 + kk;
      DF6 w;
      if (n < d.nb && kg < ke) {
        const float* src = d.LA6 + 6 * (int64_t(kg) * d.nb + n);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          w.h[q] = src[2 * q];
          w.l[q] = src[2 * q + 1];
        }
      } else {
#pragma unroll
        for (int q = 0; q < 3; ++q) w.h[q] = w.l[q] = 0.f;
      }
      as[kk][nn] = w;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kGK; ++kk) {
      const DF6 x[2] = {xs[kk][tc], xs[kk][tc + 16]};
      const DF6 l[2] = {as[kk][tn], as[kk][tn + 16]};
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          // P: (a + b) c, Q: b (c + d), S: a (d - c)
          dot2_step(l[b].h[0], l[b].l[0], x[a].h[0], x[a].l[0], hs[a][b][0], hc[a][b][0]);
          dot2_step(l[b].h[1], l[b].l[1], x[a].h[1], x[a].l[1], hs[a][b][1], hc[a][b][1]);
          dot2_step(l[b].h[2], l[b].l[2], x[a].h[2], x[a].l[2], hs[a][b][2], hc[a][b][2]);
        }
    }
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int c = c0 + tc + 16 * a, n = n0 + tn + 16 * b;
      const double P = double(hs[a][b][0]) + double(hc[a][b][0]);
      const double Q = double(hs[a][b][1]) + double(hc[a][b][1]);
      const double U = double(hs[a][b][2]) + double(hc[a][b][2]);
      if (c < d.nocc && n < d.nb) d.part[(int64_t(sl) * d.nocc + c) * d.nb + n] = make_double2(P - Q, P + U);
    }
}

template <typename T>
__global__ void __launch_bounds__(kT3) k3_reduce(ApplyData3<T> d, int S) {
  const int64_t n = int64_t(d.nocc) * d.nb;
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    T v = d.part[e];
    for (int sl = 1; sl < S; ++sl) v = cadd(v, d.part[int64_t(sl) * n + e]);
    d.gamma[e] = v;
  }
}

// slices of K for the local GEMM: about 8 blocks per SM in all, each slice at
// least a few K steps long
__host__ __device__ inline int local_slices(int nocc, int nb, int K) {
  const int tiles = ((nocc + kGC - 1) / kGC) * ((nb + kGN - 1) / kGN);
  int S = (152 * 8 + tiles - 1) / tiles;
  const int smax = K / (4 * kGK) > 1 ? K / (4 * kGK) : 1;
  if (S > smax) S = smax;
  if (S > kLocalSlicesMax) S = kLocalSlicesMax;
  if (S < 1) S = 1;
  // whole K steps per slice (no step half padded with zeros), then as few
  // slices as cover K with that length
  const int len = slice_len(K, S);
  return (K + len - 1) / len;
}

// warp per row: stored adjacent part (CSR) and the local expansion of the
// row's cell, then out_q = u_q + kappa^2 (near + far)
template <typename T>
__global__ void __launch_bounds__(kT3) k3_near(ApplyData3<T> d, const T* __restrict__ u, T* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (q >= d.N) return;
  T acc = czero(T());
  if constexpr (sizeof(T) == 16) {
    // three FMAs per complex product: P += (a + b) c, Q += b (c + d), S += a (d - c);
    // Re = P - Q, Im = P + S (GB300's FP64 pipe, not HBM, bounds this loop)
    double P = 0, Q = 0, S = 0;
    for (int64_t e = d.rowptr[q] + lane; e < d.rowptr[q + 1]; e += 32) {
      const double* w = d.val3 + 3 * e;
      const double* x = d.u3 + 3 * int64_t(d.col[e]);
      P = fma(w[0], x[0], P);
      Q = fma(w[1], x[1], Q);
      S = fma(w[2], x[2], S);
    }
    acc = mk(P - Q, P + S);
  } else {
    // complex64: the cell's dense block over its 9 neighbour node ranges
    // (row r of cell k), then the CSR remainder
    const int k = d.occ_of_node[q];
    const int* sg = d.blk_seg + 18 * k;
    int nblk = 0;
#pragma unroll
    for (int s9 = 0; s9 < 9; ++s9) nblk += sg[2 * s9 + 1];
    const T* w = d.Wb + d.blk_off[k] + (q - d.occ_start[k]) * nblk;
    T acc2 = czero(T());                 // two chains: loads of the next entries overlap the FMAs
#pragma unroll 1
    for (int s9 = 0; s9 < 9; ++s9) {
      const int n0 = sg[2 * s9], len = sg[2 * s9 + 1];
      const T* uu = u + n0;
      int e = lane;
#pragma unroll 2
      for (; e + 32 < len; e += 64) {
        acc = cfma(w[e], uu[e], acc);
        acc2 = cfma(w[e + 32], uu[e + 32], acc2);
      }
      if (e < len) acc = cfma(w[e], uu[e], acc);
      w += len;
    }
    acc = cadd(acc, acc2);
    for (int64_t e = d.rowptr[q] + lane; e < d.rowptr[q + 1]; e += 32) acc = cfma(d.val[e], u[d.col[e]], acc);
  }
  const T* ph = d.Phi + q * d.nb;
  const T* g = d.gamma + int64_t(d.occ_of_node[q]) * d.nb;
  for (int n = lane; n < d.nb; n += 32) acc = cfma(ph[n], g[n], acc);
  acc = warp_sum(acc);
  if (lane == 0) {
    using R = decltype(acc.x);
    const R k2 = R(d.kappa2);
    const T uq = u[q];
    out[q] = mk(uq.x + k2 * acc.x, uq.y + k2 * acc.y);
  }
}

__global__ void __launch_bounds__(kT3) k3_farfield(int64_t N, const double* __restrict__ xyz,
                                                  const double* __restrict__ ffw, const double2* __restrict__ u,
                                                  int nrhs, const double* __restrict__ dirs, int ndir, double kappa,
                                                  double2 c, double2* __restrict__ A) {
  // block = (direction, right-hand side); threads stride over the nodes
  const int dd = blockIdx.x % ndir, r = blockIdx.x / ndir;
  const double dx = dirs[3 * dd], dy = dirs[3 * dd + 1], dz = dirs[3 * dd + 2];
  double2 acc = make_double2(0, 0);
  for (int64_t q = threadIdx.x; q < N; q += blockDim.x) {
    double sn, cs;
    sincos(-kappa * (dx * xyz[3 * q] + dy * xyz[3 * q + 1] + dz * xyz[3 * q + 2]), &sn, &cs);
    const double2 v = u[int64_t(r) * N + q];
    acc = cfma(make_double2(ffw[q] * cs, ffw[q] * sn), v, acc);
  }
  __shared__ double2 red[kT3 / 32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0, 0);
    for (int w = 0; w < kT3 / 32; ++w) s = cadd(s, red[w]);
    A[int64_t(r) * ndir + dd] = cmul(c, s);
  }
}

// complex64 <-> complex128 copies of the strengths and coefficients
__global__ void __launch_bounds__(kT3) k3_widen(const float2* __restrict__ a, double2* __restrict__ b, int64_t n) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    b[e] = make_double2(a[e].x, a[e].y);
}
__global__ void __launch_bounds__(kT3) k3_narrow(const double2* __restrict__ a, float2* __restrict__ b, int64_t n) {
  for (int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    b[e] = make_float2(float(a[e].x), float(a[e].y));
}

int grid_for(int64_t n) {
  const int64_t b = (n + kT3 - 1) / kT3;
  return int(b < 152 * 16 ? b : 152 * 16);
}

size_t fft_smem_bytes(int M, int lpb, size_t elem) { return elem * size_t(lpb) * (M + 1); }

// lines per block of a line-transform launch over `lines` lines: a power of
// two between 32 / (M / 8) (whole warps) and 2048 / M, as large as leaves at
// least two blocks per SM
int lines_per_block(int M, int64_t lines) {
  const int G = M / 8, lo = G >= 32 ? 1 : 32 / G, hi = kT3 / G;
  int lpb = hi;
  while (lpb > lo && (lines + lpb - 1) / lpb < 2 * 152) lpb /= 2;
  return lpb;
}

template <typename T>
cudaError_t fft_box(T* x, T* x1, int M, int logM, const T* tw, bool inverse, LineBox bx, cudaStream_t st) {
  static unsigned long long attr = 0;
  if (first_on_device(attr)) {
    const cudaError_t e = cudaFuncSetAttribute(k3_fft_axis<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    if (e != cudaSuccess) return e;
  }
  const int64_t lines = int64_t(bx.n_out) * bx.n_in;
  const int LPB = lines_per_block(M, lines);
  const dim3 grid(unsigned((lines + LPB - 1) / LPB), x1 ? 2 : 1);
  k3_fft_axis<T><<<grid, LPB * (M / 8), fft_smem_bytes(M, LPB, sizeof(T)), st>>>(x, x1, M, logM, tw, inverse, bx);
  return cudaGetLastError();
}

// lattice convolution and local coefficients: sigma -> gamma on one
// precision's data.  The sources sit on the x1-face planes a = f N_eq
// (f = 0..L) inside [0, L N_eq]^3 and V is read inside [0, L N_eq]^3 only, so
// the forward c and b stages run on the face planes' lines alone, the inverse
// b and c stages on the lines with a (and b) <= L N_eq; the a stage (every
// (b, c) line) carries the spectral product.
template <typename T>
cudaError_t lattice_local(const ApplyData3<T>& d, cudaStream_t st, bool df = false) {
  const int64_t n3 = int64_t(d.M) * d.M * d.M;
  const int M = d.M, nl = d.L * d.Ne;
  k3_fill<T><<<grid_for(n3), kT3, 0, st>>>(d);
  cudaError_t e = cudaSuccess;
  // forward c and b passes of both arrays, two launches
  e = fft_box<T>(d.Sm, d.Sd, M, d.logM, d.tw, false, LineBox{2, d.L + 1, d.Ne, nl + 1}, st);
  if (e == cudaSuccess) e = fft_box<T>(d.Sm, d.Sd, M, d.logM, d.tw, false, LineBox{1, d.L + 1, d.Ne, M}, st);
  if (e != cudaSuccess) return e;
  if (M <= 1024) {
    static unsigned long long attr = 0;
    if (first_on_device(attr)) {
      e = cudaFuncSetAttribute(k3_conv_a<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
      if (e != cudaSuccess) return e;
    }
    const int LPB = std::max(2, lines_per_block(M, 2 * int64_t(M) * M)), H = LPB / 2;
    k3_conv_a<T><<<int(int64_t(M) * M / H), LPB * (M / 8), fft_smem_bytes(M, LPB, sizeof(T)), st>>>(
        d.Sm, d.Sd, d.Gs, d.Ds, M, d.logM, d.tw, nl);
  } else {
    e = fft_box<T>(d.Sm, d.Sd, M, d.logM, d.tw, false, LineBox{0, M, 1, M}, st);
    if (e != cudaSuccess) return e;
    k3_spectral<T><<<grid_for(n3), kT3, 0, st>>>(d.Sm, d.Sd, d.Gs, d.Ds, n3);
    e = fft_box<T>(d.Sm, nullptr, M, d.logM, d.tw, true, LineBox{0, M, 1, M}, st);
  }
  if (e == cudaSuccess) e = fft_box<T>(d.Sm, nullptr, M, d.logM, d.tw, true, LineBox{1, nl + 1, 1, M}, st);
  if (e == cudaSuccess) e = fft_box<T>(d.Sm, nullptr, M, d.logM, d.tw, true, LineBox{2, nl + 1, 1, nl + 1}, st);
  if (e != cudaSuccess) return e;
  const int K = d.n_loc + 27 * d.n_es, S = local_slices(d.nocc, d.nb, K);
  k3_gather<T><<<d.nocc, kT3, 0, st>>>(d, df);
  const dim3 grid((d.nocc + kGC - 1) / kGC, (d.nb + kGN - 1) / kGN, S);
  if constexpr (sizeof(T) == 16) {
    if (df) k3_gemm_df<<<grid, kT3, 0, st>>>(d, S);
    else k3_gemm<T><<<grid, kT3, 0, st>>>(d, S);
  } else {
    k3_gemm<T><<<grid, kT3, 0, st>>>(d, S);
  }
  k3_reduce<T><<<grid_for(int64_t(d.nocc) * d.nb), kT3, 0, st>>>(d, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t apply3_one(const ApplyData3<T>& d, const T* u, T* out, cudaStream_t st) {
  k3_project<T><<<d.nocc, kTP, 0, st>>>(d, u);
  cudaError_t e;
  if constexpr (sizeof(T) == 8) {
    // complex64: the strengths widened to FP64 for the lattice and the local
    // step (ApplyData3::lattice64), the coefficients narrowed back
    const ApplyData3<double2>& w = *d.lattice64;
    const int64_t ns = int64_t(d.nocc) * d.n_es, ng = int64_t(d.nocc) * d.nb;
    k3_widen<<<grid_for(ns), kT3, 0, st>>>(d.sigma, w.sigma, ns);
    e = lattice_local(w, st, true);
    if (e != cudaSuccess) return e;
    k3_narrow<<<grid_for(ng), kT3, 0, st>>>(w.gamma, d.gamma, ng);
  } else {
    e = lattice_local(d, st);
    if (e != cudaSuccess) return e;
  }
  k3_near<T><<<int((d.N * 32 + kT3 - 1) / kT3), kT3, 0, st>>>(d, u, out);
  return cudaGetLastError();
}

// position of node c in a row's dense block (its 9 ranges (start, length)
// concatenated in order), or -1 outside them
__device__ __forceinline__ int block_pos(const int (&sg)[18], int c) {
  int o = 0;
#pragma unroll
  for (int s9 = 0; s9 < 9; ++s9) {
    if (c >= sg[2 * s9] && c < sg[2 * s9] + sg[2 * s9 + 1]) return o + c - sg[2 * s9];
    o += sg[2 * s9 + 1];
  }
  return -1;
}

// thread per row: its entries in order (one-time plan construction)
__global__ void __launch_bounds__(kT3) k3_near_forms(int64_t N, const int64_t* __restrict__ occ_start,
                                                     const int* __restrict__ occ_of_node,
                                                     const int64_t* __restrict__ rowptr, const int* __restrict__ col,
                                                     const double2* __restrict__ val,
                                                     const int64_t* __restrict__ blk_off,
                                                     const int* __restrict__ blk_seg, double* __restrict__ val3,
                                                     float2* __restrict__ Wb, int64_t* __restrict__ rem_count) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const int k = occ_of_node[q];
  int sg[18], nblk = 0;
#pragma unroll
  for (int i = 0; i < 18; ++i) sg[i] = blk_seg[18 * k + i];
#pragma unroll
  for (int s9 = 0; s9 < 9; ++s9) nblk += sg[2 * s9 + 1];
  float2* w = Wb + blk_off[k] + (q - occ_start[k]) * nblk;
  int64_t cnt = 0;
  for (int64_t e = rowptr[q]; e < rowptr[q + 1]; ++e) {
    const double2 v = val[e];
    val3[3 * e] = v.x + v.y;
    val3[3 * e + 1] = v.y;
    val3[3 * e + 2] = v.x;
    const int pos = block_pos(sg, col[e]);
    if (pos >= 0) {
      const float2 o = w[pos];
      w[pos] = make_float2(o.x + float(v.x), o.y + float(v.y));
    } else {
      ++cnt;
    }
  }
  rem_count[q] = cnt;
}

__global__ void __launch_bounds__(kT3) k3_near_remainder(int64_t N, const int* __restrict__ occ_of_node,
                                                         const int64_t* __restrict__ rowptr,
                                                         const int* __restrict__ col, const double2* __restrict__ val,
                                                         const int* __restrict__ blk_seg,
                                                         const int64_t* __restrict__ rem_row, int* __restrict__ rem_col,
                                                         float2* __restrict__ rem_val) {
  const int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const int k = occ_of_node[q];
  int sg[18];
#pragma unroll
  for (int i = 0; i < 18; ++i) sg[i] = blk_seg[18 * k + i];
  int64_t o = rem_row[q];
  for (int64_t e = rowptr[q]; e < rowptr[q + 1]; ++e)
    if (block_pos(sg, col[e]) < 0) {
      rem_col[o] = col[e];
      rem_val[o] = make_float2(float(val[e].x), float(val[e].y));
      ++o;
    }
}

}  // namespace

int local3_slices(int nocc, int nb, int K) { return local_slices(nocc, nb, K); }

template <typename T>
cudaError_t fft3d(T* x, int M, int logM, const T* tw, bool inverse, cudaStream_t st) {
  if (M < 16 || M > 2048 || (M & (M - 1))) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  for (int axis = 2; axis >= 0 && e == cudaSuccess; --axis)
    e = fft_box<T>(x, nullptr, M, logM, tw, inverse, LineBox{axis, M, 1, M}, st);
  return e;
}

template <typename T>
cudaError_t apply3_batch(const ApplyData3<T>& d, const T* u, T* out, int nr, cudaStream_t st) {
  if (sizeof(T) == 8 && !d.lattice64) return cudaErrorInvalidValue;
  for (int r = 0; r < nr; ++r) {
    const cudaError_t e = apply3_one(d, u + int64_t(r) * d.N, out + int64_t(r) * d.N, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t near3_forms(int64_t N, const int64_t* occ_start, const int* occ_of_node, const int64_t* rowptr,
                        const int* col, const double2* val, const int64_t* blk_off, const int* blk_seg, double* val3,
                        float2* Wb, int64_t* rem_count, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  k3_near_forms<<<unsigned((N + kT3 - 1) / kT3), kT3, 0, st>>>(N, occ_start, occ_of_node, rowptr, col, val, blk_off,
                                                               blk_seg, val3, Wb, rem_count);
  return cudaGetLastError();
}

cudaError_t near3_remainder(int64_t N, const int* occ_of_node, const int64_t* rowptr, const int* col,
                            const double2* val, const int* blk_seg, const int64_t* rem_row, int* rem_col,
                            float2* rem_val, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  k3_near_remainder<<<unsigned((N + kT3 - 1) / kT3), kT3, 0, st>>>(N, occ_of_node, rowptr, col, val, blk_seg,
                                                                   rem_row, rem_col, rem_val);
  return cudaGetLastError();
}

cudaError_t farfield3(int64_t N, const double* xyz, const double* ffw, const double2* u, int nrhs,
                      const double* dirs, int ndir, double kappa, double2 c, double2* A, cudaStream_t st) {
  if (ndir <= 0 || nrhs <= 0) return cudaSuccess;
  k3_farfield<<<ndir * nrhs, kT3, 0, st>>>(N, xyz, ffw, u, nrhs, dirs, ndir, kappa, c, A);
  return cudaGetLastError();
}

template cudaError_t fft3d<double2>(double2*, int, int, const double2*, bool, cudaStream_t);
template cudaError_t fft3d<float2>(float2*, int, int, const float2*, bool, cudaStream_t);
template cudaError_t apply3_batch<double2>(const ApplyData3<double2>&, const double2*, double2*, int, cudaStream_t);
template cudaError_t apply3_batch<float2>(const ApplyData3<float2>&, const float2*, float2*, int, cudaStream_t);

}  // namespace lsd
