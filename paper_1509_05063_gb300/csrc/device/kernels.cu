// sm_103a kernels of the LS apply (Section 3.2 accelerator + near field) and
// of the GMRES solve.  One template per arithmetic precision: T = double2
// (complex128 path) or float2 (complex64 inner path of mixed precision).
//
// Apply pipeline for one or more right-hand sides (Eq. VolInt-Adj-NonAdj):
//   k_es_project      sigma_c = P_c u_c            (equivalent-source fit)
//   k_src_rows        sigma -> monopole / dipole face rows of the lattice, FFT along b
//   k_conv_cols       column FFTs, product with the spectra of G and dG/dz_1, inverse
//   k_inv_rows        inverse FFT along b of the kept rows (lattice values V)
//   k_local_coeffs    gamma_c = B^+ V_c - sum_o (B^+ T_o) sigma_{c+o}
//   k_near_eval       out_q = u_q + kappa^2 (sum_l W_ql u_l + Phi_q . gamma_c)
//                     (k_near_tc: the same for 8 or 16 complex64 RHS on the tensor cores)
#include <cstdio>

#include "cplx.cuh"
#include "fft.cuh"
#include "kernels.cuh"

namespace lsd {

template <typename T> struct RealOf;
template <> struct RealOf<double2> { using R = double; };
template <> struct RealOf<float2> { using R = float; };

// ------------------------------------------------------------ per-cell contractions
// The projection and the local coefficients are small dense contractions per
// cell, Y (n_out x R) = A (n_out x n_in) X (n_in x R), with A stored transposed
// ([n_in][n_out]) and X staged in shared memory.  Thread t of the block owns
// output o = t % n_out of segment s = t / n_out (S = blockDim / n_out segments)
// and sums the inputs j = s, s + S, ... in increasing order; the S partial sums
// are then added in segment order through shared memory.  No warp reductions,
// every lane does useful work, and each output is summed the same way whatever R.
//
// Staged inputs: complex64 as is; complex128 as c = Re x and (c + d, d - c),
// with the sum Re a + Im a of each matrix entry stored beside A, so that every
// complex product takes three FP64 FMAs (Gauss's form, as in the near field).
template <typename T> struct Staged;
template <> struct Staged<float2> {
  static constexpr int kBytes = 8;
  float2* x;
  int ld;
  __device__ Staged(unsigned char* raw, int ld_) : x(reinterpret_cast<float2*>(raw)), ld(ld_) {}
  __device__ void put(int r, int j, float2 v) const { x[r * ld + j] = v; }
};
template <> struct Staged<double2> {
  static constexpr int kBytes = 24;
  double* c;
  double2* ef;
  int ld;
  // ld * R doubles of c first, then the pairs (16-byte aligned: ld is even)
  __device__ Staged(unsigned char* raw, int ld_, int R)
      : c(reinterpret_cast<double*>(raw)), ef(reinterpret_cast<double2*>(raw + size_t(R) * ld_ * 8)), ld(ld_) {}
  __device__ void put(int r, int j, double2 v) const {
    c[r * ld + j] = v.x;
    ef[r * ld + j] = make_double2(v.x + v.y, v.y - v.x);
  }
};

template <typename T> struct CAcc;
template <> struct CAcc<float2> {
  float2 v;
  __device__ void zero() { v = make_float2(0.f, 0.f); }
  __device__ void mac(float2 a, double, const Staged<float2>& X, int r, int j) { v = cfma(a, X.x[r * X.ld + j], v); }
  __device__ float2 value() const { return v; }
};
template <> struct CAcc<double2> {
  double p, q, s;   // sum (a + b) c, sum b (c + d), sum a (d - c)
  __device__ void zero() { p = q = s = 0.0; }
  __device__ void mac(double2 a, double sa, const Staged<double2>& X, int r, int j) {
    const double c = X.c[r * X.ld + j];
    const double2 ef = X.ef[r * X.ld + j];
    p = fma(sa, c, p);
    q = fma(a.y, ef.x, q);
    s = fma(a.x, ef.y, s);
  }
  __device__ double2 value() const { return make_double2(p - q, p + s); }
};

template <typename T>
__device__ __forceinline__ Staged<T> staged_at(unsigned char* raw, int ld, int R) {
  if constexpr (sizeof(T) == 16) return Staged<T>(raw, ld, R);
  else return Staged<T>(raw, ld);
}

__device__ __forceinline__ const double* sa_base(const double* p, int64_t off) { return p ? p + off : nullptr; }

// acc[r] += sum over j = j1, j1 + S, ... < j_end of A[j][o] X[r][j] (A row
// length n_out; As = Re + Im of A for complex128).  Loads go out four at a
// time; the sum runs in increasing j whatever R.
template <typename T, int R>
__device__ __forceinline__ void contract_segment(const T* __restrict__ A, const double* __restrict__ As, int n_out,
                                                 int o, int j1, int j_end, int S, const Staged<T>& X,
                                                 CAcc<T> (&acc)[R]) {
  constexpr bool kC128 = sizeof(T) == 16;
  constexpr int U = 4;
  int j = j1;
  for (; j + (U - 1) * S < j_end; j += U * S) {
    T a[U];
    double sa[U];
#pragma unroll
    for (int v = 0; v < U; ++v) {
      const int64_t e = int64_t(j + v * S) * n_out + o;
      a[v] = A[e];
      sa[v] = kC128 ? As[e] : 0.0;
    }
#pragma unroll
    for (int v = 0; v < U; ++v)
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r].mac(a[v], sa[v], X, r, j + v * S);
  }
  for (; j < j_end; j += S) {
    const int64_t e = int64_t(j) * n_out + o;
    const T a = A[e];
    const double sa = kC128 ? As[e] : 0.0;
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r].mac(a, sa, X, r, j);
  }
}

// the S partial sums of every (r, o) in segment order; red = [S][R][n_out]
template <typename T, int R>
__device__ __forceinline__ void segment_sums_out(const CAcc<T> (&acc)[R], unsigned char* raw, int n_out, int o, int sg,
                                                 int S, T* __restrict__ out, int64_t r_stride) {
  T* red = reinterpret_cast<T*>(raw);
  __syncthreads();                                    // the staged inputs are no longer read
  if (sg < S) {
#pragma unroll
    for (int r = 0; r < R; ++r) red[(sg * R + r) * n_out + o] = acc[r].value();
  }
  __syncthreads();
  for (int e = threadIdx.x; e < R * n_out; e += blockDim.x) {
    const int r = e / n_out, oo = e - r * n_out;
    T v = red[r * n_out + oo];
    for (int g = 1; g < S; ++g) v = cadd(v, red[(g * R + r) * n_out + oo]);
    out[int64_t(r) * r_stride + oo] = v;
  }
}

// bytes of staged inputs per chunk of the projection (the cell's nodes): a
// whole piece of kProjPiece nodes for up to 4 complex128 or 16 complex64 RHS
constexpr int kProjStage = 32768;
static_assert(kProjPiece <= (kProjStage / (kMaxRhs64 * 24) & ~1) && kProjPiece <= kProjStage / (kMaxRhs32 * 8),
              "a projection piece fits one staging chunk");

// shared memory of a 256-thread contraction block: the staged inputs, then the
// S x R x n_out <= 256 R partial sums in the same space
template <typename T>
size_t contraction_smem(int R, size_t stage_bytes) {
  const size_t red = size_t(256) * R * sizeof(T);
  return red > stage_bytes ? red : stage_bytes;
}

// ------------------------------------------------------------ ES projection
// sigma_c = P_c u_c (P_c: n_es x nc, stored [nc][n_es], Ps = Re + Im of P_c for
// complex128).  The body sums the nodes [jb, je) of cell k into out[r * r_stride
// + i]; the nodes are staged in chunks of CJ (the inputs of thread segment s stay
// j - jb = s mod S across chunks).
template <typename T, int R>
__device__ __forceinline__ void es_project_body(int k, int jb, int je, const int64_t* __restrict__ occ_start,
                                                const int64_t* __restrict__ P_off, const T* __restrict__ P,
                                                const double* __restrict__ Ps, const T* __restrict__ u, int64_t N,
                                                T* __restrict__ out, int64_t r_stride, int n_es,
                                                double* __restrict__ utc, double2* __restrict__ utef) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int CJ = kProjStage / (R * Staged<T>::kBytes) & ~1;
  const int64_t s0 = occ_start[k] + jb;
  const int nc = je - jb;
  const int64_t pk = P_off[k] + int64_t(jb) * n_es;
  const T* Pk = P + pk;
  const double* Psk = sizeof(T) == 16 ? Ps + pk : nullptr;   // null for complex64
  const int S = blockDim.x / n_es, t = threadIdx.x, o = t % n_es, sg = t / n_es;
  const Staged<T> X = staged_at<T>(smem_raw, CJ, R);
  CAcc<T> acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r].zero();
  for (int j0 = 0; j0 < nc; j0 += CJ) {
    const int cl = min(CJ, nc - j0);
    __syncthreads();
    for (int e = t; e < R * cl; e += blockDim.x) {
      const int r = e / cl, j = e - r * cl;
      const int64_t q = int64_t(r) * N + s0 + j0 + j;
      const T v = u[q];
      X.put(r, j, v);
      if constexpr (sizeof(T) == 16) {
        if (utc) {                                 // the near field's staged forms of the input
          utc[q] = v.x;
          utef[q] = make_double2(v.x + v.y, v.y - v.x);
        }
      }
    }
    __syncthreads();
    if (sg < S) contract_segment<T, R>(Pk + int64_t(j0) * n_es, sa_base(Psk, int64_t(j0) * n_es), n_es, o,
                                       (sg - j0 % S + S) % S, cl, S, X, acc);
  }
  segment_sums_out<T, R>(acc, smem_raw, n_es, o, sg, S, out, r_stride);
}

// One block per piece (cell k, nodes [jb, je), piece p of np), pieces of at most
// kProjPiece nodes, the largest first.  A cell of one piece writes sigma
// directly; otherwise each piece writes its partial sums to its slot, and the
// last piece of the cell to finish (counted on count[k]) adds the slots in piece
// order and resets the count: the result does not depend on which piece ends
// last, nor on R.
template <typename T, int R>
__device__ __forceinline__ void es_project_piece(const int4 pc, const int* __restrict__ piece_off, int nocc,
                                                 const int64_t* __restrict__ occ_start,
                                                 const int64_t* __restrict__ P_off, const T* __restrict__ P,
                                                 const double* __restrict__ Ps, const T* __restrict__ u, int64_t N,
                                                 T* __restrict__ sigma, T* __restrict__ part, int* __restrict__ count,
                                                 int n_es, double* __restrict__ utc, double2* __restrict__ utef) {
  const int k = pc.x, p = pc.w >> 16, np = pc.w & 0xffff;
  if (np == 1) {
    es_project_body<T, R>(k, pc.y, pc.z, occ_start, P_off, P, Ps, u, N, sigma + int64_t(k) * n_es,
                          int64_t(nocc) * n_es, n_es, utc, utef);
    return;
  }
  T* slots = part + int64_t(piece_off[k]) * R * n_es;          // [piece][r][i]
  es_project_body<T, R>(k, pc.y, pc.z, occ_start, P_off, P, Ps, u, N, slots + int64_t(p) * R * n_es, n_es, n_es,
                        utc, utef);
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(count + k, 1) == np - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int e = threadIdx.x; e < R * n_es; e += blockDim.x) {
    T v = __ldcg(slots + e);
    for (int q = 1; q < np; ++q) v = cadd(v, __ldcg(slots + int64_t(q) * R * n_es + e));
    const int r = e / n_es, i = e - r * n_es;
    sigma[(int64_t(r) * nocc + k) * n_es + i] = v;
  }
  if (threadIdx.x == 0) count[k] = 0;
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_es_project(const int4* __restrict__ pieces, const int* __restrict__ piece_off,
                                                    int nocc, const int64_t* __restrict__ occ_start,
                                                    const int64_t* __restrict__ P_off, const T* __restrict__ P,
                                                    const double* __restrict__ Ps, const T* __restrict__ u, int64_t N,
                                                    T* __restrict__ sigma, T* __restrict__ part,
                                                    int* __restrict__ count, int n_es, double* __restrict__ utc,
                                                    double2* __restrict__ utef) {
  es_project_piece<T, R>(pieces[blockIdx.x], piece_off, nocc, occ_start, P_off, P, Ps, u, N, sigma, part, count,
                         n_es, utc, utef);
}

// ------------------------------------------------------------ Stockham FFT
// fft_smem (device/fft.cuh): in-place radix-4/2 Stockham transform in shared memory.

constexpr int kFftCols = 4;       // columns per block of the column pass
constexpr int kFftMaxM = 2048;    // column pass: 4 x M / 8 threads <= 1024

// one row per block, M / 8 threads
template <typename T>
__global__ void __launch_bounds__(kFftMaxM / 8) k_fft_rows(T* __restrict__ X, int M, int logM,
                                                           const T* __restrict__ tw, bool inv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  T* row = X + int64_t(blockIdx.x) * M;
  for (int i = threadIdx.x; i < M; i += blockDim.x) s[i] = row[i];
  __syncthreads();
  fft_smem<T>(s, M, logM, inv, tw, threadIdx.x);
  for (int i = threadIdx.x; i < M; i += blockDim.x) row[i] = s[i];
}

// kFftCols adjacent columns per block, each held contiguously in shared memory;
// M / 8 threads per column.
template <typename T>
__global__ void __launch_bounds__(kFftCols * kFftMaxM / 8) k_fft_cols(T* __restrict__ X, int M, int logM,
                                                                      const T* __restrict__ tw, bool inv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);
  const int c0 = blockIdx.x * kFftCols;
  for (int e = threadIdx.x; e < kFftCols * M; e += blockDim.x) {
    const int r = e / kFftCols, c = e % kFftCols;
    s[c * M + r] = X[int64_t(r) * M + c0 + c];
  }
  __syncthreads();
  const int G = M / 8;
  const int c = threadIdx.x / G, t = threadIdx.x % G;
  fft_smem<T>(s + c * M, M, logM, inv, tw, t);
  for (int e = threadIdx.x; e < kFftCols * M; e += blockDim.x) {
    const int r = e / kFftCols, cc = e % kFftCols;
    X[int64_t(r) * M + c0 + cc] = s[cc * M + r];
  }
}

template <typename T>
cudaError_t fft2d(T* x, int M, int logM, const T* tw, bool inverse, cudaStream_t st) {
  if (M < 256 || M > kFftMaxM || (M & (M - 1))) return cudaErrorInvalidValue;
  const size_t srow = size_t(M) * sizeof(T), scol = size_t(M) * kFftCols * sizeof(T);
  static unsigned long long attr_done = 0;
  if (first_on_device(attr_done)) {
    cudaFuncSetAttribute(k_fft_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kFftMaxM * sizeof(T)));
    cudaFuncSetAttribute(k_fft_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(kFftMaxM * kFftCols * sizeof(T)));
  }
  k_fft_rows<T><<<M, M / 8, srow, st>>>(x, M, logM, tw, inverse);
  k_fft_cols<T><<<M / kFftCols, kFftCols * M / 8, scol, st>>>(x, M, logM, tw, inverse);
  return cudaGetLastError();
}

// The lattice transforms' FFT per precision.  complex64: the radix-16
// transform (fft16_smem, M / 16 threads a transform, padded layout), a third
// faster on the 16-RHS lattice convolution than radix 4.  complex128: the
// radix-4 transform (fft_smem, M / 8 threads, plain layout): FP64 values
// sixteen a thread spill, and the FP64 pipe bounds these kernels either way
// (the radix-16 form measured 0.197 against 0.173 ms for the FP64 convolution).
template <typename T>
struct LatFft;
template <>
struct LatFft<float2> {
  static constexpr int kDiv = 16;              // values per thread and transform
  static constexpr int kColThreads = 256;      // launch bound of the column pass (at most 4 columns at M = 1024)
  static constexpr int kColBlocks = 3;         // 80 registers: 3 blocks of 256 per SM instead of 2 at 128
  __host__ __device__ static constexpr int len(int N) { return fft16_len(N); }
  __device__ static int at(int i) { return fpad(i); }
  __device__ static void run(float2* x, int N, int logN, bool inv, const float2* tw, int t) {
    (void)logN;
    fft16_smem<float2>(x, N, inv, tw, t);
  }
};
// The radix-4 transform for either precision (complex64: the autotuner's
// alternative to radix 16, ApplyData::fft_r4).
template <typename T>
struct LatFft4 {
  static constexpr int kDiv = 8;
  static constexpr int kColThreads = 1024;
  static constexpr int kColBlocks = 1;
  __host__ __device__ static constexpr int len(int N) { return N; }
  __device__ static int at(int i) { return i; }
  __device__ static void run(T* x, int N, int logN, bool inv, const T* tw, int t) {
    fft_smem<T>(x, N, logN, inv, tw, t);
  }
};
template <>
struct LatFft<double2> : LatFft4<double2> {};

// ------------------------------------------------------------ pruned, fused lattice convolution
// Sources live only on the L + 1 face rows a = k Ne (k = 0..L) of the M x M
// padded lattice, and only the n_lat x n_lat corner of the result is read.
//  k_src_rows  : gather sigma of face row k (monopole or dipole) into shared
//                memory and FFT it along b              -> R[k][b], (L+1) x M x 2
//                (face point (k Ne, b) takes the strengths of the left face of
//                cell k and the right face of cell k - 1; the top point of a
//                face is shared with the cell above)
//  k_conv_cols : per column b, scatter the L + 1 rows to a, FFT along a (both
//                source kinds), multiply by the kernel spectra (stored as a
//                quarter using the even / odd symmetry of the tables), inverse
//                FFT along a, keep a < n_lat            -> Vt[a][b], n_lat x M
//  k_inv_rows  : inverse FFT along b of rows a < n_lat, keep b < n_lat -> V
// face row k of one right-hand side (sigma and R of that RHS), kind 0 monopole / 1 dipole
template <typename T, class F>
__device__ __forceinline__ void src_row_body(int M, int logM, int n_lat, int Ne, int L,
                                             const int* __restrict__ occ_of_cell, const T* __restrict__ sigma,
                                             int n_es, const T* __restrict__ tw, T* __restrict__ R, int k, int kind) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);       // F layout
  for (int b = threadIdx.x; b < M; b += blockDim.x) {
    T v = czero(T{});
    if (b < n_lat) {
      for (int side = 0; side < 2; ++side) {        // left face of cell k, right face of cell k - 1
        const int ci = k - side;
        if (ci < 0 || ci >= L) continue;
        const int cjb = b / Ne, kb = b % Ne;
        for (int t = 0; t < 2; ++t) {
          if (t == 1 && kb != 0) break;
          const int cj = cjb - t, kk = kb + t * Ne;
          if (cj < 0 || cj >= L) continue;
          const int occ = occ_of_cell[cj * L + ci];
          if (occ >= 0) v = cadd(v, sigma[int64_t(occ) * n_es + (2 * kind + side) * (Ne + 1) + kk]);
        }
      }
    }
    s[F::at(b)] = v;
  }
  __syncthreads();
  F::run(s, M, logM, false, tw, threadIdx.x);
  __syncthreads();
  T* out = R + (int64_t(kind) * (L + 1) + k) * M;
  for (int b = threadIdx.x; b < M; b += blockDim.x) out[b] = s[F::at(b)];
}

template <typename T, class F = LatFft<T>>
__global__ void __launch_bounds__(kFftMaxM / F::kDiv) k_src_rows(int M, int logM, int n_lat, int Ne, int L,
                                                            const int* __restrict__ occ_of_cell,
                                                            const T* __restrict__ sigma_all, int n_es, int nocc,
                                                            const T* __restrict__ tw, T* __restrict__ R_all,
                                                            int64_t stride) {
  src_row_body<T, F>(M, logM, n_lat, Ne, L, occ_of_cell, sigma_all + int64_t(blockIdx.z) * nocc * n_es, n_es, tw,
                  R_all + int64_t(blockIdx.z) * stride, blockIdx.x, blockIdx.y);
}

// spectra quarter layout: Q[l][k] for l, k in [0, M/2] (k fastest).
// The sources of a column sit only at a = k Ne (k = 0..L), so when Ne divides M
// the length-M forward transform is a length-M/Ne transform of the L + 1 values
// repeated Ne times: X[f] = Y[f mod (M/Ne)].  Ms = M/Ne (0: use the full
// length), logMs its log2.
// columns b0 .. b0 + TC - 1 of one right-hand side (R and Vt of that RHS)
template <typename T, class F>
__device__ __forceinline__ void conv_cols_body(int M, int logM, int n_lat, int Ne, int L, int TC, int Ms, int logMs,
                                               const T* __restrict__ R, const T* __restrict__ Gq,
                                               const T* __restrict__ Dq, const T* __restrict__ tw,
                                               T* __restrict__ Vt, int b0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int PM = F::len(M);            // one column in the F layout
  T* xm = reinterpret_cast<T*>(smem_raw);      // [TC][PM]
  T* xd = xm + TC * PM;                        // [TC][PM]
  const int half = M / 2;
  constexpr int kDiv = F::kDiv;
  const int G = M / kDiv;                      // threads per column
  const int c = threadIdx.x / G, t = threadIdx.x % G;
  // the spectral product of column element e (column e >> logM, row e & (M - 1)):
  // monopole value vm times G^, plus dipole value vd times D^ (odd in the a offset)
  auto product = [&](auto value_of) {
#pragma unroll
    for (int h2 = 0; h2 < kDiv / 8; ++h2) {    // kDiv products per thread, eight loads at a time
      T gq[8], dq[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = threadIdx.x + (8 * h2 + q) * blockDim.x, cc = e >> logM, a = e & (M - 1), b = b0 + cc;
        const int kq = a <= half ? a : M - a, lq = b <= half ? b : M - b;
        const int64_t qi = int64_t(lq) * (half + 1) + kq;
        gq[q] = Gq[qi];
        dq[q] = Dq[qi];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int e = threadIdx.x + (8 * h2 + q) * blockDim.x, cc = e >> logM, a = e & (M - 1);
        const T d = a > half ? mk(-dq[q].x, -dq[q].y) : dq[q];
        T vm, vd;
        value_of(cc, a, vm, vd);
        xm[cc * PM + F::at(a)] = cfma(vd, d, cmul(vm, gq[q]));
      }
    }
  };
  if (Ms > 0) {
    // short spectra: monopole in xd[c][0, Ms), dipole in xd[c][Ms, 2 Ms) (plain layout)
    for (int e = threadIdx.x; e < TC * Ms; e += blockDim.x) {
      const int cc = e / Ms, k = e % Ms;
      T vm = czero(T{}), vd = czero(T{});
      if (k <= L) {
        vm = R[int64_t(k) * M + b0 + cc];
        vd = R[(int64_t(L + 1) + k) * M + b0 + cc];
      }
      xd[cc * PM + k] = vm;
      xd[cc * PM + Ms + k] = vd;
    }
    __syncthreads();
    // two transforms of length Ms per column, by the column's first 2 Ms / 8 threads
    const int Gs = Ms / 8;
    const bool act = t < 2 * Gs;
    const int which = t / Gs;                  // 0 monopole, 1 dipole
    fft_smem<T>(xd + c * PM + (act ? which : 0) * Ms, Ms, logMs, false, tw, act ? t % Gs : 0, M / Ms, act);
    product([&](int cc, int a, T& vm, T& vd) {
      const int f = a & (Ms - 1);
      vm = xd[cc * PM + f];
      vd = xd[cc * PM + Ms + f];
    });
    __syncthreads();
  } else {
    for (int e = threadIdx.x; e < TC * M; e += blockDim.x) {
      const int cc = e / M, a = e % M;
      T vm = czero(T{}), vd = czero(T{});
      if (a % Ne == 0 && a / Ne <= L) {
        const int k = a / Ne;
        vm = R[int64_t(k) * M + b0 + cc];
        vd = R[(int64_t(L + 1) + k) * M + b0 + cc];
      }
      xm[cc * PM + F::at(a)] = vm;
      xd[cc * PM + F::at(a)] = vd;
    }
    __syncthreads();
    F::run(xm + c * PM, M, logM, false, tw, t);
    __syncthreads();
    F::run(xd + c * PM, M, logM, false, tw, t);
    __syncthreads();
    product([&](int cc, int a, T& vm, T& vd) {
      vm = xm[cc * PM + F::at(a)];
      vd = xd[cc * PM + F::at(a)];
    });
    __syncthreads();
  }
  F::run(xm + c * PM, M, logM, true, tw, t);
  __syncthreads();
  for (int e = threadIdx.x; e < TC * n_lat; e += blockDim.x) {
    const int a = e / TC, cc = e % TC;
    Vt[int64_t(a) * M + b0 + cc] = xm[cc * PM + F::at(a)];
  }
}

template <typename T, class F = LatFft<T>>
__global__ void __launch_bounds__(F::kColThreads, F::kColBlocks) k_conv_cols(int M, int logM, int n_lat, int Ne, int L, int TC, int Ms,
                                                    int logMs, const T* __restrict__ R_all,
                                                    const T* __restrict__ Gq, const T* __restrict__ Dq,
                                                    const T* __restrict__ tw, T* __restrict__ Vt_all,
                                                    int64_t stride) {
  conv_cols_body<T, F>(M, logM, n_lat, Ne, L, TC, Ms, logMs, R_all + int64_t(blockIdx.y) * stride, Gq, Dq, tw,
                    Vt_all + int64_t(blockIdx.y) * stride, blockIdx.x * TC);
}

// kept row a of one right-hand side (Vt and V of that RHS)
template <typename T, class F>
__device__ __forceinline__ void inv_row_body(int M, int logM, int n_lat, const T* __restrict__ tw,
                                             const T* __restrict__ Vt, T* __restrict__ V, int64_t a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s = reinterpret_cast<T*>(smem_raw);       // F layout
  constexpr int kDiv = F::kDiv;
  T v[kDiv];                                   // M / kDiv threads: kDiv loads each, issued together
#pragma unroll
  for (int q = 0; q < kDiv; ++q) v[q] = Vt[a * M + threadIdx.x + q * blockDim.x];
#pragma unroll
  for (int q = 0; q < kDiv; ++q) s[F::at(threadIdx.x + q * blockDim.x)] = v[q];
  __syncthreads();
  F::run(s, M, logM, true, tw, threadIdx.x);
  __syncthreads();
  for (int b = threadIdx.x; b < n_lat; b += blockDim.x) V[a * M + b] = s[F::at(b)];
}

template <typename T, class F = LatFft<T>>
__global__ void __launch_bounds__(kFftMaxM / F::kDiv) k_inv_rows(int M, int logM, int n_lat, const T* __restrict__ tw,
                                                            const T* __restrict__ Vt_all, T* __restrict__ V_all,
                                                            int64_t stride) {
  inv_row_body<T, F>(M, logM, n_lat, tw, Vt_all + int64_t(blockIdx.y) * stride, V_all + int64_t(blockIdx.y) * stride,
                  blockIdx.x);
}

// Length of the short forward column transforms (0: none, full length): the
// source rows sit on every Ne-th lattice row, so when Ne divides M the column
// transform is a length-M/Ne transform repeated; it needs 2 (M/Ne) / 8 threads
// of the column's M / kDiv.
__host__ __device__ inline int short_len(int M, int Ne, int L, int kDiv, int& logMs) {
  logMs = 0;
  if (M % Ne != 0 || L + 1 > M / Ne) return 0;
  const int m = M / Ne;
  if (m < 16 || m > 4 * M / kDiv || (m & (m - 1)) != 0) return 0;
  while ((1 << logMs) < m) ++logMs;
  return m;
}

// columns per block of the column pass: one, so that the M blocks of M / kDiv
// threads are all resident at once, several per SM (wider blocks left SMs idle:
// complex64 with 8 columns ran 128 blocks; complex128 with 4 ran 1.7 waves)
template <typename T>
int conv_cols_tc(int) {
  return 1;
}

// whether the lattice passes run at size M with TC columns per block of the
// column pass (threads within the launch bound, shared memory within 200 KB)
template <typename T, class F>
bool lattice_fits(int M, int TC) {
  if (M < 256 || M > kFftMaxM || (M & (M - 1)) || TC < 1 || M % TC != 0) return false;
  const size_t pm = size_t(F::len(M)) * sizeof(T);
  return TC * (M / F::kDiv) <= F::kColThreads && 2 * TC * pm <= 200 * 1024;
}

bool lattice_cols_fit(bool fp64, bool radix4, int M, int TC) {
  if (fp64) return lattice_fits<double2, LatFft<double2>>(M, TC);
  return radix4 ? lattice_fits<float2, LatFft4<float2>>(M, TC) : lattice_fits<float2, LatFft<float2>>(M, TC);
}

template <typename T, class F>
cudaError_t lattice_conv_f(const ApplyData<T>& d, int nr, cudaStream_t st) {
  const int M = d.M;
  const int TC = d.conv_tc > 0 ? d.conv_tc : conv_cols_tc<T>(M);
  if (!lattice_fits<T, F>(M, TC)) return cudaErrorInvalidValue;
  constexpr int kDiv = F::kDiv;
  const size_t pm = size_t(F::len(M)) * sizeof(T);   // one column or row in the F layout
  static unsigned long long attr_done = 0;
  if (first_on_device(attr_done)) {
    const int prow = int(F::len(kFftMaxM) * sizeof(T));
    cudaFuncSetAttribute(k_src_rows<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, prow);
    cudaFuncSetAttribute(k_inv_rows<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, prow);
    cudaFuncSetAttribute(k_conv_cols<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  }
  // R (2 (L+1) x M) lives in Sd, Vt (n_lat x M) in Sm, V (n_lat x M) back in Sd
  const int64_t stride = d.lattice_rows() * M;
  k_src_rows<T, F><<<dim3(d.L + 1, 2, nr), M / kDiv, pm, st>>>(M, d.logM, d.n_lat, d.Ne, d.L, d.occ_of_cell,
                                                                     d.sigma, d.n_es, d.nocc, d.tw, d.Sd, stride);
  int logMs = 0;
  const int Ms = short_len(M, d.Ne, d.L, kDiv, logMs);
  k_conv_cols<T, F><<<dim3(M / TC, nr), TC * (M / kDiv), 2 * TC * pm, st>>>(
      M, d.logM, d.n_lat, d.Ne, d.L, TC, Ms, logMs, d.Sd, d.Gq, d.Dq, d.tw, d.Sm, stride);
  k_inv_rows<T, F><<<dim3(d.n_lat, nr), M / kDiv, pm, st>>>(M, d.logM, d.n_lat, d.tw, d.Sm, d.Sd, stride);
  return cudaGetLastError();
}

template <typename T>
cudaError_t lattice_conv(const ApplyData<T>& d, int nr, cudaStream_t st) {
  if constexpr (sizeof(T) == 8) {
    if (d.fft_r4) return lattice_conv_f<T, LatFft4<T>>(d, nr, st);
  }
  return lattice_conv_f<T, LatFft<T>>(d, nr, st);
}

// The lattice convolutions of several instances of one lattice size at once
// (one right-hand side each): work lists of (instance, face row), (instance,
// column) and (instance, kept row); every block runs the same body as the
// single-instance kernels on its instance's arrays, so each instance's result
// is the single apply's bit for bit.
template <typename T>
__global__ void __launch_bounds__(kFftMaxM / LatFft<T>::kDiv) k_src_rows_multi(const int2* __restrict__ work,
                                                                              const InstData<T>* __restrict__ I) {
  const int2 w = work[blockIdx.x];
  const ApplyData<T>& d = I[w.x].d;
  src_row_body<T, LatFft<T>>(d.M, d.logM, d.n_lat, d.Ne, d.L, d.occ_of_cell, d.sigma, d.n_es, d.tw, d.Sd, w.y, blockIdx.y);
}

template <typename T>
__global__ void __launch_bounds__(kFftMaxM / LatFft<T>::kDiv) k_conv_cols_multi(const int2* __restrict__ work,
                                                                               const InstData<T>* __restrict__ I) {
  const int2 w = work[blockIdx.x];
  const ApplyData<T>& d = I[w.x].d;
  int logMs = 0;
  const int Ms = short_len(d.M, d.Ne, d.L, LatFft<T>::kDiv, logMs);
  conv_cols_body<T, LatFft<T>>(d.M, d.logM, d.n_lat, d.Ne, d.L, 1, Ms, logMs, d.Sd, d.Gq, d.Dq, d.tw, d.Sm, w.y);
}

template <typename T>
__global__ void __launch_bounds__(kFftMaxM / LatFft<T>::kDiv) k_inv_rows_multi(const int2* __restrict__ work,
                                                                              const InstData<T>* __restrict__ I) {
  const int2 w = work[blockIdx.x];
  const ApplyData<T>& d = I[w.x].d;
  inv_row_body<T, LatFft<T>>(d.M, d.logM, d.n_lat, d.tw, d.Sm, d.Sd, w.y);
}

template <typename T>
cudaError_t lattice_conv_multi(const InstData<T>* I, const LatWork& w, cudaStream_t st) {
  const int M = w.M;
  if (M < 256 || M > kFftMaxM || (M & (M - 1))) return cudaErrorInvalidValue;
  constexpr int kDiv = LatFft<T>::kDiv;
  const size_t pm = size_t(LatFft<T>::len(M)) * sizeof(T);
  static unsigned long long attr_done = 0;
  if (first_on_device(attr_done)) {
    const int prow = int(LatFft<T>::len(kFftMaxM) * sizeof(T));
    cudaFuncSetAttribute(k_src_rows_multi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, prow);
    cudaFuncSetAttribute(k_conv_cols_multi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * prow);
    cudaFuncSetAttribute(k_inv_rows_multi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, prow);
  }
  if (w.n_src > 0) k_src_rows_multi<T><<<dim3(w.n_src, 2), M / kDiv, pm, st>>>(w.src, I);
  if (w.n_cols > 0) k_conv_cols_multi<T><<<w.n_cols, M / kDiv, 2 * pm, st>>>(w.cols, I);
  if (w.n_rows > 0) k_inv_rows_multi<T><<<w.n_rows, M / kDiv, pm, st>>>(w.rows, I);
  return cudaGetLastError();
}

// ------------------------------------------------------------ local expansion
// gamma_c = B^+ V_c - sum_o (B^+ T_o) sigma_{c+o} as one contraction per cell
//   gamma_c (nfb2 x R) = LA (nfb2 x K) X_c (K x R),  K = n_loc + 9 n_es,
// where X_c stacks the cell's (Ne+1)^2 lattice values and the strengths of its
// 3 x 3 neighbours (zero for empty or missing neighbours).  LA is stored
// transposed ([K][nfb2], LAs = Re + Im for complex128) and shared by every cell.
// One block per occupied cell and all R right-hand sides: X_c is staged once,
// then the per-cell contraction above (thread per output row and segment).
template <typename T, int R>
__device__ __forceinline__ void local_coeffs_body(int k, int nocc, const int* __restrict__ occ_cells,
                                                  const int* __restrict__ occ_of_cell, int L, int Ne, int M,
                                                  const T* __restrict__ V_all, const T* __restrict__ LA,
                                                  const double* __restrict__ LAs, const T* __restrict__ sigma_all,
                                                  int n_es, int nfb2, T* __restrict__ gamma_all, int64_t stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n_loc = (Ne + 1) * (Ne + 1);
  const int n_nb = 9 * n_es;
  const int K = n_loc + n_nb;
  const int ld = (K + 1) & ~1;
  const Staged<T> X = staged_at<T>(smem_raw, ld, R);
  const int c = occ_cells[k], ci = c % L, cj = c / L;
  for (int e = threadIdx.x; e < R * n_loc; e += blockDim.x) {
    const int r = e / n_loc, p = e - r * n_loc;
    const int a = p / (Ne + 1), b = p - a * (Ne + 1);
    X.put(r, p, V_all[int64_t(r) * stride + int64_t(ci * Ne + a) * M + cj * Ne + b]);
  }
  for (int e = threadIdx.x; e < R * n_nb; e += blockDim.x) {
    const int r = e / n_nb, q = e - r * n_nb;
    const int o = q / n_es, l = q - o * n_es;
    const int ni = ci + o / 3 - 1, nj = cj + o % 3 - 1;
    T v = czero(T{});
    if (ni >= 0 && ni < L && nj >= 0 && nj < L) {
      const int occ = occ_of_cell[nj * L + ni];
      if (occ >= 0) v = sigma_all[(int64_t(r) * nocc + occ) * n_es + l];
    }
    X.put(r, n_loc + q, v);
  }
  __syncthreads();
  const int S = blockDim.x / nfb2, t = threadIdx.x, o = t % nfb2, sg = t / nfb2;
  CAcc<T> acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r].zero();
  if (sg < S) contract_segment<T, R>(LA, LAs, nfb2, o, sg, K, S, X, acc);
  segment_sums_out<T, R>(acc, smem_raw, nfb2, o, sg, S, gamma_all + int64_t(k) * nfb2, int64_t(nocc) * nfb2);
}

// shared memory of the local-coefficient kernels (K = n_loc + 9 n_es inputs)
template <typename T>
size_t local_smem(int R, int K) {
  return contraction_smem<T>(R, size_t(R) * ((K + 1) & ~1) * Staged<T>::kBytes);
}

template <typename T, int R>
__global__ void __launch_bounds__(256) k_local_coeffs(int nocc, const int* __restrict__ occ_cells,
                                                      const int* __restrict__ occ_of_cell, int L, int Ne, int M,
                                                      const T* __restrict__ V_all, const T* __restrict__ LA,
                                                      const double* __restrict__ LAs, const T* __restrict__ sigma_all,
                                                      int n_es, int nfb2, T* __restrict__ gamma_all, int64_t stride) {
  local_coeffs_body<T, R>(blockIdx.x, nocc, occ_cells, occ_of_cell, L, Ne, M, V_all, LA, LAs, sigma_all, n_es, nfb2,
                          gamma_all, stride);
}

// ------------------------------------------------------------ near field + assembly
// One warp per target row q: the dense block row of q's cell against the three
// contiguous column ranges of the 3 x 3 neighbourhood (coalesced, no column
// indices), the CSR remainder, the local expansion Phi_q . gamma_c, and the
// assembly out_q = u_q + kappa^2 (near + far).
// One block per work item = (occupied cell, chunk of 8 NRW target rows), so
// that the large cells near the boundary are spread over many SMs.  Each warp
// owns NRW rows of the chunk and R right-hand sides at once: for every column of
// the cell's 3 x 3 neighbourhood it loads the NRW weights from HBM and the R
// input values from shared memory (staged chunk by chunk, one contiguous run
// per RHS, zero in the padding), so one pass over the weights serves all R
// right-hand sides and every staged value serves NRW rows.
// Every row is summed in the same order whatever R and NRW (lane l takes the
// columns l, l + 32, ... (pairs for complex64) in chunks that start at multiples
// of 64 columns, then one warp reduction), so a batched apply reproduces the
// single-RHS results bit for bit.
constexpr int kNearSmem = 32768;   // bytes of staged input values per chunk

// complex128: a complex product with three real multiplications (Gauss's
// form).  Weight w = a + ib comes with s = a + b (Ws), the staged value x = c + id
// as c and (c + d, d - c).  P += s c, Q += b (c + d), S += a (d - c); then
// Re(w x) = P - Q and Im(w x) = P + S.  Three FP64 FMAs per product instead of
// four: the kernel is bound by the FP64 pipe, not by the extra 8 bytes read.
// Sums run over the chunk's columns t of W[row_i][c0 + t] x_r[t] for the first
// NR rows of the warp.
template <int R, int NRW, int NR>
__device__ __forceinline__ void near_chunk_gauss(const double2* __restrict__ wk, const double* __restrict__ wsk,
                                                 const int* rows, int nblk, int c0, int cl,
                                                 const double* usc, const double2* usef, int CH, int lane,
                                                 double (&P)[NRW][R], double (&Q)[NRW][R], double (&S)[NRW][R]) {
  const double2* w[NR];
  const double* ws[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) {
    w[i] = wk + int64_t(rows[i]) * nblk + c0;
    ws[i] = wsk + int64_t(rows[i]) * nblk + c0;
  }
#pragma unroll 2
  for (int t = lane; t < cl; t += 32) {
    double2 a[NR];
    double sa[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      a[i] = w[i][t];
      sa[i] = ws[i][t];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const double c = usc[r * CH + t];
      const double2 ef = usef[r * CH + t];
#pragma unroll
      for (int i = 0; i < NR; ++i) {
        P[i][r] = fma(sa[i], c, P[i][r]);
        Q[i][r] = fma(a[i].y, ef.x, Q[i][r]);
        S[i][r] = fma(a[i].x, ef.y, S[i][r]);
      }
    }
  }
}

// complex64: two columns per lane and 16-byte loads (rows, chunk starts and
// chunk lengths are even, so every pair is 16-byte aligned)
template <int R, int NRW>
__device__ __forceinline__ void near_chunk_pairs(const float2* __restrict__ wk, const int* rows, int nblk, int c0,
                                                 int cl, const float2* us, int CH, int lane,
                                                 float2 (&acc)[NRW][R]) {
  const float4* w[NRW];
#pragma unroll
  for (int i = 0; i < NRW; ++i) w[i] = reinterpret_cast<const float4*>(wk + int64_t(rows[i]) * nblk + c0);
  const int np = cl >> 1;
  constexpr int kUnroll = NRW * R >= 32 ? 1 : 2;     // the largest accumulator sets keep to 128 registers
#pragma unroll kUnroll
  for (int t = lane; t < np; t += 32) {
    float4 a[NRW];
#pragma unroll
    for (int i = 0; i < NRW; ++i) a[i] = w[i][t];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 x = reinterpret_cast<const float4*>(us + r * CH)[t];
      const float2 x0 = make_float2(x.x, x.y), x1 = make_float2(x.z, x.w);
#pragma unroll
      for (int i = 0; i < NRW; ++i)
        acc[i][r] = cfma(make_float2(a[i].z, a[i].w), x1, cfma(make_float2(a[i].x, a[i].y), x0, acc[i][r]));
    }
  }
}

template <typename T, int R, int NRW>
__device__ __forceinline__ void near_eval_body(const int2 item, const int64_t* __restrict__ occ_start,
                                               const int64_t* __restrict__ blk_off, const int* __restrict__ blk_seg,
                                               const T* __restrict__ Wb, const double* __restrict__ Ws,
                                               const int64_t* __restrict__ rem_row,
                                               const int* __restrict__ rem_col, const T* __restrict__ rem_val,
                                               const T* __restrict__ u, const double* __restrict__ utc,
                                               const double2* __restrict__ utef, int64_t N,
                                               const T* __restrict__ Phi,
                                               const T* __restrict__ gamma, int nocc, int nfb2,
                                               typename RealOf<T>::R kappa2, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr bool kC128 = sizeof(T) == 16;
  // columns per chunk (a multiple of 64); complex128 stages 24 bytes per value
  constexpr int CH = kC128 ? kNearSmem / (R * 24) / 64 * 64 : kNearSmem / int(R * sizeof(T));
  static_assert(CH % 64 == 0 && CH > 0, "chunks must start at multiples of 64 columns");
  T* us = reinterpret_cast<T*>(smem_raw);               // complex64: [rhs][column]
  double* usc = reinterpret_cast<double*>(smem_raw);    // complex128: c = Re x, [rhs][column]
  double2* usef = reinterpret_cast<double2*>(smem_raw + size_t(R) * CH * sizeof(double));   // (c + d, d - c)
  auto put = [&](int r, int col, T v) {
    if constexpr (kC128) {
      usc[r * CH + col] = v.x;
      usef[r * CH + col] = make_double2(v.x + v.y, v.y - v.x);
    } else {
      us[r * CH + col] = v;
    }
  };
  const int k = item.x;
  const int* sg = blk_seg + 6 * k;
  const int l0 = sg[1], l1 = sg[3], l2 = sg[5];
  const int p0 = (l0 + 1) & ~1, p1 = (l1 + 1) & ~1;
  const int nblk = p0 + p1 + ((l2 + 1) & ~1);
  const int64_t r0 = occ_start[k];
  const int nrow = int(occ_start[k + 1] - r0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* wk = Wb + blk_off[k];
  int rows[NRW];
  bool valid[NRW];
#pragma unroll
  for (int i = 0; i < NRW; ++i) {
    const int r = item.y + warp + 8 * i;
    valid[i] = r < nrow;
    rows[i] = valid[i] ? r : item.y;
  }
  T acc[NRW][R];
#pragma unroll
  for (int i = 0; i < NRW; ++i)
#pragma unroll
    for (int r = 0; r < R; ++r) acc[i][r] = czero(T{});
  constexpr int GN = kC128 ? NRW : 1, GR = kC128 ? R : 1;    // three-multiplication sums (complex128)
  double gP[GN][GR], gQ[GN][GR], gS[GN][GR];
#pragma unroll
  for (int i = 0; i < GN; ++i)
#pragma unroll
    for (int r = 0; r < GR; ++r) gP[i][r] = gQ[i][r] = gS[i][r] = 0.0;
  for (int c0 = 0; c0 < nblk; c0 += CH) {
    const int cl = min(CH, nblk - c0);
    __syncthreads();
    // node index of column cc of the block (-1: padding)
    auto node_of = [&](int cc) -> int {
      if (cc < p0) return cc < l0 ? sg[0] + cc : -1;
      if (cc < p0 + p1) { const int o = cc - p0; return o < l1 ? sg[2] + o : -1; }
      const int o = cc - p0 - p1;
      return o < l2 ? sg[4] + o : -1;
    };
    if (kC128 && utc) {
      // complex128 with the staged forms written by the projection: plain copies
#pragma unroll 1
      for (int r = 0; r < R; ++r)
        for (int col = threadIdx.x; col < cl; col += blockDim.x) {
          const int q = node_of(c0 + col);
          usc[r * CH + col] = q >= 0 ? utc[int64_t(r) * N + q] : 0.0;
          usef[r * CH + col] = q >= 0 ? utef[int64_t(r) * N + q] : make_double2(0.0, 0.0);
        }
    } else if constexpr (R == 1) {
      for (int col = threadIdx.x; col < cl; col += blockDim.x) {   // us[col]
        const int cc = c0 + col;
        T v = czero(T{});
        if (cc < p0) { if (cc < l0) v = u[sg[0] + cc]; }
        else if (cc < p0 + p1) { const int o = cc - p0; if (o < l1) v = u[sg[2] + o]; }
        else { const int o = cc - p0 - p1; if (o < l2) v = u[sg[4] + o]; }
        put(0, col, v);
      }
    } else {
      // us[r * CH + col]: one contiguous run per RHS (conflict-free reads)
#pragma unroll 1
      for (int r = 0; r < R; ++r) {
        const T* ur = u + int64_t(r) * N;
        for (int col = threadIdx.x; col < cl; col += blockDim.x) {
          const int cc = c0 + col;
          T v = czero(T{});
          if (cc < p0) { if (cc < l0) v = ur[sg[0] + cc]; }
          else if (cc < p0 + p1) { const int o = cc - p0; if (o < l1) v = ur[sg[2] + o]; }
          else { const int o = cc - p0 - p1; if (o < l2) v = ur[sg[4] + o]; }
          put(r, col, v);
        }
      }
    }
    __syncthreads();
    if constexpr (kC128) {
      // FP64 is bound by the FP64 pipe: a warp skips its rows past the end of the cell
      static_assert(NRW == 2, "the FP64 variant takes two rows per warp");
      const double* wsk = Ws + blk_off[k];
      if (valid[1]) near_chunk_gauss<R, NRW, 2>(wk, wsk, rows, nblk, c0, cl, usc, usef, CH, lane, gP, gQ, gS);
      else if (valid[0]) near_chunk_gauss<R, NRW, 1>(wk, wsk, rows, nblk, c0, cl, usc, usef, CH, lane, gP, gQ, gS);
    } else {
      // complex64 is bound by HBM: a row past the end re-reads cached weights
      near_chunk_pairs<R, NRW>(wk, rows, nblk, c0, cl, us, CH, lane, acc);
    }
  }
  if constexpr (kC128) {
#pragma unroll
    for (int i = 0; i < NRW; ++i)
#pragma unroll
      for (int r = 0; r < R; ++r) acc[i][r] = mk(gP[i][r] - gQ[i][r], gP[i][r] + gS[i][r]);
  }
#pragma unroll
  for (int i = 0; i < NRW; ++i) {
    if (!valid[i]) continue;                      // warp-uniform
    const int64_t q = r0 + rows[i];
    for (int64_t e = rem_row[q] + lane; e < rem_row[q + 1]; e += 32) {
      const T w = rem_val[e];
      const int c = rem_col[e];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[i][r] = cfma(w, u[r * N + c], acc[i][r]);
    }
    const T* ph = Phi + q * nfb2;
    for (int n = lane; n < nfb2; n += 32) {
      const T p = ph[n];
#pragma unroll
      for (int r = 0; r < R; ++r) acc[i][r] = cfma(p, gamma[(int64_t(r) * nocc + k) * nfb2 + n], acc[i][r]);
    }
    if constexpr (!kC128) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const T v = warp_sum(acc[i][r]);
        if (lane == 0) {
          const T uq = u[r * N + q];
          out[r * N + q] = mk(uq.x + kappa2 * v.x, uq.y + kappa2 * v.y);
        }
      }
    }
  }
  if constexpr (kC128) {
    // One transposed warp reduction per RHS over the four values (Re, Im of the
    // two rows): exchange halves across lanes 16 apart, then one value across
    // lanes 8 apart, then butterflies; 6 FP64 adds per lane instead of 20.
    // Lane 8 j ends up with the whole sum of value j.
    const bool hi16 = lane & 16, hi8 = lane & 8;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      double a = hi16 ? acc[1][r].x : acc[0][r].x, b = hi16 ? acc[1][r].y : acc[0][r].y;
      const double c = hi16 ? acc[0][r].x : acc[1][r].x, d = hi16 ? acc[0][r].y : acc[1][r].y;
      a += __shfl_xor_sync(0xffffffffu, c, 16);
      b += __shfl_xor_sync(0xffffffffu, d, 16);
      double x = hi8 ? b : a;
      x += __shfl_xor_sync(0xffffffffu, hi8 ? a : b, 8);
      x += __shfl_xor_sync(0xffffffffu, x, 4);
      x += __shfl_xor_sync(0xffffffffu, x, 2);
      x += __shfl_xor_sync(0xffffffffu, x, 1);
      const int comp = (lane >> 3) & 1;
      if ((lane & 7) == 0 && (hi16 ? valid[1] : valid[0])) {
        const int64_t q = r0 + (hi16 ? rows[1] : rows[0]);
        const double uq = reinterpret_cast<const double*>(u + r * N + q)[comp];
        reinterpret_cast<double*>(out + r * N + q)[comp] = uq + kappa2 * x;
      }
    }
  }
}

#define LS_NEAR_ARGS                                                                                          \
  const int2 *__restrict__ items, const int64_t *__restrict__ occ_start, const int64_t *__restrict__ blk_off,     \
      const int *__restrict__ blk_seg, const T *__restrict__ Wb, const double *__restrict__ Ws,                   \
      const int64_t *__restrict__ rem_row,                                                                        \
      const int *__restrict__ rem_col, const T *__restrict__ rem_val, const T *__restrict__ u,                    \
      const double *__restrict__ utc, const double2 *__restrict__ utef, int64_t N,                                \
      const T *__restrict__ Phi, const T *__restrict__ gamma, int nocc, int nfb2,                                 \
      typename RealOf<T>::R kappa2, T *__restrict__ out
#define LS_NEAR_PASS items[blockIdx.x], occ_start, blk_off, blk_seg, Wb, Ws, rem_row, rem_col, rem_val, u, utc, utef, N, Phi, gamma, nocc, nfb2, \
                     kappa2, out
// two rows per warp, 16-row items: registers left to the compiler
template <typename T, int R>
__global__ void __launch_bounds__(256) k_near_eval(LS_NEAR_ARGS) {
  near_eval_body<T, R, 2>(LS_NEAR_PASS);
}
// single-RHS complex128: five blocks per SM (the FP64 pipe hides more latency)
template <typename T, int R>
__global__ void __launch_bounds__(256, 5) k_near_eval5(LS_NEAR_ARGS) {
  near_eval_body<T, R, 2>(LS_NEAR_PASS);
}
// four rows per warp, 32-row items: two blocks per SM
template <typename T, int R>
__global__ void __launch_bounds__(256, 2) k_near_eval4(LS_NEAR_ARGS) {
  near_eval_body<T, R, 4>(LS_NEAR_PASS);
}
#undef LS_NEAR_ARGS
#undef LS_NEAR_PASS

// rows per warp: 2, or 4 for multi-RHS complex64 (every staged value then
// serves four rows; 32-row work items)
template <typename T, int R>
constexpr int near_rows_per_warp() { return sizeof(T) == 8 && R >= 2 ? 4 : 2; }

template <typename T, int R>
cudaError_t apply_r(const ApplyData<T>& d, const T* u, T* out, cudaStream_t st, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], st);
  bool proj_done = false;
  if constexpr (sizeof(T) == 8 && R >= 8) {
    if (!d.proj_cuda && d.n_es <= 64) {     // tensor cores (device/contract_tc.cu)
      const cudaError_t e0 = project_tc<R>(d, u, st);
      if (e0 != cudaSuccess) return e0;
      proj_done = true;
    }
  }
  if (!proj_done)
    k_es_project<T, R><<<d.n_pieces, 256, contraction_smem<T>(R, kProjStage), st>>>(
        d.pieces, d.piece_off, d.nocc, d.occ_start, d.P_off, d.P, d.Ps, u, d.N, d.sigma, d.proj_part, d.proj_count,
        d.n_es, d.utc, d.utef);
  if (ev) cudaEventRecord(ev[1], st);
  if (ev) cudaEventRecord(ev[2], st);        // the lattice fill is fused into k_src_rows
  cudaError_t e = lattice_conv(d, R, st);
  if (e != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[3], st);
  const size_t sm_local = local_smem<T>(R, d.n_loc + 9 * d.n_es);
  static unsigned long long local_attr = 0;     // X_c above 48 KB (large N_eq with many RHS)
  if (first_on_device(local_attr)) {
    cudaFuncSetAttribute(k_local_coeffs<T, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  }
  if (sm_local > 160 * 1024) return cudaErrorInvalidValue;
  bool local_done = false;
  if constexpr (sizeof(T) == 8 && R >= 8) {
    if (!d.local_cuda && d.LAt) {           // tensor cores (device/contract_tc.cu)
      const cudaError_t e3 = local_coeffs_tc<R>(d, st);
      if (e3 != cudaSuccess) return e3;
      local_done = true;
    }
  }
  if (!local_done)
    k_local_coeffs<T, R><<<d.nocc, 256, sm_local, st>>>(d.nocc, d.occ_cells, d.occ_of_cell, d.L, d.Ne, d.M, d.Sd,
                                                         d.LA, d.LAs, d.sigma, d.n_es, d.nfb2, d.gamma,
                                                         d.lattice_rows() * d.M);
  if (ev) cudaEventRecord(ev[4], st);
  if constexpr (sizeof(T) == 8 && R >= 8) {
    if (!d.near_cuda) {
      const cudaError_t e2 = near_eval_tc<R>(d, u, out, st);
      if (e2 != cudaSuccess) return e2;
    } else {
      k_near_eval4<T, R><<<d.n_items32, 256, kNearSmem, st>>>(d.items32, d.occ_start, d.blk_off, d.blk_seg, d.Wb,
                                                              d.Ws, d.rem_row, d.rem_col, d.rem_val, u, d.utc, d.utef,
                                                              d.N, d.Phi, d.gamma, d.nocc, d.nfb2,
                                                              typename RealOf<T>::R(d.kappa2), out);
    }
  } else if constexpr (near_rows_per_warp<T, R>() == 4)
    k_near_eval4<T, R><<<d.n_items32, 256, kNearSmem, st>>>(d.items32, d.occ_start, d.blk_off, d.blk_seg, d.Wb,
                                                            d.Ws, d.rem_row, d.rem_col, d.rem_val, u, d.utc, d.utef, d.N, d.Phi,
                                                            d.gamma, d.nocc, d.nfb2,
                                                            typename RealOf<T>::R(d.kappa2), out);
  else if constexpr (sizeof(T) == 16 && R == 1)
    k_near_eval5<T, R><<<d.n_items, 256, kNearSmem, st>>>(d.items, d.occ_start, d.blk_off, d.blk_seg, d.Wb,
                                                          d.Ws, d.rem_row, d.rem_col, d.rem_val, u, d.utc, d.utef,
                                                          d.N, d.Phi, d.gamma, d.nocc, d.nfb2,
                                                          typename RealOf<T>::R(d.kappa2), out);
  else
    k_near_eval<T, R><<<d.n_items, 256, kNearSmem, st>>>(d.items, d.occ_start, d.blk_off, d.blk_seg, d.Wb,
                                                         d.Ws, d.rem_row, d.rem_col, d.rem_val, u, d.utc, d.utef, d.N, d.Phi, d.gamma,
                                                         d.nocc, d.nfb2, typename RealOf<T>::R(d.kappa2), out);
  if (ev) cudaEventRecord(ev[5], st);
  return cudaGetLastError();
}

// ------------------------------------------------------------ multi-instance batch
// work = (instance, projection piece of that instance): the same pieces as the
// single-instance apply, so every instance sums as it does alone
// blocks per SM the multi-instance projection and local step are compiled for:
// reading the instance's fields from memory costs registers (48 against 32 in
// the single-instance kernels); these caps keep the complex64 kernels near the
// single-instance occupancy with at most 8 bytes spilled (the FP64 projection
// keeps four blocks: at six it would spill 80 bytes)
template <typename T>
constexpr int kProjMultiBlocks = sizeof(T) == 8 ? 6 : 4;
constexpr int kLocalMultiBlocks = 7;

template <typename T>
__global__ void __launch_bounds__(256, kProjMultiBlocks<T>) k_es_project_multi(const int2* __restrict__ work,
                                                          const InstData<T>* __restrict__ I, const T* __restrict__ u) {
  const int2 w = work[blockIdx.x];
  const ApplyData<T>& d = I[w.x].d;
  es_project_piece<T, 1>(d.pieces[w.y], d.piece_off, d.nocc, d.occ_start, d.P_off, d.P, d.Ps, u + I[w.x].off, d.N,
                         d.sigma, d.proj_part, d.proj_count, d.n_es, d.utc, d.utef);
}

template <typename T>
__global__ void __launch_bounds__(256, kLocalMultiBlocks) k_local_coeffs_multi(const int2* __restrict__ cells,
                                                            const InstData<T>* __restrict__ I) {
  const int2 c = cells[blockIdx.x];
  const ApplyData<T>& d = I[c.x].d;
  local_coeffs_body<T, 1>(c.y, d.nocc, d.occ_cells, d.occ_of_cell, d.L, d.Ne, d.M, d.Sd, d.LA, d.LAs, d.sigma,
                          d.n_es, d.nfb2, d.gamma, d.lattice_rows() * d.M);
}

// five blocks per SM, as the single-instance kernels: the instance's fields
// come from memory here, and at 52 registers the kernel fit only four blocks
// and streamed the weights at 63% of HBM
template <typename T>
__global__ void __launch_bounds__(256, 5) k_near_eval_multi(const int4* __restrict__ items,
                                                         const InstData<T>* __restrict__ I, const T* __restrict__ u,
                                                         T* __restrict__ out) {
  const int4 it = items[blockIdx.x];
  const ApplyData<T>& d = I[it.x].d;
  const int64_t off = I[it.x].off;
  near_eval_body<T, 1, 2>(make_int2(it.y, it.z), d.occ_start, d.blk_off, d.blk_seg, d.Wb, d.Ws, d.rem_row,
                          d.rem_col, d.rem_val, u + off, d.utc, d.utef, d.N, d.Phi, d.gamma, d.nocc, d.nfb2,
                          typename RealOf<T>::R(d.kappa2), out + off);
}

template <typename T>
cudaError_t apply_multi(const InstData<T>* dev_inst, int n_ids,
                        const int2* pieces, int n_pieces, const int2* cells, int n_cells, const int4* items,
                        int n_items, int max_K, const LatWork* lat, int n_lat_groups, const T* u, T* out,
                        cudaStream_t st) {
  if (n_ids <= 0 || n_pieces <= 0 || n_cells <= 0 || n_items <= 0) return cudaSuccess;
  k_es_project_multi<T><<<n_pieces, 256, contraction_smem<T>(1, kProjStage), st>>>(pieces, dev_inst, u);
  for (int g = 0; g < n_lat_groups; ++g) {
    const cudaError_t e = lattice_conv_multi(dev_inst, lat[g], st);
    if (e != cudaSuccess) return e;
  }
  const size_t sm_local = local_smem<T>(1, max_K);
  static unsigned long long attr = 0;
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(k_local_coeffs_multi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  }
  if (sm_local > 160 * 1024) return cudaErrorInvalidValue;
  k_local_coeffs_multi<T><<<n_cells, 256, sm_local, st>>>(cells, dev_inst);
  k_near_eval_multi<T><<<n_items, 256, kNearSmem, st>>>(items, dev_inst, u, out);
  return cudaGetLastError();
}

template cudaError_t apply_multi<double2>(const InstData<double2>*, int,
                                          const int2*, int, const int2*, int, const int4*, int, int, const LatWork*,
                                          int, const double2*, double2*, cudaStream_t);
template cudaError_t apply_multi<float2>(const InstData<float2>*, int,
                                         const int2*, int, const int2*, int, const int4*, int, int, const LatWork*,
                                         int, const float2*, float2*, cudaStream_t);

template <typename T>
cudaError_t apply_batch(const ApplyData<T>& d, const T* u, T* out, int nr, cudaStream_t st, cudaEvent_t* ev) {
  switch (nr) {
    case 1: return apply_r<T, 1>(d, u, out, st, ev);
    case 2: return apply_r<T, 2>(d, u, out, st, ev);
    case 4: return apply_r<T, 4>(d, u, out, st, ev);
    case 8:
      if constexpr (sizeof(T) == 8) return apply_r<T, 8>(d, u, out, st, ev);
      return cudaErrorInvalidValue;
    case 16:
      if constexpr (sizeof(T) == 8) return apply_r<T, 16>(d, u, out, st, ev);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t apply_one(const ApplyData<T>& d, const T* u, T* out, cudaStream_t st, cudaEvent_t* ev) {
  return apply_batch(d, u, out, 1, st, ev);
}

template cudaError_t apply_one<double2>(const ApplyData<double2>&, const double2*, double2*, cudaStream_t,
                                        cudaEvent_t*);
template cudaError_t apply_one<float2>(const ApplyData<float2>&, const float2*, float2*, cudaStream_t,
                                       cudaEvent_t*);
template cudaError_t apply_batch<double2>(const ApplyData<double2>&, const double2*, double2*, int, cudaStream_t,
                                          cudaEvent_t*);
template cudaError_t apply_batch<float2>(const ApplyData<float2>&, const float2*, float2*, int, cudaStream_t,
                                         cudaEvent_t*);
template cudaError_t fft2d<double2>(double2*, int, int, const double2*, bool, cudaStream_t);
template cudaError_t fft2d<float2>(float2*, int, int, const float2*, bool, cudaStream_t);

// ------------------------------------------------------------ GMRES helpers
constexpr int kRedThreads = 256;

// chunks of about 1024 elements (16 KB of shared memory), at least 64 each
int gram_blocks(int64_t N) {
  int64_t b = (N + 1023) / 1024;
  if (b > 4096) b = 4096;
  if ((N + b - 1) / b > 4096) b = (N + 4095) / 4096;
  if (b < 1) b = 1;
  return int(b);
}

__device__ __forceinline__ double2 block_sum(double2 v, double2* red) {
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double2 r = make_double2(0, 0);
  if (threadIdx.x < 32) {
    r = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : make_double2(0, 0);
    r = warp_sum(r);
  }
  return r;
}

// h[j] = <V_j, w> for j < nv and h[nv].x = ||w||^2, in one pass over V: each
// block owns a contiguous chunk of the index range (w chunk in shared memory),
// each warp reduces whole vectors with shuffles only.
template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_gram_partial(const T* __restrict__ V, int nv,
                                                              int64_t vstride, const T* __restrict__ w,
                                                              int64_t N, int64_t chunk,
                                                              double2* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ws = reinterpret_cast<T*>(smem_raw);
  const int64_t i0 = int64_t(blockIdx.x) * chunk;
  const int n = int(i0 < N ? (N - i0 < chunk ? N - i0 : chunk) : 0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) ws[i] = w[i0 + i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = blockIdx.y * nw + warp; j <= nv && j < (blockIdx.y + 1) * nw; j += nw) {
    T acc = czero(T{});
    if (j < nv) {
      const T* vj = V + int64_t(j) * vstride + i0;
      T a1 = czero(T{}), a2 = czero(T{}), a3 = czero(T{});
      int i = lane;
      for (; i + 96 < n; i += 128) {
        const T v0 = vj[i], v1 = vj[i + 32], v2 = vj[i + 64], v3 = vj[i + 96];
        acc = cfma(cconj(v0), ws[i], acc);
        a1 = cfma(cconj(v1), ws[i + 32], a1);
        a2 = cfma(cconj(v2), ws[i + 64], a2);
        a3 = cfma(cconj(v3), ws[i + 96], a3);
      }
      for (; i < n; i += 32) acc = cfma(cconj(vj[i]), ws[i], acc);
      acc = cadd(cadd(acc, a1), cadd(a2, a3));
    } else {
      for (int i = lane; i < n; i += 32) acc.x = fma(ws[i].x, ws[i].x, fma(ws[i].y, ws[i].y, acc.x));
    }
    acc = warp_sum(acc);
    if (lane == 0) partial[int64_t(blockIdx.x) * (nv + 1) + j] = make_double2(acc.x, acc.y);
  }
}

// Complex128 Gram coefficients against a basis stored with S_j = Re V_j + Im V_j:
// conj(v) w = conj(conj(w) v), and conj(w) v takes three real multiplications
// with the staged w-side values (c, c - d, -c - d) (w = c + i d, v = a + i b):
// P += (a + b) c, Q += b (c - d), T += a (-c - d); Re = P - Q, Im = -(P + T).
// Row nv is ||w||^2 = ((c - d)^2 + (c + d)^2) / 2.
__global__ void __launch_bounds__(kRedThreads) k_gram3_partial(const double2* __restrict__ V,
                                                               const double* __restrict__ S, int nv,
                                                               int64_t vstride, const double2* __restrict__ w,
                                                               int64_t N, int64_t chunk,
                                                               double2* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* wq = reinterpret_cast<double2*>(smem_raw);              // (c - d, -c - d)
  double* wc = reinterpret_cast<double*>(smem_raw + chunk * sizeof(double2));   // c
  const int64_t i0 = int64_t(blockIdx.x) * chunk;
  const int n = int(i0 < N ? (N - i0 < chunk ? N - i0 : chunk) : 0);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 v = w[i0 + i];
    wc[i] = v.x;
    wq[i] = make_double2(v.x - v.y, -v.x - v.y);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = blockIdx.y * nw + warp; j <= nv && j < (blockIdx.y + 1) * nw; j += nw) {
    double2 acc = make_double2(0, 0);
    if (j < nv) {
      const double2* vj = V + int64_t(j) * vstride + i0;
      const double* sj = S + int64_t(j) * vstride + i0;
      double P[4] = {0, 0, 0, 0}, Q[4] = {0, 0, 0, 0}, T[4] = {0, 0, 0, 0};
      int i = lane;
      for (; i + 96 < n; i += 128) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const double2 v = vj[i + 32 * u];
          const double sv = sj[i + 32 * u];
          const double2 q = wq[i + 32 * u];
          P[u] = fma(sv, wc[i + 32 * u], P[u]);
          Q[u] = fma(v.y, q.x, Q[u]);
          T[u] = fma(v.x, q.y, T[u]);
        }
      }
      for (; i < n; i += 32) {
        const double2 v = vj[i];
        const double2 q = wq[i];
        P[0] = fma(sj[i], wc[i], P[0]);
        Q[0] = fma(v.y, q.x, Q[0]);
        T[0] = fma(v.x, q.y, T[0]);
      }
      const double p = (P[0] + P[1]) + (P[2] + P[3]), q = (Q[0] + Q[1]) + (Q[2] + Q[3]);
      const double t = (T[0] + T[1]) + (T[2] + T[3]);
      acc = make_double2(p - q, -(p + t));
    } else {
      for (int i = lane; i < n; i += 32) acc.x = fma(wq[i].x, wq[i].x, fma(wq[i].y, wq[i].y, acc.x));
      acc.x *= 0.5;
    }
    acc = warp_sum(acc);
    if (lane == 0) partial[int64_t(blockIdx.x) * (nv + 1) + j] = acc;
  }
}

// one warp per dot product: lanes stride over the per-block partial sums; with
// h3, also the triplet (Re h, Im h - Re h, Re h + Im h) of every coefficient
__global__ void k_gram_reduce(const double2* __restrict__ partial, int nblk, int nv1, double2* __restrict__ h,
                              double* __restrict__ h3 = nullptr) {
  const int j = blockIdx.x;
  double2 s = make_double2(0, 0);
  for (int b = threadIdx.x; b < nblk; b += 32) s = cadd(s, partial[int64_t(b) * nv1 + j]);
  s = warp_sum(s);
  if (threadIdx.x == 0) {
    h[j] = s;
    if (h3) {
      h3[3 * j] = s.x;
      h3[3 * j + 1] = s.y - s.x;
      h3[3 * j + 2] = s.x + s.y;
    }
  }
}

static int64_t gram_chunk(int64_t N) {
  const int nb = gram_blocks(N);
  return (N + nb - 1) / nb;
}

template <typename T>
cudaError_t gram_t(const T* V, int nv, int64_t vstride, const T* w, int64_t N, double2* partial, double2* h,
                   cudaStream_t st) {
  const int nb = gram_blocks(N);
  const int64_t chunk = gram_chunk(N);
  static unsigned long long attr = 0;
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(k_gram_partial<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  }
  // blockIdx.y selects 8 of the nv + 1 dot products: enough warps to hide the
  // FP64 latency (the complex multiply-adds of this kernel run on GB300's
  // narrow FP64 pipe)
  const int ng = (nv + 1 + kRedThreads / 32 - 1) / (kRedThreads / 32);
  k_gram_partial<T><<<dim3(nb, ng), kRedThreads, chunk * sizeof(T), st>>>(V, nv, vstride, w, N, chunk, partial);
  k_gram_reduce<<<nv + 1, 32, 0, st>>>(partial, nb, nv + 1, h);
  return cudaGetLastError();
}
cudaError_t gram(const double2* V, int nv, int64_t vstride, const double2* w, int64_t N, double2* partial,
                 double2* h, cudaStream_t st) {
  return gram_t(V, nv, vstride, w, N, partial, h, st);
}
cudaError_t gram(const float2* V, int nv, int64_t vstride, const float2* w, int64_t N, double2* partial, double2* h,
                 cudaStream_t st) {
  return gram_t(V, nv, vstride, w, N, partial, h, st);
}
cudaError_t gram3(const double2* V, const double* S, int nv, int64_t vstride, const double2* w, int64_t N,
                  double2* partial, double2* h, double* h3, cudaStream_t st) {
  const int nb = gram_blocks(N);
  const int64_t chunk = gram_chunk(N);
  static unsigned long long attr = 0;
  if (first_on_device(attr)) {
    cudaFuncSetAttribute(k_gram3_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
  }
  const int ng = (nv + 1 + kRedThreads / 32 - 1) / (kRedThreads / 32);
  k_gram3_partial<<<dim3(nb, ng), kRedThreads, chunk * 24, st>>>(V, S, nv, vstride, w, N, chunk, partial);
  k_gram_reduce<<<nv + 1, 32, 0, st>>>(partial, nb, nv + 1, h, h3);
  return cudaGetLastError();
}

// w -= sum_j h_j V_j, the sum over j split into G groups (blockIdx.y) so that
// G x N threads keep GB300's FP64 pipe and HBM busy; group sums go to
// part[g][i] and k_axpy_finish adds them in a fixed order (deterministic).
// coefficient h (always complex128) in the arithmetic of T
template <typename T> __device__ __forceinline__ T coef(double2 h);
template <> __device__ __forceinline__ double2 coef<double2>(double2 h) { return h; }
template <> __device__ __forceinline__ float2 coef<float2>(double2 h) { return make_float2(float(h.x), float(h.y)); }

template <typename T>
__global__ void __launch_bounds__(256) k_axpy_multi(const T* __restrict__ V, int nv, int64_t vstride,
                                                    const double2* __restrict__ h, T* __restrict__ part, int64_t N) {
  const int G = gridDim.y, g = blockIdx.y;
  const int j0 = (nv * g) / G, j1 = (nv * (g + 1)) / G;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
    T a0 = czero(T{}), a1 = czero(T{});
    int j = j0;
    for (; j + 1 < j1; j += 2) {
      const T v0 = V[int64_t(j) * vstride + i], v1 = V[int64_t(j + 1) * vstride + i];
      a0 = cfma(coef<T>(h[j]), v0, a0);
      a1 = cfma(coef<T>(h[j + 1]), v1, a1);
    }
    if (j < j1) a0 = cfma(coef<T>(h[j]), V[int64_t(j) * vstride + i], a0);
    part[int64_t(g) * N + i] = cadd(a0, a1);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_axpy_finish(const T* __restrict__ part, int G, T* __restrict__ w,
                                                     int64_t N) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
    T s = part[i];
    for (int g = 1; g < G; ++g) s = cadd(s, part[int64_t(g) * N + i]);
    w[i] = csub(w[i], s);
  }
}

static unsigned grid_for(int64_t N) {
  int64_t b = (N + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return unsigned(b < 1 ? 1 : b);
}

template <typename T>
cudaError_t axpy_multi_t(const T* V, int nv, int64_t vstride, const double2* h, T* w, T* part, int64_t N,
                         cudaStream_t st) {
  const int G = nv >= 32 ? kAxpyGroups : (nv >= 8 ? 2 : 1);
  k_axpy_multi<T><<<dim3(grid_for(N), G), 256, 0, st>>>(V, nv, vstride, h, part, N);
  k_axpy_finish<T><<<grid_for(N), 256, 0, st>>>(part, G, w, N);
  return cudaGetLastError();
}
cudaError_t axpy_multi(const double2* V, int nv, int64_t vstride, const double2* h, double2* w, double2* part,
                       int64_t N, cudaStream_t st) {
  return axpy_multi_t(V, nv, vstride, h, w, part, N, st);
}
cudaError_t axpy_multi(const float2* V, int nv, int64_t vstride, const double2* h, float2* w, float2* part,
                       int64_t N, cudaStream_t st) {
  return axpy_multi_t(V, nv, vstride, h, w, part, N, st);
}

// w -= sum_j h_j V_j with the basis sums S_j and the coefficient triplets h3
// (e, f - e, e + f) of h_j = e + i f: P += e S, Q += (e + f) Im V, T += (f - e) Re V;
// h_j V_j summed = (P - Q) + i (P + T).  Groups as in k_axpy_multi.
__global__ void __launch_bounds__(256) k_axpy3_multi(const double2* __restrict__ V, const double* __restrict__ S,
                                                     int nv, int64_t vstride, const double* __restrict__ h3,
                                                     double2* __restrict__ part, int64_t N) {
  const int G = gridDim.y, g = blockIdx.y;
  const int j0 = (nv * g) / G, j1 = (nv * (g + 1)) / G;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
    double P0 = 0, Q0 = 0, T0 = 0, P1 = 0, Q1 = 0, T1 = 0;
    int j = j0;
    for (; j + 1 < j1; j += 2) {
      const double2 v0 = V[int64_t(j) * vstride + i], v1 = V[int64_t(j + 1) * vstride + i];
      const double s0 = S[int64_t(j) * vstride + i], s1 = S[int64_t(j + 1) * vstride + i];
      P0 = fma(h3[3 * j], s0, P0);
      Q0 = fma(h3[3 * j + 2], v0.y, Q0);
      T0 = fma(h3[3 * j + 1], v0.x, T0);
      P1 = fma(h3[3 * j + 3], s1, P1);
      Q1 = fma(h3[3 * j + 5], v1.y, Q1);
      T1 = fma(h3[3 * j + 4], v1.x, T1);
    }
    if (j < j1) {
      const double2 v0 = V[int64_t(j) * vstride + i];
      P0 = fma(h3[3 * j], S[int64_t(j) * vstride + i], P0);
      Q0 = fma(h3[3 * j + 2], v0.y, Q0);
      T0 = fma(h3[3 * j + 1], v0.x, T0);
    }
    const double p = P0 + P1;
    part[int64_t(g) * N + i] = make_double2(p - (Q0 + Q1), p + (T0 + T1));
  }
}

cudaError_t axpy3_multi(const double2* V, const double* S, int nv, int64_t vstride, const double* h3, double2* w,
                        double2* part, int64_t N, cudaStream_t st) {
  const int G = nv >= 32 ? kAxpyGroups : (nv >= 8 ? 2 : 1);
  k_axpy3_multi<<<dim3(grid_for(N), G), 256, 0, st>>>(V, S, nv, vstride, h3, part, N);
  k_axpy_finish<double2><<<grid_for(N), 256, 0, st>>>(part, G, w, N);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(kRedThreads) k_norm_partial(const T* __restrict__ w, int64_t N,
                                                              double* __restrict__ partial) {
  __shared__ double2 red[32];
  T acc = czero(T{});
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
    acc.x = fma(w[i].x, w[i].x, fma(w[i].y, w[i].y, acc.x));
  const double2 s = block_sum(make_double2(acc.x, 0.0), red);
  if (threadIdx.x == 0) partial[blockIdx.x] = s.x;
}

__global__ void k_norm_reduce(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  double2 s = make_double2(0, 0);
  for (int b = threadIdx.x; b < nb; b += 32) s.x += partial[b];
  s = warp_sum(s);
  if (threadIdx.x == 0) out[0] = sqrt(s.x);
}

template <typename T>
cudaError_t norm2_t(const T* w, int64_t N, double* partial, double* out, cudaStream_t st) {
  const int nb = gram_blocks(N);
  k_norm_partial<T><<<nb, kRedThreads, 0, st>>>(w, N, partial);
  k_norm_reduce<<<1, 32, 0, st>>>(partial, nb, out);
  return cudaGetLastError();
}
cudaError_t norm2(const double2* w, int64_t N, double* partial, double* out, cudaStream_t st) {
  return norm2_t(w, N, partial, out, st);
}
cudaError_t norm2(const float2* w, int64_t N, double* partial, double* out, cudaStream_t st) {
  return norm2_t(w, N, partial, out, st);
}

template <typename T>
__global__ void k_scale_into(const T* __restrict__ w, const double* __restrict__ nrm, T* __restrict__ v, int64_t N) {
  const typename RealOf<T>::R s(nrm[0] > 0 ? 1.0 / nrm[0] : 0.0);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
    v[i] = cscale(w[i], s);
}
cudaError_t scale_into(const double2* w, const double* nrm, double2* v, int64_t N, cudaStream_t st) {
  k_scale_into<double2><<<grid_for(N), 256, 0, st>>>(w, nrm, v, N);
  return cudaGetLastError();
}
cudaError_t scale_into(const float2* w, const double* nrm, float2* v, int64_t N, cudaStream_t st) {
  k_scale_into<float2><<<grid_for(N), 256, 0, st>>>(w, nrm, v, N);
  return cudaGetLastError();
}

__global__ void k_scale_into_sums(const double2* __restrict__ w, const double* __restrict__ nrm,
                                  double2* __restrict__ v, double* __restrict__ S, int64_t N) {
  const double s = nrm[0] > 0 ? 1.0 / nrm[0] : 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
    const double2 x = cscale(w[i], s);
    v[i] = x;
    S[i] = x.x + x.y;
  }
}
cudaError_t scale_into_sums(const double2* w, const double* nrm, double2* v, double* S, int64_t N, cudaStream_t st) {
  k_scale_into_sums<<<grid_for(N), 256, 0, st>>>(w, nrm, v, S, N);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_combine(const T* __restrict__ V, int k, int64_t vstride, const double2* __restrict__ y,
                          T* __restrict__ x, int64_t N) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x) {
    T acc = x[i];
    for (int j = 0; j < k; ++j) acc = cfma(coef<T>(y[j]), V[int64_t(j) * vstride + i], acc);
    x[i] = acc;
  }
}
cudaError_t combine(const double2* V, int k, int64_t vstride, const double2* y, double2* x, int64_t N,
                    cudaStream_t st) {
  k_combine<double2><<<grid_for(N), 256, 0, st>>>(V, k, vstride, y, x, N);
  return cudaGetLastError();
}
cudaError_t combine(const float2* V, int k, int64_t vstride, const double2* y, float2* x, int64_t N,
                    cudaStream_t st) {
  k_combine<float2><<<grid_for(N), 256, 0, st>>>(V, k, vstride, y, x, N);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_sub(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ o, int64_t N) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
    o[i] = csub(a[i], b[i]);
}
cudaError_t sub(const double2* a, const double2* b, double2* out, int64_t N, cudaStream_t st) {
  k_sub<double2><<<grid_for(N), 256, 0, st>>>(a, b, out, N);
  return cudaGetLastError();
}
cudaError_t sub(const float2* a, const float2* b, float2* out, int64_t N, cudaStream_t st) {
  k_sub<float2><<<grid_for(N), 256, 0, st>>>(a, b, out, N);
  return cudaGetLastError();
}

__global__ void k_to_c64(const double2* __restrict__ a, float2* __restrict__ b, int64_t N) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = make_float2(float(a[i].x), float(a[i].y));
}
cudaError_t to_c64(const double2* a, float2* b, int64_t N, cudaStream_t st) {
  k_to_c64<<<grid_for(N), 256, 0, st>>>(a, b, N);
  return cudaGetLastError();
}
__global__ void k_to_c128(const float2* __restrict__ a, double2* __restrict__ b, int64_t N) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = make_double2(double(a[i].x), double(a[i].y));
}
cudaError_t to_c128(const float2* a, double2* b, int64_t N, cudaStream_t st) {
  k_to_c128<<<grid_for(N), 256, 0, st>>>(a, b, N);
  return cudaGetLastError();
}
__global__ void k_add(double2* __restrict__ x, const double2* __restrict__ e, int64_t N) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < N; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = cadd(x[i], e[i]);
}
cudaError_t add_inplace(double2* x, const double2* e, int64_t N, cudaStream_t st) {
  k_add<<<grid_for(N), 256, 0, st>>>(x, e, N);
  return cudaGetLastError();
}

__global__ void k_weight_sums(const double2* __restrict__ w, double* __restrict__ sum, int64_t n) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double2 v = w[i];
    sum[i] = v.x + v.y;
  }
}

cudaError_t weight_sums(const double2* w, double* s, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_weight_sums<<<grid_for(n), 256, 0, st>>>(w, s, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------ far field
__global__ void __launch_bounds__(kRedThreads) k_farfield(int64_t N, const double* __restrict__ x,
                                                          const double* __restrict__ y,
                                                          const double* __restrict__ ffw,
                                                          const double2* __restrict__ u,
                                                          const double* __restrict__ dirs, int ndir, double kappa,
                                                          double2 c, double2* __restrict__ A) {
  __shared__ double2 red[32];
  const int j = blockIdx.x, r = blockIdx.y;
  const double dx = dirs[2 * j], dy = dirs[2 * j + 1];
  const double2* ur = u + int64_t(r) * N;
  double2 acc = make_double2(0, 0);
  for (int64_t l = threadIdx.x; l < N; l += blockDim.x) {
    double s, co;
    sincos(-kappa * (dx * x[l] + dy * y[l]), &s, &co);
    acc = cfma(cscale(make_double2(co, s), ffw[l]), ur[l], acc);
  }
  const double2 t = block_sum(acc, red);
  if (threadIdx.x == 0) A[int64_t(r) * ndir + j] = cmul(c, t);
}

cudaError_t farfield(int64_t N, const double* x, const double* y, const double* ffw, const double2* u, int nrhs,
                     const double* dirs, int ndir, double kappa, double2 c, double2* A, cudaStream_t st) {
  k_farfield<<<dim3(ndir, nrhs), kRedThreads, 0, st>>>(N, x, y, ffw, u, dirs, ndir, kappa, c, A);
  return cudaGetLastError();
}

}  // namespace lsd
