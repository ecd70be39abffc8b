// Launchers of the sm_103a kernels of the LS apply / solve (device/kernels.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lsd {

// True the first time it is called for the current device with this mask
// (kernel attributes such as the shared-memory limit are per device).
inline bool first_on_device(unsigned long long& mask) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return true;
  const unsigned long long bit = 1ull << dev;
  if (mask & bit) return false;
  mask |= bit;
  return true;
}

// Device-resident pieces of a plan for one arithmetic precision R.
template <typename T>
struct ApplyData {
  int64_t N = 0;
  int nocc = 0, L = 0, Ne = 0, n_es = 0, n_loc = 0, nfb2 = 0, M = 0, n_lat = 0, logM = 0;
  const int64_t* occ_start = nullptr;   // nocc + 1: node range of each occupied cell
  const int* occ_cells = nullptr;       // nocc: cell id
  const int* occ_of_cell = nullptr;     // L*L: occupied index or -1
  const int* occ_of_node = nullptr;     // N: occupied index of the node's cell
  const int64_t* P_off = nullptr;       // nocc + 1
  const T* P = nullptr;                 // projections, per cell [node][n_es]
  const double* Ps = nullptr;           // complex128 only: Re + Im of every entry of P
  const int4* pieces = nullptr;         // projection work: (cell, first node, end node, piece | pieces << 16)
  int n_pieces = 0;                     // ... at most kProjPiece nodes each, largest first
  const int* piece_off = nullptr;       // nocc: first partial-sum slot of a cell cut into several pieces
  int* proj_count = nullptr;            // nocc: pieces of the cell finished in this apply (0 between applies)
  T* proj_part = nullptr;               // partial sums: slots x max_rhs x n_es
  const int4* cell_pieces = nullptr;    // nocc pieces of one whole cell each (no partial sums), largest first
  const T* LA = nullptr;                // [B^+ | -B^+ T_0 ... -B^+ T_8] (nfb2 x (n_loc + 9 n_es)) stored transposed
  const double* LAs = nullptr;          // complex128 only: Re + Im of every entry of LA
  const T* Phi = nullptr;               // N x nfb2
  const T* Gq = nullptr;                // (M/2+1)^2 quarter spectra, [l][k], scaled by 1/M^2
  const T* Dq = nullptr;
  const T* tw = nullptr;                // M twiddles exp(-2 pi i m / M)
  // near field: one dense block per occupied cell (rows = the cell's nodes,
  // columns = the nodes of its 3 x 3 neighbourhood, i.e. three contiguous node
  // ranges), plus a CSR remainder for the few interpolation-stencil entries
  // that fall outside the neighbourhood
  const int64_t* blk_off = nullptr;     // nocc: offset of the cell's block
  const int* blk_seg = nullptr;         // nocc x 6: (first node, length) of the 3 column ranges
  int max_nblk = 0;                     // longest padded block row
  const int2* items = nullptr;          // near-field work items (occupied cell, first row), 16 rows
  int n_items = 0;
  const int2* items32 = nullptr;        // the same with 32 rows per item (multi-RHS complex64)
  int n_items32 = 0;
  const int2* items128 = nullptr;       // 128-row items (tensor-core near field, 8 or 16 complex64 RHS)
  int n_items128 = 0;
  const int64_t* tile_off = nullptr;    // complex64 only: offset of each 128-row item in Wt
  const int* tc_bptr = nullptr;         // tensor-core grid: block b walks items tc_blist[tc_bptr[b] .. tc_bptr[b + 1])
  const int* tc_blist = nullptr;
  int tc_grid = 0;                      // blocks of the tensor-core grid (one per SM of the plan's device)
  // variants picked by ls_plan_autotune (same result up to rounding)
  int conv_tc = 0;                      // columns per block of the lattice column pass (0: default, 1)
  bool near_cuda = false;               // complex64, 8 or 16 RHS: CUDA-core near field instead of tensor cores
  bool local_cuda = false;              // complex64, 8 or 16 RHS: CUDA-core local coefficients instead of tensor cores
  bool proj_cuda = false;               // complex64, 8 or 16 RHS: CUDA-core projection instead of tensor cores
  bool fft_r4 = false;                  // complex64: radix-4 lattice transforms instead of radix 16 (single plans)
  const unsigned char* LAt = nullptr;   // complex64 only: LA in the tensor-core tile layout (local_tc_tiles)
  const T* Wt = nullptr;                // complex64 only: the blocks in the tensor-core tile layout
  const float* tc_rscale = nullptr;     // complex64 only: 1 / (power-of-two scale) of each near-field row
  unsigned* tc_tmax = nullptr;          // complex64 only: per-RHS largest |Re|, |Im| of one apply (float bits)
  int* tc_err = nullptr;                // set by the tensor-core near field when a wait times out
  int tc_spin = 1 << 22;                // polls of each mbarrier wait before it gives up
  const T* Wb = nullptr;                // blocks, row-major per cell
  const double* Ws = nullptr;           // complex128 only: Re + Im of every block weight (same layout as Wb)
  double* utc = nullptr;                // complex128 only (null: formed in the near field): the input's
  double2* utef = nullptr;              // staged forms c and (c + d, d - c), written by the projection
  const int64_t* rem_row = nullptr;     // N + 1
  const int* rem_col = nullptr;
  const T* rem_val = nullptr;
  double kappa2 = 0;
  // work space
  T* sigma = nullptr;                   // max_rhs x nocc x n_es
  T* Sm = nullptr;                      // max_rhs x lattice_rows() x M
  T* Sd = nullptr;                      // max_rhs x lattice_rows() x M
  __host__ __device__ int64_t lattice_rows() const { return (2 * (L + 1) > n_lat ? 2 * (L + 1) : n_lat); }
  T* gamma = nullptr;                   // max_rhs x nocc x nfb2
};

// Stage boundaries of one apply, for event timing: projection, (unused: the
// lattice fill is fused into the convolution), lattice convolution, local
// coefficients, near field + assembly.
constexpr int kStages = 5;

// out = A u for one right-hand side (u, out: N complex).  When ev is not null
// it holds kStages + 1 events recorded at the stage boundaries.  Returns the
// first launch error (cudaSuccess otherwise).
template <typename T>
cudaError_t apply_one(const ApplyData<T>& d, const T* u, T* out, cudaStream_t st, cudaEvent_t* ev = nullptr);

// out = A u for nr right-hand sides at once (nr in {1, 2, 4} for complex128,
// {1, 2, 4, 8, 16} for complex64, 8 and 16 with the tensor-core near field; u, out: nr vectors of length N one after
// another): one pass over the near-field weights serves all of them.  The work
// arrays must hold max_rhs right-hand sides.
template <typename T>
cudaError_t apply_batch(const ApplyData<T>& d, const T* u, T* out, int nr, cudaStream_t st,
                        cudaEvent_t* ev = nullptr);
constexpr int kMaxRhs64 = 4, kMaxRhs32 = 16;
constexpr int kProjPiece = 128;    // nodes per projection block at most

// Near field + evaluation + assembly of R complex64 right-hand sides (R = 8 or
// 16) on the tensor cores (tcgen05, split FP16 with power-of-two scaling; device/near_tc.cu); same result as
// the CUDA-core kernel up to FP32 rounding.
template <int R>
cudaError_t near_eval_tc(const ApplyData<float2>& d, const float2* u, float2* out, cudaStream_t st);
// Elements (complex64) of one 128-row item of nrow rows and nblk padded columns
// in the tile layout of the tensor-core near field, and the plan-time kernel
// that writes that layout (d.items128, d.tile_off, d.Wb set) into Wt.
int64_t tc_tile_elems(int nrow, int nblk);
cudaError_t tile_weights(const ApplyData<float2>& d, float2* Wt, float* rscale, cudaStream_t st);
// Local coefficients of 8 or 16 complex64 RHS on the tensor cores (device/contract_tc.cu, 3xTF32):
// the same contraction as k_local_coeffs with LA in the tile layout that local_tc_tiles writes at
// plan time (local_tc_bytes(K) bytes, K = n_loc + 9 n_es; nfb2 <= 32).
int local_tc_chunks(int K);
size_t local_tc_bytes(int K);
cudaError_t local_tc_tiles(const float2* LA, int K, int nfb2, unsigned char* LAt, cudaStream_t st);
template <int R>
cudaError_t local_coeffs_tc(const ApplyData<float2>& d, cudaStream_t st);
// Whether a plan's lattice passes run with TC columns per block of the column
// pass at lattice size M (FP64; complex64 with the radix-4 or radix-16 FFT):
// the same test the passes make before they launch.
bool lattice_cols_fit(bool fp64, bool radix4, int M, int TC);
// Equivalent-source projection of 8 or 16 complex64 RHS on the tensor cores (device/contract_tc.cu,
// 3xTF32): the sums of k_es_project, one block per whole cell (d.cell_pieces), P_c read as stored;
// n_es <= 64.
template <int R>
cudaError_t project_tc(const ApplyData<float2>& d, const float2* u, cudaStream_t st);

// Device-resident pieces of a 3-D plan (Section 5: ball, cube cells of side H,
// L per axis) for one arithmetic precision.  Vectors are in the plan's node
// order (grouped by cell).
template <typename T>
struct ApplyData3 {
  int64_t N = 0;
  int nocc = 0, L = 0, Ne = 0, n_es = 0, n_loc = 0, nb = 0, M = 0, logM = 0;
  const int64_t* occ_start = nullptr;   // nocc + 1: node range of each occupied cell
  const int* occ_cells = nullptr;       // nocc: cell id (k L + j) L + i
  const int* occ_of_cell = nullptr;     // L^3: occupied index or -1
  const int* occ_of_node = nullptr;     // N: occupied index of the node's cell
  const int64_t* P_off = nullptr;       // nocc + 1: element offset of each cell's projection
  const T* P = nullptr;                 // P_c stored [node][n_es] (w omega m folded in)
  const T* LA = nullptr;                // [n_loc + 27 n_es][nb]: B^+ transposed, then -(B^+ T_o) transposed
  const float* LA6 = nullptr;           // FP64 data only: LA = a + ib as (a + b, b, a), each split into
                                        // FP32 hi + lo, [K][nb][6] (the double-float local GEMM)
  const T* Phi = nullptr;               // N x nb: local basis at each node about its cell centre
  const T* Gs = nullptr;                // M^3 spectra of the G and dG/dz_1 lattice tables, / M^3
  const T* Ds = nullptr;
  const T* tw = nullptr;                // M twiddles exp(-2 pi i m / M)
  const int64_t* rowptr = nullptr;      // adjacent part: CSR over the nodes (contrast folded into val)
  const int* col = nullptr;
  const T* val = nullptr;               // complex64 data only: the CSR holds the remainder of the blocks
  const T* Wb = nullptr;                // complex64 only: per cell a dense block [row][27-neighbour columns]
  const int64_t* blk_off = nullptr;     // nocc: element offset of each cell's block in Wb
  const int* blk_seg = nullptr;         // nocc x 9 x (first node, count): the neighbour column ranges
  const double* val3 = nullptr;         // FP64 data only: (a + b, b, a) per entry of the values a + ib
  double kappa2 = 0;
  // work space (one right-hand side)
  double* u3 = nullptr;                 // FP64 data only: N x (c, c + d, d - c) of the input c + id
  T* sigma = nullptr;                   // nocc x n_es
  T* Sm = nullptr;                      // M^3: monopole lattice, then the lattice field V
  T* Sd = nullptr;                      // M^3: dipole lattice
  T* gamma = nullptr;                   // nocc x nb
  T* X = nullptr;                       // FP64 data only: nocc x (n_loc + 27 n_es), inputs of the local step
  float* X6 = nullptr;                  // FP64 data only: the same in the double-float GEMM's split forms
  T* part = nullptr;                    // FP64 data only: local3_slices x nocc x nb partial products
  // complex64 only (host pointer): the FP64 data whose lattice convolution
  // (FP64) and local coefficients (double-float GEMM) the complex64 apply
  // uses.  On a cell's own lattice points the 27 neighbours' fields dominate
  // and cancel in the neighbour subtraction; complex64 rounding of the lattice
  // field or of the local step's sums would be magnified by that cancellation
  // and by the ill-conditioned local fit.
  const ApplyData3<double2>* lattice64 = nullptr;
};

// K slices of the 3-D local-coefficient GEMM (sizes its partial-product array)
constexpr int kLocalSlicesMax = 64;
int local3_slices(int nocc, int nb, int K);

// out = A u for nr right-hand sides of a 3-D plan (one after another through
// the same work space; u, out: nr vectors of length N).
template <typename T>
cudaError_t apply3_batch(const ApplyData3<T>& d, const T* u, T* out, int nr, cudaStream_t st);
// 3-D FFT of an M x M x M array in place ([a][b][c], c contiguous), forward or
// inverse (unscaled): three passes of batched line transforms.
template <typename T>
cudaError_t fft3d(T* x, int M, int logM, const T* tw, bool inverse, cudaStream_t st);
// Plan-time construction, on the device, of the 3-D adjacent part's stored
// forms from its CSR (plan order; rowptr, col, val = a + ib, all device):
// near3_forms writes val3 = (a + b, b, a) per entry, adds the entries that
// fall in a row's 9 neighbour node ranges (blk_seg) into the complex64 dense
// block Wb (zeroed by the caller; same order and rounding as a host loop over
// the row) and counts the others per row (rem_count, N entries);
// near3_remainder then writes those others, in row order, at rem_row (the
// exclusive prefix sums of the counts).
cudaError_t near3_forms(int64_t N, const int64_t* occ_start, const int* occ_of_node, const int64_t* rowptr,
                        const int* col, const double2* val, const int64_t* blk_off, const int* blk_seg, double* val3,
                        float2* Wb, int64_t* rem_count, cudaStream_t st);
cudaError_t near3_remainder(int64_t N, const int* occ_of_node, const int64_t* rowptr, const int* col,
                            const double2* val, const int* blk_seg, const int64_t* rem_row, int* rem_col,
                            float2* rem_val, cudaStream_t st);
// Far-field pattern of a 3-D plan's solution: A[r][d] = c sum_q ffw_q u_r[q]
// exp(-i kappa dir_d . x_q) (dirs: ndir x 3 unit vectors, device).
cudaError_t farfield3(int64_t N, const double* xyz, const double* ffw, const double2* u, int nrhs,
                      const double* dirs, int ndir, double kappa, double2 c, double2* A, cudaStream_t st);

// One scatterer of a multi-instance batch: its apply data and the offset of
// its nodes in the batch's concatenated vectors.
template <typename T>
struct InstData {
  ApplyData<T> d;
  int64_t off = 0;
};

// The lattice convolutions of a batch's instances whose lattice size is M, as
// three launches over work lists: src = (instance, face row k <= L), cols =
// (instance, column b < M), rows = (instance, kept row a < n_lat).
struct LatWork {
  int M = 0;
  const int2* src = nullptr;
  int n_src = 0;
  const int2* cols = nullptr;
  int n_cols = 0;
  const int2* rows = nullptr;
  int n_rows = 0;
};

// out = A_i u_i for the n_ids active instances of a batch at once (one
// right-hand side each; u, out: the concatenated vectors; the other instances'
// parts of out are left untouched).  The projection, the local expansion and
// the near field each run as ONE launch walking work lists over those
// instances -- pieces = (instance, projection piece of the instance), cells =
// (instance, occupied cell), items = (instance, occupied cell, first of 16
// rows, unused) -- and the lattice convolution as three launches per lattice
// size (lat[0..n_lat_groups), covering the same instances).  dev_inst: the
// batch's instance table on the device; max_K is the largest n_loc + 9 n_es.
// No plan may appear twice among the instances (they would share its work
// arrays).
template <typename T>
cudaError_t apply_multi(const InstData<T>* dev_inst, int n_ids,
                        const int2* pieces, int n_pieces, const int2* cells, int n_cells, const int4* items,
                        int n_items, int max_K, const LatWork* lat, int n_lat_groups, const T* u, T* out,
                        cudaStream_t st);

// 2-D FFT of an M x M array in place (rows then columns), forward or inverse
// (unscaled).
template <typename T>
cudaError_t fft2d(T* x, int M, int logM, const T* tw, bool inverse, cudaStream_t st);

// GMRES helpers (complex128).  h[j] = <V_j, w> for j < nv (V: nv vectors of
// length N, stride N) and h[nv].x = ||w||^2; partial needs blocks * (nv + 1)
// elements, h needs nv + 1.
// (basis vector j starts at V + j * vstride)
cudaError_t gram(const double2* V, int nv, int64_t vstride, const double2* w, int64_t N, double2* partial,
                 double2* h, cudaStream_t st);
// w -= sum_j h_j V_j; part needs kAxpyGroups x N elements of scratch
constexpr int kAxpyGroups = 4;
cudaError_t axpy_multi(const double2* V, int nv, int64_t vstride, const double2* h, double2* w, double2* part,
                       int64_t N, cudaStream_t st);
cudaError_t norm2(const double2* w, int64_t N, double* partial, double* out, cudaStream_t st);
cudaError_t scale_into(const double2* w, const double* nrm, double2* v, int64_t N, cudaStream_t st);
cudaError_t combine(const double2* V, int k, int64_t vstride, const double2* y, double2* x, int64_t N,
                    cudaStream_t st);
cudaError_t sub(const double2* a, const double2* b, double2* out, int64_t N, cudaStream_t st);
// Complex128 Gram-Schmidt on a basis stored with S_j = Re V_j + Im V_j beside
// every vector (three FP64 FMAs per complex product instead of four): gram3
// also writes h3 = (Re h_j, Im h_j - Re h_j, Re h_j + Im h_j), which axpy3_multi
// takes; scale_into_sums writes v = w / nrm and its sums S.
cudaError_t gram3(const double2* V, const double* S, int nv, int64_t vstride, const double2* w, int64_t N,
                  double2* partial, double2* h, double* h3, cudaStream_t st);
cudaError_t axpy3_multi(const double2* V, const double* S, int nv, int64_t vstride, const double* h3, double2* w,
                        double2* part, int64_t N, cudaStream_t st);
cudaError_t scale_into_sums(const double2* w, const double* nrm, double2* v, double* S, int64_t N, cudaStream_t st);
// The same on complex64 vectors (the LS_MIXED32 correction solves): complex64
// arithmetic per element, the Gram and norm partial sums and the coefficients
// h, y, nrm in FP64.
cudaError_t gram(const float2* V, int nv, int64_t vstride, const float2* w, int64_t N, double2* partial, double2* h,
                 cudaStream_t st);
cudaError_t axpy_multi(const float2* V, int nv, int64_t vstride, const double2* h, float2* w, float2* part,
                       int64_t N, cudaStream_t st);
cudaError_t norm2(const float2* w, int64_t N, double* partial, double* out, cudaStream_t st);
cudaError_t scale_into(const float2* w, const double* nrm, float2* v, int64_t N, cudaStream_t st);
cudaError_t combine(const float2* V, int k, int64_t vstride, const double2* y, float2* x, int64_t N,
                    cudaStream_t st);
cudaError_t sub(const float2* a, const float2* b, float2* out, int64_t N, cudaStream_t st);
cudaError_t to_c64(const double2* a, float2* b, int64_t N, cudaStream_t st);
cudaError_t to_c128(const float2* a, double2* b, int64_t N, cudaStream_t st);
cudaError_t add_inplace(double2* x, const double2* e, int64_t N, cudaStream_t st);
// s[i] = Re w[i] + Im w[i] (the third weight of the three-multiplication complex product)
cudaError_t weight_sums(const double2* w, double* s, int64_t n, cudaStream_t st);

cudaError_t farfield(int64_t N, const double* x, const double* y, const double* ffw,
                     const double2* u, int nrhs, const double* dirs, int ndir, double kappa,
                     double2 c, double2* A, cudaStream_t st);

int gram_blocks(int64_t N);

// Measured throughput of this GPU (device/peaks.cu): FP64 FMA on the CUDA
// cores and TF32 tcgen05 MMA (M = 128, N = 256), in TFLOP/s (2 per FMA);
// tf32 is -1 if a wait of the MMA probe gave up.
cudaError_t measure_peaks(double* fp64_tflops, double* tf32_tflops);

}  // namespace lsd
