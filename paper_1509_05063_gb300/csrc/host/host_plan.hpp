// Host-side plan construction for the 2-D Lippmann-Schwinger Nystrom operator.
//
// Everything here runs once per plan (ls_plan_create): the charts and the
// partition of unity (Section 2), the node set and its quadrature weights,
// the localised singular rules of Section 3.1 composed with the Lagrange
// interpolation into a sparse near-field matrix, and the dense pieces of the
// Section 3.2 accelerator (equivalent-source fits, local expansions, kernel
// lattice tables).  Plain C++17 with std::thread; no CUDA types.
#pragma once
#include <complex>
#include <atomic>
#include <functional>
#include <cstdint>
#include <string>
#include <vector>

#include "ls.h"

namespace lsh {

using cd = std::complex<double>;

// ---------------------------------------------------------------- geometry
struct Geometry {
  ls_geometry g{};
  // gamma(s), gamma'(s), gamma''(s)
  void curve(double s, double* gm, double* g1, double* g2) const;
  // collar chart X(a, b) and |det DX| in grid-index units
  void collar_map(double a, double b, double* X, double* J) const;
};

// Closest boundary point of x: foot parameter s and signed depth d (d > 0
// inside).  `found` is false when no boundary sample lies within `reach`
// (then only the inside/outside flag is meaningful).
struct ClosestPoint {
  ClosestPoint(const Geometry& geo, double reach);
  // Newton from the nearest of ns equispaced boundary samples; found = false
  // when no sample lies within `reach` of (x, y).
  void query(double x, double y, double* s, double* d, bool* found) const;
  // x-coordinates (sorted) where the horizontal line at height y crosses the
  // sampled boundary polygon: a point is inside iff an odd number lie left of it.
  std::vector<double> crossings(double y) const;

 private:
  const Geometry& geo_;
  int ns_ = 16384;
  double reach_, x0_, y0_;
  int nbx_, nby_;
  std::vector<double> ss_, sx_, sy_;
  std::vector<int> bstart_, bidx_;
};

double smooth_step(double u);                 // 1 -> 0 C-infinity step on [0, 1]
double cutoff(double s, double s0);           // chi: 1 on [0, s0], 0 beyond 1
std::vector<double> newton_cotes(int Q);      // closed rule, unit spacing

// The Nystrom node set in the plan's order (grouped by accelerator cell).
struct Nodes {
  int64_t N = 0, n_collar = 0, n_cart = 0;
  std::vector<double> x, y;        // coordinates
  std::vector<double> w;           // quadrature weight (Jacobian x rule)
  std::vector<double> omega, n2;   // partition of unity, refractive index squared
  std::vector<double> phifac;      // m omega  (density phi = m omega u)
  std::vector<double> wfac;        // w m omega
  std::vector<double> ca, cb;      // collar index coordinates (Cartesian nodes: inverse map)
  std::vector<double> ga, gb;      // Cartesian index coordinates
  std::vector<int8_t> chart;       // 0 collar, 1 Cartesian
  std::vector<int32_t> gi, gj;     // own-chart grid indices
  std::vector<int64_t> canon;      // canonical id (collar i n2 + j, then Cartesian rank)
  std::vector<int64_t> collar_pos; // canonical collar id -> plan index
  std::vector<int64_t> cart_pos;   // ix * ny + iy -> plan index or -1
  // accelerator cells
  int L = 0;
  std::vector<int32_t> cell;        // cell id (cj L + ci) per node
  std::vector<int64_t> cell_start;  // L*L + 1, nodes of cell c are [start[c], start[c+1])
};

struct Plan2D {
  Geometry geo;
  ls_options opt{};
  double kappa = 0;
  int n_threads = 1;
  Nodes nodes;
  // near field (CSR over plan order)
  std::vector<int64_t> rowptr;
  std::vector<int32_t> col;
  std::vector<cd> val;
  // accelerator
  int Ne = 0, n_es = 0, n_loc = 0, nfb2 = 0, M = 0, n_lat = 0;
  std::vector<int32_t> occ_cells;       // occupied cell ids
  std::vector<int64_t> P_off;           // offsets into P (per occupied cell), size nocc+1
  std::vector<cd> P64, P32;             // P_c (n_es x n_c, row-major), w m omega folded in
  std::vector<cd> Bpinv;                // nfb2 x n_loc
  std::vector<cd> BT;                   // 9 x nfb2 x n_es : Bpinv T_o, o = (oi+1)*3 + (oj+1)
  std::vector<cd> Bpinv32, BT32;        // from the complex64 fits
  std::vector<cd> Phi;                  // N x nfb2 (row q: basis at node q, its cell centre)
  std::vector<cd> Gtab, Dtab;           // M x M kernel lattice tables (row-major, [da][db])
  std::vector<double> ffw;              // far-field weights w omega (n^2 - 1)
  std::string err;
};

// Builders; each returns false and sets plan.err on failure.
bool build_nodes(Plan2D& plan, ls_n2_fn n2, void* ctx);
bool build_near(Plan2D& plan);
// cheap validity check of a cell layout (cut-off support inside N(x) for every
// node) and the number of near-field block entries one apply would stream
bool check_cells(Plan2D& plan, int64_t* block_entries);
bool build_accel(Plan2D& plan);

// Dense pieces of the 3-D accelerator (Section 5) for a node set with weights
// w m omega: cube cells of side H from corner box0, L per axis.
struct Accel3 {
  double kappa = 0, H = 0, box0[3] = {0, 0, 0}, rcond = 0;
  int L = 0, Ne = 0, p = 0, m_coll = 0, n_threads = 1;
  int n_es = 0, nb = 0, n_loc = 0, n_lat = 0, M = 0;
  std::vector<int64_t> node_order;      // nodes grouped by cell (stable)
  std::vector<int32_t> occ_cells;       // occupied cell ids (k L + j) L + i
  std::vector<int64_t> P_off;           // per occupied cell, size nocc + 1
  std::vector<cd> P;                    // P_c (n_es x n_c row-major), columns in node_order
  std::vector<cd> Bpinv;                // nb x n_loc
  std::vector<cd> BT;                   // 27 x nb x n_es
  std::vector<cd> Phi;                  // N x nb (input node order)
  std::vector<cd> Gtab, Dtab;           // M^3 kernel lattice tables ([da][db][dc])
  std::string err;
};
bool build_accel3(Accel3& a, const double* xyz, const double* wfac, int64_t N);

// 3-D discretisation of a ball (Section 5): six blended cubed-sphere shell
// faces, then the interior Cartesian grid.
struct Ball3 {
  double a = 1, w = 0.5, delta = 0.25, h = 0.1, tau0 = 0.3, tau1 = 0.95;
  int n_f = 17, n_s = 9, Q = 5;
  int64_t N = 0, n_shell = 0, n_cart = 0;
  int grid_m = 0;                 // interior grid indices -m..m per axis
  std::vector<double> x;          // N x 3
  std::vector<double> w_q;        // quadrature weight
  std::vector<double> omega, psi; // depth partition of unity, surface share (0 on the interior grid)
  std::vector<double> psi_omega;  // psi omega (the shell's density factor)
  std::vector<int8_t> face;       // shell face 0..5, -1 interior
  std::vector<int32_t> grid;      // N x 3: shell (i, j, k) on its face grid, interior (ix, iy, iz) + m
  std::vector<int64_t> face_node; // [F][i][j][k] -> node or -1 (6 n_f n_f n_s)
  std::vector<int64_t> cart_node; // [ix][iy][iz] -> node or -1 ((2m + 1)^3)
  // near-field rows (ball3_near): CSR over the requested rows
  std::vector<int64_t> near_rows, near_rowptr;
  std::vector<int32_t> near_col;
  std::vector<cd> near_val;
  std::string err;
};
bool build_ball3(Ball3& b);
// Parameters of the 3-D singular rules (index units of the grids).
struct Rules3 {
  double R = 3.0;                          // interior cut-off radius (grid units)
  int p = 5, q = 3, n_rho = 16, n_mu = 16, n_phi = 32;
  double rc = 6.0, rs = 6.0;               // shell cut-off: along the surface / across the depth
  int n_sig = 20, n_th = 32;
  double chi_s0 = 0.1;
};
// Row of the 3-D operator K at node qn: K[u](x_q) = sum_n row[n] u[n] (contrast
// folded in by the caller); eta (optional, N) receives the cut-off values of
// every rule applied.
bool ball3_row(const Ball3& b, double kappa, const Rules3& ru, int64_t qn, cd* row, double* eta, std::string* err);
// Adjacent part of the 3-D operator for the given rows (all rows when rows is
// NULL): every singular rule plus the regular (1 - eta) terms of the nodes in
// the 3 x 3 x 3 block of cells (side H, L per axis from box0) around the
// target; fails when a cut-off reaches outside that block.  Stored in b.near_*.
// stencils_only: store only the singular parts and the sparse correction
// -eta w omega G, leaving the block's plain regular sum w omega G to the caller.
bool ball3_near(Ball3& b, double kappa, const Rules3& ru, const double* box0, double H, int L, const int64_t* rows,
                int64_t n_rows, bool stencils_only, int n_threads, std::string* err);
// Window (2 Wn + 1)^3 of the interior singular rule's coefficients over grid
// offsets ([di][dj][dk], offsets -Wn..Wn) for a grid-point target.
bool interior_window3(double kappa, double h, double R, int p, int q, int n_rho, int n_mu, int n_phi, double chi_s0,
                      std::vector<cd>& win, int* Wn, std::string* err);

// Truncated thin SVD of a complex m x n matrix (m >= n), one-sided Jacobi.
struct SVD {
  int m = 0, n = 0, k = 0;
  std::vector<cd> U;      // m x k (column-major)
  std::vector<double> s;  // k
  std::vector<cd> V;      // n x k (column-major)
};
SVD svd_truncated(const std::vector<cd>& A_rowmajor, int m, int n, double rcond);
// The same factorisation by column-pivoted Householder QR followed by one-sided
// Jacobi on R^H (fewer, shorter sweeps; for the larger 3-D fits).
SVD svd_truncated_qr(const std::vector<cd>& A_rowmajor, int m, int n, double rcond);
// X = V S^-1 U^H B, B is m x nb row-major; result n x nb row-major.
std::vector<cd> svd_solve(const SVD& f, const std::vector<cd>& B, int nb);

// Parallel for over [0, n) in chunks.
void parallel_for(int n_threads, int64_t n, int64_t chunk, const std::function<void(int64_t, int64_t)>& fn);

}  // namespace lsh
