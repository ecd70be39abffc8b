// Dense pieces of the Section 3.2 accelerator, built once per plan.
//
//  * equivalent sources: monopoles and d/dz_1 dipoles at the N_eq + 1 lattice
//    points of each of the cell's two x_1-faces (Eq. equiv-conv-loc); the fit
//    matrix A (collocation points on the boundary of the 3 x 3 block, n_coll
//    of them) is shared by all cells and factorised once by a truncated SVD;
//    P_c = A^+ G(coll, y in c) diag(w m omega) maps u_c to sigma_c.
//  * local expansion (Eq. PWE in its Fourier-Bessel form):
//    b_n(x) = J_n(kappa r) e^{i n theta} / J_|n|(kappa H / sqrt 2), |n| <= n_fb,
//    about the cell centre; B = [b_n(lattice points of the closed cell)],
//    gamma_c = B^+ (V_c - sum_o T_o sigma_{c+o}), so BT_o = B^+ T_o.
//  * kernel lattice tables G(delta (da, db)) and dG/dz_1, zero at the origin,
//    laid out circularly on an M x M grid for the zero-padded FFT convolution.
#include <cmath>

#include "host_plan.hpp"

namespace lsh {

static inline cd h0(double z) { return cd(::j0(z), ::y0(z)); }
static inline cd h1(double z) { return cd(::j1(z), ::y1(z)); }

static inline cd mono(double kappa, double dx, double dy) {
  return cd(0.0, 0.25) * h0(kappa * std::hypot(dx, dy));
}
static inline cd dip(double kappa, double dx, double dy) {
  const double r = std::hypot(dx, dy);
  return cd(0.0, 0.25) * kappa * h1(kappa * r) * (dx / r);
}

// J_n(x) for integer n of either sign
static inline double besselj(int n, double x) {
  const double v = ::jn(std::abs(n), x);
  return (n < 0 && (std::abs(n) % 2)) ? -v : v;
}

bool build_accel(Plan2D& plan) {
  const ls_options& o = plan.opt;
  const Nodes& nd = plan.nodes;
  const double kappa = plan.kappa, H = o.H;
  const int Ne = plan.Ne = o.N_eq, L = o.L;
  const double delta = H / Ne;
  if (kappa * H / std::sqrt(2.0) >= 2.4) { plan.err = "kappa H / sqrt 2 must stay below 2.4"; return false; }
  if (o.n_fb < 0 || 2 * o.n_fb + 1 > (Ne + 1) * (Ne + 1)) { plan.err = "bad n_fb"; return false; }
  // equivalent sources (corner frame, lattice units)
  const int n_es = plan.n_es = 4 * (Ne + 1);
  std::vector<int> es_a(n_es), es_b(n_es), es_k(n_es);
  for (int f = 0; f < 4; ++f)
    for (int k = 0; k <= Ne; ++k) {
      const int l = f * (Ne + 1) + k;
      es_a[l] = (f % 2) ? Ne : 0;
      es_b[l] = k;
      es_k[l] = f / 2;   // 0 monopole, 1 dipole
    }
  auto es_field = [&](double px, double py, int l) {
    const double dx = px - es_a[l] * delta, dy = py - es_b[l] * delta;
    return es_k[l] == 0 ? mono(kappa, dx, dy) : dip(kappa, dx, dy);
  };
  // collocation on the 3H x 3H square around the cell
  const int ncoll = o.n_coll ? o.n_coll : 4 * n_es;
  const int mside = ncoll / 4;
  std::vector<double> colx, coly;
  for (int side = 0; side < 4; ++side)
    for (int k = 0; k < mside; ++k) {
      const double t = (k + 0.5) / mside * 3 * H - H;
      const double tr = (mside - 1 - k + 0.5) / mside * 3 * H - H;
      switch (side) {
        case 0: colx.push_back(t); coly.push_back(-H); break;
        case 1: colx.push_back(2 * H); coly.push_back(t); break;
        case 2: colx.push_back(tr); coly.push_back(2 * H); break;
        default: colx.push_back(-H); coly.push_back(tr); break;
      }
    }
  const int m = int(colx.size());
  std::vector<cd> A(size_t(m) * n_es);
  for (int q = 0; q < m; ++q)
    for (int l = 0; l < n_es; ++l) A[size_t(q) * n_es + l] = es_field(colx[q], coly[q], l);
  const double rc64 = o.rcond > 0 ? o.rcond : 1e-13;
  const double rc32 = o.rcond_mixed > 0 ? o.rcond_mixed : 1e-7;
  const SVD fA = svd_truncated(A, m, n_es, rc64);
  const SVD fA32 = svd_truncated(A, m, n_es, rc32);

  // occupied cells and P_c
  plan.occ_cells.clear();
  for (int c = 0; c < L * L; ++c)
    if (nd.cell_start[c + 1] > nd.cell_start[c]) plan.occ_cells.push_back(c);
  const int nocc = int(plan.occ_cells.size());
  plan.P_off.assign(nocc + 1, 0);
  for (int k = 0; k < nocc; ++k) {
    const int c = plan.occ_cells[k];
    plan.P_off[k + 1] = plan.P_off[k] + int64_t(n_es) * (nd.cell_start[c + 1] - nd.cell_start[c]);
  }
  plan.P64.assign(plan.P_off[nocc], cd(0.0));
  plan.P32.assign(plan.P_off[nocc], cd(0.0));
  parallel_for(plan.n_threads, nocc, 4, [&](int64_t k0, int64_t k1) {
    for (int64_t k = k0; k < k1; ++k) {
      const int c = plan.occ_cells[k];
      const int ci = c % L, cj = c / L;
      const int64_t s0 = nd.cell_start[c];
      const int nc = int(nd.cell_start[c + 1] - s0);
      std::vector<cd> Gc(size_t(m) * nc);
      for (int q = 0; q < m; ++q)
        for (int j = 0; j < nc; ++j) {
          const double rx = nd.x[s0 + j] - (o.box_x0 + ci * H);
          const double ry = nd.y[s0 + j] - (o.box_y0 + cj * H);
          Gc[size_t(q) * nc + j] = mono(kappa, colx[q] - rx, coly[q] - ry);
        }
      const std::vector<cd> X = svd_solve(fA, Gc, nc);
      const std::vector<cd> X32 = svd_solve(fA32, Gc, nc);
      for (int i = 0; i < n_es; ++i)
        for (int j = 0; j < nc; ++j) {
          plan.P64[plan.P_off[k] + size_t(i) * nc + j] = X[size_t(i) * nc + j] * nd.wfac[s0 + j];
          plan.P32[plan.P_off[k] + size_t(i) * nc + j] = X32[size_t(i) * nc + j] * nd.wfac[s0 + j];
        }
    }
  });

  // local Fourier-Bessel expansion
  const int nfb = o.n_fb, nfb2 = plan.nfb2 = 2 * nfb + 1;
  const int n_loc = plan.n_loc = (Ne + 1) * (Ne + 1);
  const double Rref = H / std::sqrt(2.0);
  std::vector<double> jref(nfb + 1);
  for (int n = 0; n <= nfb; ++n) jref[n] = ::jn(n, kappa * Rref);
  auto fb_row = [&](double x, double y, cd* out) {
    const double r = std::hypot(x, y), th = std::atan2(y, x);
    for (int n = -nfb; n <= nfb; ++n)
      out[n + nfb] = besselj(n, kappa * r) / jref[std::abs(n)] * std::polar(1.0, n * th);
  };
  std::vector<cd> B(size_t(n_loc) * nfb2);
  for (int a = 0; a <= Ne; ++a)
    for (int b = 0; b <= Ne; ++b) fb_row(a * delta - H / 2, b * delta - H / 2, &B[size_t(a * (Ne + 1) + b) * nfb2]);
  const SVD fB = svd_truncated(B, n_loc, nfb2, rc64);
  std::vector<cd> I(size_t(n_loc) * n_loc, cd(0.0));
  for (int i = 0; i < n_loc; ++i) I[size_t(i) * n_loc + i] = 1.0;
  plan.Bpinv = svd_solve(fB, I, n_loc);           // nfb2 x n_loc
  // neighbour tables and BT_o = B^+ T_o
  auto table = [&](int da, int db, int kind) -> cd {
    if (da == 0 && db == 0) return cd(0.0);
    const double dx = da * delta, dy = db * delta;
    return kind == 0 ? mono(kappa, dx, dy) : dip(kappa, dx, dy);
  };
  plan.BT.assign(size_t(9) * nfb2 * n_es, cd(0.0));
  for (int oi = -1; oi <= 1; ++oi)
    for (int oj = -1; oj <= 1; ++oj) {
      const int o9 = (oi + 1) * 3 + (oj + 1);
      std::vector<cd> T(size_t(n_loc) * n_es);
      for (int a = 0; a <= Ne; ++a)
        for (int b = 0; b <= Ne; ++b)
          for (int l = 0; l < n_es; ++l)
            T[size_t(a * (Ne + 1) + b) * n_es + l] =
                table(a - (es_a[l] + oi * Ne), b - (es_b[l] + oj * Ne), es_k[l]);
      for (int n = 0; n < nfb2; ++n)
        for (int l = 0; l < n_es; ++l) {
          cd s = 0;
          for (int p = 0; p < n_loc; ++p) s += plan.Bpinv[size_t(n) * n_loc + p] * T[size_t(p) * n_es + l];
          plan.BT[(size_t(o9) * nfb2 + n) * n_es + l] = s;
        }
    }
  // evaluation rows at the nodes
  plan.Phi.assign(size_t(nd.N) * nfb2, cd(0.0));
  parallel_for(plan.n_threads, nd.N, 4096, [&](int64_t q0, int64_t q1) {
    for (int64_t q = q0; q < q1; ++q) {
      const int c = nd.cell[q], ci = c % L, cj = c / L;
      fb_row(nd.x[q] - (o.box_x0 + ci * H) - H / 2, nd.y[q] - (o.box_y0 + cj * H) - H / 2,
             &plan.Phi[size_t(q) * nfb2]);
    }
  });
  // kernel lattice tables on the padded grid
  plan.n_lat = L * Ne + 1;
  int M = 256;                          // power of two >= 2 n_lat - 1 (linear convolution)
  while (M < 2 * plan.n_lat - 1) M *= 2;
  if (M > 2048) { plan.err = "lattice too large: need 2 (L N_eq + 1) - 1 <= 2048"; return false; }
  plan.M = M;
  // Offsets wrap at M/2, so the tables are exactly even (G) / odd in a (dG/dz_1)
  // on the circle; the gap |offset| >= n_lat is never reached by the linear
  // convolution.  The odd table is zero at a = M/2.
  plan.Gtab.assign(size_t(M) * M, cd(0.0));
  plan.Dtab.assign(size_t(M) * M, cd(0.0));
  parallel_for(plan.n_threads, M, 8, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      const int da = i <= M / 2 ? int(i) : int(i) - M;
      for (int j = 0; j < M; ++j) {
        const int db = j <= M / 2 ? j : j - M;
        plan.Gtab[size_t(i) * M + j] = table(da, db, 0);
        plan.Dtab[size_t(i) * M + j] = i == M / 2 ? cd(0.0) : table(da, db, 1);
      }
    }
  });
  return true;
}

}  // namespace lsh
