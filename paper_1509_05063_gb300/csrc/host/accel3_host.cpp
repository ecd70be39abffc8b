// Dense pieces of the three-dimensional accelerator (Section 5: two-face
// equivalent sources on cube cells and a 3-D lattice FFT), built once on the
// host for a node set with per-node weights w m omega.
//
//  * equivalent sources: monopoles and d/dz_1 dipoles at the (N_eq + 1)^2
//    lattice points of each of the cell's two x_1-faces; the fit matrix A
//    (m_coll^2 face midpoints on each face of the 3H cube around the cell) is
//    shared by all cells and factorised once; P_c = A^+ G(coll, y in c)
//    diag(w m omega) maps u_c to sigma_c.
//  * local expansion: spherical waves j_l(kappa r) Ybar_l^m(theta, phi) /
//    j_l(kappa R_ref), l <= p, R_ref = sqrt(3) H / 2, about the cell centre,
//    fitted on the closed cell's (N_eq + 1)^3 lattice points:
//    gamma_c = B^+ (V_c - sum_o T_o sigma_{c+o}), so BT_o = B^+ T_o.
//  * kernel lattice tables G(delta d) and dG/dz_1, zero at the origin, laid
//    out circularly on an M^3 grid (M a power of two >= 2 (L N_eq + 1) - 1).
#include <cmath>

#include "host_plan.hpp"

namespace lsh {

static inline cd mono3(double kappa, double dx, double dy, double dz) {
  const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
  return std::polar(1.0 / (4 * M_PI * r), kappa * r);
}
static inline cd dip3(double kappa, double dx, double dy, double dz) {
  const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
  return std::polar(1.0, kappa * r) * cd(1.0, -kappa * r) * (dx / (4 * M_PI * r * r * r));
}

// Fully normalised associated Legendre functions Ybar_l^m(theta) =
// sqrt((2l + 1)/(4 pi) (l - m)!/(l + m)!) P_l^m(cos theta) (Condon-Shortley
// phase included) for 0 <= m <= l <= p, by the standard three-term recurrence
// in l; out[l (l + 1) / 2 + m].
static void legendre_normalised(int p, double x, double* out) {
  const double s = std::sqrt(std::max(0.0, 1.0 - x * x));
  auto at = [&](int l, int m) -> double& { return out[l * (l + 1) / 2 + m]; };
  at(0, 0) = std::sqrt(1.0 / (4 * M_PI));
  for (int m = 1; m <= p; ++m) at(m, m) = -std::sqrt((2.0 * m + 1) / (2.0 * m)) * s * at(m - 1, m - 1);
  for (int m = 0; m < p; ++m) at(m + 1, m) = std::sqrt(2.0 * m + 3) * x * at(m, m);
  for (int m = 0; m <= p; ++m)
    for (int l = m + 2; l <= p; ++l) {
      const double a = std::sqrt((4.0 * l * l - 1) / (double(l) * l - double(m) * m));
      const double b = std::sqrt((double(l - 1) * (l - 1) - double(m) * m) / (4.0 * (l - 1) * (l - 1) - 1));
      at(l, m) = a * (x * at(l - 1, m) - b * at(l - 2, m));
    }
}

bool build_accel3(Accel3& A3, const double* xyz, const double* wfac, int64_t N) {
  const double kappa = A3.kappa, H = A3.H;
  const int L = A3.L, Ne = A3.Ne;
  const double delta = H / Ne;
  const double Rref = std::sqrt(3.0) * H / 2;
  if (kappa * Rref >= M_PI) { A3.err = "kappa sqrt(3) H / 2 must stay below pi (first zero of j_0)"; return false; }
  const int p = A3.p = A3.p > 0 ? A3.p : 2 * Ne + 1;
  const int nb = A3.nb = (p + 1) * (p + 1);
  const int n_loc = A3.n_loc = (Ne + 1) * (Ne + 1) * (Ne + 1);
  if (nb > n_loc) { A3.err = "local expansion has more terms than fit points"; return false; }
  // cells of the nodes, nodes grouped by cell (stable)
  const int64_t ncell = int64_t(L) * L * L;
  std::vector<int64_t> cell(N);
  for (int64_t q = 0; q < N; ++q) {
    int64_t c3[3];
    for (int k = 0; k < 3; ++k) {
      const double t = std::floor((xyz[3 * q + k] - A3.box0[k]) / H);
      if (!(t >= 0 && t < L)) { A3.err = "nodes outside the cell box"; return false; }
      c3[k] = int64_t(t);
    }
    cell[q] = (c3[2] * L + c3[1]) * L + c3[0];
  }
  std::vector<int64_t> start(ncell + 1, 0);
  for (int64_t q = 0; q < N; ++q) ++start[cell[q] + 1];
  for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
  A3.node_order.assign(N, 0);
  {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t q = 0; q < N; ++q) A3.node_order[fill[cell[q]]++] = q;
  }
  auto corner = [&](int64_t c, double* x0) {
    x0[0] = A3.box0[0] + H * double(c % L);
    x0[1] = A3.box0[1] + H * double((c / L) % L);
    x0[2] = A3.box0[2] + H * double(c / (int64_t(L) * L));
  };
  // equivalent sources (corner frame, lattice units): face a = 0 then a = Ne,
  // (b, c) row-major; monopoles then dipoles
  const int nf = (Ne + 1) * (Ne + 1);
  const int n_es = A3.n_es = 4 * nf;
  std::vector<int> ea(n_es), eb(n_es), ec(n_es), ek(n_es);
  for (int l = 0; l < n_es; ++l) {
    const int f = (l / nf) % 2, r = l % nf;
    ea[l] = f ? Ne : 0;
    eb[l] = r / (Ne + 1);
    ec[l] = r % (Ne + 1);
    ek[l] = l / (2 * nf);
  }
  auto es_field = [&](const double* x, int l) {
    const double dx = x[0] - ea[l] * delta, dy = x[1] - eb[l] * delta, dz = x[2] - ec[l] * delta;
    return ek[l] == 0 ? mono3(kappa, dx, dy, dz) : dip3(kappa, dx, dy, dz);
  };
  // collocation: m x m face midpoints on each face of [-H, 2H]^3
  const int m = A3.m_coll > 0 ? A3.m_coll : int(std::ceil(std::sqrt(2.0 * n_es / 6.0))) + 1;
  std::vector<double> coll;
  for (int ax = 0; ax < 3; ++ax)
    for (int side = 0; side < 2; ++side)
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
          double q[3];
          q[ax] = side ? 2 * H : -H;
          q[(ax + 1) % 3] = -H + (i + 0.5) / m * 3 * H;
          q[(ax + 2) % 3] = -H + (j + 0.5) / m * 3 * H;
          coll.insert(coll.end(), q, q + 3);
        }
  const int mc = int(coll.size() / 3);
  std::vector<cd> Amat(size_t(mc) * n_es);
  for (int q = 0; q < mc; ++q)
    for (int l = 0; l < n_es; ++l) Amat[size_t(q) * n_es + l] = es_field(&coll[3 * q], l);
  const double rc = A3.rcond > 0 ? A3.rcond : 1e-13;
  const SVD fA = svd_truncated_qr(Amat, mc, n_es, rc);
  // occupied cells and P_c (columns in node_order within the cell)
  A3.occ_cells.clear();
  for (int64_t c = 0; c < ncell; ++c)
    if (start[c + 1] > start[c]) A3.occ_cells.push_back(int32_t(c));
  const int nocc = int(A3.occ_cells.size());
  A3.P_off.assign(nocc + 1, 0);
  for (int k = 0; k < nocc; ++k) {
    const int64_t c = A3.occ_cells[k];
    A3.P_off[k + 1] = A3.P_off[k] + int64_t(n_es) * (start[c + 1] - start[c]);
  }
  A3.P.assign(A3.P_off[nocc], cd(0.0));
  parallel_for(A3.n_threads, nocc, 1, [&](int64_t k0, int64_t k1) {
    for (int64_t k = k0; k < k1; ++k) {
      const int64_t c = A3.occ_cells[k], s0 = start[c];
      const int nc = int(start[c + 1] - s0);
      double x0[3];
      corner(c, x0);
      std::vector<cd> Gc(size_t(mc) * nc);
      for (int q = 0; q < mc; ++q)
        for (int j = 0; j < nc; ++j) {
          const double* y = xyz + 3 * A3.node_order[s0 + j];
          Gc[size_t(q) * nc + j] = mono3(kappa, coll[3 * q] - (y[0] - x0[0]), coll[3 * q + 1] - (y[1] - x0[1]),
                                         coll[3 * q + 2] - (y[2] - x0[2]));
        }
      const std::vector<cd> X = svd_solve(fA, Gc, nc);
      for (int i = 0; i < n_es; ++i)
        for (int j = 0; j < nc; ++j)
          A3.P[A3.P_off[k] + size_t(i) * nc + j] = X[size_t(i) * nc + j] * wfac[A3.node_order[s0 + j]];
    }
  });
  // local spherical-wave expansion
  std::vector<double> jref(p + 1);
  for (int l = 0; l <= p; ++l) jref[l] = std::sph_bessel(unsigned(l), kappa * Rref);
  auto basis_row = [&](double x, double y, double z, cd* out) {
    const double r = std::sqrt(x * x + y * y + z * z);
    const double ct = r > 0 ? z / r : 1.0, ph = std::atan2(y, x);
    std::vector<double> Pn((p + 1) * (p + 2) / 2);
    legendre_normalised(p, ct, Pn.data());
    for (int l = 0; l <= p; ++l) {
      const double jl = std::sph_bessel(unsigned(l), kappa * r) / jref[l];
      for (int mm = -l; mm <= l; ++mm)
        out[l * l + l + mm] = jl * Pn[l * (l + 1) / 2 + std::abs(mm)] * std::polar(1.0, mm * ph);
    }
  };
  std::vector<cd> B(size_t(n_loc) * nb);
  auto loc_index = [&](int a, int b, int c) { return (a * (Ne + 1) + b) * (Ne + 1) + c; };
  for (int a = 0; a <= Ne; ++a)
    for (int b = 0; b <= Ne; ++b)
      for (int c = 0; c <= Ne; ++c)
        basis_row(a * delta - H / 2, b * delta - H / 2, c * delta - H / 2, &B[size_t(loc_index(a, b, c)) * nb]);
  const SVD fB = svd_truncated_qr(B, n_loc, nb, rc);
  std::vector<cd> I(size_t(n_loc) * n_loc, cd(0.0));
  for (int i = 0; i < n_loc; ++i) I[size_t(i) * n_loc + i] = 1.0;
  A3.Bpinv = svd_solve(fB, I, n_loc);   // nb x n_loc
  // neighbour tables T_o and BT_o = B^+ T_o, o index (oi + 1) 9 + (oj + 1) 3 + (ok + 1)
  auto table = [&](int da, int db, int dc, int kind) -> cd {
    if (da == 0 && db == 0 && dc == 0) return cd(0.0);
    const double dx = da * delta, dy = db * delta, dz = dc * delta;
    return kind == 0 ? mono3(kappa, dx, dy, dz) : dip3(kappa, dx, dy, dz);
  };
  A3.BT.assign(size_t(27) * nb * n_es, cd(0.0));
  parallel_for(A3.n_threads, 27, 1, [&](int64_t o0, int64_t o1) {
    for (int64_t o = o0; o < o1; ++o) {
      const int oi = int(o / 9) - 1, oj = int((o / 3) % 3) - 1, ok = int(o % 3) - 1;
      std::vector<cd> T(size_t(n_loc) * n_es);
      for (int a = 0; a <= Ne; ++a)
        for (int b = 0; b <= Ne; ++b)
          for (int c = 0; c <= Ne; ++c)
            for (int l = 0; l < n_es; ++l)
              T[size_t(loc_index(a, b, c)) * n_es + l] =
                  table(a - (ea[l] + oi * Ne), b - (eb[l] + oj * Ne), c - (ec[l] + ok * Ne), ek[l]);
      const std::vector<cd> X = svd_solve(fB, T, n_es);
      std::copy(X.begin(), X.end(), A3.BT.begin() + size_t(o) * nb * n_es);
    }
  });
  // evaluation rows at the nodes (input order)
  A3.Phi.assign(size_t(N) * nb, cd(0.0));
  parallel_for(A3.n_threads, N, 256, [&](int64_t q0, int64_t q1) {
    for (int64_t q = q0; q < q1; ++q) {
      double x0[3];
      corner(cell[q], x0);
      basis_row(xyz[3 * q] - x0[0] - H / 2, xyz[3 * q + 1] - x0[1] - H / 2, xyz[3 * q + 2] - x0[2] - H / 2,
                &A3.Phi[size_t(q) * nb]);
    }
  });
  // kernel lattice tables on the padded grid (offsets wrap at M / 2)
  A3.n_lat = L * Ne + 1;
  int M = 16;
  while (M < 2 * A3.n_lat - 1) M *= 2;
  if (M > 512) { A3.err = "lattice too large: need 2 (L N_eq + 1) - 1 <= 512"; return false; }
  A3.M = M;
  const size_t M3 = size_t(M) * M * M;
  A3.Gtab.assign(M3, cd(0.0));
  A3.Dtab.assign(M3, cd(0.0));
  parallel_for(A3.n_threads, M, 1, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i) {
      const int da = i <= M / 2 ? int(i) : int(i) - M;
      for (int j = 0; j < M; ++j) {
        const int db = j <= M / 2 ? j : j - M;
        for (int k = 0; k < M; ++k) {
          const int dc = k <= M / 2 ? k : k - M;
          const size_t idx = (size_t(i) * M + j) * M + k;
          A3.Gtab[idx] = table(da, db, dc, 0);
          A3.Dtab[idx] = i == M / 2 ? cd(0.0) : table(da, db, dc, 1);
        }
      }
    }
  });
  return true;
}

}  // namespace lsh
