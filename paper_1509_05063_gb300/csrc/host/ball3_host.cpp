// Three-dimensional discretisation of a penetrable ball (Section 5) and the
// translation-invariant window of the interior singular rule, built on the
// host.
//
// Shell: the six faces of a cubed sphere in equiangular coordinates
// (xi, eta) in [-pi/4 - delta, pi/4 + delta]^2, blended on the sphere by a
// C-infinity partition of unity psi_F (normalised products of cut-offs that
// vanish to all orders at the extended edges); depth s in [0, 1], radius
// r = a - s w; trapezoid rule in xi and eta, composite Q-point Newton-Cotes in
// s; omega_B(s) = S((s - tau0) / (tau1 - tau0)).  Interior: the Cartesian grid
// of spacing h with omega_I = 1 - omega_B(depth / w), kept where omega_I > 0.
//
// Interior singular rule: for a grid-point target the cut-off part of the
// patch integral is taken in spherical coordinates about the target,
// rho = R s^q (grid units), trapezoid rule in s, Gauss-Legendre in cos(theta),
// trapezoid rule in the azimuth; the density at the off-grid points comes
// from degree-p tensor-product Lagrange interpolation on the grid, so the rule
// is a fixed window of coefficients over grid offsets.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>

#include "host_plan.hpp"

namespace lsh {

namespace {

// face frames (e1, e2, e3); e3 is the face centre direction
const double kFaces[6][3][3] = {
    {{0, 1, 0}, {0, 0, 1}, {1, 0, 0}},  {{0, 0, 1}, {0, 1, 0}, {-1, 0, 0}}, {{0, 0, 1}, {1, 0, 0}, {0, 1, 0}},
    {{1, 0, 0}, {0, 0, 1}, {0, -1, 0}}, {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}},  {{0, 1, 0}, {1, 0, 0}, {0, 0, -1}},
};

inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// direction of (xi, eta) on face F and the solid-angle element per dxi deta
void face_direction(int F, double xi, double eta, double* d, double* dom) {
  const double t1 = std::tan(xi), t2 = std::tan(eta);
  const double nrm = std::sqrt(1.0 + t1 * t1 + t2 * t2);
  for (int k = 0; k < 3; ++k) d[k] = (kFaces[F][2][k] + t1 * kFaces[F][0][k] + t2 * kFaces[F][1][k]) / nrm;
  *dom = (1.0 + t1 * t1) * (1.0 + t2 * t2) / (nrm * nrm * nrm);
}

double face_bump(double xi, double eta, double delta) {
  const double lo = M_PI / 4 - delta, hi = M_PI / 4 + delta;
  return smooth_step((std::fabs(xi) - lo) / (hi - lo)) * smooth_step((std::fabs(eta) - lo) / (hi - lo));
}

// psi_F(d): face F's share of the partition of unity on the sphere
double surface_pou(int F, const double* d, double delta) {
  double num = 0, den = 0;
  for (int G = 0; G < 6; ++G) {
    const double z = dot3(d, kFaces[G][2]);
    if (!(z > 1e-12)) continue;
    const double b = face_bump(std::atan2(dot3(d, kFaces[G][0]), z), std::atan2(dot3(d, kFaces[G][1]), z), delta);
    den += b;
    if (G == F) num = b;
  }
  return num / den;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n from the
// Chebyshev-like first guesses), ascending.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute the derivative at the converged root
    double p0 = 1, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Lagrange weights of the integer nodes s..s+p at t
void lagrange_row(double t, int64_t s, int p, double* L) {
  constexpr int kMax = 16;
  if (p >= kMax) {
    for (int k = 0; k <= p; ++k) {
      double v = 1;
      for (int m = 0; m <= p; ++m)
        if (m != k) v *= (t - double(s + m)) / double(k - m);
      L[k] = v;
    }
    return;
  }
  // L_k = prod_{m != k} (t - s - m) / (k - m): prefix and suffix products of the
  // differences d_m = t - s - m over the denominator (-1)^(p - k) k! (p - k)!
  // (exact in double for p < 16), one division per weight instead of p
  double d[kMax], suf[kMax + 1], fact[kMax];
  fact[0] = 1;
  for (int m = 1; m <= p; ++m) fact[m] = fact[m - 1] * m;
  for (int m = 0; m <= p; ++m) d[m] = t - double(s + m);
  suf[p + 1] = 1;
  for (int m = p; m >= 0; --m) suf[m] = suf[m + 1] * d[m];
  double pre = 1;
  for (int k = 0; k <= p; ++k) {
    const double den = ((p - k) & 1 ? -1.0 : 1.0) * fact[k] * fact[p - k];
    L[k] = pre * suf[k + 1] / den;
    pre *= d[k];
  }
}

}  // namespace

bool build_ball3(Ball3& B) {
  const int nf = B.n_f, ns = B.n_s, Q = B.Q;
  if (!(B.a > 0 && B.w > 0 && B.w < B.a && B.h > 0)) { B.err = "need a > 0, 0 < w < a, h > 0"; return false; }
  if (nf < 2 || ns < 2 || Q < 2 || Q > 5 || (ns - 1) % (Q - 1)) {
    B.err = "need n_f >= 2, 2 <= Q <= 5 and n_s - 1 a multiple of Q - 1";
    return false;
  }
  if (!(B.delta > 0 && B.delta < M_PI / 4)) { B.err = "need 0 < delta < pi / 4"; return false; }
  if (!(B.tau0 > 0 && B.tau0 < B.tau1 && B.tau1 < 1)) { B.err = "need 0 < tau0 < tau1 < 1"; return false; }
  const double half = M_PI / 4 + B.delta;
  const double dg = (2 * half) / (nf - 1);
  const double ds = 1.0 / (ns - 1);
  std::vector<double> g(nf), s(ns), ws(ns, 0.0);
  for (int i = 0; i < nf; ++i) g[i] = i * dg - half;
  g[nf - 1] = half;
  for (int k = 0; k < ns; ++k) s[k] = k * ds;
  s[ns - 1] = 1.0;
  const std::vector<double> nc = newton_cotes(Q);
  for (int blk = 0; blk < (ns - 1) / (Q - 1); ++blk)
    for (int k = 0; k < Q; ++k) ws[blk * (Q - 1) + k] += nc[k];
  for (double& v : ws) v *= (s[1] - s[0]);
  auto clear = [&]() {
    B.x.clear(); B.w_q.clear(); B.omega.clear(); B.psi.clear(); B.face.clear(); B.grid.clear(); B.psi_omega.clear();
  };
  clear();
  for (int F = 0; F < 6; ++F)
    for (int i = 0; i < nf; ++i)
      for (int j = 0; j < nf; ++j) {
        double d[3], dom;
        face_direction(F, g[i], g[j], d, &dom);
        const double psi = surface_pou(F, d, B.delta);
        for (int k = 0; k < ns; ++k) {
          const double r = B.a - s[k] * B.w;
          const double wq = dg * dg * ws[k] * B.w * r * r * dom * psi;
          if (!(wq > 0.0)) continue;
          for (int c = 0; c < 3; ++c) B.x.push_back(r * d[c]);
          B.w_q.push_back(wq);
          B.omega.push_back(smooth_step((s[k] - B.tau0) / (B.tau1 - B.tau0)));
          B.psi.push_back(psi);
          B.face.push_back(int8_t(F));
          B.grid.insert(B.grid.end(), {i, j, k});
        }
      }
  B.n_shell = int64_t(B.w_q.size());
  const int m = B.grid_m = int(std::ceil(B.a / B.h));
  const double h3 = B.h * B.h * B.h;
  for (int ix = -m; ix <= m; ++ix)
    for (int iy = -m; iy <= m; ++iy)
      for (int iz = -m; iz <= m; ++iz) {
        const double p[3] = {B.h * ix, B.h * iy, B.h * iz};
        const double depth = (B.a - std::sqrt(dot3(p, p))) / B.w;
        const double om = depth > 0 ? 1.0 - smooth_step((depth - B.tau0) / (B.tau1 - B.tau0)) : 0.0;
        if (!(om > 0.0)) continue;
        B.x.insert(B.x.end(), p, p + 3);
        B.w_q.push_back(h3);
        B.omega.push_back(om);
        B.psi.push_back(0.0);
        B.face.push_back(int8_t(-1));
        B.grid.insert(B.grid.end(), {ix + m, iy + m, iz + m});
      }
  B.N = int64_t(B.w_q.size());
  B.n_cart = B.N - B.n_shell;
  B.psi_omega.resize(B.N);
  for (int64_t n = 0; n < B.N; ++n) B.psi_omega[n] = B.psi[n] * B.omega[n];
  B.face_node.assign(size_t(6) * nf * nf * ns, -1);
  const int side = 2 * m + 1;
  B.cart_node.assign(size_t(side) * side * side, -1);
  for (int64_t n = 0; n < B.N; ++n) {
    const int32_t* gi = &B.grid[3 * n];
    if (n < B.n_shell)
      B.face_node[((size_t(B.face[n]) * nf + gi[0]) * nf + gi[1]) * ns + gi[2]] = n;
    else
      B.cart_node[(size_t(gi[0]) * side + gi[1]) * side + gi[2]] = n;
  }
  return true;
}

bool interior_window3(double kappa, double h, double R, int p, int q, int n_rho, int n_mu, int n_phi, double chi_s0,
                      std::vector<cd>& win, int* Wn_out, std::string* err) {
  if (!(kappa >= 0 && h > 0 && R > 0) || p < 1 || q < 1 || n_rho < 2 || n_mu < 1 || n_phi < 1 ||
      !(chi_s0 >= 0 && chi_s0 < 1)) {
    *err = "invalid interior rule parameters";
    return false;
  }
  const int Wn = int(std::ceil(R)) + p / 2 + 2;
  const int side = 2 * Wn + 1;
  *Wn_out = Wn;
  win.assign(size_t(side) * side * side, cd(0.0));
  std::vector<double> mu, wmu;
  gauss_legendre(n_mu, mu, wmu);
  std::vector<double> La(p + 1), Lb(p + 1), Lc(p + 1);
  for (int ir = 1; ir < n_rho; ++ir) {
    const double sv = double(ir) / n_rho;
    const double rho = R * std::pow(sv, q);
    const double wr = (1.0 / n_rho) * R * q * std::pow(sv, q - 1) * cutoff(std::pow(sv, q), chi_s0);
    if (wr == 0.0) continue;
    // rho^2 h^3 G(rho h) = rho h^2 exp(i kappa rho h) / (4 pi)
    const cd kern = std::polar(rho * h * h / (4 * M_PI), kappa * rho * h);
    for (int im = 0; im < n_mu; ++im) {
      const double st = std::sqrt(1 - mu[im] * mu[im]);
      for (int ip = 0; ip < n_phi; ++ip) {
        const double ph = 2 * M_PI * ip / n_phi;
        const double o[3] = {rho * st * std::cos(ph), rho * st * std::sin(ph), rho * mu[im]};
        const cd f = (wr * wmu[im] * (2 * M_PI / n_phi)) * kern;
        int64_t s0[3];
        for (int k = 0; k < 3; ++k) s0[k] = int64_t(std::floor(o[k])) - p / 2;
        lagrange_row(o[0], s0[0], p, La.data());
        lagrange_row(o[1], s0[1], p, Lb.data());
        lagrange_row(o[2], s0[2], p, Lc.data());
        for (int i = 0; i <= p; ++i)
          for (int j = 0; j <= p; ++j) {
            const cd fij = f * (La[i] * Lb[j]);
            const size_t base = (size_t(s0[0] + i + Wn) * side + size_t(s0[1] + j + Wn)) * side;
            for (int k = 0; k <= p; ++k) win[base + size_t(s0[2] + k + Wn)] += fij * Lc[k];
          }
      }
    }
  }
  return true;
}

namespace {

// Split Newton-Cotes lines and weights across the depth for a target on line
// j of lines 0..nb-1 (Eq. VolInt-Adj-Sing-MultiSplit): composite Q-point
// blocks outward from j, and each interval left over near an end gets a
// Q-point rule on fractional lines.
std::map<double, double> split_nc(int j, int nb, int Q) {
  const std::vector<double> nc = newton_cotes(Q);
  std::map<double, double> out;
  const int L1 = j / (Q - 1);
  for (int l = 1; l <= L1; ++l)
    for (int mm = 0; mm < Q; ++mm) out[double(j - l * (Q - 1) + mm)] += nc[mm];
  const int I1 = j - L1 * (Q - 1);
  for (int i = 1; i <= I1; ++i)
    for (int mm = 0; mm < Q; ++mm) out[(j - L1 * (Q - 1) - i) + double(mm) / (Q - 1)] += nc[mm] / (Q - 1);
  const int top = nb - 1;
  const int L2 = (top - j) / (Q - 1);
  for (int l = 1; l <= L2; ++l)
    for (int mm = 0; mm < Q; ++mm) out[double(j + (l - 1) * (Q - 1) + mm)] += nc[mm];
  const int I2 = (top - j) - L2 * (Q - 1);
  for (int i = 1; i <= I2; ++i)
    for (int mm = 0; mm < Q; ++mm) out[(j + L2 * (Q - 1) + (i - 1)) + double(mm) / (Q - 1)] += nc[mm] / (Q - 1);
  return out;
}

// Sparse accumulator over node ids: a dense scratch with a list of the
// entries touched, for the singular parts of one row and their cut-offs.
struct RowAcc {
  std::vector<cd> v;
  std::vector<double> eta;
  std::vector<char> seen, eseen;
  std::vector<int64_t> idx, eidx;
  explicit RowAcc(int64_t N) : v(N, cd(0.0)), eta(N, 0.0), seen(N, 0), eseen(N, 0) {}
  void add(int64_t n, cd x) {
    if (!seen[n]) { seen[n] = 1; idx.push_back(n); }
    v[n] += x;
  }
  void set_eta(int64_t n, double e) {
    if (!eseen[n]) { eseen[n] = 1; eidx.push_back(n); }
    eta[n] = e;
  }
  void clear() {
    for (int64_t n : idx) { v[n] = 0.0; seen[n] = 0; }
    for (int64_t n : eidx) { eta[n] = 0.0; eseen[n] = 0; }
    idx.clear();
    eidx.clear();
  }
};

// acc[node] += f * La Lb Lc * factor[node] over the tensor stencil of one
// point; node_of maps grid (na, nb, nc) to a node id or -1.
inline void scatter(RowAcc& acc, const int64_t* node_of, int na, int nb, int nc, const int64_t* st, const double* La,
                    const double* Lb, const double* Lc, int pa, int pc, cd f, const std::vector<double>& factor) {
  for (int i = 0; i <= pa; ++i) {
    const int64_t ia = st[0] + i;
    if (ia < 0 || ia >= na) continue;
    for (int j = 0; j <= pa; ++j) {
      const int64_t ib = st[1] + j;
      if (ib < 0 || ib >= nb) continue;
      const cd fij = f * (La[i] * Lb[j]);
      for (int k = 0; k <= pc; ++k) {
        const int64_t ic = st[2] + k;
        if (ic < 0 || ic >= nc) continue;
        const int64_t n = node_of[(size_t(ia) * nb + size_t(ib)) * nc + size_t(ic)];
        if (n >= 0) acc.add(n, fij * Lc[k] * factor[n]);
      }
    }
  }
}

// Dense accumulation window over grid indices [o, o + n) per axis: the rule
// points' interpolation stencils land here without node lookups; flush()
// hands the nonzero cells to the row (skipping indices outside the grid and
// grid points that are not nodes).  A stencil that leaves the window (never
// expected: the window is sized from the rule's reach) goes to the row
// directly.
struct Win3 {
  int64_t o[3] = {0, 0, 0};
  int n[3] = {0, 0, 0};
  std::vector<double> re, im;      // real and imaginary parts apart: the stencil loops vectorise
  void reset(int64_t o0, int64_t o1, int64_t o2, int n0, int n1, int n2) {
    o[0] = o0; o[1] = o1; o[2] = o2;
    n[0] = n0; n[1] = n1; n[2] = n2;
    re.assign(size_t(n0) * n1 * n2, 0.0);
    im.assign(size_t(n0) * n1 * n2, 0.0);
  }
  bool inside(const int64_t* st, int pa, int pc) const {
    return st[0] >= o[0] && st[0] + pa < o[0] + n[0] && st[1] >= o[1] && st[1] + pa < o[1] + n[1] &&
           st[2] >= o[2] && st[2] + pc < o[2] + n[2];
  }
  // a[i][j][k] += f La[i] Lb[j] Lc[k] over the stencil starting at st
  void add(const int64_t* st, const double* La, const double* Lb, const double* Lc, int pa, int pc, cd f) {
    for (int i = 0; i <= pa; ++i) {
      const size_t bi = size_t(st[0] + i - o[0]) * n[1];
      for (int j = 0; j <= pa; ++j) {
        const cd fij = f * (La[i] * Lb[j]);
        const double fr = fij.real(), fi = fij.imag();
        const size_t r0 = (bi + size_t(st[1] + j - o[1])) * n[2] + size_t(st[2] - o[2]);
        double* __restrict__ rr = &re[r0];
        double* __restrict__ ri = &im[r0];
        for (int k = 0; k <= pc; ++k) {
          rr[k] += fr * Lc[k];
          ri[k] += fi * Lc[k];
        }
      }
    }
  }
  void flush(RowAcc& acc, const int64_t* node_of, int na, int nb, int nc, const std::vector<double>& factor) const {
    for (int i = 0; i < n[0]; ++i) {
      const int64_t gi = o[0] + i;
      if (gi < 0 || gi >= na) continue;
      for (int j = 0; j < n[1]; ++j) {
        const int64_t gj = o[1] + j;
        if (gj < 0 || gj >= nb) continue;
        for (int k = 0; k < n[2]; ++k) {
          const int64_t gk = o[2] + k;
          if (gk < 0 || gk >= nc) continue;
          const size_t e = (size_t(i) * n[1] + j) * n[2] + k;
          const cd v(re[e], im[e]);
          if (v == 0.0) continue;
          const int64_t nd = node_of[(size_t(gi) * nb + size_t(gj)) * nc + size_t(gk)];
          if (nd >= 0) acc.add(nd, v * factor[nd]);
        }
      }
    }
  }
};

bool check_rules(const Rules3& ru, std::string* err) {
  if (!(ru.R > 0 && ru.rc > 0 && ru.rs > 0) || ru.p < 1 || ru.q < 1 || ru.n_rho < 2 || ru.n_mu < 1 ||
      ru.n_phi < 1 || ru.n_sig < 2 || ru.n_th < 1 || !(ru.chi_s0 >= 0 && ru.chi_s0 < 1)) {
    *err = "invalid rule parameters";
    return false;
  }
  return true;
}

// Index range [lo, hi] of a window |i - c| <= r clipped to 0..n-1.
inline void window(double c, double r, int n, int* lo, int* hi) {
  *lo = std::max(0, int(std::floor(c - r)));
  *hi = std::min(n - 1, int(std::ceil(c + r)));
}

// The singular parts of row qn (every rule that reaches x_q) and the cut-off
// values eta of the rules applied, accumulated sparsely.
// iwin: the interior rule's window for grid-point targets (interior_window3 with
// the same rule), or null to evaluate the rule about each target.
void singular_parts(const Ball3& B, double kappa, const Rules3& ru, int64_t qn, RowAcc& acc,
                    const std::vector<cd>* iwin = nullptr, int iwn = 0) {
  const int nf = B.n_f, ns = B.n_s, p = ru.p, ps = std::min(ru.p, ns - 1);
  const double h = B.h;
  const double half = M_PI / 4 + B.delta, dg = (2 * half) / (nf - 1), ds = 1.0 / (ns - 1);
  const double* x = &B.x[3 * qn];
  const std::vector<double>& fac_shell = B.psi_omega;   // phi_F / u on the face grids
  const std::vector<double>& fac_cart = B.omega;        // phi_I / u on the interior grid
  std::vector<double> mu, wmu;
  gauss_legendre(ru.n_mu, mu, wmu);
  std::vector<double> La(p + 1), Lb(p + 1), Lc(p + 1);
  auto chi = [&](double v) { return cutoff(v, ru.chi_s0); };
  // ---- interior patch: spherical rule about x, if its ball reaches interior nodes
  const int side = 2 * B.grid_m + 1;
  double cg[3];
  int lo[3], hi[3];
  for (int k = 0; k < 3; ++k) {
    cg[k] = x[k] / h + B.grid_m;
    window(cg[k], ru.R, side, &lo[k], &hi[k]);
  }
  bool reach = false;
  for (int i = lo[0]; i <= hi[0]; ++i)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int k = lo[2]; k <= hi[2]; ++k) {
        const int64_t n = B.cart_node[(size_t(i) * side + j) * side + k];
        if (n < 0) continue;
        const double dx = B.x[3 * n] - x[0], dy = B.x[3 * n + 1] - x[1], dz = B.x[3 * n + 2] - x[2];
        reach = reach || std::sqrt(dx * dx + dy * dy + dz * dz) < ru.R * h;
      }
  if (reach && iwin && qn >= B.n_shell) {
    // a grid-point target: the rule is the shared window, shifted
    const int ws = 2 * iwn + 1;
    const int64_t g[3] = {B.grid[3 * qn], B.grid[3 * qn + 1], B.grid[3 * qn + 2]};
    for (int i = 0; i < ws; ++i) {
      const int64_t gi = g[0] + i - iwn;
      if (gi < 0 || gi >= side) continue;
      for (int j = 0; j < ws; ++j) {
        const int64_t gj = g[1] + j - iwn;
        if (gj < 0 || gj >= side) continue;
        for (int k = 0; k < ws; ++k) {
          const int64_t gk = g[2] + k - iwn;
          if (gk < 0 || gk >= side) continue;
          const cd c = (*iwin)[(size_t(i) * ws + j) * ws + k];
          if (c == 0.0) continue;
          const int64_t n = B.cart_node[(size_t(gi) * side + size_t(gj)) * side + size_t(gk)];
          if (n >= 0) acc.add(n, c * fac_cart[n]);
        }
      }
    }
  } else if (reach) {
    Win3 w;
    const int wn = 2 * int(std::ceil(ru.R)) + p + 4;
    w.reset(int64_t(std::floor(cg[0] - ru.R)) - p / 2 - 1, int64_t(std::floor(cg[1] - ru.R)) - p / 2 - 1,
            int64_t(std::floor(cg[2] - ru.R)) - p / 2 - 1, wn, wn, wn);
    for (int ir = 1; ir < ru.n_rho; ++ir) {
      const double sv = double(ir) / ru.n_rho, rho = ru.R * std::pow(sv, ru.q);
      const double wr = (1.0 / ru.n_rho) * ru.R * ru.q * std::pow(sv, ru.q - 1) * chi(std::pow(sv, ru.q));
      const cd kern = std::polar(rho * h * h / (4 * M_PI), kappa * rho * h);
      for (int im = 0; im < ru.n_mu; ++im) {
        const double st = std::sqrt(1 - mu[im] * mu[im]);
        for (int ip = 0; ip < ru.n_phi; ++ip) {
          const double ph = 2 * M_PI * ip / ru.n_phi;
          const double d[3] = {st * std::cos(ph), st * std::sin(ph), mu[im]};
          const cd f = (wr * wmu[im] * (2 * M_PI / ru.n_phi)) * kern;
          double c[3];
          int64_t s0[3];
          for (int k = 0; k < 3; ++k) {
            c[k] = cg[k] + rho * d[k];
            s0[k] = int64_t(std::floor(c[k])) - p / 2;
          }
          lagrange_row(c[0], s0[0], p, La.data());
          lagrange_row(c[1], s0[1], p, Lb.data());
          lagrange_row(c[2], s0[2], p, Lc.data());
          if (w.inside(s0, p, p)) w.add(s0, La.data(), Lb.data(), Lc.data(), p, p, f);
          else
            scatter(acc, B.cart_node.data(), side, side, side, s0, La.data(), Lb.data(), Lc.data(), p, p, f,
                    fac_cart);
        }
      }
    }
    w.flush(acc, B.cart_node.data(), side, side, side, fac_cart);
  }
  if (reach) {
    for (int i = lo[0]; i <= hi[0]; ++i)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int k = lo[2]; k <= hi[2]; ++k) {
          const int64_t n = B.cart_node[(size_t(i) * side + j) * side + k];
          if (n < 0) continue;
          const double dx = B.x[3 * n] - x[0], dy = B.x[3 * n + 1] - x[1], dz = B.x[3 * n + 2] - x[2];
          const double e = chi(std::sqrt(dx * dx + dy * dy + dz * dz) / (ru.R * h));
          if (e > 0) acc.set_eta(n, e);
        }
  }
  // ---- shell patches: a rule on every face whose extended chart holds x
  const double r_x = std::sqrt(dot3(x, x));
  const double s_x = (B.a - r_x) / B.w;
  const bool is_shell = qn < B.n_shell;
  if (!(s_x < 1.0)) return;
  const double dirx[3] = {x[0] / r_x, x[1] / r_x, x[2] / r_x};
  for (int G = 0; G < 6; ++G) {
    const double zc = dot3(dirx, kFaces[G][2]);
    if (zc <= 1e-12) continue;
    const double xi = std::atan2(dot3(dirx, kFaces[G][0]), zc), et = std::atan2(dot3(dirx, kFaces[G][1]), zc);
    const double cx = (xi + half) / dg, cy = (et + half) / dg;
    if (!(cx >= 0.0 && cx <= nf - 1 && cy >= 0.0 && cy <= nf - 1)) continue;
    // rule points in face-grid index coordinates (ti, tj, tk) and weights wq
    std::vector<double> ti, tj, tk, wq;
    const int k0 = is_shell ? B.grid[3 * qn + 2] : 0;
    const double cz = s_x / ds, rsp = std::min(ru.rs, B.tau0 * (ns - 1));
    if (is_shell) {
      const std::map<double, double> lines = split_nc(k0, ns, B.Q);
      for (const auto& [t, wl] : lines) {
        if (!(std::fabs(t - k0) < ru.rs)) continue;
        const double wsl = wl * chi((t - k0) / ru.rs);
        for (int is = 1; is < ru.n_sig; ++is) {
          const double sg = double(is) / ru.n_sig, rho = ru.rc * std::pow(sg, ru.q);
          const double wsg = (1.0 / ru.n_sig) * ru.rc * ru.q * std::pow(sg, ru.q - 1) * chi(std::pow(sg, ru.q));
          for (int it = 0; it < ru.n_th; ++it) {
            const double th = 2 * M_PI * it / ru.n_th;
            ti.push_back(cx + rho * std::cos(th));
            tj.push_back(cy + rho * std::sin(th));
            tk.push_back(t);
            wq.push_back(wsl * wsg * (2 * M_PI / ru.n_th) * rho);
          }
        }
      }
    } else {
      for (int ir = 1; ir < ru.n_rho; ++ir) {
        const double sv = double(ir) / ru.n_rho, rho = std::pow(sv, ru.q);
        const double wr = (1.0 / ru.n_rho) * ru.q * std::pow(sv, ru.q - 1) * chi(rho);
        for (int im = 0; im < ru.n_mu; ++im) {
          const double st = std::sqrt(1 - mu[im] * mu[im]);
          for (int ip = 0; ip < ru.n_phi; ++ip) {
            const double ph = 2 * M_PI * ip / ru.n_phi;
            const double tkv = cz + rsp * rho * mu[im];
            ti.push_back(cx + ru.rc * rho * st * std::cos(ph));
            tj.push_back(cy + ru.rc * rho * st * std::sin(ph));
            tk.push_back(tkv);
            // past the chart's bottom line phi_F is exactly zero: drop the point
            const double wv = wr * wmu[im] * (2 * M_PI / ru.n_phi) * rho * rho * ru.rc * ru.rc * rsp;
            wq.push_back(tkv <= ns - 1 ? wv : 0.0);
          }
        }
      }
    }
    const int64_t* node_of = &B.face_node[size_t(G) * nf * nf * ns];
    Win3 w;
    const int wn = 2 * int(std::ceil(ru.rc)) + p + 4;
    w.reset(int64_t(std::floor(cx - ru.rc)) - p / 2 - 1, int64_t(std::floor(cy - ru.rc)) - p / 2 - 1, 0, wn, wn, ns);
    // plane accumulator for the points of one depth line (boundary rule)
    std::vector<cd> plane(size_t(wn) * wn, cd(0.0));
    double line_t = -1.0;
    int64_t line_s = 0;
    std::vector<double> Lline(ps + 1);
    bool plane_used = false;
    auto spread_line = [&]() {
      if (!plane_used) return;
      for (int i = 0; i < wn; ++i)
        for (int j = 0; j < wn; ++j) {
          cd& v = plane[size_t(i) * wn + j];
          if (v == 0.0) continue;
          const size_t d0 = (size_t(i) * wn + j) * ns + size_t(line_s);
          for (int k = 0; k <= ps; ++k) {
            w.re[d0 + k] += v.real() * Lline[k];
            w.im[d0 + k] += v.imag() * Lline[k];
          }
          v = 0.0;
        }
      plane_used = false;
    };
    for (size_t r = 0; r < wq.size(); ++r) {
      double dd[3], dom;
      face_direction(G, ti[r] * dg - half, tj[r] * dg - half, dd, &dom);
      const double rp = B.a - tk[r] * ds * B.w;
      const double y[3] = {rp * dd[0], rp * dd[1], rp * dd[2]};
      const double J = B.w * rp * rp * dom * dg * dg * ds;
      const double dist = std::sqrt((y[0] - x[0]) * (y[0] - x[0]) + (y[1] - x[1]) * (y[1] - x[1]) +
                                    (y[2] - x[2]) * (y[2] - x[2]));
      const cd f = std::polar(wq[r] * J / (4 * M_PI * dist), kappa * dist);
      int64_t s0[3];
      s0[0] = int64_t(std::floor(ti[r])) - p / 2;
      s0[1] = int64_t(std::floor(tj[r])) - p / 2;
      s0[2] = std::min<int64_t>(std::max<int64_t>(int64_t(std::floor(tk[r])) - ps / 2, 0), ns - 1 - ps);
      lagrange_row(ti[r], s0[0], p, La.data());
      lagrange_row(tj[r], s0[1], p, Lb.data());
      if (!w.inside(s0, p, ps)) {
        lagrange_row(tk[r], s0[2], ps, Lc.data());
        scatter(acc, node_of, nf, nf, ns, s0, La.data(), Lb.data(), Lc.data(), p, ps, f, fac_shell);
      } else if (is_shell) {
        if (tk[r] != line_t) {
          spread_line();
          line_t = tk[r];
          line_s = s0[2];
          lagrange_row(tk[r], s0[2], ps, Lline.data());
        }
        for (int i = 0; i <= p; ++i) {
          cd* prow = &plane[size_t(s0[0] + i - w.o[0]) * wn + size_t(s0[1] - w.o[1])];
          const cd fi = f * La[i];
          for (int j = 0; j <= p; ++j) prow[j] += fi * Lb[j];
        }
        plane_used = true;
      } else {
        lagrange_row(tk[r], s0[2], ps, Lc.data());
        w.add(s0, La.data(), Lb.data(), Lc.data(), p, ps, f);
      }
    }
    spread_line();
    w.flush(acc, node_of, nf, nf, ns, fac_shell);
    // cut-off values on this face's nodes (zero outside the windows)
    int ilo, ihi, jlo, jhi, klo, khi;
    window(cx, ru.rc, nf, &ilo, &ihi);
    window(cy, ru.rc, nf, &jlo, &jhi);
    if (is_shell) window(double(k0), ru.rs, ns, &klo, &khi);
    else window(cz, rsp, ns, &klo, &khi);
    for (int i = ilo; i <= ihi; ++i)
      for (int j = jlo; j <= jhi; ++j)
        for (int k = klo; k <= khi; ++k) {
          const int64_t n = node_of[(size_t(i) * nf + j) * ns + k];
          if (n < 0) continue;
          double e;
          if (is_shell) {
            e = chi(std::hypot(i - cx, j - cy) / ru.rc) * chi(double(k - k0) / ru.rs);
          } else {
            const double a = (i - cx) / ru.rc, b = (j - cy) / ru.rc, c = (k - cz) / rsp;
            e = chi(std::sqrt(a * a + b * b + c * c));
          }
          if (e > 0) acc.set_eta(n, e);
        }
  }
}

}  // namespace

bool ball3_row(const Ball3& B, double kappa, const Rules3& ru, int64_t qn, cd* row, double* eta_out,
               std::string* err) {
  if (qn < 0 || qn >= B.N) { *err = "node index out of range"; return false; }
  if (!check_rules(ru, err)) return false;
  RowAcc acc(B.N);
  singular_parts(B, kappa, ru, qn, acc);
  const double* x = &B.x[3 * qn];
  for (int64_t n = 0; n < B.N; ++n) {
    row[n] = acc.v[n];
    const double dx = B.x[3 * n] - x[0], dy = B.x[3 * n + 1] - x[1], dz = B.x[3 * n + 2] - x[2];
    const double dist = std::sqrt(dx * dx + dy * dy + dz * dz);
    if (dist > 0)
      row[n] += std::polar(B.w_q[n] * B.omega[n] * (1.0 - acc.eta[n]) / (4 * M_PI * dist), kappa * dist);
  }
  if (eta_out) std::copy(acc.eta.begin(), acc.eta.end(), eta_out);
  return true;
}

bool ball3_near(Ball3& B, double kappa, const Rules3& ru, const double* box0, double H, int L, const int64_t* rows,
                int64_t n_rows, bool stencils_only, int n_threads, std::string* err) {
  if (!check_rules(ru, err)) return false;
  if (!(H > 0) || L < 1) { *err = "invalid cell box"; return false; }
  const int64_t N = B.N;
  // cells of the nodes and the nodes of each cell
  const int64_t ncell = int64_t(L) * L * L;
  std::vector<int32_t> cijk(3 * N);
  std::vector<int64_t> start(ncell + 1, 0), members(N);
  for (int64_t n = 0; n < N; ++n) {
    for (int k = 0; k < 3; ++k) {
      const double t = std::floor((B.x[3 * n + k] - box0[k]) / H);
      if (!(t >= 0 && t < L)) { *err = "nodes outside the cell box"; return false; }
      cijk[3 * n + k] = int32_t(t);
    }
    ++start[(int64_t(cijk[3 * n + 2]) * L + cijk[3 * n + 1]) * L + cijk[3 * n] + 1];
  }
  for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
  {
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    for (int64_t n = 0; n < N; ++n)
      members[fill[(int64_t(cijk[3 * n + 2]) * L + cijk[3 * n + 1]) * L + cijk[3 * n]]++] = n;
  }
  std::vector<int64_t> all;
  if (!rows) {
    all.resize(N);
    for (int64_t n = 0; n < N; ++n) all[n] = n;
    rows = all.data();
    n_rows = N;
  }
  for (int64_t r = 0; r < n_rows; ++r)
    if (rows[r] < 0 || rows[r] >= N) { *err = "row index out of range"; return false; }
  std::vector<std::vector<int32_t>> cols(n_rows);
  std::vector<std::vector<cd>> vals(n_rows);
  std::atomic<bool> bad(false);
  std::vector<cd> iwin;
  int iwn = 0;
  if (!interior_window3(kappa, B.h, ru.R, ru.p, ru.q, ru.n_rho, ru.n_mu, ru.n_phi, ru.chi_s0, iwin, &iwn, err))
    return false;
  parallel_for(n_threads, n_rows, 16, [&](int64_t r0, int64_t r1) {
    RowAcc acc(N);
    std::vector<char> in_block(N, 0);
    std::vector<int64_t> block;
    for (int64_t r = r0; r < r1 && !bad; ++r) {
      const int64_t qn = rows[r];
      const double* x = &B.x[3 * qn];
      acc.clear();
      singular_parts(B, kappa, ru, qn, acc, &iwin, iwn);
      // regular (1 - eta) terms over the 3 x 3 x 3 cell block N(x)
      block.clear();
      for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj)
          for (int dk = -1; dk <= 1; ++dk) {
            const int i = cijk[3 * qn] + di, j = cijk[3 * qn + 1] + dj, k = cijk[3 * qn + 2] + dk;
            if (i < 0 || j < 0 || k < 0 || i >= L || j >= L || k >= L) continue;
            const int64_t c = (int64_t(k) * L + j) * L + i;
            for (int64_t t = start[c]; t < start[c + 1]; ++t) block.push_back(members[t]);
          }
      for (int64_t n : block) in_block[n] = 1;
      if (stencils_only) {
        // the sparse correction -eta w omega G; the caller adds w omega G over the block
        for (int64_t n : acc.eidx) {
          const double dx = B.x[3 * n] - x[0], dy = B.x[3 * n + 1] - x[1], dz = B.x[3 * n + 2] - x[2];
          const double dist = std::sqrt(dx * dx + dy * dy + dz * dz);
          if (dist > 0 && acc.eta[n] > 0)
            acc.add(n, std::polar(-B.w_q[n] * B.omega[n] * acc.eta[n] / (4 * M_PI * dist), kappa * dist));
        }
      } else {
        for (int64_t n : block) {
          const double dx = B.x[3 * n] - x[0], dy = B.x[3 * n + 1] - x[1], dz = B.x[3 * n + 2] - x[2];
          const double dist = std::sqrt(dx * dx + dy * dy + dz * dz);
          if (dist > 0)
            acc.add(n, std::polar(B.w_q[n] * B.omega[n] * (1.0 - acc.eta[n]) / (4 * M_PI * dist), kappa * dist));
        }
      }
      for (int64_t n : acc.eidx)
        if (acc.eta[n] > 0 && !in_block[n]) bad = true;
      for (int64_t n : block) in_block[n] = 0;
      std::vector<int64_t> idx = acc.idx;
      std::sort(idx.begin(), idx.end());
      cols[r].reserve(idx.size());
      vals[r].reserve(idx.size());
      for (int64_t n : idx) {
        cols[r].push_back(int32_t(n));
        vals[r].push_back(acc.v[n]);
      }
    }
  });
  if (bad) { *err = "cut-off support leaves the 3 x 3 x 3 cell block: enlarge H or shrink the rules"; return false; }
  // assemble into fresh arrays and swap them in, so that a failed call leaves
  // the previous result intact
  std::vector<int64_t> nrows(rows, rows + n_rows), rowptr(n_rows + 1, 0);
  for (int64_t r = 0; r < n_rows; ++r) rowptr[r + 1] = rowptr[r] + int64_t(cols[r].size());
  std::vector<int32_t> col(rowptr[n_rows]);
  std::vector<cd> val(rowptr[n_rows]);
  for (int64_t r = 0; r < n_rows; ++r) {
    std::copy(cols[r].begin(), cols[r].end(), col.begin() + rowptr[r]);
    std::copy(vals[r].begin(), vals[r].end(), val.begin() + rowptr[r]);
  }
  B.near_rows.swap(nrows);
  B.near_rowptr.swap(rowptr);
  B.near_col.swap(col);
  B.near_val.swap(val);
  return true;
}

}  // namespace lsh
