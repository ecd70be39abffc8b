// Near-field matrix: localised singular quadratures (Section 3.1) plus the
// adjacent regular terms (first two terms of Eq. VolInt-Adj-NonAdj-I).
//
// For every target x_q the row holds
//   sum over nodes l in the 3 x 3 cell block N(x_q) of
//        w_l m_l omega_l G(x_q, y_l) (1 - eta_{k(l)}(y_l; x_q))      (regular)
//   + the singular rule of every patch whose cut-off reaches x_q,
//     each written as coefficients of grid values phi = m omega u via
//     tensor-product Lagrange interpolation of degree p:
//   * Cartesian patch: polar rule (Eq. K-Int-Sing-Polar) about x_q with
//     rho = s^q on [0, 1] scaled by R_cart, trapezoid in s and theta;
//   * collar, collar target (i, j): rectangular cut-off, tangential integral
//     with t_1 = t_1^x + varrho(tau), varrho = R_a tau^(M+1) (Eqs. I,
//     POLYCOB, I-inTau), transverse integral by the split Newton-Cotes rule of
//     Eq. VolInt-Adj-Sing-MultiSplit (extra fractional lines near the ends);
//   * collar, Cartesian target inside the collar: polar rule on the collar
//     chart with semi-axes (R_a, min(R_b, tau0 (n2-1))).
// Everything is in grid-index units; eta must vanish outside N(x_q).
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>

#include "host_plan.hpp"

namespace lsh {

static const double kPi = 3.14159265358979323846;

static inline cd green(double kappa, double dx, double dy) {
  const double z = kappa * std::sqrt(dx * dx + dy * dy);
  return cd(0.0, 0.25) * cd(::j0(z), ::y0(z));
}

// 1 / prod_{m != k} (k - m) = (-1)^(p-k) / (k! (p-k)!) for the integer nodes 0..p
struct LagrangeDen {
  double c[32][32] = {};
  LagrangeDen() {
    double f[32];
    f[0] = 1.0;
    for (int i = 1; i < 32; ++i) f[i] = f[i - 1] * double(i);
    for (int p = 0; p < 32; ++p)
      for (int k = 0; k <= p; ++k) c[p][k] = ((p - k) % 2 ? -1.0 : 1.0) / (f[k] * f[p - k]);
  }
};
static const LagrangeDen kLagDen;

// Lagrange basis on the integer nodes start..start+p at x:
// l_k(x) = prod_{m != k} (x - x_m) / prod_{m != k} (k - m), the numerator from
// prefix and suffix products (no division)
static void lagrange(double x, int64_t start, int p, double* out) {
  double d[32], pre[33], suf[33];
  for (int m = 0; m <= p; ++m) d[m] = x - double(start + m);
  pre[0] = 1.0;
  for (int m = 0; m <= p; ++m) pre[m + 1] = pre[m] * d[m];
  suf[p + 1] = 1.0;
  for (int m = p; m >= 0; --m) suf[m] = suf[m + 1] * d[m];
  for (int k = 0; k <= p; ++k) out[k] = pre[k] * suf[k + 1] * kLagDen.c[p][k];
}

namespace {

struct Window {
  int64_t oa = 0, ob = 0;
  int Wa = 0, Wb = 0;
  std::vector<cd> v;
  void reset(int64_t oa_, int64_t ob_, int Wa_, int Wb_) {
    oa = oa_; ob = ob_; Wa = Wa_; Wb = Wb_;
    v.assign(size_t(Wa) * Wb, cd(0.0));
  }
  void add(int p, double a, double b, int64_t sa, int64_t sb, cd f) {
    double la[32], lb[32];
    lagrange(a, sa, p, la);
    lagrange(b, sb, p, lb);
    for (int k = 0; k <= p; ++k) {
      const cd fk = f * la[k];
      cd* row = &v[size_t(sa - oa + k) * Wb + (sb - ob)];
      for (int l = 0; l <= p; ++l) row[l] += fk * lb[l];
    }
  }
};

struct RowBuilder {
  const Plan2D& P;
  const Nodes& nd;
  const ls_geometry& g;
  const ls_options& o;
  double Rbc;                      // collar transverse semi-axis for Cartesian targets
  std::vector<std::pair<int64_t, cd>> ents;
  Window win;
  // polar template (relative offsets in unit disc) for the radial/angular rule
  std::vector<double> tr, tc, ts, tw;   // rho, cos, sin, weight (without Ra Rb)
  // regular term G(h d) (1 - eta) of a Cartesian target and a Cartesian source
  // at grid offset d = (da, db), |da|, |db| <= D: both factors depend on d only
  int D = 0;
  std::vector<cd> gcart;

  explicit RowBuilder(const Plan2D& plan)
      : P(plan), nd(plan.nodes), g(plan.geo.g), o(plan.opt) {
    Rbc = std::min(o.R_b, g.tau0 * (g.n2 - 1));
    // the 3 x 3 block spans less than two cells each way from a target's cell
    D = int(std::ceil(2.0 * o.H / g.h)) + 2;
    gcart.assign(size_t(2 * D + 1) * (2 * D + 1), cd(0.0));
    for (int da = -D; da <= D; ++da)
      for (int db = -D; db <= D; ++db) {
        const double ome = (da == 0 && db == 0) ? 0.0 : 1.0 - cutoff(std::hypot(double(da), double(db)) / o.R_cart,
                                                                        o.chi_s0);
        if (ome != 0.0) gcart[size_t(da + D) * (2 * D + 1) + (db + D)] = green(P.kappa, da * g.h, db * g.h) * ome;
      }
    const int q = o.q_polar;
    for (int ks = 1; ks < o.n_rho; ++ks) {
      const double s = double(ks) / o.n_rho;
      const double rho = std::pow(s, q);
      const double wq = (2.0 * kPi / o.n_theta) * (1.0 / o.n_rho) * q * std::pow(s, 2 * q - 1) *
                        cutoff(rho, o.chi_s0);
      if (wq == 0.0) continue;
      for (int mt = 0; mt < o.n_theta; ++mt) {
        const double th = 2.0 * kPi * mt / o.n_theta;
        tr.push_back(rho); tc.push_back(std::cos(th)); ts.push_back(std::sin(th)); tw.push_back(wq);
      }
    }
  }

  void flush_window(int chart) {
    for (int i = 0; i < win.Wa; ++i)
      for (int j = 0; j < win.Wb; ++j) {
        const cd c = win.v[size_t(i) * win.Wb + j];
        if (c == 0.0) continue;
        int64_t col = -1;
        if (chart == 0) {
          const int64_t ib = win.ob + j;
          if (ib < 0 || ib >= g.n2) continue;
          int64_t ia = (win.oa + i) % g.n1;
          if (ia < 0) ia += g.n1;
          col = nd.collar_pos[ia * g.n2 + ib];
        } else {
          const int64_t ia = win.oa + i, ib = win.ob + j;
          if (ia < 0 || ia >= g.cart_nx || ib < 0 || ib >= g.cart_ny) continue;
          col = nd.cart_pos[ia * g.cart_ny + ib];
        }
        if (col < 0) continue;
        ents.emplace_back(col, c * nd.phifac[col]);
      }
  }

  // interior-type (polar) rule on chart 0 (collar) or 1 (Cartesian)
  void polar(int chart, int64_t q, double ax, double bx) {
    const double Ra = chart == 0 ? o.R_a : o.R_cart;
    const double Rb = chart == 0 ? Rbc : o.R_cart;
    const int p = o.p;
    const int64_t oa = int64_t(std::floor(ax - Ra)) - p / 2 - 1;
    const int Wa = 2 * int(std::ceil(Ra)) + p + 4;
    int64_t ob;
    int Wb;
    if (chart == 0) { ob = 0; Wb = g.n2; }
    else { ob = int64_t(std::floor(bx - Rb)) - p / 2 - 1; Wb = 2 * int(std::ceil(Rb)) + p + 4; }
    win.reset(oa, ob, Wa, Wb);
    const double xq = nd.x[q], yq = nd.y[q];
    for (size_t t = 0; t < tr.size(); ++t) {
      const double a = ax + Ra * tr[t] * tc[t];
      const double b = bx + Rb * tr[t] * ts[t];
      double X[2], J;
      int64_t sb = int64_t(std::floor(b)) - p / 2;
      if (chart == 0) {
        if (b < 0.0 || b > g.n2 - 1) continue;
        P.geo.collar_map(a, b, X, &J);
        sb = std::min<int64_t>(std::max<int64_t>(sb, 0), g.n2 - 1 - p);
      } else {
        X[0] = g.cart_x0 + a * g.h; X[1] = g.cart_y0 + b * g.h; J = g.h * g.h;
      }
      const cd f = (tw[t] * Ra * Rb) * J * green(P.kappa, xq - X[0], yq - X[1]);
      win.add(p, a, b, int64_t(std::floor(a)) - p / 2, sb, f);
    }
    flush_window(chart);
  }

  // The Cartesian polar rule about a target on a Cartesian grid point: the
  // template offsets, their Lagrange weights and G(x_q - y) depend only on the
  // offset from the target, so the window (relative to the target) is computed
  // once and shifted; only the node ids and the m omega factors differ per target.
  std::vector<cd> cart_win;
  int64_t cw_oa = 0, cw_ob = 0;
  int cw_Wa = 0, cw_Wb = 0;

  void polar_cart_grid(int64_t ia, int64_t ib) {
    if (cart_win.empty()) {
      const double R = o.R_cart;
      const int p = o.p;
      win.reset(int64_t(std::floor(-R)) - p / 2 - 1, int64_t(std::floor(-R)) - p / 2 - 1,
                2 * int(std::ceil(R)) + p + 4, 2 * int(std::ceil(R)) + p + 4);
      for (size_t t = 0; t < tr.size(); ++t) {
        const double a = R * tr[t] * tc[t], b = R * tr[t] * ts[t];
        const cd f = (tw[t] * R * R) * (g.h * g.h) * green(P.kappa, -a * g.h, -b * g.h);
        win.add(p, a, b, int64_t(std::floor(a)) - p / 2, int64_t(std::floor(b)) - p / 2, f);
      }
      cart_win = win.v;
      cw_oa = win.oa; cw_ob = win.ob; cw_Wa = win.Wa; cw_Wb = win.Wb;
    }
    win.oa = ia + cw_oa;
    win.ob = ib + cw_ob;
    win.Wa = cw_Wa;
    win.Wb = cw_Wb;
    win.v = cart_win;
    flush_window(1);
  }

  // split Newton-Cotes nodes across the collar for a target on line j
  std::map<double, double> split_nc(int j) const {
    const std::vector<double> nc = newton_cotes(o.Q);
    const int Q = o.Q, top = g.n2 - 1;
    std::map<double, double> out;
    const int L1 = j / (Q - 1);
    for (int l = 1; l <= L1; ++l) {
      const int lo = j - l * (Q - 1);
      for (int m = 0; m < Q; ++m) out[double(lo + m)] += nc[m];
    }
    const int I1 = j - L1 * (Q - 1);
    for (int i = 1; i <= I1; ++i) {
      const int lo = j - L1 * (Q - 1) - i;
      for (int m = 0; m < Q; ++m) out[lo + double(m) / (Q - 1)] += nc[m] / (Q - 1);
    }
    const int L2 = (top - j) / (Q - 1);
    for (int l = 1; l <= L2; ++l) {
      const int lo = j + (l - 1) * (Q - 1);
      for (int m = 0; m < Q; ++m) out[double(lo + m)] += nc[m];
    }
    const int I2 = (top - j) - L2 * (Q - 1);
    for (int i = 1; i <= I2; ++i) {
      const int lo = j + L2 * (Q - 1) + (i - 1);
      for (int m = 0; m < Q; ++m) out[lo + double(m) / (Q - 1)] += nc[m] / (Q - 1);
    }
    return out;
  }

  void boundary(int64_t q, int i, int j) {
    const double Ra = o.R_a, Rb = o.R_b;
    const int p = o.p;
    const int64_t oa = int64_t(i) - int64_t(std::ceil(Ra)) - p / 2 - 1;
    const int Wa = 2 * int(std::ceil(Ra)) + p + 4;
    win.reset(oa, 0, Wa, g.n2);
    const double xq = nd.x[q], yq = nd.y[q];
    const std::map<double, double> tb = split_nc(j);
    for (const auto& kv : tb) {
      const double b = kv.first;
      if (!(std::fabs(b - j) < Rb)) continue;
      const double wb = kv.second * cutoff((b - j) / Rb, o.chi_s0);
      if (wb == 0.0) continue;
      const int64_t sb = std::min<int64_t>(std::max<int64_t>(int64_t(std::floor(b)) - p / 2, 0), g.n2 - 1 - p);
      for (int k = 0; k < o.N_tau; ++k) {
        const double tau = -1.0 + 2.0 * k / o.N_tau;
        const double rho = Ra * std::pow(tau, o.M + 1);
        const double drho = Ra * (o.M + 1) * std::pow(tau, o.M);
        const double wt = (2.0 / o.N_tau) * drho * cutoff(rho / Ra, o.chi_s0);
        const double w1 = wb * wt;
        if (w1 == 0.0) continue;
        const double a = i + rho;
        double X[2], J;
        P.geo.collar_map(a, b, X, &J);
        const cd f = w1 * J * green(P.kappa, xq - X[0], yq - X[1]);
        win.add(p, a, b, int64_t(std::floor(a)) - p / 2, sb, f);
      }
    }
    flush_window(0);
  }

  bool needs_cart_rule(int64_t q) const {
    const double reach = o.R_cart + o.p / 2.0 + 2.0;
    const double ga = nd.ga[q], gb = nd.gb[q];
    const int64_t lo_a = int64_t(std::max(std::floor(ga - reach), 0.0));
    const int64_t hi_a = int64_t(std::min(std::ceil(ga + reach), double(g.cart_nx - 1)));
    const int64_t lo_b = int64_t(std::max(std::floor(gb - reach), 0.0));
    const int64_t hi_b = int64_t(std::min(std::ceil(gb + reach), double(g.cart_ny - 1)));
    for (int64_t ia = lo_a; ia <= hi_a; ++ia)
      for (int64_t ib = lo_b; ib <= hi_b; ++ib)
        if (nd.cart_pos[ia * g.cart_ny + ib] >= 0) return true;
    return false;
  }

  double eta(int64_t q, int64_t l) const {
    if (nd.chart[l] == 1) {
      const double da = nd.ga[l] - nd.ga[q], db = nd.gb[l] - nd.gb[q];
      return cutoff(std::hypot(da, db) / o.R_cart, o.chi_s0);
    }
    double da = std::fmod(nd.ca[l] - nd.ca[q] + g.n1 / 2.0, double(g.n1));
    if (da < 0) da += g.n1;
    da -= g.n1 / 2.0;
    const double db = nd.cb[l] - nd.cb[q];
    if (nd.chart[q] == 0) return cutoff(da / o.R_a, o.chi_s0) * cutoff(db / o.R_b, o.chi_s0);
    if (nd.cb[q] <= g.n2 - 1) return cutoff(std::hypot(da / o.R_a, db / Rbc), o.chi_s0);
    return 0.0;
  }

  // true when every node with eta != 0 lies in the 3 x 3 block of q
  bool eta_inside_block(int64_t q, int ci, int cj) const {
    auto in_block = [&](int64_t l) {
      const int c = nd.cell[l], li = c % nd.L, lj = c / nd.L;
      return std::abs(li - ci) <= 1 && std::abs(lj - cj) <= 1;
    };
    const double R = o.R_cart;
    for (int64_t ia = int64_t(std::floor(nd.ga[q] - R)); ia <= int64_t(std::ceil(nd.ga[q] + R)); ++ia)
      for (int64_t ib = int64_t(std::floor(nd.gb[q] - R)); ib <= int64_t(std::ceil(nd.gb[q] + R)); ++ib) {
        if (ia < 0 || ib < 0 || ia >= g.cart_nx || ib >= g.cart_ny) continue;
        const int64_t l = nd.cart_pos[ia * g.cart_ny + ib];
        if (l >= 0 && eta(q, l) != 0.0 && !in_block(l)) return false;
      }
    if (nd.chart[q] == 1 && !(nd.cb[q] <= g.n2 - 1)) return true;
    const double Rb = nd.chart[q] == 0 ? o.R_b : Rbc;
    for (int64_t ia = int64_t(std::floor(nd.ca[q] - o.R_a)); ia <= int64_t(std::ceil(nd.ca[q] + o.R_a)); ++ia)
      for (int64_t ib = int64_t(std::floor(nd.cb[q] - Rb)); ib <= int64_t(std::ceil(nd.cb[q] + Rb)); ++ib) {
        if (ib < 0 || ib >= g.n2) continue;
        int64_t iw = ia % g.n1;
        if (iw < 0) iw += g.n1;
        const int64_t l = nd.collar_pos[iw * g.n2 + ib];
        if (eta(q, l) != 0.0 && !in_block(l)) return false;
      }
    return true;
  }

  // build row q into ents (sorted, merged); returns false if eta leaves N(x)
  bool row(int64_t q) {
    ents.clear();
    const int c = nd.cell[q], ci = c % nd.L, cj = c / nd.L;
    if (!eta_inside_block(q, ci, cj)) return false;
    // regular adjacent part
    for (int dj = -1; dj <= 1; ++dj) {
      const int nj = cj + dj;
      if (nj < 0 || nj >= nd.L) continue;
      for (int di = -1; di <= 1; ++di) {
        const int ni = ci + di;
        if (ni < 0 || ni >= nd.L) continue;
        const int nc = nj * nd.L + ni;
        for (int64_t l = nd.cell_start[nc]; l < nd.cell_start[nc + 1]; ++l) {
          if (nd.wfac[l] == 0.0) continue;
          if (nd.chart[q] == 1 && nd.chart[l] == 1) {
            const int64_t da = std::llround(nd.ga[l] - nd.ga[q]), db = std::llround(nd.gb[l] - nd.gb[q]);
            if (std::abs(da) <= D && std::abs(db) <= D) {
              const cd v = gcart[size_t(da + D) * (2 * D + 1) + (db + D)];
              if (v != 0.0) ents.emplace_back(l, v * nd.wfac[l]);
              continue;
            }
          }
          const double ome = 1.0 - eta(q, l);
          if (ome == 0.0) continue;
          ents.emplace_back(l, green(P.kappa, nd.x[q] - nd.x[l], nd.y[q] - nd.y[l]) * (nd.wfac[l] * ome));
        }
      }
    }
    // The regular entries are in increasing column order (neighbour cells in
    // increasing id, each cell's nodes contiguous): only the singular rules'
    // entries need sorting before the merge.
    const size_t nreg = ents.size();
    // singular rules
    if (needs_cart_rule(q)) {
      if (nd.chart[q] == 1) polar_cart_grid(std::llround(nd.ga[q]), std::llround(nd.gb[q]));
      else polar(1, q, nd.ga[q], nd.gb[q]);
    }
    if (nd.chart[q] == 0) boundary(q, nd.gi[q], nd.gj[q]);
    else if (nd.cb[q] <= g.n2 - 1) polar(0, q, nd.ca[q], nd.cb[q]);
    auto by_col = [](const std::pair<int64_t, cd>& a, const std::pair<int64_t, cd>& b) { return a.first < b.first; };
    std::sort(ents.begin() + nreg, ents.end(), by_col);
    std::inplace_merge(ents.begin(), ents.begin() + nreg, ents.end(), by_col);
    size_t w = 0;
    for (size_t r = 0; r < ents.size(); ++r) {
      if (w > 0 && ents[w - 1].first == ents[r].first) ents[w - 1].second += ents[r].second;
      else ents[w++] = ents[r];
    }
    ents.resize(w);
    return true;
  }
};

}  // namespace

bool check_cells(Plan2D& plan, int64_t* block_entries) {
  const Nodes& nd = plan.nodes;
  const int64_t N = nd.N;
  std::atomic<bool> ok(true);
  parallel_for(plan.n_threads, N, 1024, [&](int64_t q0, int64_t q1) {
    RowBuilder rb(plan);
    for (int64_t q = q0; q < q1 && ok; ++q) {
      const int c = nd.cell[q];
      if (!rb.eta_inside_block(q, c % nd.L, c / nd.L)) ok = false;
    }
  });
  if (!ok) {
    plan.err = "cut-off support leaves the 3 x 3 cell block N(x): enlarge H or shrink the radii";
    return false;
  }
  // entries of the padded per-cell near-field blocks (what one apply streams)
  const int L = nd.L;
  int64_t tot = 0;
  for (int c = 0; c < L * L; ++c) {
    const int64_t nc = nd.cell_start[c + 1] - nd.cell_start[c];
    if (!nc) continue;
    const int ci = c % L, cj = c / L;
    int64_t nblk = 0;
    for (int dj = -1; dj <= 1; ++dj) {
      const int nj = cj + dj;
      if (nj < 0 || nj >= L) continue;
      const int lo = nj * L + std::max(ci - 1, 0), hi = nj * L + std::min(ci + 1, L - 1);
      nblk += ((nd.cell_start[hi + 1] - nd.cell_start[lo]) + 1) & ~int64_t(1);
    }
    tot += nc * nblk;
  }
  *block_entries = tot;
  return true;
}

bool build_near(Plan2D& plan) {
  const int64_t N = plan.nodes.N;
  const int64_t chunk = 256;
  const int64_t nchunks = (N + chunk - 1) / chunk;
  std::vector<std::vector<int32_t>> ccol(nchunks);
  std::vector<std::vector<cd>> cval(nchunks);
  std::vector<std::vector<int64_t>> clen(nchunks);
  std::atomic<bool> ok(true);
  std::mutex mu;
  std::string err;
  parallel_for(plan.n_threads, nchunks, 1, [&](int64_t c0, int64_t c1) {
    RowBuilder rb(plan);
    for (int64_t ck = c0; ck < c1; ++ck) {
      for (int64_t q = ck * chunk; q < std::min(N, (ck + 1) * chunk); ++q) {
        if (!rb.row(q)) {
          ok = false;
          std::lock_guard<std::mutex> lk(mu);
          err = "cut-off support leaves the 3 x 3 cell block N(x): enlarge H or shrink the radii";
          return;
        }
        clen[ck].push_back(int64_t(rb.ents.size()));
        for (const auto& e : rb.ents) {
          ccol[ck].push_back(int32_t(e.first));
          cval[ck].push_back(e.second);
        }
      }
    }
  });
  if (!ok) { plan.err = err; return false; }
  plan.rowptr.assign(N + 1, 0);
  int64_t q = 0;
  for (int64_t ck = 0; ck < nchunks; ++ck)
    for (int64_t len : clen[ck]) { plan.rowptr[q + 1] = plan.rowptr[q] + len; ++q; }
  const int64_t nnz = plan.rowptr[N];
  plan.col.resize(nnz);
  plan.val.resize(nnz);
  std::vector<int64_t> pos(nchunks + 1, 0);
  for (int64_t ck = 0; ck < nchunks; ++ck) pos[ck + 1] = pos[ck] + int64_t(ccol[ck].size());
  parallel_for(plan.n_threads, nchunks, 16, [&](int64_t c0, int64_t c1) {
    for (int64_t ck = c0; ck < c1; ++ck) {
      std::copy(ccol[ck].begin(), ccol[ck].end(), plan.col.begin() + pos[ck]);
      std::copy(cval[ck].begin(), cval[ck].end(), plan.val.begin() + pos[ck]);
      std::vector<int32_t>().swap(ccol[ck]);
      std::vector<cd>().swap(cval[ck]);
    }
  });
  return true;
}

}  // namespace lsh
