// Charts, partition of unity and the Nystrom node set (Section 2).
//
// Boundary chart ("collar"): X(a, b) = gamma(s) - t w nu(s), s = 2 pi a / n1,
// t = b / (n2 - 1), nu the outward unit normal; t = 0 is the boundary.
// Interior chart: Cartesian grid.  Partition of unity omega_B(t) =
// S((t - tau0)/(tau1 - tau0)), omega_I = 1 - omega_B, with S(u) =
// f(1 - u) / (f(1 - u) + f(u)), f(u) = exp(-1/u) (a C-infinity step).
// Quadrature weights: collar = |det DX| (index units) x composite Q-point
// Newton-Cotes weight across; Cartesian = h^2.
#include <algorithm>
#include <cmath>
#include <exception>
#include <mutex>
#include <numeric>
#include <thread>

#include "host_plan.hpp"

namespace lsh {

static const double kPi = 3.14159265358979323846;

void Geometry::curve(double s, double* gm, double* g1, double* g2) const {
  const double c1 = std::cos(s), s1 = std::sin(s);
  if (g.shape == LS_DISC) {
    const double a = g.params[0], cx = g.params[1], cy = g.params[2];
    gm[0] = cx + a * c1; gm[1] = cy + a * s1;
    g1[0] = -a * s1;     g1[1] = a * c1;
    g2[0] = -a * c1;     g2[1] = -a * s1;
  } else if (g.shape == LS_FOURIER_STAR) {
    // r(s) = a0 + sum_k c_k cos(k s), gamma = c + r (cos s, sin s)
    double r = g.params[0], r1 = 0, r2 = 0;
    for (int k = 1; k <= 5; ++k) {
      const double ck = g.params[2 + k], ckc = std::cos(k * s), cks = std::sin(k * s);
      r += ck * ckc;
      r1 -= k * ck * cks;
      r2 -= double(k) * k * ck * ckc;
    }
    const double cx = g.params[1], cy = g.params[2];
    gm[0] = cx + r * c1;                 gm[1] = cy + r * s1;
    g1[0] = r1 * c1 - r * s1;            g1[1] = r1 * s1 + r * c1;
    g2[0] = r2 * c1 - 2 * r1 * s1 - r * c1;
    g2[1] = r2 * s1 + 2 * r1 * c1 - r * s1;
  } else {  // kite
    const double sc = g.params[0], cx = g.params[1], cy = g.params[2];
    const double c2 = std::cos(2 * s), s2 = std::sin(2 * s);
    gm[0] = cx + sc * (c1 + 0.65 * c2 - 0.65); gm[1] = cy + sc * 1.5 * s1;
    g1[0] = sc * (-s1 - 1.3 * s2);             g1[1] = sc * 1.5 * c1;
    g2[0] = sc * (-c1 - 2.6 * c2);             g2[1] = -sc * 1.5 * s1;
  }
}

// outward normal nu = (g1_y, -g1_x)/|g1| and its s-derivative
static void normal_and_derivative(const double* g1, const double* g2, double* nu, double* dnu) {
  const double sp = std::sqrt(g1[0] * g1[0] + g1[1] * g1[1]);
  const double dot = g1[0] * g2[0] + g1[1] * g2[1];
  nu[0] = g1[1] / sp;
  nu[1] = -g1[0] / sp;
  const double k = dot / (sp * sp * sp);
  dnu[0] = g2[1] / sp - g1[1] * k;
  dnu[1] = -g2[0] / sp + g1[0] * k;
}

void Geometry::collar_map(double a, double b, double* X, double* J) const {
  const double s = 2.0 * kPi * a / g.n1;
  const double t = b / (g.n2 - 1);
  double gm[2], g1[2], g2[2], nu[2], dnu[2];
  curve(s, gm, g1, g2);
  normal_and_derivative(g1, g2, nu, dnu);
  const double tw = t * g.collar_w;
  X[0] = gm[0] - tw * nu[0];
  X[1] = gm[1] - tw * nu[1];
  const double xs0 = g1[0] - tw * dnu[0], xs1 = g1[1] - tw * dnu[1];
  const double xt0 = -g.collar_w * nu[0], xt1 = -g.collar_w * nu[1];
  *J = std::fabs(xs0 * xt1 - xs1 * xt0) * (2.0 * kPi / g.n1) / (g.n2 - 1);
}

// ---------------------------------------------------------------- closest point
ClosestPoint::ClosestPoint(const Geometry& geo, double reach) : geo_(geo), reach_(reach) {
  ss_.resize(ns_); sx_.resize(ns_); sy_.resize(ns_);
  double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
  for (int k = 0; k < ns_; ++k) {
    double gm[2], g1[2], g2[2];
    ss_[k] = 2.0 * kPi * k / ns_;
    geo.curve(ss_[k], gm, g1, g2);
    sx_[k] = gm[0]; sy_[k] = gm[1];
    xmin = std::min(xmin, gm[0]); xmax = std::max(xmax, gm[0]);
    ymin = std::min(ymin, gm[1]); ymax = std::max(ymax, gm[1]);
  }
  x0_ = xmin - reach_; y0_ = ymin - reach_;
  nbx_ = int((xmax - xmin) / reach_) + 3;
  nby_ = int((ymax - ymin) / reach_) + 3;
  std::vector<int> cnt(nbx_ * nby_ + 1, 0);
  std::vector<int> bk(ns_);
  for (int k = 0; k < ns_; ++k) {
    int bx = int((sx_[k] - x0_) / reach_), by = int((sy_[k] - y0_) / reach_);
    bk[k] = by * nbx_ + bx;
    cnt[bk[k] + 1]++;
  }
  for (int i = 0; i < nbx_ * nby_; ++i) cnt[i + 1] += cnt[i];
  bstart_ = cnt;
  bidx_.resize(ns_);
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (int k = 0; k < ns_; ++k) bidx_[fill[bk[k]]++] = k;
}

void ClosestPoint::query(double x, double y, double* s_out, double* d_out, bool* found) const {
  int bx = int(std::floor((x - x0_) / reach_)), by = int(std::floor((y - y0_) / reach_));
  double best = 1e300;
  int kbest = -1;
  for (int j = by - 1; j <= by + 1; ++j) {
    if (j < 0 || j >= nby_) continue;
    for (int i = bx - 1; i <= bx + 1; ++i) {
      if (i < 0 || i >= nbx_) continue;
      const int b = j * nbx_ + i;
      for (int t = bstart_[b]; t < bstart_[b + 1]; ++t) {
        const int k = bidx_[t];
        const double dx = x - sx_[k], dy = y - sy_[k];
        const double d2 = dx * dx + dy * dy;
        if (d2 < best || (d2 == best && k < kbest)) { best = d2; kbest = k; }
      }
    }
  }
  if (kbest < 0 || best > reach_ * reach_) { *found = false; return; }
  *found = true;
  double s = ss_[kbest];
  double gm[2], g1[2], g2[2];
  for (int it = 0; it < 40; ++it) {
    geo_.curve(s, gm, g1, g2);
    const double dx = x - gm[0], dy = y - gm[1];
    const double f = dx * g1[0] + dy * g1[1];
    const double fp = -(g1[0] * g1[0] + g1[1] * g1[1]) + dx * g2[0] + dy * g2[1];
    const double ds = std::fabs(fp) > 1e-300 ? f / fp : 0.0;
    s -= ds;
    if (std::fabs(ds) < 1e-15) break;
  }
  s = std::fmod(s, 2.0 * kPi);
  if (s < 0) s += 2.0 * kPi;
  double nu[2], dnu[2];
  geo_.curve(s, gm, g1, g2);
  normal_and_derivative(g1, g2, nu, dnu);
  *s_out = s;
  *d_out = (gm[0] - x) * nu[0] + (gm[1] - y) * nu[1];
}

std::vector<double> ClosestPoint::crossings(double y) const {
  std::vector<double> xs;
  for (int k = 0; k < ns_; ++k) {
    const int k2 = (k + 1) % ns_;
    const double ya = sy_[k], yb = sy_[k2];
    if ((ya <= y && y < yb) || (yb <= y && y < ya)) {
      const double t = (y - ya) / (yb - ya);
      xs.push_back(sx_[k] + t * (sx_[k2] - sx_[k]));
    }
  }
  std::sort(xs.begin(), xs.end());
  return xs;
}

// ---------------------------------------------------------------- POU, rules
double smooth_step(double u) {
  if (u <= 0.0) return 1.0;
  if (u >= 1.0) return 0.0;
  const double f1 = std::exp(-1.0 / (1.0 - u));
  const double f0 = std::exp(-1.0 / u);
  return f1 / (f1 + f0);
}

double cutoff(double s, double s0) {
  s = std::fabs(s);
  if (s <= s0) return 1.0;
  if (s >= 1.0) return 0.0;
  const double u = (s - s0) / (1.0 - s0);
  return std::exp(2.0 * std::exp(-1.0 / u) / (u - 1.0));
}

std::vector<double> newton_cotes(int Q) {
  switch (Q) {
    case 2: return {0.5, 0.5};
    case 3: return {1.0 / 3, 4.0 / 3, 1.0 / 3};
    case 4: return {3.0 / 8, 9.0 / 8, 9.0 / 8, 3.0 / 8};
    case 5: return {14.0 / 45, 64.0 / 45, 24.0 / 45, 64.0 / 45, 14.0 / 45};
  }
  return {};
}

void parallel_for(int n_threads, int64_t n, int64_t chunk,
                  const std::function<void(int64_t, int64_t)>& fn) {
  if (n <= 0) return;
  if (n_threads <= 1 || n <= chunk) { fn(0, n); return; }
  // An exception in a worker (an allocation failure) stops the remaining
  // chunks and is rethrown here, in the calling thread.
  std::atomic<int64_t> next(0);
  std::exception_ptr first;
  std::mutex mu;
  std::vector<std::thread> th;
  for (int t = 0; t < n_threads; ++t)
    th.emplace_back([&]() {
      try {
        for (;;) {
          const int64_t s = next.fetch_add(chunk);
          if (s >= n) break;
          fn(s, std::min(n, s + chunk));
        }
      } catch (...) {
        next = n;
        std::lock_guard<std::mutex> lk(mu);
        if (!first) first = std::current_exception();
      }
    });
  for (auto& t : th) t.join();
  if (first) std::rethrow_exception(first);
}

// ---------------------------------------------------------------- node set
bool build_nodes(Plan2D& plan, ls_n2_fn n2fn, void* ctx) {
  const ls_geometry& g = plan.geo.g;
  const ls_options& o = plan.opt;
  Nodes& nd = plan.nodes;
  const int n1 = g.n1, n2 = g.n2;
  if ((n2 - 1) % (o.Q - 1)) { plan.err = "n2 - 1 must be a multiple of Q - 1"; return false; }
  if (n2 < o.p + 1) { plan.err = "collar needs at least p + 1 transverse lines"; return false; }
  if (!(g.tau0 > 0 && g.tau0 < g.tau1 && g.tau1 < 1)) { plan.err = "need 0 < tau0 < tau1 < 1"; return false; }
  // composite Newton-Cotes across the collar
  std::vector<double> ncw(n2, 0.0);
  const std::vector<double> nc = newton_cotes(o.Q);
  for (int blk = 0; blk < (n2 - 1) / (o.Q - 1); ++blk)
    for (int m = 0; m < o.Q; ++m) ncw[blk * (o.Q - 1) + m] += nc[m];

  // canonical collar nodes
  const int64_t nc_nodes = int64_t(n1) * n2;
  std::vector<double> cx(nc_nodes), cy(nc_nodes), cw(nc_nodes), com(nc_nodes);
  parallel_for(plan.n_threads, n1, 16, [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i)
      for (int j = 0; j < n2; ++j) {
        double X[2], J;
        plan.geo.collar_map(double(i), double(j), X, &J);
        const int64_t id = i * n2 + j;
        cx[id] = X[0]; cy[id] = X[1];
        cw[id] = J * ncw[j];
        com[id] = smooth_step((double(j) / (n2 - 1) - g.tau0) / (g.tau1 - g.tau0));
      }
  });
  // Cartesian candidates: keep omega_I > 0 (inside, t > tau0)
  ClosestPoint cp(plan.geo, 2.5 * g.collar_w);
  const int nx = g.cart_nx, ny = g.cart_ny;
  std::vector<double> tt(int64_t(nx) * ny, -1.0), sa(int64_t(nx) * ny, 0.0);
  std::vector<char> keep(int64_t(nx) * ny, 0);
  parallel_for(plan.n_threads, ny, 4, [&](int64_t j0, int64_t j1) {
    for (int64_t iy = j0; iy < j1; ++iy) {
      const double y = g.cart_y0 + iy * g.h;
      const std::vector<double> xs = cp.crossings(y);
      for (int ix = 0; ix < nx; ++ix) {
        const double x = g.cart_x0 + ix * g.h;
        double s, d;
        bool found;
        cp.query(x, y, &s, &d, &found);
        const int64_t id = int64_t(ix) * ny + iy;
        if (found) {
          const double t = d / g.collar_w;
          tt[id] = t; sa[id] = s;
          keep[id] = t > g.tau0;
        } else {
          const int left = int(std::lower_bound(xs.begin(), xs.end(), x) - xs.begin());
          if (left % 2 == 1) { tt[id] = 1e30; keep[id] = 1; }
        }
      }
    }
  });
  std::vector<int64_t> cart_ids;
  for (int64_t id = 0; id < int64_t(nx) * ny; ++id)
    if (keep[id]) cart_ids.push_back(id);
  nd.n_collar = nc_nodes;
  nd.n_cart = int64_t(cart_ids.size());
  nd.N = nd.n_collar + nd.n_cart;
  const int64_t N = nd.N;

  // canonical arrays
  std::vector<double> X(N), Y(N), W(N), OM(N), CA(N), CB(N), GA(N), GB(N);
  std::vector<int8_t> CH(N);
  std::vector<int32_t> GI(N), GJ(N);
  for (int64_t id = 0; id < nc_nodes; ++id) {
    X[id] = cx[id]; Y[id] = cy[id]; W[id] = cw[id]; OM[id] = com[id];
    CH[id] = 0; GI[id] = int32_t(id / n2); GJ[id] = int32_t(id % n2);
    CA[id] = GI[id]; CB[id] = GJ[id];
    GA[id] = (X[id] - g.cart_x0) / g.h; GB[id] = (Y[id] - g.cart_y0) / g.h;
  }
  for (int64_t r = 0; r < nd.n_cart; ++r) {
    const int64_t gid = cart_ids[r], id = nc_nodes + r;
    const int ix = int(gid / ny), iy = int(gid % ny);
    X[id] = g.cart_x0 + ix * g.h; Y[id] = g.cart_y0 + iy * g.h;
    W[id] = g.h * g.h;
    OM[id] = 1.0 - smooth_step((tt[gid] - g.tau0) / (g.tau1 - g.tau0));
    CH[id] = 1; GI[id] = ix; GJ[id] = iy;
    CA[id] = sa[gid] * n1 / (2.0 * kPi);
    CB[id] = tt[gid] * (n2 - 1);
    GA[id] = ix; GB[id] = iy;
  }
  // refractive index at the nodes (host callback, canonical order)
  std::vector<double> xy(2 * N), N2(N);
  for (int64_t i = 0; i < N; ++i) { xy[2 * i] = X[i]; xy[2 * i + 1] = Y[i]; }
  if (!n2fn) { plan.err = "n2 callback is NULL"; return false; }
  if (n2fn(N, xy.data(), N2.data(), ctx) != 0) { plan.err = "n2 callback failed"; return false; }

  // cells of the accelerator; plan order = stable sort by cell.  With L <= 0
  // the box is chosen here: it covers every node, its faces lie half a
  // Cartesian spacing off the grid lines (H should be a multiple of h), and
  // L = number of cells per side.
  if (plan.opt.L <= 0) {
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int64_t i = 0; i < N; ++i) {
      xmin = std::min(xmin, X[i]); xmax = std::max(xmax, X[i]);
      ymin = std::min(ymin, Y[i]); ymax = std::max(ymax, Y[i]);
    }
    const double H0 = plan.opt.H;
    plan.opt.box_x0 = g.cart_x0 + (std::floor((xmin - g.cart_x0) / g.h) - 0.5) * g.h;
    plan.opt.box_y0 = g.cart_y0 + (std::floor((ymin - g.cart_y0) / g.h) - 0.5) * g.h;
    const int Lx = int(std::floor((xmax - plan.opt.box_x0) / H0)) + 1;
    const int Ly = int(std::floor((ymax - plan.opt.box_y0) / H0)) + 1;
    plan.opt.L = std::max(Lx, Ly);
  }
  const int L = plan.opt.L;
  const double H = o.H;
  nd.L = L;
  std::vector<int32_t> cellc(N);
  for (int64_t i = 0; i < N; ++i) {
    const double fx = std::floor((X[i] - plan.opt.box_x0) / H), fy = std::floor((Y[i] - plan.opt.box_y0) / H);
    if (fx < 0 || fy < 0 || fx >= L || fy >= L) { plan.err = "nodes outside the cell box"; return false; }
    cellc[i] = int32_t(fy) * L + int32_t(fx);
  }
  std::vector<int64_t> order(N);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return cellc[a] < cellc[b]; });
  auto take = [&](auto& dst, const auto& src) {
    dst.resize(N);
    for (int64_t k = 0; k < N; ++k) dst[k] = src[order[k]];
  };
  take(nd.x, X); take(nd.y, Y); take(nd.w, W); take(nd.omega, OM); take(nd.n2, N2);
  take(nd.ca, CA); take(nd.cb, CB); take(nd.ga, GA); take(nd.gb, GB);
  take(nd.chart, CH); take(nd.gi, GI); take(nd.gj, GJ); take(nd.cell, cellc);
  nd.canon = order;
  nd.phifac.resize(N); nd.wfac.resize(N);
  for (int64_t k = 0; k < N; ++k) {
    nd.phifac[k] = nd.omega[k] * (1.0 - nd.n2[k]);
    nd.wfac[k] = nd.w[k] * nd.phifac[k];
  }
  nd.collar_pos.assign(nc_nodes, -1);
  nd.cart_pos.assign(int64_t(nx) * ny, -1);
  for (int64_t k = 0; k < N; ++k) {
    const int64_t c = order[k];
    if (c < nc_nodes) nd.collar_pos[c] = k;
    else nd.cart_pos[cart_ids[c - nc_nodes]] = k;
  }
  nd.cell_start.assign(int64_t(L) * L + 1, 0);
  for (int64_t k = 0; k < N; ++k) nd.cell_start[nd.cell[k] + 1]++;
  for (int64_t c = 0; c < int64_t(L) * L; ++c) nd.cell_start[c + 1] += nd.cell_start[c];
  plan.ffw.resize(N);
  for (int64_t k = 0; k < N; ++k) plan.ffw[k] = nd.w[k] * nd.omega[k] * (nd.n2[k] - 1.0);
  return true;
}

}  // namespace lsh
