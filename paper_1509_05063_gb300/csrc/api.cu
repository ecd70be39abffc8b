// C ABI of the library (include/ls.h): plan creation and upload, apply,
// GMRES solve (FP64 and mixed complex64 + FP64 refinement) and far field.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <climits>
#include <cstdint>
#include <map>
#include <new>
#include <mutex>
#include <set>
#include <tuple>
#include <string>
#include <thread>
#include <queue>
#include <vector>

#include "device/kernels.cuh"
#include "host/host_plan.hpp"
#include "ls.h"

namespace {

thread_local std::string g_create_error;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

// Owner of device allocations and of the last error message (plans, batches).
struct DevOwner {
  std::vector<DevBuf> bufs;
  int64_t device_bytes = 0;
  std::string err;

  template <typename T>
  T* alloc(size_t n, ls_status* st) {
    void* p = nullptr;
    if (n == 0) n = 1;
    if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      *st = LS_ERR_NOMEM;
      err = "cudaMalloc of " + std::to_string(n * sizeof(T)) + " bytes failed";
      return nullptr;
    }
    bufs.push_back({p, n * sizeof(T)});
    device_bytes += int64_t(n * sizeof(T));
    return static_cast<T*>(p);
  }
  template <typename T, typename S>
  T* upload(const std::vector<S>& v, ls_status* st) {
    static_assert(sizeof(T) == sizeof(S), "layout");
    T* d = alloc<T>(v.size(), st);
    if (!d) return nullptr;
    if (!v.empty() && cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
      *st = LS_ERR_CUDA;
      err = "cudaMemcpy upload failed";
      return nullptr;
    }
    return d;
  }
  // free one buffer obtained from alloc / upload (nullptr: nothing)
  void release(const void* p) {
    if (!p) return;
    for (size_t i = 0; i < bufs.size(); ++i)
      if (bufs[i].p == p) {
        cudaFree(bufs[i].p);
        device_bytes -= int64_t(bufs[i].bytes);
        bufs.erase(bufs.begin() + i);
        return;
      }
  }
  void free_bufs() {
    for (auto& b : bufs) cudaFree(b.p);
    bufs.clear();
  }
};

// Work space of lock-step GMRES and of the mixed refinement, for R right-hand
// sides whose vectors occupy `total` elements together (grown on demand).
struct Krylov {
  int restart = -1, R = 0;
  int64_t total = 0, max_len = 0;
  double2 *V = nullptr, *w = nullptr, *r = nullptr, *e = nullptr, *cor = nullptr, *h = nullptr, *partial = nullptr;
  double2* apart = nullptr;     // kAxpyGroups x max_len partial sums of the Arnoldi update
  double* vs = nullptr;         // FP64 solve: Re + Im of every basis entry (same layout as V)
  double* h3 = nullptr;         // FP64 solve: coefficient triplets of the update, R x (restart + 3) x 3
  double* dnorm = nullptr;
  double* dpartial = nullptr;
  float2 *c64a = nullptr, *c64b = nullptr;
  double2* pin_h = nullptr;     // pinned host copies of h and the norms (async D2H)
  double* pin_n = nullptr;
  // pipelined GMRES: Gram-Schmidt coefficients (two passes) and norms of every
  // iteration of a cycle, on the device and mirrored in pinned memory
  double2* hk = nullptr;        // [iteration][pass][RHS][restart + 3]
  double* nk = nullptr;         // [iteration][RHS]
  double2* pin_hk = nullptr;
  double* pin_nk = nullptr;
  static constexpr int kEvents = 4;
  cudaEvent_t ev[kEvents] = {};
  void free_pinned() {
    if (pin_h) cudaFreeHost(pin_h);
    if (pin_n) cudaFreeHost(pin_n);
    if (pin_hk) cudaFreeHost(pin_hk);
    if (pin_nk) cudaFreeHost(pin_nk);
    pin_h = nullptr;
    pin_n = nullptr;
    pin_hk = nullptr;
    pin_nk = nullptr;
    for (auto& e : ev)
      if (e) { cudaEventDestroy(e); e = nullptr; }
  }
};

// CUDA graphs of a launch sequence keyed by (precision, batch, input, output):
// the first call with a key launches directly, the second captures the
// sequence on a private stream and launches the graph, later calls replay it.
struct GraphCache {
  using Key = std::tuple<int, int, const void*, void*>;
  std::map<Key, cudaGraphExec_t> graphs;
  std::set<Key> seen;
  cudaStream_t cap_stream = nullptr;
  bool off = false;

  template <typename F>
  cudaError_t run(const Key& key, F launch, cudaStream_t st) {
    if (off) return launch(st);
    auto it = graphs.find(key);
    if (it != graphs.end()) return cudaGraphLaunch(it->second, st);
    if (!seen.count(key)) {
      if (seen.size() > 4096) seen.clear();
      seen.insert(key);
      return launch(st);
    }
    if (!cap_stream && cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      off = true;
      return launch(st);
    }
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t e1 = launch(cap_stream);
      e = cudaStreamEndCapture(cap_stream, &g);
      if (e1 != cudaSuccess) e = e1;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      cudaGetLastError();
      off = true;
      return launch(st);
    }
    if (graphs.size() >= 512) clear();
    graphs[key] = ex;
    return cudaGraphLaunch(ex, st);
  }
  void clear() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
  }
  void release() {
    clear();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
  }
};

struct ls_plan_s : DevOwner {
  lsh::Plan2D host;                 // kept for node queries (large arrays are released)
  lsd::ApplyData<double2> d64;
  lsd::ApplyData<float2> d32;
  // plan-wide device arrays
  double *x = nullptr, *y = nullptr, *ffw = nullptr;
  Krylov K;                         // solve work space (lazily sized)
  double2 *seed_h = nullptr, *seed_part = nullptr;   // initial guesses from earlier right-hand sides
  int seed_cap = 0;
  double* dirs = nullptr;
  int dirs_cap = 0;
  ls_plan_info_t info{};
  int device = -1;                  // ordinal of the GPU that holds the plan's arrays
  int dim = 2;                      // 3: a ball (ls_plan_create3); d64 / d32 then hold N only
  lsd::ApplyData3<double2> e64;     // 3-D apply data
  lsd::ApplyData3<float2> e32;
  std::vector<double> xyz3;         // 3-D: node coordinates in plan order
  std::vector<int64_t> canon3;      // 3-D: ball node id of each plan node
  double* ffw3 = nullptr;           // 3-D: w omega (n^2 - 1) per node (far field)
  GraphCache graphs;                // CUDA graphs of the apply
  int group32 = lsd::kMaxRhs32;     // complex64 right-hand sides per apply launch (ls_plan_autotune)
  // optional per-stage event timing of ls_apply
  bool timing = false;
  cudaEvent_t ev[lsd::kStages + 1] = {};
  double stage_ms[2][lsd::kStages] = {};
  int64_t stage_calls[2] = {0, 0};

  void free_all() {
    K.free_pinned();
    graphs.release();
    free_bufs();
  }
};

namespace {

using cd = std::complex<double>;

ls_status fail(DevOwner* p, ls_status s, const std::string& m) {
  if (p) p->err = m;
  else g_create_error = m;
  return s;
}

#define LS_CU(call)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(plan, LS_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
  } while (0)

// Apply through a cached CUDA graph of the whole kernel sequence (direct
// launches when timing, on the first call of a key, or if capture fails).
template <typename T> const lsd::ApplyData3<T>& data3(ls_plan p);
template <> const lsd::ApplyData3<double2>& data3<double2>(ls_plan p) { return p->e64; }
template <> const lsd::ApplyData3<float2>& data3<float2>(ls_plan p) { return p->e32; }

template <typename T>
cudaError_t run_apply(ls_plan plan, int prec, const lsd::ApplyData<T>& d, const T* u, T* out, int nr,
                      cudaStream_t st) {
  auto launch = [&](cudaStream_t s) {
    return plan->dim == 3 ? lsd::apply3_batch(data3<T>(plan), u, out, nr, s) : lsd::apply_batch(d, u, out, nr, s);
  };
  if (plan->timing) return launch(st);
  return plan->graphs.run(GraphCache::Key(prec, nr, static_cast<const void*>(u), static_cast<void*>(out)), launch,
                          st);
}

std::vector<std::complex<float>> to32(const std::vector<cd>& v) {
  std::vector<std::complex<float>> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = std::complex<float>(float(v[i].real()), float(v[i].imag()));
  return o;
}

ls_status validate(const ls_geometry* g, const ls_options* o, double kappa) {
  if (!g || !o) return LS_ERR_INVALID;
  if (g->dim != 2) return LS_ERR_UNSUPPORTED;
  if (g->shape != LS_DISC && g->shape != LS_KITE && g->shape != LS_FOURIER_STAR) return LS_ERR_INVALID;
  if (g->shape == LS_FOURIER_STAR) {
    // star-shaped: r(s) > 0 on a fine sample
    for (int i = 0; i < 4096; ++i) {
      const double s = 2.0 * M_PI * i / 4096;
      double r = g->params[0];
      for (int k = 1; k <= 5; ++k) r += g->params[2 + k] * std::cos(k * s);
      if (!(r > 0)) return LS_ERR_INVALID;
    }
  }
  if (g->n1 < 8 || g->n2 < 2 || g->collar_w <= 0 || g->h <= 0 || g->cart_nx < 1 || g->cart_ny < 1)
    return LS_ERR_INVALID;
  if (!(kappa > 0)) return LS_ERR_INVALID;
  if (o->Q < 2 || o->Q > 5 || o->p < 1 || o->p > 15 || o->R_a <= 0 || o->R_b <= 0 || o->R_cart <= 0)
    return LS_ERR_INVALID;
  if (o->M < 0 || o->N_tau < 4 || o->q_polar < 1 || o->n_rho < 2 || o->n_theta < 4) return LS_ERR_INVALID;
  if (o->N_eq < 2 || o->H <= 0 || o->n_fb < 0) return LS_ERR_INVALID;   // L <= 0: box chosen by the plan
  if (!(o->chi_s0 >= 0 && o->chi_s0 < 1)) return LS_ERR_INVALID;
  return LS_OK;
}

double secs_since(std::chrono::steady_clock::time_point t) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t).count();
}

// host plan construction; stage (may be NULL) receives the seconds of the
// nodes, near-field weights and accelerator steps
ls_status build_host(lsh::Plan2D& P, const ls_geometry* geom, ls_n2_fn n2, void* ctx, double kappa,
                     const ls_options* opt, std::string* msg, double* stage = nullptr) {
  P.geo.g = *geom;
  P.opt = *opt;
  P.kappa = kappa;
  P.n_threads = opt->n_threads > 0 ? opt->n_threads : int(std::max(1u, std::thread::hardware_concurrency()));
  try {
    auto t = std::chrono::steady_clock::now();
    bool ok = lsh::build_nodes(P, n2, ctx);
    if (stage) stage[0] = secs_since(t);
    t = std::chrono::steady_clock::now();
    ok = ok && lsh::build_near(P);
    if (stage) stage[1] = secs_since(t);
    t = std::chrono::steady_clock::now();
    ok = ok && lsh::build_accel(P);
    if (stage) stage[2] = secs_since(t);
    if (!ok) {
      *msg = P.err;
      return LS_ERR_INVALID;
    }
  } catch (const std::bad_alloc&) {
    *msg = "host allocation failed during plan construction";
    return LS_ERR_NOMEM;
  }
  return LS_OK;
}

}  // namespace

struct ls_host_plan_s {
  lsh::Plan2D P;
};

extern "C" {

ls_status ls_host_plan_create(const ls_geometry* geom, ls_n2_fn n2, void* ctx, double kappa, const ls_options* opt,
                              ls_host_plan* out) {
  if (!out) return fail(nullptr, LS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  const ls_status v = validate(geom, opt, kappa);
  if (v != LS_OK) return fail(nullptr, v, "invalid geometry or options");
  ls_host_plan h = new (std::nothrow) ls_host_plan_s;
  if (!h) return fail(nullptr, LS_ERR_NOMEM, "host allocation failed");
  std::string m;
  const ls_status s = build_host(h->P, geom, n2, ctx, kappa, opt, &m);
  if (s != LS_OK) {
    delete h;
    return fail(nullptr, s, m);
  }
  *out = h;
  return LS_OK;
}

ls_status ls_check_cells(const ls_geometry* geom, ls_n2_fn n2, void* ctx, double kappa, const ls_options* opt,
                         double* out) {
  if (!out) return fail(nullptr, LS_ERR_INVALID, "out is NULL");
  const ls_status v = validate(geom, opt, kappa);
  if (v != LS_OK) return fail(nullptr, v, "invalid geometry or options");
  lsh::Plan2D P;
  P.geo.g = *geom;
  P.opt = *opt;
  P.kappa = kappa;
  P.n_threads = opt->n_threads > 0 ? opt->n_threads : int(std::max(1u, std::thread::hardware_concurrency()));
  int64_t entries = 0;
  try {
    if (!lsh::build_nodes(P, n2, ctx)) return fail(nullptr, LS_ERR_INVALID, P.err);
    const int nlat = P.opt.L * P.opt.N_eq + 1;
    int M = 256;
    while (M < 2 * nlat - 1) M *= 2;
    if (M > 2048) return fail(nullptr, LS_ERR_INVALID, "lattice too large: need 2 (L N_eq + 1) - 1 <= 2048");
    if (kappa * P.opt.H / std::sqrt(2.0) >= 2.4) return fail(nullptr, LS_ERR_INVALID, "kappa H / sqrt 2 must stay below 2.4");
    if (!lsh::check_cells(P, &entries)) return fail(nullptr, LS_ERR_INVALID, P.err);
    int nocc = 0;
    for (int c = 0; c < P.opt.L * P.opt.L; ++c) nocc += P.nodes.cell_start[c + 1] > P.nodes.cell_start[c];
    out[0] = double(P.nodes.N);
    out[1] = nocc;
    out[2] = double(entries);
    out[3] = M;
    out[4] = P.opt.L;
    out[5] = P.opt.box_x0;
    out[6] = P.opt.box_y0;
  } catch (const std::bad_alloc&) {
    return fail(nullptr, LS_ERR_NOMEM, "host allocation failed");
  }
  return LS_OK;
}

ls_status ls_host_plan_sizes(ls_host_plan h, int64_t* sizes) {
  if (!h || !sizes) return LS_ERR_INVALID;
  const lsh::Plan2D& P = h->P;
  sizes[0] = P.nodes.N;
  sizes[1] = P.rowptr.empty() ? 0 : P.rowptr.back();
  sizes[2] = int64_t(P.occ_cells.size());
  sizes[3] = P.n_es;
  sizes[4] = P.nfb2;
  sizes[5] = P.n_loc;
  sizes[6] = P.M;
  sizes[7] = int64_t(P.P64.size());
  return LS_OK;
}

ls_status ls_host_plan_nodes(ls_host_plan h, double* xy, int64_t* canon, double* wfac) {
  if (!h) return LS_ERR_INVALID;
  const lsh::Nodes& nd = h->P.nodes;
  for (int64_t i = 0; i < nd.N; ++i) {
    if (xy) { xy[2 * i] = nd.x[i]; xy[2 * i + 1] = nd.y[i]; }
    if (canon) canon[i] = nd.canon[i];
    if (wfac) wfac[i] = nd.wfac[i];
  }
  return LS_OK;
}

ls_status ls_host_plan_near(ls_host_plan h, int64_t* rowptr, int32_t* col, double* val) {
  if (!h || !rowptr || !col || !val) return LS_ERR_INVALID;
  const lsh::Plan2D& P = h->P;
  std::copy(P.rowptr.begin(), P.rowptr.end(), rowptr);
  std::copy(P.col.begin(), P.col.end(), col);
  std::memcpy(val, P.val.data(), P.val.size() * sizeof(cd));
  return LS_OK;
}

ls_status ls_host_plan_accel(ls_host_plan h, int32_t* occ_cells, int64_t* P_off, double* Pm, double* Bpinv,
                             double* BT, double* Phi, double* Gtab, double* Dtab) {
  if (!h) return LS_ERR_INVALID;
  const lsh::Plan2D& P = h->P;
  if (occ_cells) std::copy(P.occ_cells.begin(), P.occ_cells.end(), occ_cells);
  if (P_off) std::copy(P.P_off.begin(), P.P_off.end(), P_off);
  if (Pm) std::memcpy(Pm, P.P64.data(), P.P64.size() * sizeof(cd));
  if (Bpinv) std::memcpy(Bpinv, P.Bpinv.data(), P.Bpinv.size() * sizeof(cd));
  if (BT) std::memcpy(BT, P.BT.data(), P.BT.size() * sizeof(cd));
  if (Phi) std::memcpy(Phi, P.Phi.data(), P.Phi.size() * sizeof(cd));
  if (Gtab) std::memcpy(Gtab, P.Gtab.data(), P.Gtab.size() * sizeof(cd));
  if (Dtab) std::memcpy(Dtab, P.Dtab.data(), P.Dtab.size() * sizeof(cd));
  return LS_OK;
}

ls_status ls_host_plan_destroy(ls_host_plan h) {
  delete h;
  return LS_OK;
}

}  // extern "C"

struct ls_host_accel3_s {
  lsh::Accel3 A;
};

extern "C" {

ls_status ls_host_accel3_create(const double* xyz, const double* wfac, int64_t N, double kappa, const double* box0,
                                double H, int L, int N_eq, int p, int m_coll, double rcond, int n_threads,
                                ls_host_accel3* out) {
  if (!out) return fail(nullptr, LS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!xyz || !wfac || !box0 || N <= 0) return fail(nullptr, LS_ERR_INVALID, "empty node set or NULL array");
  if (!(kappa > 0) || !(H > 0) || L < 1 || N_eq < 1 || p < 0 || m_coll < 0 || rcond < 0)
    return fail(nullptr, LS_ERR_INVALID, "invalid kappa, H, L, N_eq, p, m_coll or rcond");
  ls_host_accel3 h = new (std::nothrow) ls_host_accel3_s;
  if (!h) return fail(nullptr, LS_ERR_NOMEM, "host allocation failed");
  lsh::Accel3& A = h->A;
  A.kappa = kappa;
  A.H = H;
  A.L = L;
  A.Ne = N_eq;
  A.p = p;
  A.m_coll = m_coll;
  A.rcond = rcond;
  for (int k = 0; k < 3; ++k) A.box0[k] = box0[k];
  A.n_threads = n_threads > 0 ? n_threads : int(std::max(1u, std::thread::hardware_concurrency()));
  try {
    if (!lsh::build_accel3(A, xyz, wfac, N)) {
      const std::string m = A.err;
      delete h;
      return fail(nullptr, LS_ERR_INVALID, m);
    }
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(nullptr, LS_ERR_NOMEM, "host allocation failed");
  }
  *out = h;
  return LS_OK;
}

ls_status ls_host_accel3_sizes(ls_host_accel3 h, int64_t* sizes) {
  if (!h || !sizes) return LS_ERR_INVALID;
  const lsh::Accel3& A = h->A;
  sizes[0] = int64_t(A.occ_cells.size());
  sizes[1] = A.n_es;
  sizes[2] = A.nb;
  sizes[3] = A.n_loc;
  sizes[4] = A.M;
  sizes[5] = A.P_off.empty() ? 0 : A.P_off.back();
  sizes[6] = int64_t(A.node_order.size());
  return LS_OK;
}

ls_status ls_host_accel3_get(ls_host_accel3 h, int32_t* occ_cells, int64_t* P_off, int64_t* node_order, double* P,
                             double* Bpinv, double* BT, double* Phi, double* Gtab, double* Dtab) {
  if (!h) return LS_ERR_INVALID;
  const lsh::Accel3& A = h->A;
  auto put = [](const auto& v, auto* dst) {
    if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  put(A.occ_cells, occ_cells);
  put(A.P_off, P_off);
  put(A.node_order, node_order);
  put(A.P, P);
  put(A.Bpinv, Bpinv);
  put(A.BT, BT);
  put(A.Phi, Phi);
  put(A.Gtab, Gtab);
  put(A.Dtab, Dtab);
  return LS_OK;
}

ls_status ls_host_accel3_destroy(ls_host_accel3 h) {
  delete h;
  return LS_OK;
}

}  // extern "C"

struct ls_host_ball3_s {
  lsh::Ball3 B;
};

extern "C" {

ls_status ls_host_ball3_create(const ls_ball3* ball, ls_host_ball3* out) {
  if (!out) return fail(nullptr, LS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!ball) return fail(nullptr, LS_ERR_INVALID, "ball is NULL");
  ls_host_ball3 h = new (std::nothrow) ls_host_ball3_s;
  if (!h) return fail(nullptr, LS_ERR_NOMEM, "host allocation failed");
  lsh::Ball3& B = h->B;
  B.a = ball->a;
  B.w = ball->w;
  B.n_f = ball->n_f;
  B.n_s = ball->n_s;
  B.Q = ball->Q;
  B.delta = ball->delta;
  B.h = ball->h;
  B.tau0 = ball->tau0;
  B.tau1 = ball->tau1;
  try {
    if (!lsh::build_ball3(B)) {
      const std::string m = B.err;
      delete h;
      return fail(nullptr, LS_ERR_INVALID, m);
    }
  } catch (const std::bad_alloc&) {
    delete h;
    return fail(nullptr, LS_ERR_NOMEM, "host allocation failed");
  }
  *out = h;
  return LS_OK;
}

ls_status ls_host_ball3_sizes(ls_host_ball3 h, int64_t* sizes) {
  if (!h || !sizes) return LS_ERR_INVALID;
  sizes[0] = h->B.N;
  sizes[1] = h->B.n_shell;
  sizes[2] = h->B.n_cart;
  sizes[3] = h->B.grid_m;
  return LS_OK;
}

ls_status ls_host_ball3_nodes(ls_host_ball3 h, double* xyz, double* w, double* omega, double* psi, int8_t* face,
                              int32_t* grid) {
  if (!h) return LS_ERR_INVALID;
  const lsh::Ball3& B = h->B;
  auto put = [](const auto& v, auto* dst) {
    if (dst) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  put(B.x, xyz);
  put(B.w_q, w);
  put(B.omega, omega);
  put(B.psi, psi);
  put(B.face, face);
  put(B.grid, grid);
  return LS_OK;
}


static lsh::Rules3 rules_from(const ls_rules3* r) {
  lsh::Rules3 ru;
  if (r) {
    ru.R = r->R;
    ru.p = r->p;
    ru.q = r->q;
    ru.n_rho = r->n_rho;
    ru.n_mu = r->n_mu;
    ru.n_phi = r->n_phi;
    ru.rc = r->rc;
    ru.rs = r->rs;
    ru.n_sig = r->n_sig;
    ru.n_th = r->n_th;
    ru.chi_s0 = r->chi_s0;
  }
  return ru;
}

ls_status ls_host_ball3_row(ls_host_ball3 h, double kappa, const ls_rules3* rules, int64_t q, double* row,
                            double* eta) {
  if (!h || !row) return fail(nullptr, LS_ERR_INVALID, "NULL handle or row");
  if (!(kappa >= 0)) return fail(nullptr, LS_ERR_INVALID, "kappa must be >= 0");
  std::string m;
  try {
    if (!lsh::ball3_row(h->B, kappa, rules_from(rules), q, reinterpret_cast<lsh::cd*>(row), eta, &m))
      return fail(nullptr, LS_ERR_INVALID, m);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, LS_ERR_NOMEM, "host allocation failed");
  }
  return LS_OK;
}

ls_status ls_host_ball3_near(ls_host_ball3 h, double kappa, const ls_rules3* rules, const double* box0, double H,
                             int L, const int64_t* rows, int64_t n_rows, int stencils_only, int n_threads,
                             int64_t* nnz) {
  if (!h || !box0 || !nnz) return fail(nullptr, LS_ERR_INVALID, "NULL handle, box0 or nnz");
  if (!(kappa >= 0) || (rows && n_rows < 0)) return fail(nullptr, LS_ERR_INVALID, "invalid kappa or row count");
  const int nt = n_threads > 0 ? n_threads : int(std::max(1u, std::thread::hardware_concurrency()));
  std::string m;
  try {
    if (!lsh::ball3_near(h->B, kappa, rules_from(rules), box0, H, L, rows, n_rows, stencils_only != 0, nt, &m))
      return fail(nullptr, LS_ERR_INVALID, m);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, LS_ERR_NOMEM, "host allocation failed");
  }
  *nnz = h->B.near_rowptr.back();
  return LS_OK;
}

ls_status ls_host_ball3_near_get(ls_host_ball3 h, int64_t* rowptr, int32_t* col, double* val) {
  if (!h || h->B.near_rowptr.empty()) return fail(nullptr, LS_ERR_INVALID, "no near field built");
  const lsh::Ball3& B = h->B;
  if (rowptr) std::memcpy(rowptr, B.near_rowptr.data(), B.near_rowptr.size() * sizeof(int64_t));
  if (col) std::memcpy(col, B.near_col.data(), B.near_col.size() * sizeof(int32_t));
  if (val) std::memcpy(val, B.near_val.data(), B.near_val.size() * sizeof(lsh::cd));
  return LS_OK;
}

ls_status ls_host_ball3_destroy(ls_host_ball3 h) {
  delete h;
  return LS_OK;
}

ls_status ls_interior_window3(double kappa, double h, double R, int p, int q, int n_rho, int n_mu, int n_phi,
                              double chi_s0, double* win, int* Wn) {
  if (!Wn) return fail(nullptr, LS_ERR_INVALID, "Wn is NULL");
  std::vector<lsh::cd> w;
  std::string m;
  try {
    if (!lsh::interior_window3(kappa, h, R, p, q, n_rho, n_mu, n_phi, chi_s0, w, Wn, &m))
      return fail(nullptr, LS_ERR_INVALID, m);
  } catch (const std::bad_alloc&) {
    return fail(nullptr, LS_ERR_NOMEM, "host allocation failed");
  }
  if (win) std::memcpy(win, w.data(), w.size() * sizeof(w[0]));
  return LS_OK;
}

const char* ls_status_string(ls_status s) {
  switch (s) {
    case LS_OK: return "ok";
    case LS_ERR_INVALID: return "invalid argument";
    case LS_ERR_NOMEM: return "out of memory";
    case LS_ERR_CUDA: return "CUDA error";
    case LS_ERR_NOCONV: return "no convergence";
    case LS_ERR_TIMEOUT: return "device wait timed out";
    case LS_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* ls_last_error(ls_plan plan) { return plan ? plan->err.c_str() : g_create_error.c_str(); }

ls_status ls_plan_create(const ls_geometry* geom, ls_n2_fn n2, void* ctx, double kappa, const ls_options* opt,
                         ls_plan* out) {
  if (!out) return fail(nullptr, LS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  const ls_status v = validate(geom, opt, kappa);
  if (v != LS_OK) return fail(nullptr, v, "invalid geometry or options");
  const auto t0 = std::chrono::steady_clock::now();
  ls_plan plan = new (std::nothrow) ls_plan_s;
  if (!plan) return fail(nullptr, LS_ERR_NOMEM, "host allocation failed");
  if (cudaGetDevice(&plan->device) != cudaSuccess) {
    cudaGetLastError();
    delete plan;
    return fail(nullptr, LS_ERR_CUDA, "cudaGetDevice failed");
  }
  lsh::Plan2D& P = plan->host;
  auto bail = [&](ls_status s, const std::string& m) {
    g_create_error = m;
    plan->free_all();
    delete plan;
    return s;
  };
  double stage[4] = {0, 0, 0, 0};
  {
    std::string m;
    const ls_status hs = build_host(P, geom, n2, ctx, kappa, opt, &m, stage);
    if (hs != LS_OK) return bail(hs, m);
  }
  const auto t_dev = std::chrono::steady_clock::now();
  const lsh::Nodes& nd = P.nodes;
  const int64_t N = nd.N;
  const int nocc = int(P.occ_cells.size());
  ls_status st = LS_OK;
#define UP(T, v) plan->upload<T>(v, &st); if (st != LS_OK) return bail(st, plan->err)
  // shared integer structure
  std::vector<int64_t> occ_start(nocc + 1);
  std::vector<int> occ_of_cell(size_t(P.opt.L) * P.opt.L, -1), occ_of_node(N);
  for (int k = 0; k < nocc; ++k) {
    occ_start[k] = nd.cell_start[P.occ_cells[k]];
    occ_of_cell[P.occ_cells[k]] = k;
  }
  occ_start[nocc] = N;
  for (int64_t q = 0; q < N; ++q) occ_of_node[q] = occ_of_cell[nd.cell[q]];
  // near field: CSR -> one dense block per occupied cell + CSR remainder.
  // Each of the three column ranges of a row is stored padded to an even
  // length (zeros), so every range starts 16-byte aligned in complex64.
  const int Lc = P.opt.L;
  std::vector<int64_t> blk_off(nocc + 1, 0);
  std::vector<int> blk_seg(size_t(6) * nocc, 0);
  auto padded = [](int len) { return (len + 1) & ~1; };
  int max_nblk = 0;
  for (int k = 0; k < nocc; ++k) {
    const int c = P.occ_cells[k], ci = c % Lc, cj = c / Lc;
    int nblk = 0;
    for (int s = 0; s < 3; ++s) {
      const int nj = cj + s - 1;
      if (nj < 0 || nj >= Lc) continue;
      const int lo = nj * Lc + std::max(ci - 1, 0), hi = nj * Lc + std::min(ci + 1, Lc - 1);
      blk_seg[6 * k + 2 * s] = int(nd.cell_start[lo]);
      blk_seg[6 * k + 2 * s + 1] = int(nd.cell_start[hi + 1] - nd.cell_start[lo]);
      nblk += padded(blk_seg[6 * k + 2 * s + 1]);
    }
    max_nblk = std::max(max_nblk, nblk);
    blk_off[k + 1] = blk_off[k] + (nd.cell_start[c + 1] - nd.cell_start[c]) * int64_t(nblk);
  }
  std::vector<cd> Wb(blk_off[nocc], cd(0.0));
  std::vector<int64_t> rem_row(N + 1, 0);
  // position of column col in row q's block, or -1 (the remainder)
  auto block_pos = [&](int64_t q, int col) {
    const int* sg = &blk_seg[6 * occ_of_node[q]];
    int base = 0;
    for (int s = 0; s < 3; ++s) {
      if (col >= sg[2 * s] && col < sg[2 * s] + sg[2 * s + 1]) return base + col - sg[2 * s];
      base += padded(sg[2 * s + 1]);
    }
    return -1;
  };
  // rows in parallel (each row owns its block row); every row sums its entries in CSR order
  lsh::parallel_for(P.n_threads, N, 512, [&](int64_t q0, int64_t q1) {
    for (int64_t q = q0; q < q1; ++q) {
      const int k = occ_of_node[q];
      const int* sg = &blk_seg[6 * k];
      const int nblk = padded(sg[1]) + padded(sg[3]) + padded(sg[5]);
      cd* row = &Wb[blk_off[k] + (q - occ_start[k]) * nblk];
      int64_t rem = 0;
      for (int64_t e = P.rowptr[q]; e < P.rowptr[q + 1]; ++e) {
        const int pos = block_pos(q, P.col[e]);
        if (pos >= 0) row[pos] += P.val[e];
        else ++rem;
      }
      rem_row[q + 1] = rem;
    }
  });
  for (int64_t q = 0; q < N; ++q) rem_row[q + 1] += rem_row[q];
  std::vector<int> rem_col(rem_row[N]);
  std::vector<cd> rem_val(rem_row[N]);
  lsh::parallel_for(P.n_threads, N, 512, [&](int64_t q0, int64_t q1) {
    for (int64_t q = q0; q < q1; ++q) {
      int64_t o = rem_row[q];
      for (int64_t e = P.rowptr[q]; e < P.rowptr[q + 1]; ++e)
        if (block_pos(q, P.col[e]) < 0) {
          rem_col[o] = P.col[e];
          rem_val[o] = P.val[e];
          ++o;
        }
    }
  });
  std::vector<int32_t>().swap(P.col);
  std::vector<cd>().swap(P.val);
  const int64_t* d_occ_start = UP(int64_t, occ_start);
  const int* d_occ_cells = UP(int, P.occ_cells);
  const int* d_occ_of_cell = UP(int, occ_of_cell);
  const int* d_occ_of_node = UP(int, occ_of_node);
  const int64_t* d_P_off = UP(int64_t, P.P_off);
  // projection pieces: each cell's nodes cut into np near-equal runs of at most
  // kProjPiece, the longest runs first; cells of several pieces get np
  // partial-sum slots
  std::vector<int> pieces, piece_off(nocc, 0);
  int n_slots = 0;
  for (int k = 0; k < nocc; ++k) {
    const int nc = int(occ_start[k + 1] - occ_start[k]);
    const int np = std::max(1, (nc + lsd::kProjPiece - 1) / lsd::kProjPiece);
    if (np > 0xffff) return bail(LS_ERR_INVALID, "a cell holds too many nodes");
    piece_off[k] = n_slots;
    if (np > 1) n_slots += np;
    for (int q = 0; q < np; ++q) {
      pieces.push_back(k);
      pieces.push_back(int(int64_t(q) * nc / np));
      pieces.push_back(int(int64_t(q + 1) * nc / np));
      pieces.push_back((q << 16) | np);
    }
  }
  {
    const size_t n = pieces.size() / 4;
    std::vector<size_t> idx(n);
    for (size_t i = 0; i < n; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
      return pieces[4 * x + 2] - pieces[4 * x + 1] > pieces[4 * y + 2] - pieces[4 * y + 1];
    });
    std::vector<int> o(pieces.size());
    for (size_t i = 0; i < n; ++i)
      for (int c = 0; c < 4; ++c) o[4 * i + c] = pieces[4 * idx[i] + c];
    pieces.swap(o);
  }
  std::vector<int> cell_pieces;
  {
    std::vector<int> by_size(nocc);
    for (int k = 0; k < nocc; ++k) by_size[k] = k;
    std::stable_sort(by_size.begin(), by_size.end(), [&](int x, int y) {
      return occ_start[x + 1] - occ_start[x] > occ_start[y + 1] - occ_start[y];
    });
    for (int k : by_size) {
      cell_pieces.push_back(k);
      cell_pieces.push_back(0);
      cell_pieces.push_back(int(occ_start[k + 1] - occ_start[k]));
      cell_pieces.push_back(1);
    }
  }
  const int* d_cell_pieces_raw = UP(int, cell_pieces);
  const int4* d_cell_pieces = reinterpret_cast<const int4*>(d_cell_pieces_raw);
  const int* d_pieces_raw = UP(int, pieces);
  const int4* d_pieces = reinterpret_cast<const int4*>(d_pieces_raw);
  const int* d_piece_off = UP(int, piece_off);
  int* d_count64 = UP(int, std::vector<int>(nocc, 0));
  int* d_count32 = UP(int, std::vector<int>(nocc, 0));
  std::vector<int> items, items32, items128;   // (occupied cell, first row) pairs, 16 / 32 / 128 rows each
  for (int k = 0; k < nocc; ++k)
    for (int64_t r = 0; r < occ_start[k + 1] - occ_start[k]; r += 16) {
      items.push_back(k); items.push_back(int(r));
      if (r % 32 == 0) { items32.push_back(k); items32.push_back(int(r)); }
      if (r % 128 == 0) { items128.push_back(k); items128.push_back(int(r)); }
    }
  // heaviest work items first (rows x padded columns), so that the last wave of
  // the grid holds the short ones.  For the FP64-bound and tensor-core grids;
  // the HBM-bound complex64 grids on CUDA cores keep cell order, which streams
  // the weights in address order.
  auto heaviest_first = [&](std::vector<int>& v, int rows_per) {
    const size_t n = v.size() / 2;
    std::vector<std::pair<int64_t, size_t>> cost(n);
    for (size_t i = 0; i < n; ++i) {
      const int k = v[2 * i], r = v[2 * i + 1];
      const int* sg = &blk_seg[6 * k];
      const int64_t nblk = padded(sg[1]) + padded(sg[3]) + padded(sg[5]);
      cost[i] = {std::min<int64_t>(rows_per, occ_start[k + 1] - occ_start[k] - r) * nblk, i};
    }
    std::stable_sort(cost.begin(), cost.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    std::vector<int> o(v.size());
    for (size_t i = 0; i < n; ++i) {
      o[2 * i] = v[2 * cost[i].second];
      o[2 * i + 1] = v[2 * cost[i].second + 1];
    }
    v.swap(o);
  };
  const int* d_items_raw = UP(int, items);
  const int2* d_items = reinterpret_cast<const int2*>(d_items_raw);
  heaviest_first(items, 16);
  heaviest_first(items128, 128);
  const int* d_items64_raw = UP(int, items);
  const int2* d_items64 = reinterpret_cast<const int2*>(d_items64_raw);
  const int* d_items32_raw = UP(int, items32);
  const int2* d_items32 = reinterpret_cast<const int2*>(d_items32_raw);
  const int* d_items128_raw = UP(int, items128);
  const int2* d_items128 = reinterpret_cast<const int2*>(d_items128_raw);
  // offsets of the 128-row items in the tensor-core tile layout of the weights
  std::vector<int64_t> tile_off(items128.size() / 2 + 1, 0);
  for (size_t i = 0; i + 1 < tile_off.size(); ++i) {
    const int k = items128[2 * i], r = items128[2 * i + 1];
    const int* sg = &blk_seg[6 * k];
    const int nblk = padded(sg[1]) + padded(sg[3]) + padded(sg[5]);
    tile_off[i + 1] = tile_off[i] + lsd::tc_tile_elems(int(occ_start[k + 1] - occ_start[k] - r), nblk);
  }
  const int64_t* d_tile_off = UP(int64_t, tile_off);
  int* d_tc_err = UP(int, std::vector<int>(1, 0));
  // the persistent tensor-core grid (one block per SM) takes its 128-row items
  // from per-block lists balanced by longest-processing-time-first: an item
  // costs its chunk count times the larger of the MMA issue time (a fixed
  // number of instructions per chunk, whatever the rows) and the copy time of
  // its row groups (half the MMA time for a chunk of 16 groups)
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, plan->device) != cudaSuccess || n_sm <= 0)
    return bail(LS_ERR_CUDA, "cudaDeviceGetAttribute(multiProcessorCount) failed");
  const int n_it128 = int(items128.size() / 2);
  const int tc_grid = std::max(1, std::min(n_it128, n_sm));
  std::vector<int> tc_bptr(tc_grid + 1, 0), tc_blist(n_it128);
  {
    std::vector<std::pair<double, int>> cost(n_it128);
    for (int i = 0; i < n_it128; ++i) {
      const int k = items128[2 * i], r = items128[2 * i + 1];
      const int* sg = &blk_seg[6 * k];
      const int64_t nblk = padded(sg[1]) + padded(sg[3]) + padded(sg[5]);
      const int64_t rows = std::min<int64_t>(128, occ_start[k + 1] - occ_start[k] - r);
      cost[i] = {double((nblk + 15) / 16) * std::max(0.5, double((rows + 7) / 8) / 16.0), i};
    }
    std::stable_sort(cost.begin(), cost.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    std::priority_queue<std::pair<double, int>, std::vector<std::pair<double, int>>, std::greater<>> load;
    for (int b = 0; b < tc_grid; ++b) load.push({0.0, b});
    std::vector<std::vector<int>> per(tc_grid);
    for (const auto& c : cost) {
      auto top = load.top();
      load.pop();
      per[top.second].push_back(c.second);
      load.push({top.first + c.first, top.second});
    }
    for (int b = 0, n = 0; b < tc_grid; ++b) {
      for (int i : per[b]) tc_blist[n++] = i;
      tc_bptr[b + 1] = n;
    }
  }
  const int* d_tc_bptr = UP(int, tc_bptr);
  const int* d_tc_blist = UP(int, tc_blist);
  const int64_t* d_blk_off = UP(int64_t, blk_off);
  const int* d_blk_seg = UP(int, blk_seg);
  const int64_t* d_rem_row = UP(int64_t, rem_row);
  const int* d_rem_col = UP(int, rem_col);
  plan->x = UP(double, nd.x);
  plan->y = UP(double, nd.y);
  plan->ffw = UP(double, P.ffw);
  // twiddles and spectra
  const int M = P.M;
  int logM = 0;
  while ((1 << logM) < M) ++logM;
  std::vector<cd> tw(M);
  for (int m = 0; m < M; ++m) tw[m] = std::polar(1.0, -2.0 * M_PI * double(m) / M);
  std::vector<cd> G = P.Gtab, D = P.Dtab;
  const double sc = 1.0 / (double(M) * double(M));
  for (auto& z : G) z *= sc;
  for (auto& z : D) z *= sc;
  double2* d_tw64 = UP(double2, tw);
  // spectra: full FFT of the tables on the device, then keep the quarter
  // [l][k], k, l in [0, M/2] (even / odd symmetry of the tables)
  const int64_t MM = int64_t(M) * M;
  const int hq = M / 2 + 1;
  std::vector<cd> Gq(size_t(hq) * hq), Dq(size_t(hq) * hq);
  {
    double2* tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, MM * sizeof(double2));
    if (e != cudaSuccess) return bail(LS_ERR_NOMEM, "spectra work space");
    std::vector<cd> full(MM);
    for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
      const std::vector<cd>& tab = which == 0 ? G : D;
      e = cudaMemcpy(tmp, tab.data(), MM * sizeof(double2), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = lsd::fft2d<double2>(tmp, M, logM, d_tw64, false, 0);
      if (e == cudaSuccess) e = cudaMemcpy(full.data(), tmp, MM * sizeof(double2), cudaMemcpyDeviceToHost);
      std::vector<cd>& q = which == 0 ? Gq : Dq;
      for (int l = 0; l < hq; ++l)
        for (int k = 0; k < hq; ++k) q[size_t(l) * hq + k] = full[size_t(k) * M + l];
    }
    cudaFree(tmp);
    if (e != cudaSuccess) return bail(LS_ERR_CUDA, std::string("spectra: ") + cudaGetErrorString(e));
  }
  std::vector<cd>().swap(G);
  std::vector<cd>().swap(D);
  const double2* d_G64 = UP(double2, Gq);
  const double2* d_D64 = UP(double2, Dq);
  const float2* d_G32 = UP(float2, to32(Gq));
  const float2* d_D32 = UP(float2, to32(Dq));
  // FP64 apply data
  auto& a = plan->d64;
  a.N = N; a.nocc = nocc; a.L = P.opt.L; a.Ne = P.Ne; a.n_es = P.n_es; a.n_loc = P.n_loc; a.nfb2 = P.nfb2;
  a.M = M; a.n_lat = P.n_lat; a.logM = logM;
  a.occ_start = d_occ_start; a.occ_cells = d_occ_cells; a.occ_of_cell = d_occ_of_cell;
  a.occ_of_node = d_occ_of_node; a.P_off = d_P_off;
  a.pieces = d_pieces; a.n_pieces = int(pieces.size() / 4); a.piece_off = d_piece_off; a.proj_count = d_count64;
  a.cell_pieces = d_cell_pieces;
  a.blk_off = d_blk_off; a.blk_seg = d_blk_seg; a.rem_row = d_rem_row; a.rem_col = d_rem_col;
  a.max_nblk = max_nblk;
  a.items = d_items64; a.n_items = int(items.size() / 2);
  a.items32 = d_items32; a.n_items32 = int(items32.size() / 2);
  // projections per cell stored [node][n_es] (thread per row of P_c reads
  // consecutive entries); Re + Im of each entry for the three-multiplication product
  auto node_major = [&](std::vector<cd>& Pm) {
    std::vector<cd> t(Pm.size());
    for (int k = 0; k < nocc; ++k) {
      const int64_t base = P.P_off[k], nc = occ_start[k + 1] - occ_start[k];
      for (int i = 0; i < P.n_es; ++i)
        for (int64_t j = 0; j < nc; ++j) t[base + j * P.n_es + i] = Pm[base + i * nc + j];
    }
    Pm.swap(t);
  };
  node_major(P.P64);
  node_major(P.P32);
  a.P = UP(double2, P.P64);
  {
    double* ps = plan->alloc<double>(P.P64.size(), &st);
    if (st != LS_OK) return bail(st, plan->err);
    const cudaError_t e = lsd::weight_sums(a.P, ps, int64_t(P.P64.size()), 0);
    if (e != cudaSuccess) return bail(LS_ERR_CUDA, std::string("projection sums: ") + cudaGetErrorString(e));
    a.Ps = ps;
  }
  // local-expansion matrix [B^+ | -B^+ T_o ...]: one contraction with the cell's
  // lattice values and its 3 x 3 neighbours' strengths gives gamma_c
  const int n_lk = P.n_loc + 9 * P.n_es;
  // stored transposed, [n_lk][nfb2] (thread per row n reads consecutive entries)
  std::vector<cd> LA(size_t(P.nfb2) * n_lk);
  for (int n = 0; n < P.nfb2; ++n) {
    for (int p = 0; p < P.n_loc; ++p) LA[size_t(p) * P.nfb2 + n] = P.Bpinv[size_t(n) * P.n_loc + p];
    for (int o = 0; o < 9; ++o)
      for (int l = 0; l < P.n_es; ++l)
        LA[size_t(P.n_loc + o * P.n_es + l) * P.nfb2 + n] = -P.BT[(size_t(o) * P.nfb2 + n) * P.n_es + l];
  }
  a.LA = UP(double2, LA);
  {
    double* las = plan->alloc<double>(LA.size(), &st);
    if (st != LS_OK) return bail(st, plan->err);
    const cudaError_t e = lsd::weight_sums(a.LA, las, int64_t(LA.size()), 0);
    if (e != cudaSuccess) return bail(LS_ERR_CUDA, std::string("local matrix sums: ") + cudaGetErrorString(e));
    a.LAs = las;
  }
  a.Phi = UP(double2, P.Phi);
  a.Wb = UP(double2, Wb);
  {   // Re + Im of every block weight: the three-multiplication complex product
    double* ws = plan->alloc<double>(size_t(blk_off[nocc]), &st);
    if (st != LS_OK) return bail(st, plan->err);
    const cudaError_t e = lsd::weight_sums(a.Wb, ws, blk_off[nocc], 0);
    if (e != cudaSuccess) return bail(LS_ERR_CUDA, std::string("weight sums: ") + cudaGetErrorString(e));
    a.Ws = ws;
  }
  a.rem_val = UP(double2, rem_val);
  a.Gq = d_G64; a.Dq = d_D64; a.tw = d_tw64;
  a.kappa2 = kappa * kappa;
  a.sigma = plan->alloc<double2>(size_t(lsd::kMaxRhs64) * nocc * P.n_es, &st);
  a.proj_part = plan->alloc<double2>(size_t(lsd::kMaxRhs64) * n_slots * P.n_es, &st);
  a.Sm = plan->alloc<double2>(lsd::kMaxRhs64 * a.lattice_rows() * M, &st);
  a.Sd = plan->alloc<double2>(lsd::kMaxRhs64 * a.lattice_rows() * M, &st);
  a.gamma = plan->alloc<double2>(size_t(lsd::kMaxRhs64) * nocc * P.nfb2, &st);
  a.utc = plan->alloc<double>(size_t(lsd::kMaxRhs64) * N, &st);
  a.utef = plan->alloc<double2>(size_t(lsd::kMaxRhs64) * N, &st);
  if (st != LS_OK) return bail(st, plan->err);
  // complex64 apply data
  auto& b = plan->d32;
  b.N = a.N; b.nocc = a.nocc; b.L = a.L; b.Ne = a.Ne; b.n_es = a.n_es; b.n_loc = a.n_loc; b.nfb2 = a.nfb2;
  b.M = a.M; b.n_lat = a.n_lat; b.logM = a.logM;
  b.occ_start = a.occ_start; b.occ_cells = a.occ_cells; b.occ_of_cell = a.occ_of_cell;
  b.occ_of_node = a.occ_of_node; b.P_off = a.P_off;
  b.pieces = a.pieces; b.n_pieces = a.n_pieces; b.piece_off = a.piece_off; b.proj_count = d_count32;
  b.cell_pieces = a.cell_pieces;
  b.blk_off = a.blk_off; b.blk_seg = a.blk_seg; b.rem_row = a.rem_row; b.rem_col = a.rem_col;
  b.max_nblk = a.max_nblk;
  b.items = d_items; b.n_items = a.n_items;
  b.items32 = a.items32; b.n_items32 = a.n_items32;
  b.items128 = d_items128; b.n_items128 = int(items128.size() / 2);
  b.tile_off = d_tile_off;
  b.tc_bptr = d_tc_bptr;
  b.tc_blist = d_tc_blist;
  b.tc_grid = tc_grid;
  b.tc_err = d_tc_err;
  b.P = UP(float2, to32(P.P32));
  b.LA = UP(float2, to32(LA));
  b.Phi = UP(float2, to32(P.Phi));
  {
    std::vector<std::complex<float>> w32 = to32(Wb);
    std::vector<cd>().swap(Wb);
    b.Wb = UP(float2, w32);
  }
  {   // the same blocks in the tile layout the tensor-core near field copies in
      // bulk (split FP16, scaled per row), its row scales and per-RHS scales
    float2* wt = plan->alloc<float2>(size_t(tile_off.back()), &st);
    float* rs = plan->alloc<float>(size_t(N), &st);
    b.tc_tmax = plan->alloc<unsigned>(size_t(lsd::kMaxRhs32), &st);
    if (st != LS_OK) return bail(st, plan->err);
    const cudaError_t e = lsd::tile_weights(b, wt, rs, 0);
    if (e != cudaSuccess) return bail(LS_ERR_CUDA, std::string("tile layout: ") + cudaGetErrorString(e));
    b.Wt = wt;
    b.tc_rscale = rs;
  }
  if (P.nfb2 <= 32) {   // LA in the tile layout of the tensor-core local coefficients
    const int Kl = P.n_loc + 9 * P.n_es;
    unsigned char* lat = plan->alloc<unsigned char>(lsd::local_tc_bytes(Kl), &st);
    if (st != LS_OK) return bail(st, plan->err);
    const cudaError_t e = lsd::local_tc_tiles(b.LA, Kl, P.nfb2, lat, 0);
    if (e != cudaSuccess) return bail(LS_ERR_CUDA, std::string("local tile layout: ") + cudaGetErrorString(e));
    b.LAt = lat;
  }
  b.rem_val = UP(float2, to32(rem_val));
  b.Gq = d_G32; b.Dq = d_D32;
  b.tw = UP(float2, to32(tw));
  b.kappa2 = a.kappa2;
  b.sigma = plan->alloc<float2>(size_t(lsd::kMaxRhs32) * nocc * P.n_es, &st);
  b.proj_part = plan->alloc<float2>(size_t(lsd::kMaxRhs32) * n_slots * P.n_es, &st);
  b.Sm = plan->alloc<float2>(lsd::kMaxRhs32 * b.lattice_rows() * M, &st);
  b.Sd = plan->alloc<float2>(lsd::kMaxRhs32 * b.lattice_rows() * M, &st);
  b.gamma = plan->alloc<float2>(size_t(lsd::kMaxRhs32) * nocc * P.nfb2, &st);
  if (st != LS_OK) return bail(st, plan->err);
#undef UP
  if (cudaDeviceSynchronize() != cudaSuccess) return bail(LS_ERR_CUDA, "upload failed");
  // info, then release the large host arrays
  ls_plan_info_t& inf = plan->info;
  inf.N = N; inf.n_collar = nd.n_collar; inf.n_cart = nd.n_cart; inf.nnz_near = blk_off[nocc] + rem_row[N];
  inf.L = P.opt.L; inf.N_eq = P.Ne; inf.n_es = P.n_es; inf.n_loc = P.n_loc; inf.n_fb = P.opt.n_fb;
  inf.fft_M = M; inf.n_cells_occupied = nocc;
  inf.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  stage[3] = secs_since(t_dev);
  for (int k = 0; k < 4; ++k) inf.stage_seconds[k] = stage[k];
  inf.device_bytes = plan->device_bytes;
  std::vector<cd>().swap(P.P64);
  std::vector<cd>().swap(P.P32);
  std::vector<cd>().swap(P.Phi);
  std::vector<cd>().swap(P.Gtab);
  std::vector<cd>().swap(P.Dtab);
  *out = plan;
  return LS_OK;
}

ls_status ls_plan_create3(const ls_ball3* ball, const ls_rules3* rules, ls_n2_fn n2, void* ctx, double kappa,
                          const ls_accel3* acc, ls_plan* out) {
  if (!out) return fail(nullptr, LS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!ball || !acc || !n2) return fail(nullptr, LS_ERR_INVALID, "ball, acc or n2 is NULL");
  if (!(kappa > 0) || !(acc->H > 0) || acc->L < 1 || acc->N_eq < 1 || acc->p < 0 || acc->m_coll < 0 ||
      acc->rcond < 0)
    return fail(nullptr, LS_ERR_INVALID, "invalid kappa or accelerator options");
  const auto t0 = std::chrono::steady_clock::now();
  ls_plan plan = new (std::nothrow) ls_plan_s;
  if (!plan) return fail(nullptr, LS_ERR_NOMEM, "host allocation failed");
  if (cudaGetDevice(&plan->device) != cudaSuccess) {
    cudaGetLastError();
    delete plan;
    return fail(nullptr, LS_ERR_CUDA, "cudaGetDevice failed");
  }
  plan->dim = 3;
  auto bail = [&](ls_status st, const std::string& m) {
    g_create_error = m;
    plan->free_all();
    delete plan;
    return st;
  };
  const int nt = acc->n_threads > 0 ? acc->n_threads : int(std::max(1u, std::thread::hardware_concurrency()));
  lsh::Ball3 B;
  B.a = ball->a; B.w = ball->w; B.n_f = ball->n_f; B.n_s = ball->n_s; B.Q = ball->Q;
  B.delta = ball->delta; B.h = ball->h; B.tau0 = ball->tau0; B.tau1 = ball->tau1;
  std::vector<cd> P64, LA64, Phi64, Gs, Ds;
  std::vector<std::complex<float>> P32;
  std::vector<double> m, wfac;
  lsh::Accel3 A;
  double stage[4] = {0, 0, 0, 0};
  auto tst = std::chrono::steady_clock::now();
  try {
    if (!lsh::build_ball3(B)) return bail(LS_ERR_INVALID, B.err);
    const int64_t N = B.N;
    // contrast m = 1 - n^2 at the nodes (the callback receives 3 coordinates per point)
    std::vector<double> n2v(N, 1.0);
    if (n2(N, B.x.data(), n2v.data(), ctx) != 0) return bail(LS_ERR_INVALID, "n2 callback failed");
    m.resize(N);
    wfac.resize(N);
    for (int64_t q = 0; q < N; ++q) {
      m[q] = 1.0 - n2v[q];
      wfac[q] = B.w_q[q] * B.omega[q] * m[q];
    }
    stage[0] = secs_since(tst);
    tst = std::chrono::steady_clock::now();
    std::string em;
    if (!lsh::ball3_near(B, kappa, rules_from(rules), acc->box0, acc->H, acc->L, nullptr, 0, false, nt, &em))
      return bail(LS_ERR_INVALID, em);
    stage[1] = secs_since(tst);
    tst = std::chrono::steady_clock::now();
    A.kappa = kappa; A.H = acc->H; A.L = acc->L; A.Ne = acc->N_eq; A.p = acc->p; A.m_coll = acc->m_coll;
    A.n_threads = nt;
    for (int k = 0; k < 3; ++k) A.box0[k] = acc->box0[k];
    // one set of fits (truncation rcond, 1e-13 by default) serves both precisions
    A.rcond = acc->rcond > 0 ? acc->rcond : 1e-13;
    if (!lsh::build_accel3(A, B.x.data(), wfac.data(), N)) return bail(LS_ERR_INVALID, A.err);
    stage[2] = secs_since(tst);
    tst = std::chrono::steady_clock::now();
    const int nocc = int(A.occ_cells.size());
    const int n_es = A.n_es, nb = A.nb, n_loc = A.n_loc, M = A.M, L = acc->L;
    // plan order: the accelerator's node order (grouped by cell)
    const std::vector<int64_t>& order = A.node_order;
    std::vector<int64_t> inv(N);
    for (int64_t i = 0; i < N; ++i) inv[order[i]] = i;
    std::vector<int64_t> occ_start(nocc + 1, 0);
    for (int k = 0; k < nocc; ++k) occ_start[k + 1] = occ_start[k] + (A.P_off[k + 1] - A.P_off[k]) / n_es;
    if (occ_start[nocc] != N) return bail(LS_ERR_INVALID, "accelerator cells do not hold every node");
    std::vector<int> occ_of_cell(size_t(L) * L * L, -1), occ_of_node(N);
    for (int k = 0; k < nocc; ++k) {
      occ_of_cell[A.occ_cells[k]] = k;
      for (int64_t q = occ_start[k]; q < occ_start[k + 1]; ++q) occ_of_node[q] = k;
    }
    // projections per cell stored [node][n_es]
    auto node_major = [&](const std::vector<cd>& Pm, auto& dst) {
      dst.resize(Pm.size());
      for (int k = 0; k < nocc; ++k) {
        const int64_t base = A.P_off[k], nc = occ_start[k + 1] - occ_start[k];
        for (int i = 0; i < n_es; ++i)
          for (int64_t j = 0; j < nc; ++j) {
            const cd v = Pm[base + i * nc + j];
            dst[base + j * n_es + i] = {decltype(dst[0].real())(v.real()), decltype(dst[0].real())(v.imag())};
          }
      }
    };
    node_major(A.P, P64);
    node_major(A.P, P32);
    // [B^+ | -B^+ T_o] stored transposed: [n_loc + 27 n_es][nb]
    const int K = n_loc + 27 * n_es;
    auto local_matrix = [&](const lsh::Accel3& a, auto& dst) {
      dst.resize(size_t(K) * nb);
      for (int n = 0; n < nb; ++n) {
        for (int q = 0; q < n_loc; ++q) {
          const cd v = a.Bpinv[size_t(n) * n_loc + q];
          dst[size_t(q) * nb + n] = {decltype(dst[0].real())(v.real()), decltype(dst[0].real())(v.imag())};
        }
        for (int o = 0; o < 27; ++o)
          for (int l = 0; l < n_es; ++l) {
            const cd v = -a.BT[(size_t(o) * nb + n) * n_es + l];
            dst[size_t(n_loc + o * n_es + l) * nb + n] = {decltype(dst[0].real())(v.real()),
                                                         decltype(dst[0].real())(v.imag())};
          }
      }
    };
    local_matrix(A, LA64);
    Phi64.resize(size_t(N) * nb);
    for (int64_t i = 0; i < N; ++i)
      std::copy(A.Phi.begin() + order[i] * nb, A.Phi.begin() + (order[i] + 1) * nb, Phi64.begin() + i * nb);
    // adjacent part in plan order, contrast of the source node folded in
    std::vector<int64_t> rowptr(N + 1, 0);
    for (int64_t i = 0; i < N; ++i)
      rowptr[i + 1] = rowptr[i] + (B.near_rowptr[order[i] + 1] - B.near_rowptr[order[i]]);
    std::vector<int> col(rowptr[N]);
    std::vector<cd> val(rowptr[N]);
    lsh::parallel_for(nt, N, 256, [&](int64_t i0, int64_t i1) {
      for (int64_t i = i0; i < i1; ++i) {
        int64_t o = rowptr[i];
        for (int64_t e = B.near_rowptr[order[i]]; e < B.near_rowptr[order[i] + 1]; ++e, ++o) {
          col[o] = int(inv[B.near_col[e]]);
          val[o] = B.near_val[e] * m[B.near_col[e]];
        }
      }
    });
    std::vector<int32_t>().swap(B.near_col);
    std::vector<cd>().swap(B.near_val);
    ls_status st = LS_OK;
#define UP3(T, v) plan->upload<T>(v, &st); if (st != LS_OK) return bail(st, plan->err)
    const int64_t* d_occ_start = UP3(int64_t, occ_start);
    const int* d_occ_cells = UP3(int, A.occ_cells);
    const int* d_occ_of_cell = UP3(int, occ_of_cell);
    const int* d_occ_of_node = UP3(int, occ_of_node);
    const int64_t* d_P_off = UP3(int64_t, A.P_off);
    const int64_t* d_rowptr = UP3(int64_t, rowptr);
    const int* d_col = UP3(int, col);
    int logM = 0;
    while ((1 << logM) < M) ++logM;
    std::vector<cd> tw(M);
    for (int q = 0; q < M; ++q) tw[q] = std::polar(1.0, -2.0 * M_PI * double(q) / M);
    double2* d_tw64 = UP3(double2, tw);
    // spectra: 3-D FFT of the lattice tables on the device, scaled by 1 / M^3
    const int64_t M3 = int64_t(M) * M * M;
    {
      double2* tmp = plan->alloc<double2>(size_t(M3), &st);
      if (st != LS_OK) return bail(st, plan->err);
      Gs.resize(M3);
      Ds.resize(M3);
      const double sc = 1.0 / double(M3);
      for (int which = 0; which < 2; ++which) {
        const std::vector<cd>& tab = which == 0 ? A.Gtab : A.Dtab;
        std::vector<cd>& dst = which == 0 ? Gs : Ds;
        cudaError_t e = cudaMemcpy(tmp, tab.data(), M3 * sizeof(double2), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = lsd::fft3d<double2>(tmp, M, logM, d_tw64, false, 0);
        if (e == cudaSuccess) e = cudaMemcpy(dst.data(), tmp, M3 * sizeof(double2), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bail(LS_ERR_CUDA, std::string("3-D spectra: ") + cudaGetErrorString(e));
        for (auto& z : dst) z *= sc;
      }
      plan->release(tmp);
    }
    auto& a = plan->e64;
    a.N = N; a.nocc = nocc; a.L = L; a.Ne = acc->N_eq; a.n_es = n_es; a.n_loc = n_loc; a.nb = nb; a.M = M;
    a.logM = logM;
    a.occ_start = d_occ_start; a.occ_cells = d_occ_cells; a.occ_of_cell = d_occ_of_cell;
    a.occ_of_node = d_occ_of_node; a.P_off = d_P_off; a.rowptr = d_rowptr; a.col = d_col;
    a.P = UP3(double2, P64);
    a.LA = UP3(double2, LA64);
    {
      std::vector<float> la6(size_t(6) * LA64.size());
      for (size_t e = 0; e < LA64.size(); ++e) {
        const double f[3] = {LA64[e].real() + LA64[e].imag(), LA64[e].imag(), LA64[e].real()};
        for (int t = 0; t < 3; ++t) {
          const float hi = float(f[t]);
          la6[6 * e + 2 * t] = hi;
          la6[6 * e + 2 * t + 1] = float(f[t] - double(hi));
        }
      }
      a.LA6 = UP3(float, la6);
    }
    a.Phi = UP3(double2, Phi64);
    a.Gs = UP3(double2, Gs);
    a.Ds = UP3(double2, Ds);
    a.tw = d_tw64;
    // the FP64 adjacent part in the three-multiplication form (a + b, b, a)
    // is built on the device from the CSR values, with the complex64 blocks below
    double* d_val3 = plan->alloc<double>(size_t(3) * val.size(), &st);
    a.val3 = d_val3;
    a.u3 = plan->alloc<double>(size_t(3) * N, &st);
    a.kappa2 = kappa * kappa;
    a.sigma = plan->alloc<double2>(size_t(nocc) * n_es, &st);
    a.Sm = plan->alloc<double2>(size_t(M3), &st);
    a.Sd = plan->alloc<double2>(size_t(M3), &st);
    a.gamma = plan->alloc<double2>(size_t(nocc) * nb, &st);
    a.X = plan->alloc<double2>(size_t(nocc) * K, &st);
    a.X6 = plan->alloc<float>(size_t(6) * nocc * K, &st);
    a.part = plan->alloc<double2>(size_t(lsd::local3_slices(nocc, nb, K)) * nocc * nb, &st);
    if (st != LS_OK) return bail(st, plan->err);
    auto& b = plan->e32;
    b.N = a.N; b.nocc = a.nocc; b.L = a.L; b.Ne = a.Ne; b.n_es = a.n_es; b.n_loc = a.n_loc; b.nb = a.nb; b.M = a.M;
    b.logM = a.logM;
    b.occ_start = a.occ_start; b.occ_cells = a.occ_cells; b.occ_of_cell = a.occ_of_cell;
    b.occ_of_node = a.occ_of_node; b.P_off = a.P_off; b.rowptr = a.rowptr; b.col = a.col;
    // the complex64 apply runs the lattice convolution and the local
    // coefficients on the FP64 arrays (see apply3_batch): only the projection,
    // the adjacent part and the evaluation are complex64
    b.P = UP3(float2, P32);
    b.Phi = UP3(float2, to32(Phi64));
    b.lattice64 = &plan->e64;
    {
      // complex64 adjacent part as one dense block per cell over its 27
      // neighbours' nodes: nodes are grouped by cell in increasing cell id
      // (x fastest), so cells (i - 1 .. i + 1, j', k') hold one contiguous
      // node range; 9 ranges per cell.  Entries outside them (singular
      // stencils reaching past the block) stay in a CSR remainder.
      std::vector<int64_t> first_at(size_t(L) * L * L + 1, N);   // first node of the first cell >= id
      for (int k = nocc - 1; k >= 0; --k) first_at[A.occ_cells[k]] = occ_start[k];
      for (int64_t id = int64_t(L) * L * L - 1; id >= 0; --id)
        if (occ_of_cell[id] < 0) first_at[id] = first_at[id + 1];
      std::vector<int> seg(size_t(nocc) * 18, 0);
      std::vector<int64_t> boff(nocc + 1, 0);
      for (int k = 0; k < nocc; ++k) {
        const int c = A.occ_cells[k], ci = c % L, cj = (c / L) % L, ck = c / (L * L);
        int nblk = 0;
        for (int s9 = 0; s9 < 9; ++s9) {
          const int jj = cj + s9 % 3 - 1, kk = ck + s9 / 3 - 1;
          int st0 = 0, len = 0;
          if (jj >= 0 && jj < L && kk >= 0 && kk < L) {
            const int64_t row = (int64_t(kk) * L + jj) * L;
            const int64_t lo = first_at[row + std::max(ci - 1, 0)], hi = first_at[row + std::min(ci + 1, L - 1) + 1];
            st0 = int(lo);
            len = int(hi - lo);
          }
          seg[18 * k + 2 * s9] = st0;
          seg[18 * k + 2 * s9 + 1] = len;
          nblk += len;
        }
        boff[k + 1] = boff[k] + (occ_start[k + 1] - occ_start[k]) * nblk;
      }
      // both stored forms from the CSR on the device: val3, the dense blocks and
      // the per-row count of entries outside them; then the remainder CSR
#define CU3(call)                                                                        \
  do {                                                                                   \
    const cudaError_t e3_ = (call);                                                      \
    if (e3_ != cudaSuccess) return bail(LS_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e3_)); \
  } while (0)
      float2* d_wb = plan->alloc<float2>(size_t(boff[nocc]), &st);
      const double2* d_val = UP3(double2, val);
      std::vector<cd>().swap(val);
      const int64_t* d_boff = UP3(int64_t, boff);
      const int* d_seg = UP3(int, seg);
      int64_t* d_rcount = plan->alloc<int64_t>(size_t(N), &st);
      if (st != LS_OK) return bail(st, plan->err);
      CU3(cudaMemset(d_wb, 0, sizeof(float2) * size_t(boff[nocc])));
      CU3(lsd::near3_forms(N, d_occ_start, d_occ_of_node, d_rowptr, d_col, d_val, d_boff, d_seg, d_val3, d_wb,
                             d_rcount, 0));
      std::vector<int64_t> rrow(N + 1, 0);
      CU3(cudaMemcpy(rrow.data() + 1, d_rcount, sizeof(int64_t) * size_t(N), cudaMemcpyDeviceToHost));
      for (int64_t q = 0; q < N; ++q) rrow[q + 1] += rrow[q];
      plan->release(d_rcount);
      const int64_t* d_rrow = UP3(int64_t, rrow);
      int* d_rcol = plan->alloc<int>(size_t(rrow[N]), &st);
      float2* d_rval = plan->alloc<float2>(size_t(rrow[N]), &st);
      if (st != LS_OK) return bail(st, plan->err);
      CU3(lsd::near3_remainder(N, d_occ_of_node, d_rowptr, d_col, d_val, d_seg, d_rrow, d_rcol, d_rval, 0));
      CU3(cudaDeviceSynchronize());
#undef CU3
      plan->release(d_val);
      b.Wb = d_wb;
      b.blk_off = d_boff;
      b.blk_seg = d_seg;
      b.rowptr = d_rrow;
      b.col = d_rcol;
      b.val = d_rval;
    }
    b.kappa2 = a.kappa2;
    b.sigma = plan->alloc<float2>(size_t(nocc) * n_es, &st);
    b.gamma = plan->alloc<float2>(size_t(nocc) * nb, &st);
    if (st != LS_OK) return bail(st, plan->err);
    // coordinates and far-field weights in plan order; N in the 2-D apply data
    // (the solver and ls_apply read it there)
    plan->xyz3.resize(size_t(3) * N);
    plan->canon3 = order;
    std::vector<double> xs(N), ys(N), ffw(N);
    for (int64_t i = 0; i < N; ++i) {
      for (int k = 0; k < 3; ++k) plan->xyz3[3 * i + k] = B.x[3 * order[i] + k];
      ffw[i] = -B.w_q[order[i]] * B.omega[order[i]] * m[order[i]];      // w omega (n^2 - 1)
    }
    plan->x = UP3(double, plan->xyz3);
    plan->ffw3 = UP3(double, ffw);
#undef UP3
    plan->d64.N = N;
    plan->d32.N = N;
    plan->d64.kappa2 = plan->d32.kappa2 = kappa * kappa;
    plan->host.kappa = kappa;
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(LS_ERR_CUDA, "upload failed");
    ls_plan_info_t& inf = plan->info;
    inf.N = N; inf.n_collar = B.n_shell; inf.n_cart = B.n_cart; inf.nnz_near = rowptr[N];
    inf.L = L; inf.N_eq = acc->N_eq; inf.n_es = n_es; inf.n_loc = n_loc; inf.n_fb = nb;
    inf.fft_M = M; inf.n_cells_occupied = nocc;
    inf.plan_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    stage[3] = secs_since(tst);
    for (int k = 0; k < 4; ++k) inf.stage_seconds[k] = stage[k];
    inf.device_bytes = plan->device_bytes;
  } catch (const std::bad_alloc&) {
    return bail(LS_ERR_NOMEM, "host allocation failed");
  }
  *out = plan;
  return LS_OK;
}

ls_status ls_plan_info(ls_plan plan, ls_plan_info_t* info) {
  if (!plan || !info) return LS_ERR_INVALID;
  *info = plan->info;
  return LS_OK;
}

ls_status ls_plan_nodes(ls_plan plan, double* xy, int64_t* canon) {
  if (!plan) return LS_ERR_INVALID;
  if (plan->dim == 3) {
    if (xy) std::copy(plan->xyz3.begin(), plan->xyz3.end(), xy);
    if (canon) std::copy(plan->canon3.begin(), plan->canon3.end(), canon);
    return LS_OK;
  }
  const lsh::Nodes& nd = plan->host.nodes;
  if (xy)
    for (int64_t i = 0; i < nd.N; ++i) { xy[2 * i] = nd.x[i]; xy[2 * i + 1] = nd.y[i]; }
  if (canon) std::copy(nd.canon.begin(), nd.canon.end(), canon);
  return LS_OK;
}

ls_status ls_apply(ls_plan plan, const void* u, void* Au, int nrhs, ls_precision prec, void* stream) {
  if (!plan) return LS_ERR_INVALID;
  if (!u || !Au || nrhs < 0) return fail(plan, LS_ERR_INVALID, "ls_apply: bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t N = plan->d64.N;
  if (prec != LS_FP64 && prec != LS_MIXED) return fail(plan, LS_ERR_INVALID, "ls_apply: bad precision");
  cudaEvent_t* ev = plan->timing && plan->dim == 2 ? plan->ev : nullptr;
  const int maxr = prec == LS_FP64 ? lsd::kMaxRhs64 : plan->group32;
  for (int r = 0; r < nrhs;) {
    int nr = maxr;                       // largest power of two batch that fits
    while (nr > nrhs - r) nr /= 2;
    cudaError_t e;
    if (ev) {
      if (prec == LS_FP64)
        e = lsd::apply_batch(plan->d64, static_cast<const double2*>(u) + r * N, static_cast<double2*>(Au) + r * N,
                             nr, st, ev);
      else
        e = lsd::apply_batch(plan->d32, static_cast<const float2*>(u) + r * N, static_cast<float2*>(Au) + r * N, nr,
                             st, ev);
    } else if (prec == LS_FP64) {
      e = run_apply(plan, prec, plan->d64, static_cast<const double2*>(u) + r * N, static_cast<double2*>(Au) + r * N,
                    nr, st);
    } else {
      e = run_apply(plan, prec, plan->d32, static_cast<const float2*>(u) + r * N, static_cast<float2*>(Au) + r * N,
                    nr, st);
    }
    r += nr;
    if (e != cudaSuccess) return fail(plan, LS_ERR_CUDA, std::string("ls_apply: ") + cudaGetErrorString(e));
    if (ev) {
      LS_CU(cudaEventSynchronize(ev[lsd::kStages]));
      for (int k = 0; k < lsd::kStages; ++k) {
        float ms = 0;
        LS_CU(cudaEventElapsedTime(&ms, ev[k], ev[k + 1]));
        plan->stage_ms[prec][k] += ms;
      }
      plan->stage_calls[prec]++;
    }
  }
  return LS_OK;
}

}  // extern "C"

namespace {

// Where the R right-hand sides of a lock-step solve live: RHS r occupies
// elements [off[r], off[r] + len[r]) of every vector, and one vector of all R
// holds `total` elements (R contiguous vectors of one plan, or the
// concatenated vectors of the instances of a batch).
struct Layout {
  int R = 0;
  std::vector<int64_t> off, len;
  int64_t total = 0;
  int64_t max_len() const { return len.empty() ? 0 : *std::max_element(len.begin(), len.end()); }
};

Layout uniform_layout(int R, int64_t N) {
  Layout L;
  L.R = R;
  for (int r = 0; r < R; ++r) { L.off.push_back(int64_t(r) * N); L.len.push_back(N); }
  L.total = int64_t(R) * N;
  return L;
}

ls_status ensure_krylov(DevOwner* plan, Krylov& K, int restart, const Layout& lay) {
  const int R = lay.R;
  const int64_t total = lay.total, max_len = lay.max_len();
  if (K.restart >= restart && K.R >= R && K.total >= total && K.max_len >= max_len) return LS_OK;
  restart = std::max(restart, K.restart);
  const int Rw = std::max(R, K.R);
  const int64_t Tw = std::max(total, K.total), Lw = std::max(max_len, K.max_len);
  ls_status st = LS_OK;
  const int nb = lsd::gram_blocks(Lw);
  // the previous (smaller) work space: no solve is running (ls_solve synchronises before it returns)
  for (const void* p : {static_cast<const void*>(K.V), static_cast<const void*>(K.w), static_cast<const void*>(K.r),
                        static_cast<const void*>(K.e), static_cast<const void*>(K.cor),
                        static_cast<const void*>(K.apart), static_cast<const void*>(K.h),
                        static_cast<const void*>(K.partial), static_cast<const void*>(K.dnorm),
                        static_cast<const void*>(K.dpartial), static_cast<const void*>(K.c64a),
                        static_cast<const void*>(K.c64b), static_cast<const void*>(K.hk),
                        static_cast<const void*>(K.nk), static_cast<const void*>(K.vs),
                        static_cast<const void*>(K.h3)})
    plan->release(p);
  K.free_pinned();
  K = Krylov{};
  K.V = plan->alloc<double2>(size_t(restart + 1) * Tw, &st);
  K.w = plan->alloc<double2>(size_t(Tw), &st);
  K.r = plan->alloc<double2>(size_t(Tw), &st);
  K.e = plan->alloc<double2>(size_t(Tw), &st);
  K.cor = plan->alloc<double2>(size_t(Tw), &st);
  K.apart = plan->alloc<double2>(size_t(lsd::kAxpyGroups) * Lw, &st);
  K.vs = plan->alloc<double>(size_t(restart + 1) * Tw, &st);
  K.h3 = plan->alloc<double>(size_t(Rw) * (restart + 3) * 3, &st);
  K.h = plan->alloc<double2>(size_t(Rw) * (restart + 3), &st);
  K.partial = plan->alloc<double2>(size_t(Rw) * nb * (restart + 3), &st);
  K.dnorm = plan->alloc<double>(Rw, &st);
  K.dpartial = plan->alloc<double>(size_t(Rw) * nb, &st);
  K.c64a = plan->alloc<float2>(size_t(Tw), &st);
  K.c64b = plan->alloc<float2>(size_t(Tw), &st);
  const size_t nhk = size_t(restart) * 2 * Rw * (restart + 3), nnk = size_t(restart) * Rw;
  K.hk = plan->alloc<double2>(nhk, &st);
  K.nk = plan->alloc<double>(nnk, &st);
  if (st != LS_OK) return st;
  K.free_pinned();
  if (cudaMallocHost(&K.pin_h, size_t(Rw) * (restart + 3) * sizeof(double2)) != cudaSuccess ||
      cudaMallocHost(&K.pin_n, size_t(Rw) * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&K.pin_hk, nhk * sizeof(double2)) != cudaSuccess ||
      cudaMallocHost(&K.pin_nk, nnk * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(plan, LS_ERR_NOMEM, "pinned host staging");
  }
  for (auto& e : K.ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return fail(plan, LS_ERR_CUDA, "event creation");
    }
  K.restart = restart;
  K.R = Rw;
  K.total = Tw;
  K.max_len = Lw;
  return LS_OK;
}

// nrm[r] = ||base_r|| for every RHS of the layout (one host synchronisation)
template <typename T>
cudaError_t layout_norms(Krylov& K, const Layout& lay, const T* base, cudaStream_t st) {
  const int64_t nbmax = lsd::gram_blocks(K.max_len);
  for (int r = 0; r < lay.R; ++r) {
    cudaError_t e = lsd::norm2(base + lay.off[r], lay.len[r], K.dpartial + size_t(r) * nbmax, K.dnorm + r, st);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemcpyAsync(K.pin_n, K.dnorm, lay.R * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(st);
}

// Lock-step GMRES(m) for the R right-hand sides of a layout (FP64 Arnoldi):
// every iteration applies the operator to the R current basis vectors in ONE
// call (op(in, out, need) on whole layout vectors: a batched apply of one
// plan, or the apply of a multi-instance batch; need[r] = 0 marks RHS whose
// product is not used, nullptr means all), then runs the Arnoldi step of each RHS
// with one host synchronisation for all of them.  Classical Gram-Schmidt with
// selective re-orthogonalisation (a second pass only when the first removed
// more than 1 - 1/sqrt(2) of ||w||), Givens rotations on the host, true
// residual checked at every restart.  The basis is stored with Re + Im of
// every entry, so the Gram and update products take three FP64 FMAs each.  Stops when every RHS has
// ||b - A x|| / ||b|| <= tol; iters[r] counts the iterations of RHS r.
template <typename Op>
ls_status gmres_lockstep(DevOwner* plan, Krylov& K, const Layout& lay, Op op, const double2* B, double2* X,
                         double tol, int max_iter, int restart, cudaStream_t st, int* iters, double* relres) {
  const int R = lay.R;
  const int64_t vs = lay.total;                      // stride between basis slots
  double2* V = K.V;
  double* VS = K.vs;                                 // Re + Im of every basis entry
  double2* Wv = K.w;
  double2* Rv = K.r;
  const int m = restart;
  const int nbmax = lsd::gram_blocks(K.max_len);
  const int hstride = m + 3;
  auto h_of = [&](int r) { return K.h + size_t(r) * hstride; };
  auto h3_of = [&](int r) { return K.h3 + size_t(r) * hstride * 3; };
  auto part_of = [&](int r) { return K.partial + size_t(r) * nbmax * hstride; };
  auto dn_of = [&](int r) { return K.dnorm + r; };
  auto dp_of = [&](int r) { return K.dpartial + size_t(r) * nbmax; };
  auto O = [&](int r) { return lay.off[r]; };
  auto Ln = [&](int r) { return lay.len[r]; };
  double* nrm = K.pin_n;
  std::vector<double> bnorm(R);
  LS_CU(layout_norms(K, lay, B, st));
  bnorm.assign(nrm, nrm + R);
  for (int r = 0; r < R; ++r) {
    iters[r] = 0;
    relres[r] = 0;
    if (bnorm[r] == 0.0) LS_CU(cudaMemsetAsync(X + O(r), 0, Ln(r) * sizeof(double2), st));
  }
  std::vector<std::vector<cd>> H(R, std::vector<cd>(size_t(m + 1) * m)), cs(R, std::vector<cd>(m)),
      sn(R, std::vector<cd>(m)), g(R, std::vector<cd>(m + 1));
  cd* hcol = reinterpret_cast<cd*>(K.pin_h);
  std::vector<int> k_used(R);
  std::vector<char> done(R), active(R), again(R);
  int total = 0;
  for (;;) {
    // true residuals
    LS_CU(op(X, Wv, nullptr));
    LS_CU(lsd::sub(B, Wv, Rv, vs, st));
    LS_CU(layout_norms(K, lay, Rv, st));
    bool all_done = true;
    for (int r = 0; r < R; ++r) {
      relres[r] = bnorm[r] > 0 ? nrm[r] / bnorm[r] : 0.0;
      done[r] = relres[r] <= tol;
      all_done = all_done && done[r];
    }
    if (all_done) return LS_OK;
    if (total >= max_iter) return fail(plan, LS_ERR_NOCONV, "GMRES reached max_iter");
    for (int r = 0; r < R; ++r) {
      double2* v0 = V + O(r);
      if (done[r]) {
        LS_CU(cudaMemsetAsync(v0, 0, Ln(r) * sizeof(double2), st));
        LS_CU(cudaMemsetAsync(VS + O(r), 0, Ln(r) * sizeof(double), st));
      } else {
        LS_CU(lsd::scale_into_sums(Rv + O(r), dn_of(r), v0, VS + O(r), Ln(r), st));
        std::fill(H[r].begin(), H[r].end(), cd(0));
        std::fill(g[r].begin(), g[r].end(), cd(0));
        g[r][0] = nrm[r];
      }
      active[r] = !done[r];
      k_used[r] = 0;
    }
    for (int k = 0; k < m; ++k) {
      LS_CU(op(V + k * vs, Wv, active.data()));     // only the RHS still iterating need A v
      std::vector<double> hk1(R, 0.0);
      for (int r = 0; r < R; ++r) again[r] = active[r];
      for (int pass = 0; pass < 2; ++pass) {
        bool any = false;
        for (int r = 0; r < R; ++r) {
          if (!again[r]) continue;
          any = true;
          LS_CU(lsd::gram3(V + O(r), VS + O(r), k + 1, vs, Wv + O(r), Ln(r), part_of(r), h_of(r), h3_of(r), st));
          LS_CU(lsd::axpy3_multi(V + O(r), VS + O(r), k + 1, vs, h3_of(r), Wv + O(r), K.apart, Ln(r), st));
          LS_CU(lsd::norm2(Wv + O(r), Ln(r), dp_of(r), dn_of(r), st));
        }
        if (!any) break;
        LS_CU(cudaMemcpyAsync(hcol, K.h, size_t(R) * hstride * sizeof(double2), cudaMemcpyDeviceToHost, st));
        LS_CU(cudaMemcpyAsync(nrm, K.dnorm, R * sizeof(double), cudaMemcpyDeviceToHost, st));
        LS_CU(cudaStreamSynchronize(st));
        for (int r = 0; r < R; ++r) {
          if (!again[r]) continue;
          for (int j = 0; j <= k; ++j) H[r][size_t(j) * m + k] += hcol[size_t(r) * hstride + j];
          const double before = std::sqrt(std::max(hcol[size_t(r) * hstride + k + 1].real(), 0.0));
          hk1[r] = nrm[r];
          again[r] = hk1[r] < 0.7071067811865476 * before;
        }
      }
      bool any_active = false;
      for (int r = 0; r < R; ++r) {
        double2* vn = V + (k + 1) * vs + O(r);
        double* vsn = VS + (k + 1) * vs + O(r);
        if (!active[r]) {
          LS_CU(cudaMemsetAsync(vn, 0, Ln(r) * sizeof(double2), st));
          LS_CU(cudaMemsetAsync(vsn, 0, Ln(r) * sizeof(double), st));
          continue;
        }
        std::vector<cd>& Hr = H[r];
        Hr[size_t(k + 1) * m + k] = hk1[r];
        LS_CU(lsd::scale_into_sums(Wv + O(r), dn_of(r), vn, vsn, Ln(r), st));
        for (int j = 0; j < k; ++j) {
          const cd t = std::conj(cs[r][j]) * Hr[size_t(j) * m + k] + std::conj(sn[r][j]) * Hr[size_t(j + 1) * m + k];
          Hr[size_t(j + 1) * m + k] = -sn[r][j] * Hr[size_t(j) * m + k] + cs[r][j] * Hr[size_t(j + 1) * m + k];
          Hr[size_t(j) * m + k] = t;
        }
        const cd a = Hr[size_t(k) * m + k], bb = Hr[size_t(k + 1) * m + k];
        const double den = std::sqrt(std::norm(a) + std::norm(bb));
        cs[r][k] = den > 0 ? a / den : cd(1);
        sn[r][k] = den > 0 ? bb / den : cd(0);
        Hr[size_t(k) * m + k] = den;
        Hr[size_t(k + 1) * m + k] = 0;
        g[r][k + 1] = -sn[r][k] * g[r][k];
        g[r][k] = std::conj(cs[r][k]) * g[r][k];
        ++iters[r];
        k_used[r] = k + 1;
        if (std::abs(g[r][k + 1]) / bnorm[r] <= tol || hk1[r] == 0.0) active[r] = 0;
        any_active = any_active || active[r];
      }
      ++total;
      if (!any_active || total >= max_iter) break;
    }
    // back substitution and x_r += V_r y_r
    for (int r = 0; r < R; ++r) {
      const int ku = k_used[r];
      if (done[r] || ku == 0) continue;
      std::vector<cd> y(ku);
      for (int i = ku - 1; i >= 0; --i) {
        cd sacc = g[r][i];
        for (int j = i + 1; j < ku; ++j) sacc -= H[r][size_t(i) * m + j] * y[j];
        y[i] = sacc / H[r][size_t(i) * m + i];
      }
      LS_CU(cudaMemcpyAsync(h_of(r), y.data(), ku * sizeof(double2), cudaMemcpyHostToDevice, st));
      LS_CU(lsd::combine(V + O(r), ku, vs, h_of(r), X + O(r), Ln(r), st));
    }
  }
}

// Pipelined lock-step GMRES(m): the same iteration as gmres_lockstep, but the
// host never waits for the iteration it has just queued.  Every iteration runs
// two full classical Gram-Schmidt passes (CGS2, so that no host decision sits
// between the passes), normalises on the device (v_{k+1} = w / ||w||), and
// queues an asynchronous copy of its coefficients to pinned memory plus an
// event; the host queues up to kLag iterations ahead and builds the Hessenberg
// columns, Givens rotations and residual estimates of the earlier iterations
// while the device works.  An RHS found converged stops taking part in later
// queued applies (op's need flags); iterations queued past its convergence are
// discarded (their columns are never used).  Used for the correction solves
// of the mixed refinement (complex64 apply, FP64 basis stored with its Re + Im
// sums), where the apply is short and a host round trip per iteration would
// leave the GPU idle.
template <typename T, typename Op>
ls_status gmres_lockstep_async(DevOwner* plan, Krylov& K, const Layout& lay, Op op, const T* B, T* X,
                               double tol, int max_iter, int restart, cudaStream_t st, int* iters, double* relres) {
  constexpr int kLag = 2;
  static_assert(kLag < Krylov::kEvents, "event ring");
  const int R = lay.R;
  const int64_t vs = lay.total;
  // complex128: the buffers as allocated, the basis with its Re + Im sums;
  // complex64 (LS_MIXED32): the same storage at half the element size
  constexpr bool kC128 = sizeof(T) == 16;
  T* V = reinterpret_cast<T*>(K.V);
  double* VS = K.vs;
  T* Wv = reinterpret_cast<T*>(K.w);
  T* Rv = reinterpret_cast<T*>(K.r);
  T* apart = reinterpret_cast<T*>(K.apart);
  // basis vector v = w / nrm into slot (offset into V)
  auto new_basis = [&](const T* w, const double* nrm, int64_t slot, int64_t len) -> cudaError_t {
    if constexpr (kC128) return lsd::scale_into_sums(w, nrm, V + slot, VS + slot, len, st);
    else return lsd::scale_into(w, nrm, V + slot, len, st);
  };
  const int m = restart;
  const int nbmax = lsd::gram_blocks(K.max_len);
  const int hstride = m + 3;
  auto part_of = [&](int r) { return K.partial + size_t(r) * nbmax * hstride; };
  auto dp_of = [&](int r) { return K.dpartial + size_t(r) * nbmax; };
  auto hslot = [&](int k, int pass, int r) { return K.hk + ((size_t(k) * 2 + pass) * R + r) * hstride; };
  auto h3_of = [&](int r) { return K.h3 + size_t(r) * hstride * 3; };   // per pass, used right away
  auto O = [&](int r) { return lay.off[r]; };
  auto Ln = [&](int r) { return lay.len[r]; };
  double* nrm = K.pin_n;
  std::vector<double> bnorm(R);
  LS_CU(layout_norms(K, lay, B, st));
  bnorm.assign(nrm, nrm + R);
  for (int r = 0; r < R; ++r) {
    iters[r] = 0;
    relres[r] = 0;
    if (bnorm[r] == 0.0) LS_CU(cudaMemsetAsync(X + O(r), 0, Ln(r) * sizeof(T), st));
  }
  std::vector<std::vector<cd>> H(R, std::vector<cd>(size_t(m + 1) * m)), cs(R, std::vector<cd>(m)),
      sn(R, std::vector<cd>(m)), g(R, std::vector<cd>(m + 1));
  std::vector<int> k_used(R);
  std::vector<char> done(R), active(R);
  std::vector<std::vector<char>> queued_for(m, std::vector<char>(R));
  int total = 0;
  for (;;) {
    // true residuals
    LS_CU(op(X, Wv, nullptr));
    LS_CU(lsd::sub(B, Wv, Rv, vs, st));
    LS_CU(layout_norms(K, lay, Rv, st));
    bool all_done = true;
    for (int r = 0; r < R; ++r) {
      relres[r] = bnorm[r] > 0 ? nrm[r] / bnorm[r] : 0.0;
      done[r] = relres[r] <= tol;
      all_done = all_done && done[r];
    }
    if (all_done) return LS_OK;
    if (total >= max_iter) return fail(plan, LS_ERR_NOCONV, "GMRES reached max_iter");
    std::vector<double> beta(nrm, nrm + R);
    for (int r = 0; r < R; ++r) {
      if (done[r]) {
        LS_CU(cudaMemsetAsync(V + O(r), 0, Ln(r) * sizeof(T), st));
        if (kC128) LS_CU(cudaMemsetAsync(VS + O(r), 0, Ln(r) * sizeof(double), st));
      } else {
        LS_CU(new_basis(Rv + O(r), K.dnorm + r, O(r), Ln(r)));
        std::fill(H[r].begin(), H[r].end(), cd(0));
        std::fill(g[r].begin(), g[r].end(), cd(0));
        g[r][0] = beta[r];
      }
      active[r] = !done[r];
      k_used[r] = 0;
    }
    int queued = 0, handled = 0;
    bool stop = false;
    for (;;) {
      // queue iterations ahead of the host
      while (!stop && queued < m && queued - handled < kLag && total + (queued - handled) < max_iter) {
        const int k = queued;
        bool any = false;
        for (int r = 0; r < R; ++r) { queued_for[k][r] = active[r]; any = any || active[r]; }
        if (!any) break;
        LS_CU(op(V + k * vs, Wv, queued_for[k].data()));
        for (int r = 0; r < R; ++r) {
          if (!queued_for[k][r]) continue;
          for (int pass = 0; pass < 2; ++pass) {
            if constexpr (kC128) {
              LS_CU(lsd::gram3(V + O(r), VS + O(r), k + 1, vs, Wv + O(r), Ln(r), part_of(r), hslot(k, pass, r),
                               h3_of(r), st));
              LS_CU(lsd::axpy3_multi(V + O(r), VS + O(r), k + 1, vs, h3_of(r), Wv + O(r), apart, Ln(r), st));
            } else {
              LS_CU(lsd::gram(V + O(r), k + 1, vs, Wv + O(r), Ln(r), part_of(r), hslot(k, pass, r), st));
              LS_CU(lsd::axpy_multi(V + O(r), k + 1, vs, hslot(k, pass, r), Wv + O(r), apart, Ln(r), st));
            }
          }
          LS_CU(lsd::norm2(Wv + O(r), Ln(r), dp_of(r), K.nk + size_t(k) * R + r, st));
          LS_CU(new_basis(Wv + O(r), K.nk + size_t(k) * R + r, (k + 1) * vs + O(r), Ln(r)));
        }
        LS_CU(cudaMemcpyAsync(K.pin_hk + size_t(k) * 2 * R * hstride, hslot(k, 0, 0),
                              size_t(2) * R * hstride * sizeof(double2), cudaMemcpyDeviceToHost, st));
        LS_CU(cudaMemcpyAsync(K.pin_nk + size_t(k) * R, K.nk + size_t(k) * R, R * sizeof(double),
                              cudaMemcpyDeviceToHost, st));
        LS_CU(cudaEventRecord(K.ev[k % Krylov::kEvents], st));
        ++queued;
      }
      if (handled == queued) break;
      // the oldest queued iteration: Hessenberg column, Givens rotation, residual estimate
      const int k = handled;
      LS_CU(cudaEventSynchronize(K.ev[k % Krylov::kEvents]));
      bool any_active = false;
      for (int r = 0; r < R; ++r) {
        if (!queued_for[k][r] || !active[r]) continue;
        const double2* h1 = K.pin_hk + (size_t(k) * 2 * R + r) * hstride;
        const double2* h2 = K.pin_hk + ((size_t(k) * 2 + 1) * R + r) * hstride;
        std::vector<cd>& Hr = H[r];
        for (int j = 0; j <= k; ++j) Hr[size_t(j) * m + k] = cd(h1[j].x + h2[j].x, h1[j].y + h2[j].y);
        const double hk1 = K.pin_nk[size_t(k) * R + r];
        Hr[size_t(k + 1) * m + k] = hk1;
        for (int j = 0; j < k; ++j) {
          const cd t = std::conj(cs[r][j]) * Hr[size_t(j) * m + k] + std::conj(sn[r][j]) * Hr[size_t(j + 1) * m + k];
          Hr[size_t(j + 1) * m + k] = -sn[r][j] * Hr[size_t(j) * m + k] + cs[r][j] * Hr[size_t(j + 1) * m + k];
          Hr[size_t(j) * m + k] = t;
        }
        const cd a = Hr[size_t(k) * m + k], bb = Hr[size_t(k + 1) * m + k];
        const double den = std::sqrt(std::norm(a) + std::norm(bb));
        cs[r][k] = den > 0 ? a / den : cd(1);
        sn[r][k] = den > 0 ? bb / den : cd(0);
        Hr[size_t(k) * m + k] = den;
        Hr[size_t(k + 1) * m + k] = 0;
        g[r][k + 1] = -sn[r][k] * g[r][k];
        g[r][k] = std::conj(cs[r][k]) * g[r][k];
        ++iters[r];
        k_used[r] = k + 1;
        if (std::abs(g[r][k + 1]) / bnorm[r] <= tol || hk1 == 0.0) active[r] = 0;
      }
      for (int r = 0; r < R; ++r) any_active = any_active || active[r];
      ++handled;
      ++total;
      if (!any_active || handled == m || total >= max_iter) stop = true;
      if (stop) break;
    }
    LS_CU(cudaStreamSynchronize(st));           // iterations queued past the stop are discarded
    // back substitution and x_r += V_r y_r
    for (int r = 0; r < R; ++r) {
      const int ku = k_used[r];
      if (done[r] || ku == 0) continue;
      std::vector<cd> y(ku);
      for (int i = ku - 1; i >= 0; --i) {
        cd sacc = g[r][i];
        for (int j = i + 1; j < ku; ++j) sacc -= H[r][size_t(i) * m + j] * y[j];
        y[i] = sacc / H[r][size_t(i) * m + i];
      }
      double2* hy = K.h + size_t(r) * hstride;
      LS_CU(cudaMemcpyAsync(hy, y.data(), ku * sizeof(double2), cudaMemcpyHostToDevice, st));
      LS_CU(lsd::combine(V + O(r), ku, vs, hy, X + O(r), Ln(r), st));
    }
  }
}

struct SolveStats {
  int iterations = 0, refinements = 0;
  double worst = 0;
  std::vector<int> it_per;          // per RHS: GMRES iterations (inner iterations for mixed)
  std::vector<double> res_per;      // per RHS: final relative residual ||b - A_64 x|| / ||b||
};

// A x = B for the R right-hand sides of a layout.  FP64: lock-step GMRES on
// op64.  Mixed: FP64 iterative refinement r = b - A_64 x (op64), lock-step
// GMRES on op32 (complex64 apply) to a loose tolerance, x += correction, until
// the FP64 residual of every RHS is <= tol.
template <typename Op64, typename Op32, typename Op32f>
ls_status solve_lockstep(DevOwner* plan, Krylov& K, const Layout& lay, Op64 op64, Op32 op32, Op32f op32f,
                         ls_precision prec, const double2* B, double2* X, double tol, int max_iter, int restart,
                         cudaStream_t st, SolveStats& S) {
  const int R = lay.R;
  std::vector<int> it(R);
  std::vector<double> rr(R);
  S.it_per.assign(R, 0);
  S.res_per.assign(R, 0.0);
  if (prec == LS_FP64) {
    const ls_status s = gmres_lockstep(plan, K, lay, op64, B, X, tol, max_iter, restart, st, it.data(), rr.data());
    for (int r = 0; r < R; ++r) {
      S.iterations += it[r];
      S.it_per[r] = it[r];
      S.res_per[r] = rr[r];
      S.worst = std::max(S.worst, rr[r]);
    }
    return s;
  }
  double2* Res = K.e;
  double2* Cor = K.cor;
  std::vector<double> bn(R), rn(R);
  LS_CU(layout_norms(K, lay, B, st));
  bn.assign(K.pin_n, K.pin_n + R);
  int inner_total = 0;
  for (int ref = 0;; ++ref) {
    LS_CU(op64(X, K.w, nullptr));
    LS_CU(lsd::sub(B, K.w, Res, lay.total, st));
    LS_CU(layout_norms(K, lay, Res, st));
    rn.assign(K.pin_n, K.pin_n + R);
    double rel = 0;
    for (int r = 0; r < R; ++r) {
      S.res_per[r] = bn[r] > 0 ? rn[r] / bn[r] : 0.0;
      rel = std::max(rel, S.res_per[r]);
    }
    // RHS already at tol get a zero correction equation (GMRES skips them)
    if (rel > tol)
      for (int r = 0; r < R; ++r)
        if (S.res_per[r] <= tol) LS_CU(cudaMemsetAsync(Res + lay.off[r], 0, lay.len[r] * sizeof(double2), st));
    if (rel <= tol) { S.worst = std::max(S.worst, rel); return LS_OK; }
    if (inner_total >= max_iter || ref >= 50) {
      S.worst = std::max(S.worst, rel);
      return fail(plan, LS_ERR_NOCONV, "refinement reached max_iter");
    }
    S.refinements++;
    const double inner_tol = std::max(1e-5, 0.3 * tol / rel);
    // the correction equation A e = r with the complex64 apply; basis and
    // Gram-Schmidt in FP64 (a complex64 basis loses the small remainder of
    // w - V h near stagnation: hard instances then took four times the iterations)
    const int inner_max = std::max(1, max_iter - inner_total);
    ls_status s = LS_OK;
    if (prec == LS_MIXED32) {
      // complex64 right-hand side, correction and Krylov basis
      LS_CU(lsd::to_c64(Res, K.c64a, lay.total, st));
      LS_CU(cudaMemsetAsync(K.c64b, 0, size_t(lay.total) * sizeof(float2), st));
      s = gmres_lockstep_async<float2>(plan, K, lay, op32f, K.c64a, K.c64b, inner_tol, inner_max, restart, st,
                                       it.data(), rr.data());
      if (s == LS_OK || s == LS_ERR_NOCONV) LS_CU(lsd::to_c128(K.c64b, Cor, lay.total, st));
    } else {
      LS_CU(cudaMemsetAsync(Cor, 0, size_t(lay.total) * sizeof(double2), st));
      s = gmres_lockstep_async<double2>(plan, K, lay, op32, Res, Cor, inner_tol, inner_max, restart, st, it.data(),
                                        rr.data());
    }
    int mx = 0;
    for (int r = 0; r < R; ++r) { S.iterations += it[r]; S.it_per[r] += it[r]; mx = std::max(mx, it[r]); }
    inner_total += mx;
    if (s != LS_OK && s != LS_ERR_NOCONV) return s;
    LS_CU(lsd::add_inplace(X, Cor, lay.total, st));
  }
}

// Initial guesses for the right-hand sides [r0, r0 + R) of one ls_solve call
// from the solutions of its earlier right-hand sides [0, r0): since
// A x_j = b_j, the residual of x0 = sum_j c_j x_j is b - sum_j c_j b_j, so c
// solves the least-squares problem min || b - B_prev c || through the normal
// equations (Gram matrix of the earlier right-hand sides, regularised by
// 1e-12 of its largest diagonal entry: a guess, not a solution).  Only
// right-hand sides whose initial guess is zero are seeded; the residual never
// exceeds that of the zero guess.
ls_status seed_from_previous(ls_plan plan, const double2* B, double2* X, int r0, int R, int64_t N,
                             std::vector<cd>& G, cudaStream_t st) {
  const int nb = lsd::gram_blocks(N);
  if (plan->seed_cap < r0 + 1) {
    ls_status s = LS_OK;
    plan->seed_h = plan->alloc<double2>(size_t(r0 + 1) * 2, &s);
    plan->seed_part = plan->alloc<double2>(size_t(nb) * (r0 + 1) * 2, &s);
    if (s != LS_OK) return s;
    plan->seed_cap = (r0 + 1) * 2;
  }
  // Gram matrix G[i][j] = <b_i, b_j> of the earlier right-hand sides (columns added as r0 grows)
  const int old = int(std::lround(std::sqrt(double(G.size()))));
  std::vector<cd> Gn(size_t(r0) * r0);
  for (int i = 0; i < old; ++i)
    for (int j = 0; j < old; ++j) Gn[size_t(i) * r0 + j] = G[size_t(i) * old + j];
  std::vector<cd> col(r0 + 1);
  for (int j = old; j < r0; ++j) {
    LS_CU(lsd::gram(B, r0, N, B + int64_t(j) * N, N, plan->seed_part, plan->seed_h, st));
    LS_CU(cudaMemcpyAsync(col.data(), plan->seed_h, r0 * sizeof(double2), cudaMemcpyDeviceToHost, st));
    LS_CU(cudaStreamSynchronize(st));
    for (int i = 0; i < r0; ++i) {
      Gn[size_t(i) * r0 + j] = col[i];
      Gn[size_t(j) * r0 + i] = std::conj(col[i]);
    }
  }
  G.swap(Gn);
  // Cholesky of G + eps I
  double dmax = 0;
  for (int i = 0; i < r0; ++i) dmax = std::max(dmax, G[size_t(i) * r0 + i].real());
  std::vector<cd> Lc(G);
  for (int i = 0; i < r0; ++i) Lc[size_t(i) * r0 + i] += 1e-12 * dmax;
  for (int j = 0; j < r0; ++j) {
    double d = Lc[size_t(j) * r0 + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(Lc[size_t(j) * r0 + k]);
    if (!(d > 0)) return LS_OK;                      // degenerate: keep the zero guesses
    d = std::sqrt(d);
    Lc[size_t(j) * r0 + j] = d;
    for (int i = j + 1; i < r0; ++i) {
      cd v = Lc[size_t(i) * r0 + j];
      for (int k = 0; k < j; ++k) v -= Lc[size_t(i) * r0 + k] * std::conj(Lc[size_t(j) * r0 + k]);
      Lc[size_t(i) * r0 + j] = v / d;
    }
  }
  std::vector<double> nrm(1);
  for (int r = 0; r < R; ++r) {
    double2* x = X + int64_t(r0 + r) * N;
    LS_CU(lsd::norm2(x, N, reinterpret_cast<double*>(plan->seed_part), reinterpret_cast<double*>(plan->seed_h), st));
    LS_CU(cudaMemcpyAsync(nrm.data(), plan->seed_h, sizeof(double), cudaMemcpyDeviceToHost, st));
    LS_CU(cudaStreamSynchronize(st));
    if (nrm[0] != 0.0) continue;                     // the caller gave a guess
    LS_CU(lsd::gram(B, r0, N, B + int64_t(r0 + r) * N, N, plan->seed_part, plan->seed_h, st));
    LS_CU(cudaMemcpyAsync(col.data(), plan->seed_h, r0 * sizeof(double2), cudaMemcpyDeviceToHost, st));
    LS_CU(cudaStreamSynchronize(st));
    std::vector<cd> c(r0);
    for (int i = 0; i < r0; ++i) {                   // L y = h
      cd v = col[i];
      for (int k = 0; k < i; ++k) v -= Lc[size_t(i) * r0 + k] * c[k];
      c[i] = v / Lc[size_t(i) * r0 + i];
    }
    for (int i = r0 - 1; i >= 0; --i) {              // L^H c = y
      cd v = c[i];
      for (int k = i + 1; k < r0; ++k) v -= std::conj(Lc[size_t(k) * r0 + i]) * c[k];
      c[i] = v / Lc[size_t(i) * r0 + i].real();
    }
    LS_CU(cudaMemcpyAsync(plan->seed_h, c.data(), r0 * sizeof(double2), cudaMemcpyHostToDevice, st));
    LS_CU(lsd::combine(X, r0, N, plan->seed_h, x, N, st));
  }
  return LS_OK;
}

}  // namespace

extern "C" {

ls_status ls_solve(ls_plan plan, const void* uinc, void* u, int nrhs, double tol, int max_iter, int restart,
                   ls_precision prec, ls_solve_info* info, void* stream) {
  if (!plan) return LS_ERR_INVALID;
  if (!uinc || !u || nrhs < 0 || !(tol > 0) || max_iter < 1 || restart < 1)
    return fail(plan, LS_ERR_INVALID, "ls_solve: bad arguments");
  if (prec != LS_FP64 && prec != LS_MIXED && prec != LS_MIXED32)
    return fail(plan, LS_ERR_INVALID, "ls_solve: bad precision");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t N = plan->d64.N;
  // right-hand sides are solved in lock-step batches sharing one batched apply
  const int maxb = prec == LS_FP64 ? lsd::kMaxRhs64 : lsd::kMaxRhs32;
  const int Rb = std::max(1, std::min(nrhs, maxb));
  ls_status s = ensure_krylov(plan, plan->K, restart, uniform_layout(Rb, N));
  if (s != LS_OK) return s;
  SolveStats S;
  int total_it = 0, total_ref = 0;
  double worst = 0;
  ls_status result = LS_OK;
  std::vector<cd> G;                        // Gram matrix of the solved right-hand sides
  for (int r0 = 0; r0 < nrhs; r0 += Rb) {
    const int R = std::min(Rb, nrhs - r0);
    if (r0 > 0) {
      s = seed_from_previous(plan, static_cast<const double2*>(uinc), static_cast<double2*>(u), r0, R, N, G, st);
      if (s != LS_OK) return s;
    }
    // FP64 apply of R contiguous vectors (chunks of at most kMaxRhs64)
    auto op64 = [&](const double2* v, double2* Av, const char*) -> cudaError_t {
      for (int r = 0; r < R;) {
        int nr = lsd::kMaxRhs64;
        while (nr > R - r) nr /= 2;
        cudaError_t e = run_apply(plan, LS_FP64, plan->d64, v + r * N, Av + r * N, nr, st);
        if (e != cudaSuccess) return e;
        r += nr;
      }
      return cudaSuccess;
    };
    // complex64 apply of R contiguous complex128 vectors (cast in, batched apply, cast out)
    auto op32 = [&](const double2* v, double2* Av, const char*) -> cudaError_t {
      cudaError_t e = lsd::to_c64(v, plan->K.c64a, int64_t(R) * N, st);
      for (int r = 0; r < R && e == cudaSuccess;) {
        int nr = plan->group32;
        while (nr > R - r) nr /= 2;
        e = run_apply(plan, LS_MIXED, plan->d32, plan->K.c64a + r * N, plan->K.c64b + r * N, nr, st);
        r += nr;
      }
      if (e == cudaSuccess) e = lsd::to_c128(plan->K.c64b, Av, int64_t(R) * N, st);
      return e;
    };
    // complex64 apply of R contiguous complex64 vectors (the LS_MIXED32 correction solves)
    auto op32f = [&](const float2* v, float2* Av, const char*) -> cudaError_t {
      cudaError_t e = cudaSuccess;
      for (int r = 0; r < R && e == cudaSuccess;) {
        int nr = plan->group32;
        while (nr > R - r) nr /= 2;
        e = run_apply(plan, LS_MIXED, plan->d32, v + r * N, Av + r * N, nr, st);
        r += nr;
      }
      return e;
    };
    SolveStats Sb;
    s = solve_lockstep(plan, plan->K, uniform_layout(R, N), op64, op32, op32f, prec,
                       static_cast<const double2*>(uinc) + int64_t(r0) * N, static_cast<double2*>(u) + int64_t(r0) * N,
                       tol, max_iter, restart, st, Sb);
    total_it += Sb.iterations;
    total_ref += Sb.refinements;
    worst = std::max(worst, Sb.worst);
    if (s != LS_OK) {
      result = s;
      if (s != LS_ERR_NOCONV) break;
    }
  }
  if (info) {
    info->iterations = total_it;
    info->refinements = total_ref;
    info->residual = worst;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  const ls_status dev = ls_plan_device_status(plan);
  return dev != LS_OK ? dev : result;
}

ls_status ls_farfield(ls_plan plan, const void* u, int nrhs, const double* dirs_host, int ndir, void* A,
                      void* stream) {
  if (!plan) return LS_ERR_INVALID;
  if (!u || !dirs_host || !A || nrhs < 0 || ndir < 0) return fail(plan, LS_ERR_INVALID, "ls_farfield: bad arguments");
  if (nrhs == 0 || ndir == 0) return LS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (ndir > plan->dirs_cap) {
    ls_status s = LS_OK;
    plan->dirs = plan->alloc<double>(size_t(2) * ndir, &s);
    if (s != LS_OK) return s;
    plan->dirs_cap = ndir;
  }
  if (plan->dim == 3) {
    if (3 * ndir > 2 * plan->dirs_cap) {
      ls_status s = LS_OK;
      plan->dirs = plan->alloc<double>(size_t(3) * ndir, &s);
      if (s != LS_OK) return s;
      plan->dirs_cap = (3 * ndir + 1) / 2;
    }
    LS_CU(cudaMemcpyAsync(plan->dirs, dirs_host, sizeof(double) * 3 * ndir, cudaMemcpyHostToDevice, st));
    const double k = std::sqrt(plan->e64.kappa2);
    LS_CU(lsd::farfield3(plan->e64.N, plan->x, plan->ffw3, static_cast<const double2*>(u), nrhs, plan->dirs, ndir,
                         k, make_double2(k * k / (4 * M_PI), 0.0), static_cast<double2*>(A), st));
    LS_CU(cudaStreamSynchronize(st));
    return LS_OK;
  }
  LS_CU(cudaMemcpyAsync(plan->dirs, dirs_host, sizeof(double) * 2 * ndir, cudaMemcpyHostToDevice, st));
  const double k = plan->host.kappa;
  const std::complex<double> c = std::polar(1.0, M_PI / 4) / std::sqrt(8 * M_PI * k) * (k * k);
  LS_CU(lsd::farfield(plan->d64.N, plan->x, plan->y, plan->ffw, static_cast<const double2*>(u), nrhs, plan->dirs,
                      ndir, k, make_double2(c.real(), c.imag()), static_cast<double2*>(A), st));
  LS_CU(cudaStreamSynchronize(st));
  return LS_OK;
}

ls_status ls_measure_peaks(double* fp64_tflops, double* tf32_tflops) {
  if (!fp64_tflops || !tf32_tflops) return LS_ERR_INVALID;
  const cudaError_t e = lsd::measure_peaks(fp64_tflops, tf32_tflops);
  if (e != cudaSuccess) {
    g_create_error = std::string("ls_measure_peaks: ") + cudaGetErrorString(e);
    return LS_ERR_CUDA;
  }
  if (*tf32_tflops < 0) {
    g_create_error = "ls_measure_peaks: a wait of the tensor-core probe gave up";
    return LS_ERR_TIMEOUT;
  }
  return LS_OK;
}

ls_status ls_set_wait_limit(ls_plan plan, int polls) {
  if (!plan) return LS_ERR_INVALID;
  if (polls < 0) return fail(plan, LS_ERR_INVALID, "ls_set_wait_limit: polls must be >= 0");
  LS_CU(cudaDeviceSynchronize());   // no captured apply may still run with the old limit
  plan->d32.tc_spin = polls;
  plan->d64.tc_spin = polls;
  plan->graphs.clear();             // captured applies hold the old limit
  return LS_OK;
}

ls_status ls_plan_device_status(ls_plan plan) {
  if (!plan) return LS_ERR_INVALID;
  if (!plan->d32.tc_err) {          // no kernel of this plan waits on the device (3-D plans)
    LS_CU(cudaDeviceSynchronize());
    return LS_OK;
  }
  int flag = 0;
  LS_CU(cudaMemcpy(&flag, plan->d32.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (!flag) return LS_OK;
  LS_CU(cudaMemset(plan->d32.tc_err, 0, sizeof(int)));
  return fail(plan, LS_ERR_TIMEOUT, "a device-side wait of the tensor-core near field timed out; "
                                    "the rows of the affected work items were not written");
}

ls_status ls_plan_autotune(ls_plan plan, int nrhs, ls_tune_report* report) {
  if (!plan) return LS_ERR_INVALID;
  if (plan->dim != 2) return fail(plan, LS_ERR_UNSUPPORTED, "ls_plan_autotune: 2-D plans only");
  if (nrhs < 1 || nrhs > 64) return fail(plan, LS_ERR_INVALID, "ls_plan_autotune: nrhs must be in [1, 64]");
  int cur = -1;
  LS_CU(cudaGetDevice(&cur));
  if (cur != plan->device) return fail(plan, LS_ERR_INVALID, "ls_plan_autotune: the plan's device is not current");
  const int64_t N = plan->d64.N;
  const int n64 = std::min(nrhs, lsd::kMaxRhs64);
  ls_status st = LS_OK;
  // scratch inputs (finite, not zero) and outputs; released before returning
  double2* u64 = plan->alloc<double2>(size_t(n64) * N, &st);
  double2* o64 = plan->alloc<double2>(size_t(n64) * N, &st);
  float2* u32 = plan->alloc<float2>(size_t(nrhs) * N, &st);
  float2* o32 = plan->alloc<float2>(size_t(nrhs) * N, &st);
  cudaStream_t ts = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ts) cudaStreamDestroy(ts);
    const void* scratch[4] = {u64, o64, u32, o32};
    for (const void* p : scratch) plan->release(p);
  };
  if (st != LS_OK) {
    cleanup();
    return fail(plan, st, "ls_plan_autotune: " + plan->err);
  }
  cudaError_t ce = cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(u64, 0x3c, size_t(n64) * N * sizeof(double2), ts);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(u32, 0x3c, size_t(nrhs) * N * sizeof(float2), ts);
  // mean milliseconds of one call of f (2 untimed, 5 timed); < 0 on a launch error
  auto timed = [&](auto f) -> double {
    for (int i = 0; i < 2; ++i)
      if (f() != cudaSuccess) return -1.0;
    cudaEventRecord(e0, ts);
    for (int i = 0; i < 5; ++i)
      if (f() != cudaSuccess) return -1.0;
    cudaEventRecord(e1, ts);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / 5;
  };
  ls_tune_report r{};
  r.nrhs = nrhs;
  const int conv_opts[4] = {1, 2, 4, 8};
  if (ce == cudaSuccess) {
    // FP64: columns per block of the column pass
    const int keep = plan->d64.conv_tc;
    double best = -1;
    int best_tc = 1;
    for (int tc : conv_opts) {
      plan->d64.conv_tc = tc;
      const double ms = timed([&] { return lsd::apply_batch(plan->d64, u64, o64, n64, ts); });
      cudaGetLastError();
      ++r.n_candidates;
      if (ms < 0) continue;
      if (tc == 1) r.ms64_default = ms;
      if (best < 0 || ms < best) { best = ms; best_tc = tc; }
    }
    plan->d64.conv_tc = best > 0 ? best_tc : keep;
    r.conv_cols64 = plan->d64.conv_tc > 0 ? plan->d64.conv_tc : 1;
    r.ms64_best = best;
    // complex64: columns per block x right-hand-side group x near-field unit
    const int keep_tc = plan->d32.conv_tc, keep_group = plan->group32;
    const bool keep_cuda = plan->d32.near_cuda;
    best = -1;
    int bt = 1, bg = keep_group;
    bool bc = false;
    const bool keep_lcuda = plan->d32.local_cuda, keep_pcuda = plan->d32.proj_cuda;
    bool blc = keep_lcuda, bpc = keep_pcuda;
    for (int tc : conv_opts)
      for (int grp = 16; grp >= 4; grp /= 2)
        for (int var = 0; var < 8; ++var) {
          // var bit 0: CUDA-core near field; bit 1: CUDA-core local coefficients; bit 2: CUDA-core
          // projection (groups of 8 or 16)
          const int cuda = var & 1, lcuda = (var >> 1) & 1, pcuda = var >> 2;
          if (grp > std::max(4, nrhs) || (var && grp < 8) || (lcuda && !plan->d32.LAt) ||
              (pcuda && plan->d32.n_es > 64))
            continue;
          plan->d32.conv_tc = tc;
          plan->d32.near_cuda = cuda != 0;
          plan->d32.local_cuda = lcuda != 0;
          plan->d32.proj_cuda = pcuda != 0;
          const double ms = timed([&] {
            for (int q = 0; q < nrhs;) {
              int nr = grp;
              while (nr > nrhs - q) nr /= 2;
              const cudaError_t e = lsd::apply_batch(plan->d32, u32 + int64_t(q) * N, o32 + int64_t(q) * N, nr, ts);
              if (e != cudaSuccess) return e;
              q += nr;
            }
            return cudaSuccess;
          });
          cudaGetLastError();
          ++r.n_candidates;
          if (ms < 0) continue;
          if (tc == 1 && grp == std::min(keep_group, std::max(4, nrhs)) && var == 0) r.ms32_default = ms;
          if (best < 0 || ms < best) {
            best = ms;
            bt = tc;
            bg = grp;
            bc = cuda != 0;
            blc = lcuda != 0;
            bpc = pcuda != 0;
          }
        }
    plan->d32.conv_tc = best > 0 ? bt : keep_tc;
    plan->d32.near_cuda = best > 0 ? bc : keep_cuda;
    plan->d32.local_cuda = best > 0 ? blc : keep_lcuda;
    plan->d32.proj_cuda = best > 0 ? bpc : keep_pcuda;
    plan->group32 = best > 0 ? bg : keep_group;
    r.conv_cols32 = plan->d32.conv_tc > 0 ? plan->d32.conv_tc : 1;
    r.group32 = plan->group32;
    r.near_cuda32 = plan->d32.near_cuda ? 1 : 0;
    r.local_cuda32 = plan->d32.local_cuda ? 1 : 0;
    r.proj_cuda32 = plan->d32.proj_cuda ? 1 : 0;
    r.ms32_best = best;
    // the lattice FFT's radix (16 or 4) for the chosen variants, on the same applies
    if (best > 0) {
      const bool keep_r4 = plan->d32.fft_r4;
      double ms_r[2] = {-1, -1};
      for (int r4 = 0; r4 < 2; ++r4) {
        plan->d32.fft_r4 = r4 != 0;
        ms_r[r4] = timed([&] {
          for (int q = 0; q < nrhs;) {
            int nr = plan->group32;
            while (nr > nrhs - q) nr /= 2;
            const cudaError_t e = lsd::apply_batch(plan->d32, u32 + int64_t(q) * N, o32 + int64_t(q) * N, nr, ts);
            if (e != cudaSuccess) return e;
            q += nr;
          }
          return cudaSuccess;
        });
        cudaGetLastError();
        ++r.n_candidates;
      }
      plan->d32.fft_r4 = (ms_r[0] > 0 && ms_r[1] > 0) ? ms_r[1] < ms_r[0] : keep_r4;
      if (ms_r[0] > 0 && ms_r[1] > 0) r.ms32_best = std::min(ms_r[0], ms_r[1]);
    }
    r.fft_radix32 = plan->d32.fft_r4 ? 4 : 16;
    ce = cudaStreamSynchronize(ts);
  }
  cleanup();
  plan->graphs.clear();          // captured applies hold the previous variants
  if (ce != cudaSuccess) return fail(plan, LS_ERR_CUDA, std::string("ls_plan_autotune: ") + cudaGetErrorString(ce));
  if (plan->d32.tc_err) {
    int flag = 0;
    LS_CU(cudaMemcpy(&flag, plan->d32.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return fail(plan, LS_ERR_TIMEOUT, "ls_plan_autotune: a device-side wait of the tensor-core near field "
                                                "timed out; see ls_plan_device_status");
  }
  if (report) *report = r;
  return LS_OK;
}

ls_status ls_plan_set_variants(ls_plan plan, const ls_tune_report* v) {
  if (!plan) return LS_ERR_INVALID;
  if (plan->dim != 2) return fail(plan, LS_ERR_UNSUPPORTED, "ls_plan_set_variants: 2-D plans only");
  if (!v) return fail(plan, LS_ERR_INVALID, "ls_plan_set_variants: null report");
  auto cols_ok = [](int c) { return c == 1 || c == 2 || c == 4 || c == 8; };
  auto flag_ok = [](int f) { return f == 0 || f == 1; };
  if (!cols_ok(v->conv_cols64) || !cols_ok(v->conv_cols32) ||
      (v->group32 != 4 && v->group32 != 8 && v->group32 != 16) || !flag_ok(v->near_cuda32) ||
      !flag_ok(v->local_cuda32) || !flag_ok(v->proj_cuda32) ||
      (v->fft_radix32 != 0 && v->fft_radix32 != 4 && v->fft_radix32 != 16))
    return fail(plan, LS_ERR_INVALID, "ls_plan_set_variants: columns must be 1, 2, 4 or 8, the group 4, 8 or 16, "
                                      "the unit flags 0 or 1, the FFT radix 4 or 16");
  const bool r4 = v->fft_radix32 == 4;
  if (!lsd::lattice_cols_fit(true, false, plan->d64.M, v->conv_cols64) ||
      !lsd::lattice_cols_fit(false, r4, plan->d32.M, v->conv_cols32))
    return fail(plan, LS_ERR_INVALID, "ls_plan_set_variants: the lattice column pass does not fit " +
                                          std::to_string(v->conv_cols64) + " / " + std::to_string(v->conv_cols32) +
                                          " columns per block at lattice size " + std::to_string(plan->d64.M));
  plan->d64.conv_tc = v->conv_cols64;
  plan->d32.conv_tc = v->conv_cols32;
  plan->group32 = v->group32;
  plan->d32.near_cuda = v->near_cuda32 != 0;
  plan->d32.local_cuda = v->local_cuda32 != 0;
  plan->d32.proj_cuda = v->proj_cuda32 != 0;
  plan->d32.fft_r4 = r4;
  plan->graphs.clear();          // captured applies hold the previous variants
  return LS_OK;
}

ls_status ls_set_stage_timing(ls_plan plan, int enable) {
  if (!plan) return LS_ERR_INVALID;
  if (enable && !plan->ev[0])
    for (auto& e : plan->ev) LS_CU(cudaEventCreate(&e));
  plan->timing = enable != 0;
  for (auto& row : plan->stage_ms)
    for (double& v : row) v = 0;
  plan->stage_calls[0] = plan->stage_calls[1] = 0;
  return LS_OK;
}

ls_status ls_get_stage_times(ls_plan plan, ls_precision prec, double* ms, int64_t* calls) {
  if (!plan || !ms || (prec != LS_FP64 && prec != LS_MIXED)) return LS_ERR_INVALID;
  for (int k = 0; k < lsd::kStages; ++k) ms[k] = plan->stage_ms[prec][k];
  if (calls) *calls = plan->stage_calls[prec];
  return LS_OK;
}

ls_status ls_plan_destroy(ls_plan plan) {
  if (!plan) return LS_OK;
  cudaDeviceSynchronize();
  for (auto& e : plan->ev)
    if (e) cudaEventDestroy(e);
  plan->free_all();
  delete plan;
  return LS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free apply.
//
// Some callers cannot allocate device memory at the moment they want an
// operator application: code running under a CUDA stream capture (where a
// cudaMalloc would break the capture), code inside another library's memory
// pool that forbids outside allocations, or real-time loops that must never
// reach the allocator.  ls_apply_noalloc serves them: it works exactly like
// ls_apply for one right-hand side but keeps its intermediate arrays (the
// equivalent-source strengths, the two lattice grids and the local-expansion
// coefficients) in the fixed device array below instead of in plan memory.
// Every GPU that loads this library reserves these bytes until the process
// exits.  All calls share the array, so calls whose GPU work overlaps (two
// streams, two host threads, two plans) corrupt each other's results: order
// them on one stream or synchronise between them.  Every element the apply
// reads from the array is written earlier in the same call, so nothing has to
// start at zero.
static constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[256] = {};   // device address of the array, per device ordinal

template <typename T>
ls_status noalloc_apply(ls_plan plan, const lsd::ApplyData<T>& src, const void* u, void* Au, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return fail(plan, LS_ERR_CUDA, std::string("ls_apply_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 256)
    return fail(plan, LS_ERR_INVALID, "ls_apply_noalloc: device ordinal " + std::to_string(dev) +
                                          " is outside the 256 devices this entry point supports");
  if (dev != plan->device)
    // the fixed array of the current device and the plan's arrays would sit on
    // two different GPUs
    return fail(plan, LS_ERR_INVALID, "ls_apply_noalloc: the current device (" + std::to_string(dev) +
                                          ") is not the plan's device (" + std::to_string(plan->device) +
                                          "); make the plan's device current first");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // the name of a __device__ array is a host-side stand-in; ask the runtime
      // for its device address once per device, with that device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return fail(plan, LS_ERR_CUDA,
                    std::string("ls_apply_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_noalloc_ptr[dev] = p;
    }
    base = g_noalloc_ptr[dev];
  }
  const size_t n_sigma = size_t(src.nocc) * src.n_es, n_grid = size_t(src.lattice_rows()) * src.M;
  const size_t n_gamma = size_t(src.nocc) * src.nfb2;
  auto up256 = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t need = up256(n_sigma * sizeof(T)) + 2 * up256(n_grid * sizeof(T)) + up256(n_gamma * sizeof(T));
  if (need > kNoAllocScratchBytes)
    return fail(plan, LS_ERR_INVALID,
                "ls_apply_noalloc: this plan needs " + std::to_string(need) + " bytes of work space but the " +
                "fixed device array holds " + std::to_string(kNoAllocScratchBytes) +
                " bytes (lattice FFT size M too large); use ls_apply");
  lsd::ApplyData<T> d = src;
  unsigned char* p = static_cast<unsigned char*>(base);
  d.sigma = reinterpret_cast<T*>(p);
  p += up256(n_sigma * sizeof(T));
  d.Sm = reinterpret_cast<T*>(p);
  p += up256(n_grid * sizeof(T));
  d.Sd = reinterpret_cast<T*>(p);
  p += up256(n_grid * sizeof(T));
  d.gamma = reinterpret_cast<T*>(p);
  // the projection runs one block per whole cell (no partial sums or counters
  // in plan memory) and the near field forms its staged inputs itself
  d.pieces = src.cell_pieces;
  d.n_pieces = src.nocc;
  d.proj_part = nullptr;
  d.proj_count = nullptr;
  d.utc = nullptr;
  d.utef = nullptr;
  e = lsd::apply_one(d, static_cast<const T*>(u), static_cast<T*>(Au), st);
  if (e != cudaSuccess) return fail(plan, LS_ERR_CUDA, std::string("ls_apply_noalloc: ") + cudaGetErrorString(e));
  return LS_OK;
}
}  // namespace

extern "C" ls_status ls_apply_noalloc(ls_plan plan, const void* u, void* Au, ls_precision prec, void* stream) {
  if (!plan) return LS_ERR_INVALID;
  if (plan->dim != 2) return fail(plan, LS_ERR_UNSUPPORTED, "ls_apply_noalloc: 2-D plans only");
  if (!u || !Au) return fail(plan, LS_ERR_INVALID, "ls_apply_noalloc: null vector");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == LS_FP64) return noalloc_apply(plan, plan->d64, u, Au, st);
  if (prec == LS_MIXED) return noalloc_apply(plan, plan->d32, u, Au, st);
  return fail(plan, LS_ERR_INVALID, "ls_apply_noalloc: bad precision");
}

// ---------------------------------------------------------------- multi-instance batches
// Work lists of a subset of a batch's instances (the instances still
// iterating in a lock-step solve): device arrays owned by the set.
struct ActiveSet {
  std::vector<int> ids;
  int2* pieces = nullptr;
  int n_pieces = 0;
  int2* cells = nullptr;
  int n_cells = 0;
  int4* items = nullptr;
  int n_items = 0;
  int2* lat_lists = nullptr;           // the lattice work lists of every lattice size, back to back
  std::vector<lsd::LatWork> lat;       // one per lattice size among the active instances
  void release() {
    if (pieces) cudaFree(pieces);
    if (cells) cudaFree(cells);
    if (items) cudaFree(items);
    if (lat_lists) cudaFree(lat_lists);
    pieces = nullptr;
    cells = nullptr;
    items = nullptr;
    lat_lists = nullptr;
    lat.clear();
  }
};

struct ls_batch_s : DevOwner {
  std::vector<ls_plan> plans;
  std::vector<int64_t> off;                          // n + 1 node offsets in the concatenated vectors
  std::vector<lsd::InstData<double2>> h64;
  std::vector<lsd::InstData<float2>> h32;
  const lsd::InstData<double2>* d64 = nullptr;
  const lsd::InstData<float2>* d32 = nullptr;
  std::vector<std::vector<int>> cells_of, items_of;  // host work lists per instance (pairs / quadruples)
  std::vector<std::vector<int>> piece_len;           // node count of each projection piece, per instance
  int max_K = 0;
  std::map<std::vector<char>, int> set_of;           // instance subset -> index in sets
  std::vector<ActiveSet> sets;
  Krylov K;
  GraphCache graphs;
  void release_sets() {
    for (auto& a : sets) a.release();
    sets.clear();
    set_of.clear();
  }
};

namespace {

// Index of the work lists of the instances with need[i] != 0 (all if need is
// null), built and uploaded on first use.  A lock-step solve meets at most
// n + 1 subsets (instances only drop out); the cache is bounded.
int active_set(ls_batch b, const char* need, cudaError_t* err) {
  const int n = int(b->plans.size());
  std::vector<char> key(n, 1);
  if (need)
    for (int i = 0; i < n; ++i) key[i] = need[i] ? 1 : 0;
  auto it = b->set_of.find(key);
  if (it != b->set_of.end()) return it->second;
  if (b->sets.size() >= 256) {                       // many distinct subsets: start over
    cudaDeviceSynchronize();                         // no graph of the old lists may still run
    b->graphs.clear();
    b->release_sets();
  }
  ActiveSet a;
  std::vector<int> cells, items;
  std::vector<std::pair<int, int2>> pcs;             // (node count, (instance, piece))
  for (int i = 0; i < n; ++i) {
    if (!key[i]) continue;
    a.ids.push_back(i);
    cells.insert(cells.end(), b->cells_of[i].begin(), b->cells_of[i].end());
    items.insert(items.end(), b->items_of[i].begin(), b->items_of[i].end());
    for (size_t q = 0; q < b->piece_len[i].size(); ++q) pcs.push_back({b->piece_len[i][q], make_int2(i, int(q))});
  }
  // the largest projection pieces of all active instances first
  std::stable_sort(pcs.begin(), pcs.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
  std::vector<int2> pieces(pcs.size());
  for (size_t q = 0; q < pcs.size(); ++q) pieces[q] = pcs[q].second;
  a.n_pieces = int(pieces.size());
  a.n_cells = int(cells.size() / 2);
  a.n_items = int(items.size() / 4);
  // lattice work lists per lattice size: (instance, face row), (instance, column), (instance, kept row)
  std::map<int, std::vector<int>> by_M;
  for (int i : a.ids) by_M[b->plans[i]->d64.M].push_back(i);
  std::vector<int2> lat_lists;
  std::vector<std::array<size_t, 3>> lat_off;
  for (const auto& [M, group] : by_M) {
    lsd::LatWork w;
    w.M = M;
    std::array<size_t, 3> o{};
    o[0] = lat_lists.size();
    for (int i : group)
      for (int k = 0; k <= b->plans[i]->d64.L; ++k) lat_lists.push_back(make_int2(i, k));
    o[1] = lat_lists.size();
    for (int i : group)
      for (int c = 0; c < M; ++c) lat_lists.push_back(make_int2(i, c));
    o[2] = lat_lists.size();
    for (int i : group)
      for (int r = 0; r < b->plans[i]->d64.n_lat; ++r) lat_lists.push_back(make_int2(i, r));
    w.n_src = int(o[1] - o[0]);
    w.n_cols = int(o[2] - o[1]);
    w.n_rows = int(lat_lists.size() - o[2]);
    a.lat.push_back(w);
    lat_off.push_back(o);
  }
  *err = cudaSuccess;
  if (!lat_lists.empty()) {
    *err = cudaMalloc(&a.lat_lists, lat_lists.size() * sizeof(int2));
    if (*err == cudaSuccess)
      *err = cudaMemcpy(a.lat_lists, lat_lists.data(), lat_lists.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (*err != cudaSuccess) {
      a.release();
      return -1;
    }
    for (size_t g = 0; g < a.lat.size(); ++g) {
      a.lat[g].src = a.lat_lists + lat_off[g][0];
      a.lat[g].cols = a.lat_lists + lat_off[g][1];
      a.lat[g].rows = a.lat_lists + lat_off[g][2];
    }
  }
  if (!cells.empty()) {
    *err = cudaMalloc(&a.cells, cells.size() * sizeof(int));
    if (*err == cudaSuccess) *err = cudaMalloc(&a.items, items.size() * sizeof(int));
    if (*err == cudaSuccess) *err = cudaMalloc(&a.pieces, pieces.size() * sizeof(int2));
    if (*err == cudaSuccess)
      *err = cudaMemcpy(a.cells, cells.data(), cells.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (*err == cudaSuccess)
      *err = cudaMemcpy(a.items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (*err == cudaSuccess)
      *err = cudaMemcpy(a.pieces, pieces.data(), pieces.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (*err != cudaSuccess) {
      a.release();
      return -1;
    }
  }
  b->sets.push_back(std::move(a));
  const int idx = int(b->sets.size()) - 1;
  b->set_of[key] = idx;
  return idx;
}

// need: per-instance flags (nullptr = every instance); the apply covers only
// the instances with need != 0.
template <typename T>
cudaError_t batch_apply_t(ls_batch b, int prec, const lsd::InstData<T>* dI,
                          const T* u, T* out, cudaStream_t st, const char* need = nullptr) {
  cudaError_t err = cudaSuccess;
  const int si = active_set(b, need, &err);
  if (si < 0) return err;
  const ActiveSet& a = b->sets[si];
  if (a.ids.empty()) return cudaSuccess;
  auto launch = [&](cudaStream_t s) {
    return lsd::apply_multi<T>(dI, int(a.ids.size()), a.pieces, a.n_pieces, a.cells, a.n_cells, a.items,
                               a.n_items, b->max_K, a.lat.data(), int(a.lat.size()), u, out, s);
  };
  return b->graphs.run(GraphCache::Key(prec, si, static_cast<const void*>(u), static_cast<void*>(out)), launch, st);
}

Layout batch_layout(ls_batch b) {
  Layout L;
  L.R = int(b->plans.size());
  for (int i = 0; i < L.R; ++i) { L.off.push_back(b->off[i]); L.len.push_back(b->off[i + 1] - b->off[i]); }
  L.total = b->off.back();
  return L;
}

}  // namespace

extern "C" {

ls_status ls_batch_create(const ls_plan* plans, int n_plans, ls_batch* out) {
  if (!out) return LS_ERR_INVALID;
  *out = nullptr;
  if (!plans || n_plans < 1) return fail(nullptr, LS_ERR_INVALID, "ls_batch_create: no plans");
  // handles are compared before any is dereferenced
  for (int i = 0; i < n_plans; ++i) {
    if (!plans[i]) return fail(nullptr, LS_ERR_INVALID, "ls_batch_create: null plan");
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i])
        return fail(nullptr, LS_ERR_INVALID, "ls_batch_create: a plan appears twice (instances would share its "
                                             "work arrays)");
  }
  for (int i = 0; i < n_plans; ++i)
    if (plans[i]->dim != 2) return fail(nullptr, LS_ERR_UNSUPPORTED, "ls_batch_create: 2-D plans only");
  auto* b = new (std::nothrow) ls_batch_s();
  if (!b) return fail(nullptr, LS_ERR_NOMEM, "ls_batch_create: host allocation");
  auto bail = [&](ls_status s) {
    g_create_error = b->err;
    b->release_sets();
    b->free_bufs();
    delete b;
    return s;
  };
  b->plans.assign(plans, plans + n_plans);
  b->off.push_back(0);
  for (int i = 0; i < n_plans; ++i) {
    const ls_plan p = plans[i];
    b->h64.push_back({p->d64, b->off.back()});
    b->h32.push_back({p->d32, b->off.back()});
    b->off.push_back(b->off.back() + p->d64.N);
    b->max_K = std::max(b->max_K, p->d64.n_loc + 9 * p->d64.n_es);
    std::vector<int> cells, items;
    for (int k = 0; k < p->d64.nocc; ++k) { cells.push_back(i); cells.push_back(k); }
    std::vector<int> it(size_t(2) * p->d64.n_items);
    if (cudaMemcpy(it.data(), p->d64.items, it.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      b->err = "ls_batch_create: reading a plan's work items failed";
      return bail(LS_ERR_CUDA);
    }
    for (size_t e = 0; e < it.size(); e += 2) {
      items.push_back(i); items.push_back(it[e]); items.push_back(it[e + 1]); items.push_back(0);
    }
    std::vector<int> pc(size_t(4) * p->d64.n_pieces), len(p->d64.n_pieces);
    if (cudaMemcpy(pc.data(), p->d64.pieces, pc.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      b->err = "ls_batch_create: reading a plan's projection pieces failed";
      return bail(LS_ERR_CUDA);
    }
    for (int q = 0; q < p->d64.n_pieces; ++q) len[q] = pc[4 * q + 2] - pc[4 * q + 1];
    b->cells_of.push_back(std::move(cells));
    b->items_of.push_back(std::move(items));
    b->piece_len.push_back(std::move(len));
  }
  int64_t n_cells = 0, n_items = 0;
  for (int i = 0; i < n_plans; ++i) {
    n_cells += int64_t(b->cells_of[i].size() / 2);
    n_items += int64_t(b->items_of[i].size() / 4);
  }
  if (n_cells > INT32_MAX || n_items > INT32_MAX) {
    b->err = "ls_batch_create: work lists too long";
    return bail(LS_ERR_INVALID);
  }
  ls_status st = LS_OK;
  b->d64 = b->upload<lsd::InstData<double2>>(b->h64, &st);
  if (st != LS_OK) return bail(st);
  b->d32 = b->upload<lsd::InstData<float2>>(b->h32, &st);
  if (st != LS_OK) return bail(st);
  cudaError_t ce = cudaSuccess;
  if (active_set(b, nullptr, &ce) < 0) {
    cudaGetLastError();
    b->err = std::string("ls_batch_create: work list upload: ") + cudaGetErrorString(ce);
    return bail(LS_ERR_NOMEM);
  }
  *out = b;
  return LS_OK;
}

ls_status ls_batch_offsets(ls_batch b, int64_t* off_host) {
  if (!b || !off_host) return LS_ERR_INVALID;
  std::copy(b->off.begin(), b->off.end(), off_host);
  return LS_OK;
}

ls_status ls_batch_apply(ls_batch b, const void* u, void* Au, ls_precision prec, void* stream) {
  if (!b) return LS_ERR_INVALID;
  DevOwner* plan = b;
  if (!u || !Au) return fail(b, LS_ERR_INVALID, "ls_batch_apply: bad arguments");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == LS_FP64)
    LS_CU(batch_apply_t(b, prec, b->d64, static_cast<const double2*>(u), static_cast<double2*>(Au), st));
  else if (prec == LS_MIXED)
    LS_CU(batch_apply_t(b, prec, b->d32, static_cast<const float2*>(u), static_cast<float2*>(Au), st));
  else
    return fail(b, LS_ERR_INVALID, "ls_batch_apply: bad precision");
  return LS_OK;
}

ls_status ls_batch_solve(ls_batch b, const void* uinc, void* u, double tol, int max_iter, int restart,
                         ls_precision prec, ls_solve_info* info, ls_solve_info* per, void* stream) {
  if (!b) return LS_ERR_INVALID;
  if (!uinc || !u || !(tol > 0) || max_iter < 1 || restart < 1)
    return fail(b, LS_ERR_INVALID, "ls_batch_solve: bad arguments");
  if (prec != LS_FP64 && prec != LS_MIXED && prec != LS_MIXED32)
    return fail(b, LS_ERR_INVALID, "ls_batch_solve: bad precision");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Layout lay = batch_layout(b);
  ls_status s = ensure_krylov(b, b->K, restart, lay);
  if (s != LS_OK) return s;
  auto op64 = [&](const double2* v, double2* Av, const char* need) -> cudaError_t {
    return batch_apply_t(b, LS_FP64, b->d64, v, Av, st, need);
  };
  auto op32 = [&](const double2* v, double2* Av, const char* need) -> cudaError_t {
    cudaError_t e = lsd::to_c64(v, b->K.c64a, lay.total, st);
    if (e == cudaSuccess) e = batch_apply_t(b, LS_MIXED, b->d32, b->K.c64a, b->K.c64b, st, need);
    if (e == cudaSuccess) e = lsd::to_c128(b->K.c64b, Av, lay.total, st);
    return e;
  };
  auto op32f = [&](const float2* v, float2* Av, const char* need) -> cudaError_t {
    return batch_apply_t(b, LS_MIXED, b->d32, v, Av, st, need);
  };
  SolveStats S;
  s = solve_lockstep(b, b->K, lay, op64, op32, op32f, prec, static_cast<const double2*>(uinc), static_cast<double2*>(u), tol,
                     max_iter, restart, st, S);
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info) {
    info->iterations = S.iterations;
    info->refinements = S.refinements;
    info->residual = S.worst;
    info->seconds = secs;
  }
  if (per)
    for (int i = 0; i < lay.R; ++i) {
      per[i].iterations = S.it_per.empty() ? 0 : S.it_per[i];
      per[i].refinements = S.refinements;
      per[i].residual = S.res_per.empty() ? 0 : S.res_per[i];
      per[i].seconds = secs;
    }
  for (ls_plan p : b->plans)
    if (ls_plan_device_status(p) != LS_OK) return fail(b, LS_ERR_TIMEOUT, p->err);
  return s;
}

ls_status ls_batch_destroy(ls_batch b) {
  if (!b) return LS_OK;
  cudaDeviceSynchronize();
  b->K.free_pinned();
  b->graphs.release();
  b->release_sets();
  b->free_bufs();
  delete b;
  return LS_OK;
}

const char* ls_batch_last_error(ls_batch b) { return b ? b->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
