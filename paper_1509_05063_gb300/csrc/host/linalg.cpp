// Small dense complex linear algebra for plan construction: a one-sided
// (Hestenes) Jacobi SVD, which keeps small singular values to high relative
// accuracy, and a least-squares solve applied factor by factor.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "host_plan.hpp"

namespace lsh {

SVD svd_truncated(const std::vector<cd>& A, int m, int n, double rcond) {
  // work on columns: Uc[j] is column j (length m), Vc[j] column j of V (length n)
  std::vector<cd> Uc(size_t(m) * n), Vc(size_t(n) * n, cd(0.0));
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) Uc[size_t(j) * m + i] = A[size_t(i) * n + j];
  for (int j = 0; j < n; ++j) Vc[size_t(j) * n + j] = 1.0;
  const double eps = 2.2e-16;
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        cd* up = &Uc[size_t(p) * m];
        cd* uq = &Uc[size_t(q) * m];
        double alpha = 0, beta = 0;
        cd gamma = 0;
        for (int i = 0; i < m; ++i) {
          alpha += std::norm(up[i]);
          beta += std::norm(uq[i]);
          gamma += std::conj(up[i]) * uq[i];
        }
        const double ag = std::abs(gamma);
        if (ag == 0.0 || ag <= eps * std::sqrt(alpha * beta)) continue;
        rotated = true;
        const cd ph = gamma / ag;                       // e^{i phi}
        const double zeta = (beta - alpha) / (2.0 * ag);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        const cd sph = s * std::conj(ph);               // s e^{-i phi}
        for (int i = 0; i < m; ++i) {
          const cd a = up[i], b = uq[i];
          up[i] = c * a - sph * b;
          uq[i] = s * a + c * std::conj(ph) * b;
        }
        cd* vp = &Vc[size_t(p) * n];
        cd* vq = &Vc[size_t(q) * n];
        for (int i = 0; i < n; ++i) {
          const cd a = vp[i], b = vq[i];
          vp[i] = c * a - sph * b;
          vq[i] = s * a + c * std::conj(ph) * b;
        }
      }
    if (!rotated) break;
  }
  std::vector<double> sv(n);
  for (int j = 0; j < n; ++j) {
    double s2 = 0;
    for (int i = 0; i < m; ++i) s2 += std::norm(Uc[size_t(j) * m + i]);
    sv[j] = std::sqrt(s2);
  }
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return sv[a] > sv[b]; });
  SVD f;
  f.m = m; f.n = n;
  const double smax = sv[ord[0]];
  int k = 0;
  while (k < n && sv[ord[k]] > rcond * smax) ++k;
  f.k = k;
  f.U.resize(size_t(m) * k); f.V.resize(size_t(n) * k); f.s.resize(k);
  for (int r = 0; r < k; ++r) {
    const int j = ord[r];
    f.s[r] = sv[j];
    for (int i = 0; i < m; ++i) f.U[size_t(r) * m + i] = Uc[size_t(j) * m + i] / sv[j];
    for (int i = 0; i < n; ++i) f.V[size_t(r) * n + i] = Vc[size_t(j) * n + i];
  }
  return f;
}

// One-sided Jacobi sweeps on the columns of X (len x n, column-major),
// accumulating the rotations into J (n x n, column-major); real arithmetic in
// the inner loops.
static void jacobi_columns(std::vector<cd>& X, int len, int n, std::vector<cd>& J) {
  const double eps = 2.2e-16;
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double* up = reinterpret_cast<double*>(&X[size_t(p) * len]);
        double* uq = reinterpret_cast<double*>(&X[size_t(q) * len]);
        double alpha = 0, beta = 0, gr = 0, gi = 0;
        for (int i = 0; i < len; ++i) {
          const double ar = up[2 * i], ai = up[2 * i + 1], br = uq[2 * i], bi = uq[2 * i + 1];
          alpha += ar * ar + ai * ai;
          beta += br * br + bi * bi;
          gr += ar * br + ai * bi;                      // conj(a) b
          gi += ar * bi - ai * br;
        }
        const double ag = std::hypot(gr, gi);
        if (ag == 0.0 || ag <= eps * std::sqrt(alpha * beta)) continue;
        rotated = true;
        const double pr = gr / ag, pi = gi / ag;        // e^{i phi}
        const double zeta = (beta - alpha) / (2.0 * ag);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        // a' = c a - s e^{-i phi} b,  b' = s a + c e^{-i phi} b
        auto rot = [&](double* a, double* b, int m) {
          for (int i = 0; i < m; ++i) {
            const double ar = a[2 * i], ai = a[2 * i + 1], br = b[2 * i], bi = b[2 * i + 1];
            const double er = pr * br + pi * bi, ei = pr * bi - pi * br;   // e^{-i phi} b
            a[2 * i] = c * ar - sn * er;
            a[2 * i + 1] = c * ai - sn * ei;
            b[2 * i] = sn * ar + c * er;
            b[2 * i + 1] = sn * ai + c * ei;
          }
        };
        rot(up, uq, len);
        rot(reinterpret_cast<double*>(&J[size_t(p) * n]), reinterpret_cast<double*>(&J[size_t(q) * n]), n);
      }
    if (!rotated) break;
  }
}

SVD svd_truncated_qr(const std::vector<cd>& A, int m, int n, double rcond) {
  // Householder QR with column pivoting, A P = Q R (Businger-Golub), then
  // one-sided Jacobi on X = R^H: X J = U_x Sigma, so A = (Q J) Sigma (P U_x)^H
  // (the QR-preconditioned Jacobi SVD of Drmac and Veselic).
  std::vector<cd> W(size_t(m) * n);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) W[size_t(j) * m + i] = A[size_t(i) * n + j];
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::vector<std::vector<cd>> refl(n);
  std::vector<cd> R(size_t(n) * n, cd(0.0));   // column-major, upper triangular
  for (int j = 0; j < n; ++j) {
    int best = j;
    double bn = -1;
    for (int c = j; c < n; ++c) {
      double s2 = 0;
      for (int i = j; i < m; ++i) s2 += std::norm(W[size_t(c) * m + i]);
      if (s2 > bn) { bn = s2; best = c; }
    }
    if (best != j) {
      std::swap_ranges(W.begin() + size_t(j) * m, W.begin() + size_t(j + 1) * m, W.begin() + size_t(best) * m);
      std::swap(perm[j], perm[best]);
      for (int i = 0; i < j; ++i) std::swap(R[size_t(j) * n + i], R[size_t(best) * n + i]);
    }
    cd* x = &W[size_t(j) * m];
    const double xn = std::sqrt(bn > 0 ? bn : 0.0);
    std::vector<cd> v(x + j, x + m);
    cd alpha = 0;
    if (xn > 0) {
      const double a0 = std::abs(v[0]);
      const cd ph = a0 > 0 ? v[0] / a0 : cd(1.0);
      alpha = -ph * xn;
      v[0] -= alpha;
      double vn2 = 0;
      for (const cd& e : v) vn2 += std::norm(e);
      const double inv = vn2 > 0 ? 1.0 / std::sqrt(vn2) : 0.0;
      for (cd& e : v) e *= inv;                       // H = I - 2 v v^H
      for (int c = j + 1; c < n; ++c) {
        cd* y = &W[size_t(c) * m + j];
        cd d = 0;
        for (int i = 0; i < m - j; ++i) d += std::conj(v[i]) * y[i];
        d *= 2.0;
        for (int i = 0; i < m - j; ++i) y[i] -= d * v[i];
      }
    } else {
      std::fill(v.begin(), v.end(), cd(0.0));
    }
    R[size_t(j) * n + j] = alpha;
    for (int c = j + 1; c < n; ++c) R[size_t(c) * n + j] = W[size_t(c) * m + j];
    refl[j] = std::move(v);
  }
  // X = R^H (column j of X = conjugate of row j of R)
  std::vector<cd> X(size_t(n) * n, cd(0.0)), J(size_t(n) * n, cd(0.0));
  for (int j = 0; j < n; ++j)
    for (int i = j; i < n; ++i) X[size_t(j) * n + i] = std::conj(R[size_t(i) * n + j]);
  for (int j = 0; j < n; ++j) J[size_t(j) * n + j] = 1.0;
  jacobi_columns(X, n, n, J);
  std::vector<double> sv(n);
  for (int j = 0; j < n; ++j) {
    double s2 = 0;
    for (int i = 0; i < n; ++i) s2 += std::norm(X[size_t(j) * n + i]);
    sv[j] = std::sqrt(s2);
  }
  std::vector<int> ord(n);
  std::iota(ord.begin(), ord.end(), 0);
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return sv[a] > sv[b]; });
  SVD f;
  f.m = m; f.n = n;
  const double smax = sv[ord[0]];
  int k = 0;
  while (k < n && sv[ord[k]] > rcond * smax) ++k;
  f.k = k;
  f.U.assign(size_t(m) * k, cd(0.0)); f.V.resize(size_t(n) * k); f.s.resize(k);
  for (int r = 0; r < k; ++r) {
    const int j = ord[r];
    f.s[r] = sv[j];
    for (int i = 0; i < n; ++i) f.V[size_t(r) * n + perm[i]] = X[size_t(j) * n + i] / sv[j];
    // U column = Q (J column, zero-padded): reflectors applied last to first
    cd* u = &f.U[size_t(r) * m];
    for (int i = 0; i < n; ++i) u[i] = J[size_t(j) * n + i];
    for (int h = n - 1; h >= 0; --h) {
      const std::vector<cd>& v = refl[h];
      cd d = 0;
      for (int i = 0; i < m - h; ++i) d += std::conj(v[i]) * u[h + i];
      d *= 2.0;
      for (int i = 0; i < m - h; ++i) u[h + i] -= d * v[i];
    }
  }
  return f;
}

std::vector<cd> svd_solve(const SVD& f, const std::vector<cd>& B, int nb) {
  // C = S^-1 U^H B  (k x nb), X = V C (n x nb)
  std::vector<cd> C(size_t(f.k) * nb, cd(0.0));
  for (int r = 0; r < f.k; ++r) {
    const cd* u = &f.U[size_t(r) * f.m];
    cd* c = &C[size_t(r) * nb];
    for (int i = 0; i < f.m; ++i) {
      const cd ui = std::conj(u[i]);
      const cd* b = &B[size_t(i) * nb];
      for (int j = 0; j < nb; ++j) c[j] += ui * b[j];
    }
    for (int j = 0; j < nb; ++j) c[j] /= f.s[r];
  }
  std::vector<cd> X(size_t(f.n) * nb, cd(0.0));
  for (int r = 0; r < f.k; ++r) {
    const cd* v = &f.V[size_t(r) * f.n];
    const cd* c = &C[size_t(r) * nb];
    for (int i = 0; i < f.n; ++i) {
      cd* x = &X[size_t(i) * nb];
      const cd vi = v[i];
      for (int j = 0; j < nb; ++j) x[j] += vi * c[j];
    }
  }
  return X;
}

}  // namespace lsh
