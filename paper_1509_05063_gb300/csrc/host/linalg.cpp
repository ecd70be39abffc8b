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
