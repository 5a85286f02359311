// Host-side dense linear algebra of the driver: the symmetric eigen-decomposition
// of the residual check's Gram matrix and the SVD of the Galerkin core Z for the
// post-processing of the solution.  Plain C++ on small (m x m, j x j) matrices,
// header-only so that it also builds without the CUDA toolkit.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace cr_host {

// Host Jacobi eigen-decomposition of a symmetric n x n matrix (column-major);
// eigenvectors in V (columns), eigenvalues in w.
inline void sym_eig(int n, std::vector<double> A, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i + (size_t)i * n] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        const double x = A[a + (size_t)b * n];
        tot += x * x;
        if (a != b) off += x * x;
      }
    // converged once the off-diagonal mass is at the rounding level of the matrix
    constexpr double eps = 2.220446049250313e-16;
    if (off <= (double)n * n * eps * eps * tot || off == 0.0) break;
    for (int pp = 0; pp < n - 1; ++pp)
      for (int qq = pp + 1; qq < n; ++qq) {
        const double apq = A[pp + (size_t)qq * n];
        if (apq == 0.0) continue;
        const double app = A[pp + (size_t)pp * n], aqq = A[qq + (size_t)qq * n];
        if (std::fabs(apq) <= eps * std::sqrt(std::fabs(app) * std::fabs(aqq))) {
          // negligible against its diagonal pair: no rotation needed
          A[pp + (size_t)qq * n] = A[qq + (size_t)pp * n] = 0.0;
          continue;
        }
        const double th = (aqq - app) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double cth = 1.0 / std::sqrt(t * t + 1.0), sth = t * cth;
        for (int k = 0; k < n; ++k) {
          const double akp = A[k + (size_t)pp * n], akq = A[k + (size_t)qq * n];
          A[k + (size_t)pp * n] = cth * akp - sth * akq;
          A[k + (size_t)qq * n] = sth * akp + cth * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = A[pp + (size_t)k * n], aqk = A[qq + (size_t)k * n];
          A[pp + (size_t)k * n] = cth * apk - sth * aqk;
          A[qq + (size_t)k * n] = sth * apk + cth * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[k + (size_t)pp * n], vkq = V[k + (size_t)qq * n];
          V[k + (size_t)pp * n] = cth * vkp - sth * vkq;
          V[k + (size_t)qq * n] = sth * vkp + cth * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[i + (size_t)i * n];
}

// One-sided Jacobi SVD of an n x n matrix A (column-major), the method of
// Hestenes (1958), accurate in the relative sense shown by Demmel and Veselic
// (1992).  Plane rotations applied from the right make A's columns mutually
// orthogonal, A J1 J2 ... = U~ S; their product is V~.  A pair (p, q) is left
// alone once |a_p^T a_q| <= sqrt(n) eps |a_p| |a_q|, and the sweeps stop after
// one without a rotation.  On return A holds U~ (unit columns), s the singular
// values and V the columns of V~, ordered by descending s.  Columns of U~ whose
// singular value is exactly zero are completed to an orthonormal set.
inline void jacobi_svd(int n, std::vector<double>& A, std::vector<double>& s, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i + (size_t)i * n] = 1.0;
  constexpr double eps = 2.220446049250313e-16;
  const double tol = eps * std::sqrt((double)std::max(n, 1));
  auto col = [n](std::vector<double>& M, int c) { return M.data() + (size_t)c * n; };
  for (int sweep = 0; sweep < 80; ++sweep) {
    bool rotated = false;
    for (int pp = 0; pp < n - 1; ++pp)
      for (int qq = pp + 1; qq < n; ++qq) {
        double* x = col(A, pp);
        double* y = col(A, qq);
        double a = 0.0, b = 0.0, g = 0.0;
        for (int k = 0; k < n; ++k) {
          a += x[k] * x[k];
          b += y[k] * y[k];
          g += x[k] * y[k];
        }
        if (g == 0.0 || std::fabs(g) <= tol * std::sqrt(a * b)) continue;
        rotated = true;
        // (c, s) with c^2 - s^2 = ((b - a) / g) c s: the smaller root t = s / c
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), sn = c * t;
        for (int k = 0; k < n; ++k) {
          const double xk = x[k], yk = y[k];
          x[k] = c * xk - sn * yk;
          y[k] = sn * xk + c * yk;
        }
        double* vx = col(V, pp);
        double* vy = col(V, qq);
        for (int k = 0; k < n; ++k) {
          const double xk = vx[k], yk = vy[k];
          vx[k] = c * xk - sn * yk;
          vy[k] = sn * xk + c * yk;
        }
      }
    if (!rotated) break;
  }
  s.assign(n, 0.0);
  for (int c = 0; c < n; ++c) {
    double* x = col(A, c);
    double nr = 0.0;
    for (int k = 0; k < n; ++k) nr += x[k] * x[k];
    s[c] = std::sqrt(nr);
    if (s[c] > 0.0)
      for (int k = 0; k < n; ++k) x[k] /= s[c];
  }
  std::vector<int> order(n);
  for (int c = 0; c < n; ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&s](int u, int v) { return s[u] > s[v]; });
  std::vector<double> A2((size_t)n * n), V2((size_t)n * n), s2(n);
  for (int c = 0; c < n; ++c) {
    s2[c] = s[order[c]];
    std::copy(col(A, order[c]), col(A, order[c]) + n, A2.data() + (size_t)c * n);
    std::copy(col(V, order[c]), col(V, order[c]) + n, V2.data() + (size_t)c * n);
  }
  A.swap(A2);
  V.swap(V2);
  s.swap(s2);
  // zero singular values sort last: each of their left vectors becomes the unit
  // vector with the largest part orthogonal to the columns before it (the parts
  // of all n unit vectors add up to n - c > 0), orthogonalised twice
  std::vector<double> x(n), best(n);
  for (int c = 0; c < n; ++c) {
    if (s[c] > 0.0) continue;
    double best_nr = -1.0;
    for (int e = 0; e < n; ++e) {
      std::fill(x.begin(), x.end(), 0.0);
      x[e] = 1.0;
      for (int pass = 0; pass < 2; ++pass)
        for (int d = 0; d < c; ++d) {
          const double* y = col(A, d);
          double g = 0.0;
          for (int k = 0; k < n; ++k) g += y[k] * x[k];
          for (int k = 0; k < n; ++k) x[k] -= g * y[k];
        }
      double nr = 0.0;
      for (int k = 0; k < n; ++k) nr += x[k] * x[k];
      if (nr > best_nr) {
        best_nr = nr;
        best = x;
      }
    }
    const double inv = 1.0 / std::sqrt(best_nr);
    for (int k = 0; k < n; ++k) col(A, c)[k] = best[k] * inv;
  }
}

}  // namespace cr_host
