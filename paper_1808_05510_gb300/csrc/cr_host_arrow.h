// Eigen-decomposition of a symmetric arrowhead matrix
//
//   M = [ diag(d)  z ]      d, z in R^n (d ascending), alpha scalar,
//       [ z^T  alpha ]
//
// the step that keeps the eigenbasis of a bordered matrix up to date: if
// A = Q diag(d) Q^T and A' = [A a; a^T alpha], then in the basis
// blockdiag(Q, 1) A' is the arrowhead with z = Q^T a, so
// A' = (blockdiag(Q, 1) W) diag(mu) (blockdiag(Q, 1) W)^T with M = W diag(mu) W^T.
// The Galerkin projection (Eq. Proj_Sylv) grows U^T L_y U and V^T L_x V by one
// border per greedy step (U and V never change old columns), so their
// eigenbases follow at O(n^2) per step plus one matrix product.
//
// Method (the secular equation of a rank-one bordering, as in divide-and-
// conquer eigensolvers): entries with negligible z_i, and one of any pair of
// nearly equal d_i (after a plane rotation that zeroes its z component), are
// deflated and keep (d_i, e_i).  The remaining k poles give k + 1 eigenvalues,
// the roots of
//   f(mu) = alpha - mu - sum_i z_i^2 / (d_i - mu),
// one in each gap between consecutive poles and one beyond each end (f is
// decreasing between poles), found by Newton steps kept inside the bracket by
// bisection, to full precision.  The
// eigenvectors come from z recomputed from the computed roots (the Loewner
// construction of Gu and Eisenstat, 1995), which makes them numerically
// orthogonal whatever the spacing of the roots.
//
// Header-only and free of CUDA so that it is tested on the CPU with g++ alone.
#pragma once

#include <algorithm>
#include <cmath>
#include <numeric>
#include <thread>
#include <vector>

namespace cr_host {

// On return mu (n + 1, ascending) and W ((n + 1) x (n + 1), column-major, columns
// the eigenvectors in the order of mu).
inline void arrow_eig(int n, const std::vector<double>& d, const std::vector<double>& z, double alpha,
                      std::vector<double>& mu, std::vector<double>& W) {
  const int N = n + 1;
  mu.assign(N, 0.0);
  W.assign((size_t)N * N, 0.0);
  double scale = std::fabs(alpha);
  for (int i = 0; i < n; ++i) scale = std::max(scale, std::max(std::fabs(d[i]), std::fabs(z[i])));
  if (scale == 0.0) {
    for (int i = 0; i < N; ++i) W[i + (size_t)i * N] = 1.0;
    return;
  }
  const double eps = 2.2204460492503131e-16;
  const double tol = 8.0 * eps * scale;
  // deflation: negligible z_i, then one of each pair of nearly equal poles after a
  // plane rotation (recorded, applied to the eigenvectors at the end)
  struct Rot {
    int a, b;
    double c, s;
  };
  std::vector<Rot> rots;
  std::vector<double> zz(z.begin(), z.end());
  std::vector<char> defl(n, 0);
  for (int i = 0; i < n; ++i)
    if (std::fabs(zz[i]) <= tol) defl[i] = 1;
  int last = -1;
  for (int i = 0; i < n; ++i) {
    if (defl[i]) continue;
    if (last >= 0 && std::fabs(d[i] - d[last]) <= tol) {
      const double r = std::hypot(zz[last], zz[i]);
      const double c = zz[i] / r, s = zz[last] / r;
      // e_last' = c e_last - s e_i (z component 0), e_i' = s e_last + c e_i (z component r)
      rots.push_back({last, i, c, s});
      zz[last] = 0.0;
      zz[i] = r;
      defl[last] = 1;
    }
    last = i;
  }
  std::vector<int> live;
  for (int i = 0; i < n; ++i)
    if (!defl[i]) live.push_back(i);
  const int k = (int)live.size();
  std::vector<double> dl(k), zl(k);
  for (int t = 0; t < k; ++t) {
    dl[t] = d[live[t]];
    zl[t] = zz[live[t]];
  }
  double zn2 = 0.0;
  for (double v : zl) zn2 += v * v;
  const double zn = std::sqrt(zn2);
  // secular roots, one per gap plus one beyond each end; f decreasing on each bracket.
  // Newton steps from the bracket's midpoint, a bisection step whenever Newton leaves it.
  std::vector<double> root(k + 1);
  auto find_root = [&](int r) {
    if (k == 0) {
      root[0] = alpha;
      return;
    }
    double lo, hi;
    if (r == 0) {
      lo = std::min(dl[0], alpha) - zn - scale * eps;
      hi = dl[0];
    } else if (r == k) {
      lo = dl[k - 1];
      hi = std::max(dl[k - 1], alpha) + zn + scale * eps;
    } else {
      lo = dl[r - 1];
      hi = dl[r];
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
      double fv = alpha - x, fd = -1.0;
      for (int t = 0; t < k; ++t) {
        const double q = 1.0 / (dl[t] - x), w = zl[t] * q;
        fv -= zl[t] * w;
        fd -= w * w;
      }
      if (fv > 0.0)
        lo = x;
      else
        hi = x;
      if (fv == 0.0) break;
      double xn = x - fv / fd;
      if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
      if (xn == x || !(xn > lo && xn < hi)) break;
      if (std::fabs(xn - x) <= 4.0 * eps * std::max(std::fabs(xn), std::fabs(x))) {
        x = xn;
        break;
      }
      x = xn;
    }
    root[r] = x;
  };
  // the roots are independent: threads take interleaved ones when there are many
  const int nthr = k >= 128 ? (int)std::min<unsigned>(16u, std::max(1u, std::thread::hardware_concurrency())) : 1;
  if (nthr > 1) {
    std::vector<std::thread> th;
    for (int w = 0; w < nthr; ++w)
      th.emplace_back([&, w]() {
        for (int r = w; r <= k; r += nthr) find_root(r);
      });
    for (auto& t : th) t.join();
  } else {
    for (int r = 0; r <= k; ++r) find_root(r);
  }
  // Loewner: the z for which the computed roots are exact,
  //   zhat_t^2 = -prod_r (root_r - d_t) / prod_{s != t} (d_s - d_t)
  std::vector<double> zh(k);
  for (int t = 0; t < k; ++t) {
    double p = root[k] - dl[t];
    for (int r = 0; r < k; ++r) {
      p *= (root[r] - dl[t]);
      if (r != t) p /= (dl[r] - dl[t]);
    }
    zh[t] = std::copysign(std::sqrt(std::fabs(p)), zl[t]);
  }
  // eigenpairs in the rotated basis, then the recorded rotations, then ascending order
  std::vector<double> val(N);
  std::vector<double> V((size_t)N * N, 0.0);
  int col = 0;
  for (int i = 0; i < n; ++i)
    if (defl[i]) {
      val[col] = d[i];
      V[i + (size_t)col * N] = 1.0;
      ++col;
    }
  for (int r = 0; r <= k; ++r, ++col) {
    double* v = &V[(size_t)col * N];
    double nrm = 1.0;  // last component -1
    for (int t = 0; t < k; ++t) {
      const double y = zh[t] / (dl[t] - root[r]);
      v[live[t]] = y;
      nrm += y * y;
    }
    v[n] = -1.0;
    nrm = 1.0 / std::sqrt(nrm);
    for (int q = 0; q < N; ++q) v[q] *= nrm;
    val[col] = root[r];
  }
  for (int q = (int)rots.size() - 1; q >= 0; --q) {  // back to the original basis
    const Rot& R = rots[q];
    for (int c = 0; c < N; ++c) {
      double* v = &V[(size_t)c * N];
      const double a = v[R.a], b = v[R.b];
      v[R.a] = R.c * a + R.s * b;
      v[R.b] = -R.s * a + R.c * b;
    }
  }
  std::vector<int> ord(N);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return val[a] < val[b]; });
  for (int c = 0; c < N; ++c) {
    mu[c] = val[ord[c]];
    std::copy(&V[(size_t)ord[c] * N], &V[(size_t)ord[c] * N] + N, &W[(size_t)c * N]);
  }
}

}  // namespace cr_host
