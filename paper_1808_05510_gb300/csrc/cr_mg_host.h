// Host construction of the multigrid hierarchy that preconditions the ALS
// sub-problems (Eqs. ALS_linsys and ALS_linsys_v, Sec. 2.3).
//
// Both sub-problem operators are  lam [(L + cI)^2 + e I] + data,  a polynomial
// in one graph Laplacian L plus a data term.  The preconditioner approximates
// the inverse of  lam (L + sigma I)^2  by two V-cycles for  L + sigma I,  so
// its hierarchy depends on L alone and serves every shift sigma: each level
// keeps the coarse Laplacian L_l and the coarse mass matrix M_l separately and
// the kernel forms  L_l + sigma M_l  on the fly.
//
// Coarsening is smoothed aggregation on the graph of L (no voxel geometry is
// needed): distance-1 aggregates (a root with all its free neighbours, then
// leftovers join a neighbouring aggregate), the tentative piecewise-constant
// prolongation P0 smoothed by one damped-Jacobi step of L,
//   P = (I - omega D_L^-1 L) P0,
// which keeps the constant vector exact (L 1 = 0, so P 1 = 1), and Galerkin
// coarse matrices  L_{l+1} = P^T L_l P,  M_{l+1} = P^T M_l P  (M_0 = I).
// Coarsening stops at coarse_max rows; that level is solved densely.
//
// Header-only and free of CUDA so that the builder is tested on the CPU with
// g++ alone.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "cr_host_linalg.h"

namespace cr_mg {

// Sparse matrix in CSR form (rows x cols), columns ascending within a row.
struct Csr {
  int rows = 0, cols = 0;
  std::vector<int> rp{0}, ci;
  std::vector<double> v;
  int64_t nnz() const { return (int64_t)ci.size(); }
};

inline Csr identity(int n) {
  Csr I;
  I.rows = I.cols = n;
  I.rp.resize(n + 1);
  I.ci.resize(n);
  I.v.assign(n, 1.0);
  for (int i = 0; i <= n; ++i) I.rp[i] = i;
  for (int i = 0; i < n; ++i) I.ci[i] = i;
  return I;
}

inline Csr transpose(const Csr& A) {
  Csr T;
  T.rows = A.cols;
  T.cols = A.rows;
  T.rp.assign(A.cols + 1, 0);
  for (int c : A.ci) T.rp[c + 1] += 1;
  for (int c = 0; c < A.cols; ++c) T.rp[c + 1] += T.rp[c];
  T.ci.resize(A.ci.size());
  T.v.resize(A.v.size());
  std::vector<int> pos(T.rp.begin(), T.rp.end() - 1);
  for (int i = 0; i < A.rows; ++i)
    for (int q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      const int p = pos[A.ci[q]]++;
      T.ci[p] = i;
      T.v[p] = A.v[q];
    }
  return T;  // rows visited in order, so columns come out ascending
}

// C = A B with a dense accumulator per row (exact zeros dropped).
inline Csr multiply(const Csr& A, const Csr& B) {
  Csr C;
  C.rows = A.rows;
  C.cols = B.cols;
  C.rp.assign(A.rows + 1, 0);
  std::vector<double> acc(B.cols, 0.0);
  std::vector<int> mark(B.cols, -1), cols;
  for (int i = 0; i < A.rows; ++i) {
    cols.clear();
    for (int q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      const int k = A.ci[q];
      const double a = A.v[q];
      for (int s = B.rp[k]; s < B.rp[k + 1]; ++s) {
        const int c = B.ci[s];
        if (mark[c] != i) {
          mark[c] = i;
          acc[c] = 0.0;
          cols.push_back(c);
        }
        acc[c] += a * B.v[s];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int c : cols)
      if (acc[c] != 0.0) {
        C.ci.push_back(c);
        C.v.push_back(acc[c]);
      }
    C.rp[i + 1] = (int)C.ci.size();
  }
  return C;
}

inline std::vector<double> diagonal(const Csr& A) {
  std::vector<double> d(A.rows, 0.0);
  for (int i = 0; i < A.rows; ++i)
    for (int q = A.rp[i]; q < A.rp[i + 1]; ++q)
      if (A.ci[q] == i) d[i] += A.v[q];
  return d;
}

// Distance-1 aggregation of the graph of A's off-diagonal nonzeros, scanning
// rows in order: (1) a row whose neighbours are all free becomes the root of
// a new aggregate holding it and its neighbours; (2) each row still free joins
// the aggregate of its most strongly coupled aggregated neighbour; (3) rows
// with no aggregated neighbour become aggregates of their own.  Aggregates are
// numbered in order of creation, so they follow the row order.
inline std::vector<int> aggregate(const Csr& A, int* n_agg) {
  const int n = A.rows;
  std::vector<int> agg(n, -1);
  int na = 0;
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool free_nbhd = true;
    for (int q = A.rp[i]; q < A.rp[i + 1] && free_nbhd; ++q)
      if (A.ci[q] != i && A.v[q] != 0.0 && agg[A.ci[q]] >= 0) free_nbhd = false;
    if (!free_nbhd) continue;
    agg[i] = na;
    for (int q = A.rp[i]; q < A.rp[i + 1]; ++q)
      if (A.ci[q] != i && A.v[q] != 0.0) agg[A.ci[q]] = na;
    ++na;
  }
  std::vector<int> first(agg);  // assignments of step (1) only
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    int best = -1;
    double bw = -1.0;
    for (int q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      const int c = A.ci[q];
      if (c == i || A.v[q] == 0.0 || first[c] < 0) continue;
      const double w = std::fabs(A.v[q]);
      if (w > bw) {
        bw = w;
        best = first[c];
      }
    }
    agg[i] = best;
  }
  for (int i = 0; i < n; ++i)
    if (agg[i] < 0) agg[i] = na++;
  *n_agg = na;
  return agg;
}

// P = (I - omega D^-1 A) P0 with P0 the 0/1 aggregate indicator; rows whose
// diagonal is not positive keep their P0 row.
inline Csr prolongation(const Csr& A, const std::vector<int>& agg, int n_agg, double omega) {
  const int n = A.rows;
  Csr P0;
  P0.rows = n;
  P0.cols = n_agg;
  P0.rp.resize(n + 1);
  P0.ci.resize(n);
  P0.v.assign(n, 1.0);
  for (int i = 0; i <= n; ++i) P0.rp[i] = i;
  for (int i = 0; i < n; ++i) P0.ci[i] = agg[i];
  const std::vector<double> d = diagonal(A);
  Csr S;  // I - omega D^-1 A
  S.rows = S.cols = n;
  S.rp.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    bool diag_seen = false;
    for (int q = A.rp[i]; q < A.rp[i + 1]; ++q) {
      const int c = A.ci[q];
      double val = d[i] > 0.0 ? -omega * A.v[q] / d[i] : 0.0;
      if (c == i) {
        val += 1.0;
        diag_seen = true;
      }
      if (!diag_seen && c > i) {  // the identity entry sorts before this column
        S.ci.push_back(i);
        S.v.push_back(1.0);
        diag_seen = true;
      }
      if (val != 0.0) {
        S.ci.push_back(c);
        S.v.push_back(val);
      }
    }
    if (!diag_seen) {
      S.ci.push_back(i);
      S.v.push_back(1.0);
    }
    S.rp[i + 1] = (int)S.ci.size();
  }
  return multiply(S, P0);
}

struct Level {
  Csr L, M;  // level operators: the kernel smooths with L + sigma M
  Csr P, R;  // prolongation from the next level (rows x next rows) and R = P^T (empty on the last level)
};

struct Hierarchy {
  std::vector<Level> lev;  // lev.back() is the coarsest level (dense solve)
};

// Eigenbasis of the pencil (L_c, M_c) of the coarsest level (M_c symmetric
// positive definite): L_c Q = M_c Q diag(mu), Q^T M_c Q = I, so that
//   (L_c + sigma M_c)^-1 = Q diag(1 / (mu + sigma)) Q^T   for every shift sigma.
// Through the Cholesky factor M_c = C C^T: S = C^-1 L_c C^-T = W diag(mu) W^T,
// Q = C^-T W.  Q is column-major nc x nc.  Returns false if M_c is not positive
// definite.
inline bool pencil_basis(const Csr& Lc, const Csr& Mc, std::vector<double>& Q, std::vector<double>& mu) {
  const int n = Lc.rows;
  std::vector<double> Ld((size_t)n * n, 0.0), C((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    for (int q = Lc.rp[i]; q < Lc.rp[i + 1]; ++q) Ld[i + (size_t)Lc.ci[q] * n] += Lc.v[q];
    for (int q = Mc.rp[i]; q < Mc.rp[i + 1]; ++q) C[i + (size_t)Mc.ci[q] * n] += Mc.v[q];
  }
  // lower Cholesky factor of M_c in place (column-major, lower triangle)
  for (int k = 0; k < n; ++k) {
    double dkk = C[k + (size_t)k * n];
    for (int p = 0; p < k; ++p) dkk -= C[k + (size_t)p * n] * C[k + (size_t)p * n];
    if (!(dkk > 0.0)) return false;
    dkk = std::sqrt(dkk);
    C[k + (size_t)k * n] = dkk;
    for (int i = k + 1; i < n; ++i) {
      double s = C[i + (size_t)k * n];
      for (int p = 0; p < k; ++p) s -= C[i + (size_t)p * n] * C[k + (size_t)p * n];
      C[i + (size_t)k * n] = s / dkk;
    }
    for (int i = 0; i < k; ++i) C[i + (size_t)k * n] = 0.0;
  }
  // forward substitution C Y = B, column by column (B overwritten by Y)
  auto lower_solve = [&](std::vector<double>& B) {
    for (int col = 0; col < n; ++col)
      for (int i = 0; i < n; ++i) {
        double s = B[i + (size_t)col * n];
        for (int p = 0; p < i; ++p) s -= C[i + (size_t)p * n] * B[p + (size_t)col * n];
        B[i + (size_t)col * n] = s / C[i + (size_t)i * n];
      }
  };
  lower_solve(Ld);  // Y = C^-1 L_c
  std::vector<double> S((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) S[i + (size_t)j * n] = Ld[j + (size_t)i * n];  // Y^T
  lower_solve(S);  // C^-1 Y^T = C^-1 L_c C^-T
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) {
      const double a = 0.5 * (S[i + (size_t)j * n] + S[j + (size_t)i * n]);
      S[i + (size_t)j * n] = S[j + (size_t)i * n] = a;
    }
  std::vector<double> W;
  cr_host::sym_eig(n, S, mu, W);
  // Q = C^-T W: back substitution C^T Q = W
  Q = W;
  for (int col = 0; col < n; ++col)
    for (int i = n - 1; i >= 0; --i) {
      double s = Q[i + (size_t)col * n];
      for (int p = i + 1; p < n; ++p) s -= C[p + (size_t)i * n] * Q[p + (size_t)col * n];
      Q[i + (size_t)col * n] = s / C[i + (size_t)i * n];
    }
  return true;
}

// L: the fine-level graph Laplacian (symmetric, n x n).
inline Hierarchy build(const Csr& L, int coarse_max = 64, int max_levels = 8, double omega = 2.0 / 3.0) {
  Hierarchy h;
  Level l0;
  l0.L = L;
  l0.M = identity(L.rows);
  h.lev.push_back(std::move(l0));
  while ((int)h.lev.size() < max_levels && h.lev.back().L.rows > coarse_max) {
    Level& f = h.lev.back();
    int na = 0;
    const std::vector<int> agg = aggregate(f.L, &na);
    if (na >= f.L.rows) break;  // no coarsening possible (e.g. no edges)
    f.P = prolongation(f.L, agg, na, omega);
    f.R = transpose(f.P);
    Level c;
    c.L = multiply(f.R, multiply(f.L, f.P));
    c.M = multiply(f.R, multiply(f.M, f.P));
    h.lev.push_back(std::move(c));
  }
  return h;
}

}  // namespace cr_mg
