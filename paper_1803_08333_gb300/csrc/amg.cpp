// Smoothed-aggregation multigrid hierarchy for the cell graph Laplacian Sigma^T Sigma.
//
// The paper inverts its graph Laplacians with an algebraic multigrid library (Sec. 3.4,
// Sec. 4).  Here the hierarchy preconditions the block CG that builds the dense
// (Sigma^T Sigma)^+ once per mesh connectivity.  Setup on the host:
//  * aggregation: a node whose neighbours are all free seeds an aggregate with them; the
//    remaining nodes join a neighbouring aggregate;
//  * tentative prolongator P0[i, agg(i)] = 1 / sqrt(|agg|) (the constants, the null space);
//  * smoothed prolongator P = (I - w D^{-1} A) P0, w = 4 / (3 rho), rho the Gershgorin bound
//    of D^{-1} A;
//  * Galerkin coarse matrix P^T A P, recursively, until at most `max_coarse` nodes;
//  * coarsest level: dense pseudo-inverse from a cyclic Jacobi eigendecomposition
//    (eigenvalues below 1e-10 of the largest are dropped: the Laplacian's null space).
#include <algorithm>
#include <cmath>

#include "rfcmp_internal.h"

namespace rfcmp {

namespace {

struct Csr {
  int n = 0, m = 0;
  std::vector<int32_t> ptr, col;
  std::vector<double> val;
};

Csr transpose(const Csr& A) {
  Csr T;
  T.n = A.m;
  T.m = A.n;
  T.ptr.assign(T.n + 1, 0);
  for (int32_t c : A.col) T.ptr[c + 1]++;
  for (int i = 0; i < T.n; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(A.col.size());
  T.val.resize(A.val.size());
  std::vector<int32_t> fill(T.ptr.begin(), T.ptr.end() - 1);
  for (int i = 0; i < A.n; ++i)
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
      const int d = fill[A.col[q]]++;
      T.col[d] = i;
      T.val[d] = A.val[q];
    }
  return T;
}

// C = A B (dense accumulator per row)
Csr multiply(const Csr& A, const Csr& B) {
  Csr C;
  C.n = A.n;
  C.m = B.m;
  C.ptr.assign(C.n + 1, 0);
  std::vector<double> acc(B.m, 0.0);
  std::vector<int32_t> mark(B.m, -1), cols;
  for (int i = 0; i < A.n; ++i) {
    cols.clear();
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
      const int k = A.col[q];
      const double a = A.val[q];
      for (int r = B.ptr[k]; r < B.ptr[k + 1]; ++r) {
        const int j = B.col[r];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = 0.0;
          cols.push_back(j);
        }
        acc[j] += a * B.val[r];
      }
    }
    std::sort(cols.begin(), cols.end());
    for (int j : cols) {
      if (acc[j] != 0.0) {
        C.col.push_back(j);
        C.val.push_back(acc[j]);
      }
    }
    C.ptr[i + 1] = (int32_t)C.col.size();
  }
  return C;
}

// cyclic Jacobi eigendecomposition of a small dense symmetric matrix (row-major n x n)
void jacobi_eig(int n, std::vector<double>& a, std::vector<double>& vecs, std::vector<double>& vals) {
  vecs.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) vecs[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double v = a[(size_t)i * n + j] * a[(size_t)i * n + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * std::max(tot, 1e-300)) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[(size_t)p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        const double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        const double theta = 0.5 * (aqq - app) / apq;
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // rotate columns p, q
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = c * akp - s * akq;
          a[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rotate rows p, q
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = c * apk - s * aqk;
          a[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = vecs[(size_t)k * n + p], vkq = vecs[(size_t)k * n + q];
          vecs[(size_t)k * n + p] = c * vkp - s * vkq;
          vecs[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  vals.resize(n);
  for (int i = 0; i < n; ++i) vals[i] = a[(size_t)i * n + i];
}

double gershgorin_rho(const Csr& A, const std::vector<double>& diag) {
  double rho = 0.0;
  for (int i = 0; i < A.n; ++i) {
    double s = 0.0;
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) s += std::fabs(A.val[q]);
    rho = std::max(rho, s / diag[i]);
  }
  return rho;
}

}  // namespace

int build_amg(const std::vector<int32_t>& ptr, const std::vector<int32_t>& col, const std::vector<double>& val, int n,
              int max_coarse, AmgHierarchy& H, std::string& err) {
  H = AmgHierarchy();
  Csr A;
  A.n = A.m = n;
  A.ptr = ptr;
  A.col = col;
  A.val = val;
  while (A.n > max_coarse && (int)H.levels.size() < 12) {
    AmgLevelHost L;
    L.n = A.n;
    L.diag.assign(A.n, 0.0);
    for (int i = 0; i < A.n; ++i)
      for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
        if (A.col[q] == i) L.diag[i] = A.val[q];
    for (int i = 0; i < A.n; ++i)
      if (!(L.diag[i] > 0.0)) {
        err = "multigrid setup: non-positive diagonal";
        return RFCMP_ERR_INVALID_ARG;
      }
    const double rho = gershgorin_rho(A, L.diag);
    L.omega = 4.0 / (3.0 * rho);
    // aggregation
    std::vector<int32_t> agg(A.n, -1);
    int na = 0;
    for (int i = 0; i < A.n; ++i) {
      if (agg[i] >= 0) continue;
      bool free_all = true;
      for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q)
        if (agg[A.col[q]] >= 0) free_all = false;
      if (!free_all) continue;
      for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) agg[A.col[q]] = na;
      agg[i] = na++;
    }
    for (int i = 0; i < A.n; ++i) {
      if (agg[i] >= 0) continue;
      int best = -1;
      double bw = -1.0;
      for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) {
        const int j = A.col[q];
        if (j != i && agg[j] >= 0 && std::fabs(A.val[q]) > bw) {
          bw = std::fabs(A.val[q]);
          best = agg[j];
        }
      }
      agg[i] = best >= 0 ? best : na++;
    }
    if (na >= A.n) break;  // no coarsening possible
    std::vector<int> size(na, 0);
    for (int i = 0; i < A.n; ++i) size[agg[i]]++;
    Csr P0;
    P0.n = A.n;
    P0.m = na;
    P0.ptr.resize(A.n + 1);
    P0.col.resize(A.n);
    P0.val.resize(A.n);
    for (int i = 0; i < A.n; ++i) {
      P0.ptr[i] = i;
      P0.col[i] = agg[i];
      P0.val[i] = 1.0 / std::sqrt((double)size[agg[i]]);
    }
    P0.ptr[A.n] = A.n;
    // P = P0 - w D^{-1} A P0
    Csr AP0 = multiply(A, P0);
    Csr P;
    P.n = A.n;
    P.m = na;
    P.ptr.assign(A.n + 1, 0);
    for (int i = 0; i < A.n; ++i) {
      std::vector<std::pair<int32_t, double>> row;
      for (int q = AP0.ptr[i]; q < AP0.ptr[i + 1]; ++q) row.push_back({AP0.col[q], -L.omega * AP0.val[q] / L.diag[i]});
      bool found = false;
      for (auto& e : row)
        if (e.first == agg[i]) {
          e.second += P0.val[i];
          found = true;
        }
      if (!found) row.push_back({agg[i], P0.val[i]});
      std::sort(row.begin(), row.end());
      for (auto& e : row)
        if (e.second != 0.0) {
          P.col.push_back(e.first);
          P.val.push_back(e.second);
        }
      P.ptr[i + 1] = (int32_t)P.col.size();
    }
    Csr R = transpose(P);
    Csr Ac = multiply(R, multiply(A, P));
    L.A_ptr = A.ptr;
    L.A_col = A.col;
    L.A_val = A.val;
    L.P_ptr = P.ptr;
    L.P_col = P.col;
    L.P_val = P.val;
    L.R_ptr = R.ptr;
    L.R_col = R.col;
    L.R_val = R.val;
    L.nc = na;
    H.levels.push_back(std::move(L));
    A = std::move(Ac);
  }
  // coarsest: dense pseudo-inverse
  const int m = A.n;
  std::vector<double> dense((size_t)m * m, 0.0), vecs, vals;
  for (int i = 0; i < m; ++i)
    for (int q = A.ptr[i]; q < A.ptr[i + 1]; ++q) dense[(size_t)i * m + A.col[q]] += A.val[q];
  // symmetrise (the Galerkin product is symmetric up to rounding)
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) {
      const double s = 0.5 * (dense[(size_t)i * m + j] + dense[(size_t)j * m + i]);
      dense[(size_t)i * m + j] = dense[(size_t)j * m + i] = s;
    }
  jacobi_eig(m, dense, vecs, vals);
  double vmax = 0.0;
  for (double v : vals) vmax = std::max(vmax, std::fabs(v));
  H.coarse_n = m;
  H.coarse_inv.assign((size_t)m * m, 0.0);
  for (int e = 0; e < m; ++e) {
    if (!(vals[e] > 1e-10 * vmax)) continue;
    const double inv = 1.0 / vals[e];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) H.coarse_inv[(size_t)i * m + j] += vecs[(size_t)i * m + e] * inv * vecs[(size_t)j * m + e];
  }
  return RFCMP_OK;
}

}  // namespace rfcmp
