// symeig.cu -- dense symmetric eigensolver (host code only; see symeig.h).
//
// Two textbook stages (Golub & Van Loan, Matrix Computations, Sec. 8.3):
//  1. Householder reflections H_k = I - beta v v^T reduce A to a tridiagonal T = Q^T A Q;
//  2. implicit symmetric QR steps with the Wilkinson shift chase a bulge down each
//     unreduced block of T with Givens rotations until every off-diagonal entry is
//     negligible.
// Q is kept transposed (zt = Q^T, row k = column k of Q) so that both the reflections
// and the rotations touch contiguous rows.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "symeig.h"

namespace afmpb {

namespace {

// Stage 1.  a: n x n row-major symmetric (overwritten), zt: Q^T.  d, e: diagonal and
// super-diagonal of T (e[n-1] unused).
void householder_tridiag(int n, double *a, double *zt, double *d, double *e) {
  std::fill(zt, zt + (size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) zt[(size_t)i * n + i] = 1.0;
  std::vector<double> v(n), p(n), u(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;                       // length of x = A[k+1.., k]
    double xnorm2 = 0.0;
    for (int j = 0; j < m; ++j) {
      const double x = a[(size_t)(k + 1 + j) * n + k];
      v[j] = x;
      xnorm2 += x * x;
    }
    if (xnorm2 == 0.0) continue;                   // column already reduced
    const double alpha = -std::copysign(std::sqrt(xnorm2), v[0]);   // H x = alpha e_1
    v[0] -= alpha;                                 // no cancellation: opposite signs
    double vnorm2 = 0.0;
    for (int j = 0; j < m; ++j) vnorm2 += v[j] * v[j];
    const double beta = 2.0 / vnorm2;
    // trailing block B = A[k+1.., k+1..] <- H B H = B - v w^T - w v^T with
    // p = beta B v, w = p - (beta/2)(v.p) v
    double vp = 0.0;
    for (int i = 0; i < m; ++i) {
      const double *row = a + (size_t)(k + 1 + i) * n + (k + 1);
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += row[j] * v[j];
      p[i] = beta * s;
      vp += v[i] * p[i];
    }
    const double kk = 0.5 * beta * vp;
    for (int i = 0; i < m; ++i) p[i] -= kk * v[i];   // p is now w
    for (int i = 0; i < m; ++i) {
      double *row = a + (size_t)(k + 1 + i) * n + (k + 1);
      for (int j = 0; j < m; ++j) row[j] -= v[i] * p[j] + p[i] * v[j];
    }
    a[(size_t)(k + 1) * n + k] = a[(size_t)k * n + k + 1] = alpha;
    for (int j = 1; j < m; ++j) a[(size_t)(k + 1 + j) * n + k] = a[(size_t)k * n + k + 1 + j] = 0.0;
    // Q <- Q H: rows k+1.. of zt: zt_r -= beta v_r (sum_j v_j zt_j)
    std::fill(u.begin(), u.end(), 0.0);
    for (int j = 0; j < m; ++j) {
      const double *row = zt + (size_t)(k + 1 + j) * n;
      for (int c = 0; c < n; ++c) u[c] += v[j] * row[c];
    }
    for (int j = 0; j < m; ++j) {
      double *row = zt + (size_t)(k + 1 + j) * n;
      const double f = beta * v[j];
      for (int c = 0; c < n; ++c) row[c] -= f * u[c];
    }
  }
  for (int i = 0; i < n; ++i) {
    d[i] = a[(size_t)i * n + i];
    e[i] = i + 1 < n ? a[(size_t)i * n + i + 1] : 0.0;
  }
}

// One implicit QR step with Wilkinson shift on the unreduced block [lo, hi] of T.
void qr_step(int n, int lo, int hi, double *d, double *e, double *zt) {
  const double t = 0.5 * (d[hi - 1] - d[hi]);
  const double eh = e[hi - 1];
  const double mu = d[hi] - eh * eh / (t + std::copysign(std::hypot(t, eh), t == 0.0 ? 1.0 : t));
  double x = d[lo] - mu, z = e[lo];
  for (int k = lo; k < hi; ++k) {
    // rotation G = [[c, s], [-s, c]] on (k, k+1) with s x + c z = 0
    const double r = std::hypot(x, z);
    double c = 1.0, s = 0.0;
    if (r != 0.0) { c = x / r; s = -z / r; }
    if (k > lo) e[k - 1] = r;                       // bulge at (k-1, k+1) absorbed
    const double a0 = d[k], b0 = d[k + 1], f = e[k];
    d[k] = c * c * a0 - 2.0 * c * s * f + s * s * b0;
    d[k + 1] = s * s * a0 + 2.0 * c * s * f + c * c * b0;
    e[k] = c * s * (a0 - b0) + (c * c - s * s) * f;
    if (k + 1 < hi) {                               // new bulge at (k, k+2)
      const double g = e[k + 1];
      z = -s * g;
      e[k + 1] = c * g;
      x = e[k];
    }
    double *qa = zt + (size_t)k * n, *qb = zt + (size_t)(k + 1) * n;
    for (int i = 0; i < n; ++i) {
      const double ua = qa[i], ub = qb[i];
      qa[i] = c * ua - s * ub;
      qb[i] = s * ua + c * ub;
    }
  }
}

}  // namespace

int sym_eig_desc(int n, double *A, double *w, double *zt) {
  if (n <= 0) return 0;
  std::vector<double> d(n), e(n);
  householder_tridiag(n, A, zt, d.data(), e.data());
  const double eps = 0x1p-52;
  int hi = n - 1;
  long iter = 0;
  const long max_iter = 30L * n;
  while (hi > 0) {
    // deflate negligible off-diagonal entries
    for (int i = 0; i < hi; ++i)
      if (std::fabs(e[i]) <= eps * (std::fabs(d[i]) + std::fabs(d[i + 1]))) e[i] = 0.0;
    while (hi > 0 && e[hi - 1] == 0.0) --hi;       // trailing eigenvalues converged
    if (hi == 0) break;
    int lo = hi - 1;
    while (lo > 0 && e[lo - 1] != 0.0) --lo;       // start of the unreduced block
    if (++iter > max_iter) return -1;
    qr_step(n, lo, hi, d.data(), e.data(), zt);
  }
  // sort descending, permuting the eigenvector rows
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int i, int j) { return d[i] > d[j]; });
  std::vector<double> tmp((size_t)n * n);
  for (int k = 0; k < n; ++k) {
    w[k] = d[idx[k]];
    std::copy(zt + (size_t)idx[k] * n, zt + (size_t)(idx[k] + 1) * n, tmp.begin() + (size_t)k * n);
  }
  std::copy(tmp.begin(), tmp.end(), zt);
  return 0;
}

}  // namespace afmpb
