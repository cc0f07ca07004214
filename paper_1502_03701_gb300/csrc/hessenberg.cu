// Small dense complex Hessenberg routines for the implicit restart
// (Algorithm iram): Schur form by single-shift QR iteration with Wilkinson
// shifts and deflation, eigenvectors by back substitution on the triangular
// factor, and the sweep of shifted QR factorisations H - mu_j I = Q_j R_j,
// H <- Q_j^H H Q_j, Q <- Q Q_j.  Matrices are row-major m x m (H[i*m + j]).
#include <cmath>
#include <complex>
#include <vector>

#include "hessenberg.h"

namespace hess {

typedef std::complex<double> cd;

// Givens rotation G = [[c, s], [-conj(s), c]] with G [a; b] = [r; 0]
static void givens(cd a, cd b, double& c, cd& s) {
  double aa = std::abs(a), ab = std::abs(b);
  if (ab == 0.0) { c = 1.0; s = 0.0; return; }
  if (aa == 0.0) { c = 0.0; s = std::conj(b) / ab; return; }
  double r = std::hypot(aa, ab);
  c = aa / r;
  s = (a / aa) * std::conj(b) / r;
}

// rows k, k+1 of A (columns j0..j1-1) <- G [row k; row k+1]
static void rot_rows(cd* A, int m, int k, int j0, int j1, double c, cd s) {
  for (int j = j0; j < j1; ++j) {
    cd x = A[k * m + j], y = A[(k + 1) * m + j];
    A[k * m + j] = c * x + s * y;
    A[(k + 1) * m + j] = -std::conj(s) * x + c * y;
  }
}

// columns k, k+1 of A (rows i0..i1-1) <- [col k, col k+1] G^H
static void rot_cols(cd* A, int m, int k, int i0, int i1, double c, cd s) {
  for (int i = i0; i < i1; ++i) {
    cd x = A[i * m + k], y = A[i * m + k + 1];
    A[i * m + k] = c * x + std::conj(s) * y;
    A[i * m + k + 1] = -s * x + c * y;
  }
}

int schur(int m, cd* T, cd* Z) {
  for (int i = 0; i < m * m; ++i) Z[i] = 0.0;
  for (int i = 0; i < m; ++i) Z[i * m + i] = 1.0;
  double anorm = 0.0;
  for (int i = 0; i < m * m; ++i) anorm = std::max(anorm, std::abs(T[i]));
  if (!(anorm < INFINITY)) return -1;
  if (anorm == 0.0) return 0;
  const double ulp = 2.220446049250313e-16;
  int hi = m - 1, iter = 0, total = 0;
  while (hi > 0) {
    int lo = hi;
    while (lo > 0) {
      double s = std::abs(T[lo * m + lo]) + std::abs(T[(lo - 1) * m + lo - 1]);
      if (s == 0.0) s = anorm;
      if (std::abs(T[lo * m + lo - 1]) <= ulp * s) { T[lo * m + lo - 1] = 0.0; break; }
      --lo;
    }
    if (lo == hi) { --hi; iter = 0; continue; }
    if (++total > 60 * m) return -2;
    ++iter;
    // Wilkinson shift: eigenvalue of the trailing 2x2 block closer to T[hi][hi]
    cd a = T[(hi - 1) * m + hi - 1], b = T[(hi - 1) * m + hi], c = T[hi * m + hi - 1], d = T[hi * m + hi];
    cd mu;
    if (iter % 11 == 10) {
      mu = d + std::abs(c) * 1.5;  // exceptional shift
    } else {
      cd half = 0.5 * (a - d);
      cd disc = std::sqrt(half * half + b * c);
      cd m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
      mu = std::abs(m1 - d) < std::abs(m2 - d) ? m1 : m2;
    }
    // one implicit single-shift QR sweep on the active block lo..hi
    cd x = T[lo * m + lo] - mu, y = T[(lo + 1) * m + lo];
    for (int k = lo; k < hi; ++k) {
      double cs;
      cd sn;
      givens(x, y, cs, sn);
      rot_rows(T, m, k, k > lo ? k - 1 : lo, m, cs, sn);
      rot_cols(T, m, k, 0, std::min(k + 3, hi + 1), cs, sn);
      rot_cols(Z, m, k, 0, m, cs, sn);
      if (k > lo) T[(k + 1) * m + k - 1] = 0.0;
      if (k < hi - 1) { x = T[(k + 1) * m + k]; y = T[(k + 2) * m + k]; }
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < i; ++j) T[i * m + j] = 0.0;
  return 0;
}

int eig(int m, const cd* H, cd* theta, cd* Y) {
  std::vector<cd> T(H, H + (size_t)m * m), Z((size_t)m * m), X((size_t)m * m, 0.0);
  int rc = schur(m, T.data(), Z.data());
  if (rc) return rc;
  double tnorm = 0.0;
  for (int i = 0; i < m * m; ++i) tnorm = std::max(tnorm, std::abs(T[i]));
  const double small = tnorm * 2.220446049250313e-16 + 1e-300;
  for (int i = 0; i < m; ++i) theta[i] = T[i * m + i];
  // eigenvectors of the triangular factor, column i of X
  for (int i = 0; i < m; ++i) {
    X[i * m + i] = 1.0;
    for (int j = i - 1; j >= 0; --j) {
      cd s = 0.0;
      for (int l = j + 1; l <= i; ++l) s += T[j * m + l] * X[l * m + i];
      cd den = T[j * m + j] - theta[i];
      if (std::abs(den) < small) den = small;
      X[j * m + i] = -s / den;
    }
  }
  // Y = Z X, unit columns
  for (int i = 0; i < m; ++i) {
    double nrm = 0.0;
    for (int r = 0; r < m; ++r) {
      cd s = 0.0;
      for (int l = 0; l <= i; ++l) s += Z[r * m + l] * X[l * m + i];
      Y[r * m + i] = s;
      nrm += std::norm(s);
    }
    nrm = std::sqrt(nrm);
    for (int r = 0; r < m; ++r) Y[r * m + i] /= nrm;
  }
  return 0;
}

void shifted_qr(int m, cd* H, cd* Q, cd mu) {
  std::vector<double> c(m);
  std::vector<cd> s(m);
  for (int i = 0; i < m; ++i) H[i * m + i] -= mu;
  for (int k = 0; k < m - 1; ++k) {
    givens(H[k * m + k], H[(k + 1) * m + k], c[k], s[k]);
    rot_rows(H, m, k, 0, m, c[k], s[k]);
    H[(k + 1) * m + k] = 0.0;
  }
  for (int k = 0; k < m - 1; ++k) {
    rot_cols(H, m, k, 0, m, c[k], s[k]);
    rot_cols(Q, m, k, 0, m, c[k], s[k]);
  }
  for (int i = 0; i < m; ++i) H[i * m + i] += mu;
  // restore exact Hessenberg shape
  for (int i = 2; i < m; ++i)
    for (int j = 0; j < i - 1; ++j) H[i * m + j] = 0.0;
}

void givens_ls(cd a, cd b, double& c, cd& s) { givens(a, b, c, s); }

}  // namespace hess
