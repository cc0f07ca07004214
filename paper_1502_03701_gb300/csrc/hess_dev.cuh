// Small dense complex Hessenberg algebra of the implicit restart
// (Algorithm iram), written once for host and device: Schur form by
// single-shift QR with Wilkinson shifts and deflation, eigenvectors by back
// substitution, the exact-shift QR sweep H - mu I = Q1 R, H <- Q1^H H Q1,
// Q <- Q Q1, and the Ritz-estimate test of Eq. ritz_estimate.  Row-major m x m.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

namespace hd {

struct zc {
  double re, im;
};
__host__ __device__ __forceinline__ zc mk(double r, double i = 0.0) { return zc{r, i}; }
__host__ __device__ __forceinline__ zc operator+(zc a, zc b) { return mk(a.re + b.re, a.im + b.im); }
__host__ __device__ __forceinline__ zc operator-(zc a, zc b) { return mk(a.re - b.re, a.im - b.im); }
__host__ __device__ __forceinline__ zc operator-(zc a) { return mk(-a.re, -a.im); }
__host__ __device__ __forceinline__ zc operator*(zc a, zc b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__host__ __device__ __forceinline__ zc operator*(double s, zc a) { return mk(s * a.re, s * a.im); }
__host__ __device__ __forceinline__ zc conj(zc a) { return mk(a.re, -a.im); }
__host__ __device__ __forceinline__ double abs2(zc a) { return a.re * a.re + a.im * a.im; }
__host__ __device__ __forceinline__ double zabs(zc a) { return hypot(a.re, a.im); }
__host__ __device__ __forceinline__ zc operator/(zc a, zc b) {
  // scaled division (Smith's method)
  if (fabs(b.re) >= fabs(b.im)) {
    double r = b.im / b.re, d = b.re + b.im * r;
    return mk((a.re + a.im * r) / d, (a.im - a.re * r) / d);
  }
  double r = b.re / b.im, d = b.re * r + b.im;
  return mk((a.re * r + a.im) / d, (a.im * r - a.re) / d);
}
__host__ __device__ __forceinline__ zc zsqrt(zc z) {
  double r = zabs(z);
  if (r == 0.0) return mk(0.0);
  double t = sqrt(0.5 * (r + fabs(z.re)));
  if (z.re >= 0.0) return mk(t, z.im / (2.0 * t));
  return mk(fabs(z.im) / (2.0 * t), copysign(t, z.im));
}

// G = [[c, s], [-conj(s), c]],  G [a; b] = [r; 0]
__host__ __device__ __forceinline__ void givens(zc a, zc b, double& c, zc& s) {
  double aa = zabs(a), ab = zabs(b);
  if (ab == 0.0) { c = 1.0; s = mk(0.0); return; }
  if (aa == 0.0) { c = 0.0; s = (1.0 / ab) * conj(b); return; }
  double r = hypot(aa, ab);
  c = aa / r;
  s = (1.0 / (aa * r)) * (a * conj(b));
}
__host__ __device__ __forceinline__ void rot_rows(zc* A, int m, int k, int j0, int j1, double c, zc s) {
  for (int j = j0; j < j1; ++j) {
    zc x = A[k * m + j], y = A[(k + 1) * m + j];
    A[k * m + j] = c * x + s * y;
    A[(k + 1) * m + j] = c * y - conj(s) * x;
  }
}
__host__ __device__ __forceinline__ void rot_cols(zc* A, int m, int k, int i0, int i1, double c, zc s) {
  for (int i = i0; i < i1; ++i) {
    zc x = A[i * m + k], y = A[i * m + k + 1];
    A[i * m + k] = c * x + conj(s) * y;
    A[i * m + k + 1] = c * y - s * x;
  }
}

// Schur form in place: T (upper Hessenberg) -> upper triangular, Z accumulates.
__host__ __device__ inline int schur(int m, zc* T, zc* Z) {
  for (int i = 0; i < m * m; ++i) Z[i] = mk(0.0);
  for (int i = 0; i < m; ++i) Z[i * m + i] = mk(1.0);
  double anorm = 0.0;
  for (int i = 0; i < m * m; ++i) anorm = fmax(anorm, zabs(T[i]));
  if (!(anorm < INFINITY)) return -1;
  if (anorm == 0.0) return 0;
  const double ulp = 2.220446049250313e-16;
  int hi = m - 1, iter = 0, total = 0;
  while (hi > 0) {
    int lo = hi;
    while (lo > 0) {
      double s = zabs(T[lo * m + lo]) + zabs(T[(lo - 1) * m + lo - 1]);
      if (s == 0.0) s = anorm;
      if (zabs(T[lo * m + lo - 1]) <= ulp * s) { T[lo * m + lo - 1] = mk(0.0); break; }
      --lo;
    }
    if (lo == hi) { --hi; iter = 0; continue; }
    if (++total > 60 * m) return -2;
    ++iter;
    zc a = T[(hi - 1) * m + hi - 1], b = T[(hi - 1) * m + hi], c = T[hi * m + hi - 1], d = T[hi * m + hi];
    zc mu;
    if (iter % 11 == 10) {
      mu = d + mk(1.5 * zabs(c));  // exceptional shift
    } else {
      zc half = 0.5 * (a - d);
      zc disc = zsqrt(half * half + b * c);
      zc m1 = 0.5 * (a + d) + disc, m2 = 0.5 * (a + d) - disc;
      mu = abs2(m1 - d) < abs2(m2 - d) ? m1 : m2;
    }
    zc x = T[lo * m + lo] - mu, y = T[(lo + 1) * m + lo];
    for (int k = lo; k < hi; ++k) {
      double cs;
      zc sn;
      givens(x, y, cs, sn);
      rot_rows(T, m, k, k > lo ? k - 1 : lo, m, cs, sn);
      rot_cols(T, m, k, 0, (k + 3 < hi + 1 ? k + 3 : hi + 1), cs, sn);
      rot_cols(Z, m, k, 0, m, cs, sn);
      if (k > lo) T[(k + 1) * m + k - 1] = mk(0.0);
      if (k < hi - 1) { x = T[(k + 1) * m + k]; y = T[(k + 2) * m + k]; }
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < i; ++j) T[i * m + j] = mk(0.0);
  return 0;
}

// Eigenvalues theta and unit right eigenvectors Y (column i) of H; T, Z, X are
// m x m workspaces.
__host__ __device__ inline int eig(int m, const zc* H, zc* theta, zc* Y, zc* T, zc* Z, zc* X) {
  for (int i = 0; i < m * m; ++i) { T[i] = H[i]; X[i] = mk(0.0); }
  int rc = schur(m, T, Z);
  if (rc) return rc;
  double tnorm = 0.0;
  for (int i = 0; i < m * m; ++i) tnorm = fmax(tnorm, zabs(T[i]));
  const double small = tnorm * 2.220446049250313e-16 + 1e-300;
  for (int i = 0; i < m; ++i) theta[i] = T[i * m + i];
  for (int i = 0; i < m; ++i) {
    X[i * m + i] = mk(1.0);
    for (int j = i - 1; j >= 0; --j) {
      zc s = mk(0.0);
      for (int l = j + 1; l <= i; ++l) s = s + T[j * m + l] * X[l * m + i];
      zc den = T[j * m + j] - theta[i];
      if (zabs(den) < small) den = mk(small);
      X[j * m + i] = -(s / den);
    }
  }
  for (int i = 0; i < m; ++i) {
    double nrm = 0.0;
    for (int r = 0; r < m; ++r) {
      zc s = mk(0.0);
      for (int l = 0; l <= i; ++l) s = s + Z[r * m + l] * X[l * m + i];
      Y[r * m + i] = s;
      nrm += abs2(s);
    }
    nrm = sqrt(nrm);
    for (int r = 0; r < m; ++r) Y[r * m + i] = (1.0 / nrm) * Y[r * m + i];
  }
  return 0;
}

// One exact-shift QR sweep; cs/sn are m-long workspaces.
__host__ __device__ inline void shifted_qr(int m, zc* H, zc* Q, zc mu, double* cs, zc* sn) {
  for (int i = 0; i < m; ++i) H[i * m + i] = H[i * m + i] - mu;
  for (int k = 0; k < m - 1; ++k) {
    givens(H[k * m + k], H[(k + 1) * m + k], cs[k], sn[k]);
    rot_rows(H, m, k, 0, m, cs[k], sn[k]);
    H[(k + 1) * m + k] = mk(0.0);
  }
  for (int k = 0; k < m - 1; ++k) {
    rot_cols(H, m, k, 0, m, cs[k], sn[k]);
    rot_cols(Q, m, k, 0, m, cs[k], sn[k]);
  }
  for (int i = 0; i < m; ++i) H[i * m + i] = H[i * m + i] + mu;
  for (int i = 2; i < m; ++i)
    for (int j = 0; j < i - 1; ++j) H[i * m + j] = mk(0.0);
}

__host__ __device__ __forceinline__ zc cayley_lambda(zc th, zc sigma, zc tau) {
  return (sigma * th - tau) / (th - mk(1.0));
}

// Wanted order: decreasing |theta|, ties by larger Re lambda, then Im lambda.
__host__ __device__ inline bool before(zc ta, zc tb, zc sigma, zc tau) {
  double aa = abs2(ta), ab = abs2(tb);
  if (aa != ab) return aa > ab;
  zc la = cayley_lambda(ta, sigma, tau), lb = cayley_lambda(tb, sigma, tau);
  if (la.re != lb.re) return la.re > lb.re;
  return la.im > lb.im;
}

}  // namespace hd
