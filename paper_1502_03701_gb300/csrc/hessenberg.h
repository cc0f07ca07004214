// Host-side small dense complex Hessenberg routines (see hessenberg.cu).
#pragma once
#include <complex>

namespace hess {
// Schur form T = Z^H H Z of an upper Hessenberg T (in place); 0 on success.
int schur(int m, std::complex<double>* T, std::complex<double>* Z);
// Eigenvalues theta and unit right eigenvectors Y (column i at Y[r*m + i]); 0 on success.
int eig(int m, const std::complex<double>* H, std::complex<double>* theta, std::complex<double>* Y);
// H - mu I = Q1 R, H <- Q1^H H Q1, Q <- Q Q1 (Givens, H upper Hessenberg).
void shifted_qr(int m, std::complex<double>* H, std::complex<double>* Q, std::complex<double> mu);
// Rotation G = [[c, s], [-conj(s), c]] with G [a; b] = [r; 0].
void givens_ls(std::complex<double> a, std::complex<double> b, double& c, std::complex<double>& s);
}  // namespace hess
