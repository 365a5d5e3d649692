// symeig.h -- dense symmetric eigensolver (host, FP64) for the compressed M2L basis.
#pragma once

namespace afmpb {

// Eigen-decomposition of the symmetric n x n matrix A (row-major; destroyed):
// Householder reduction to tridiagonal form, then implicit QR steps with Wilkinson shifts
// on the tridiagonal matrix, both accumulated into the eigenvector matrix.
// On return w[0..n) holds the eigenvalues in descending order and row k of zt (n x n,
// row-major) the unit eigenvector of w[k].  Returns 0, or -1 when the QR iteration did
// not converge within 30 n sweeps.
int sym_eig_desc(int n, double *A, double *w, double *zt);

}  // namespace afmpb
