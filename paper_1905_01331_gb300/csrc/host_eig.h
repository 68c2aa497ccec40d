// Host-side setup arithmetic (step a0): the bond shift.
#pragma once

namespace ttn {

// Largest eigenvalue of the bond term 1/2 (o (x) I + I (x) o) + sum_k A_k (x) B_k
// (symmetrised), a d0^2 x d0^2 matrix built from host FP64 row-major terms.
// Householder reduction to tridiagonal form, then Sturm-sequence bisection.
double bond_lambda_max(const double* o, const double* A, const double* B, int d0, int K);

}  // namespace ttn
