// krylov.h -- device-resident solver state shared by the Krylov kernels.
#pragma once

// status: 0 running, 1 converged, 2 converged once x += alpha p is applied,
// negative: an MPSPMV_E* code.  The first member is read by the gated SpMV
// kernels, which skip their work unless it is 0.
struct KrylovState {
  int status;
  int iter;
  int maxit;
  int exact;      // 1: inner products summed exactly (MPSPMV_EXACT_ACC handles)
  double tol;     // rtol * ||b|| + atol
  double bnorm;   // ||b||_2 (binary64)
  double relres;  // ||b - A x|| / ||b|| at exit
  double sc[8][8];  // MP scalars: [slot][0..3] real components, [4..7] imaginary components
  double hist[16];  // CG: ||r_k|| / ||b|| (recurrence residual) for k = 1..16
};
