// krylov_ops.h -- per-precision entry points of the Krylov solvers and
// vector operations, defined in krylov_impl.cuh and instantiated in several
// translation units (krylov_L<L>*.cu) that compile in parallel: the quad- and
// triple-double instantiations of the larger methods take minutes each.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct mpspmv_mat;

namespace mpkry {

enum Method : int { KRY_BICGSTAB = 0, KRY_BICG = 1, KRY_CGS = 2, KRY_GPBICG = 3 };

template <int L>
struct KrylovOps {
  // CG (real); hist (may be null) receives ||r_k|| / ||b|| for k = 1..16
  static int cg(mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                double* relres, cudaStream_t s, double* hist);
  static int dot(mpspmv_mat* h, int64_t n, const double* u, const double* v, double* out, cudaStream_t s);
  static int axpy(mpspmv_mat* h, int64_t n, const double* alpha, const double* u, const double* v, double* w,
                  cudaStream_t s);
  static int scalar_sum(mpspmv_mat* h, int count, const double* parts, double* out, cudaStream_t s);
  static int scalar_div(mpspmv_mat* h, const double* a, const double* b, double* out, cudaStream_t s);
};

// one nonsymmetric method (Method) for real or complex data
template <int L, bool CPLX, int M>
struct KrylovSolve {
  static int run(mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                 double* relres, cudaStream_t s);
};

}  // namespace mpkry
