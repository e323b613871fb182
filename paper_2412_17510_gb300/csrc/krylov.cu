// krylov.cu -- C entry points of the Krylov solvers and vector operations,
// the precision ladder and the learned selector's solve entry points
// (arXiv 2412.17510, Section 4.2).  The solver kernels live in
// krylov_impl.cuh, compiled once per precision (krylov_L1.cu .. krylov_L4.cu).
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "krylov.h"
#include "krylov_ops.h"

using mpkry::KrylovOps;

namespace {

bool args_ok(mpspmv_mat* h, const double* b, const double* x, double rtol, double atol, int maxit) {
  return h && b && x && h->nrows == h->ncols && rtol >= 0.0 && atol >= 0.0 && maxit >= 0 && !h->mixed &&
         std::isfinite(rtol) && std::isfinite(atol);
}

}  // namespace

// Run `call` with Ops = KrylovOps<L> for the precision L.
#define MPS_BY_L(L, call)                      \
  switch (L) {                                 \
    case 1: {                                  \
      using Ops = KrylovOps<1>;                \
      return call;                             \
    }                                          \
    case 2: {                                  \
      using Ops = KrylovOps<2>;                \
      return call;                             \
    }                                          \
    case 3: {                                  \
      using Ops = KrylovOps<3>;                \
      return call;                             \
    }                                          \
    case 4: {                                  \
      using Ops = KrylovOps<4>;                \
      return call;                             \
    }                                          \
  }                                            \
  return MPSPMV_ENOTSUP

// Run method M for the handle's precision and data type.
template <int M>
int run_method(mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
          double* relres, cudaStream_t s) {
  using mpkry::KrylovSolve;
  switch (h->L * 2 + (h->cplx ? 1 : 0)) {
    case 2: return KrylovSolve<1, false, M>::run(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 3: return KrylovSolve<1, true, M>::run(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 4: return KrylovSolve<2, false, M>::run(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 5: return KrylovSolve<2, true, M>::run(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 6: return KrylovSolve<3, false, M>::run(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 7: return KrylovSolve<3, true, M>::run(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 8: return KrylovSolve<4, false, M>::run(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 9: return KrylovSolve<4, true, M>::run(h, b, x, rtol, atol, maxit, iters, relres, s);
  }
  return MPSPMV_ENOTSUP;
}

extern "C" int mpspmv_cg(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                         double* relres, void* stream) {
  if (!args_ok(h, b, x, rtol, atol, maxit)) return MPSPMV_EINVAL;
  if (h->cplx) return MPSPMV_ENOTSUP;
  cudaStream_t s = mps_stream(stream);
  MPS_BY_L(h->L, Ops::cg(h, b, x, rtol, atol, maxit, iters, relres, s, nullptr));
}

extern "C" int mpspmv_bicgstab(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit,
                               int* iters, double* relres, void* stream) {
  if (!args_ok(h, b, x, rtol, atol, maxit)) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  return run_method<mpkry::KRY_BICGSTAB>(h, b, x, rtol, atol, maxit, iters, relres, s);
}

extern "C" int mpspmv_bicg(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                           double* relres, void* stream) {
  if (!args_ok(h, b, x, rtol, atol, maxit)) return MPSPMV_EINVAL;
  if (!h->tr) return MPSPMV_ENOTSUP;
  cudaStream_t s = mps_stream(stream);
  return run_method<mpkry::KRY_BICG>(h, b, x, rtol, atol, maxit, iters, relres, s);
}

extern "C" int mpspmv_cgs(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                          double* relres, void* stream) {
  if (!args_ok(h, b, x, rtol, atol, maxit)) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  return run_method<mpkry::KRY_CGS>(h, b, x, rtol, atol, maxit, iters, relres, s);
}

extern "C" int mpspmv_gpbicg(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit,
                             int* iters, double* relres, void* stream) {
  if (!args_ok(h, b, x, rtol, atol, maxit)) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  return run_method<mpkry::KRY_GPBICG>(h, b, x, rtol, atol, maxit, iters, relres, s);
}

extern "C" int mpspmv_dot(mpspmv_h h, int64_t n, const double* u, const double* v, double* out, void* stream) {
  if (!h || n < 0 || !out || (n > 0 && (!u || !v))) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  MPS_BY_L(h->L, Ops::dot(h, n, u, v, out, s));
}

extern "C" int mpspmv_axpy(mpspmv_h h, int64_t n, const double* alpha, const double* u, const double* v, double* w,
                           void* stream) {
  if (!h || n < 0 || (n > 0 && (!alpha || !u || !v || !w))) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  MPS_BY_L(h->L, Ops::axpy(h, n, alpha, u, v, w, s));
}

extern "C" int mpspmv_scalar_sum(mpspmv_h h, int count, const double* parts, double* out, void* stream) {
  if (!h || count < 1 || !parts || !out) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  MPS_BY_L(h->L, Ops::scalar_sum(h, count, parts, out, s));
}

extern "C" int mpspmv_scalar_div(mpspmv_h h, const double* a, const double* b, double* out, void* stream) {
  if (!h || !a || !b || !out) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  MPS_BY_L(h->L, Ops::scalar_div(h, a, b, out, s));
}

// ---------------------------------------------------------------------------
// Precision ladder and the learned selector's entry points.
// ---------------------------------------------------------------------------
namespace {

int cg_level(int L, mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit, int* it,
             double* rr, cudaStream_t s, double* hist = nullptr) {
  MPS_BY_L(L, Ops::cg(h, b, x, rtol, atol, maxit, it, rr, s, hist));
}

bool ladder_ok(const mpspmv_h* hs, int64_t* n) {
  *n = -1;
  for (int l = 0; l < 4; l++) {
    const mpspmv_mat* h = hs[l];
    if (!h) continue;
    if (h->L != l + 1 || h->cplx || h->mixed || h->nrows != h->ncols) return false;
    if (*n >= 0 && h->nrows != *n) return false;
    *n = h->nrows;
  }
  return *n >= 0;
}

// b (one binary64 plane) expanded to four planes with zero lower components
int expand_b(const double* b, int64_t n, double** out, cudaStream_t s) {
  if (cudaMalloc(out, sizeof(double) * 4 * std::max<int64_t>(n, 1)) != cudaSuccess) {
    cudaGetLastError();
    return MPSPMV_ENOMEM;
  }
  MPS_CUDA(cudaMemsetAsync(*out, 0, sizeof(double) * 4 * n, s));
  MPS_CUDA(cudaMemcpyAsync(*out, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  return MPSPMV_OK;
}

int ladder_run(const mpspmv_h* hs, int start, const double* b4, double* x, int64_t n, double rtol, double atol,
               int maxit, int* final_L, int* iters, double* relres, cudaStream_t s) {
  if (iters)
    for (int l = 0; l < 4; l++) iters[l] = 0;
  MPS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * 4 * n, s));
  int st = MPSPMV_ENOCONV;
  double rr = INFINITY;
  int last = 0;
  for (int L = std::max(start, 1); L <= 4; L++) {
    mpspmv_mat* h = hs[L - 1];
    if (!h) continue;
    int it = 0;
    // continue from the current x: its components beyond the previous level
    // are zero, so the promotion is exact; r is recomputed at this level
    int e = cg_level(L, h, b4, x, rtol, atol, maxit, &it, &rr, s);
    last = L;
    if (iters) iters[L - 1] = it;
    if (e != MPSPMV_OK && e != MPSPMV_ENOCONV && e != MPSPMV_EBREAKDOWN) return e;
    // success means the residual recomputed at this level meets the target
    if (e == MPSPMV_OK && rr <= rtol + atol) {
      st = MPSPMV_OK;
      break;
    }
  }
  if (final_L) *final_L = last;
  if (relres) *relres = rr;
  return st;
}

}  // namespace

int mps_features(mpspmv_mat* h, const double* cg_hist, float* feat, cudaStream_t s);
int mps_mlp_classify(const float* params, int C, const float* feat, int* cls, cudaStream_t s);

extern "C" int mpspmv_ladder_solve(const mpspmv_h* hs, int start_L, const double* b, double* x, double rtol,
                                   double atol, int maxit, int* final_L, int* iters, double* relres,
                                   void* stream) {
  int64_t n;
  if (!hs || !b || !x || start_L < 1 || start_L > 4 || !ladder_ok(hs, &n) || !(rtol >= 0) || !(atol >= 0) ||
      maxit < 0)
    return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  double* b4 = nullptr;
  int st = expand_b(b, n, &b4, s);
  if (!st) st = ladder_run(hs, start_L, b4, x, n, rtol, atol, maxit, final_L, iters, relres, s);
  cudaStreamSynchronize(s);
  cudaFree(b4);
  return st;
}

extern "C" int mpspmv_cg_history(mpspmv_h h, const double* b, int k, double* hist, void* stream) {
  if (!h || !b || !hist || k < 1 || k > 16 || h->cplx || h->mixed || h->nrows != h->ncols) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  double* x = nullptr;
  if (cudaMalloc(&x, sizeof(double) * h->L * std::max<int64_t>(h->nrows, 1)) != cudaSuccess) return MPSPMV_ENOMEM;
  cudaMemsetAsync(x, 0, sizeof(double) * h->L * h->nrows, s);
  double hh[16];
  int it = 0;
  double rr;
  int st = cg_level(h->L, h, b, x, 0.0, 0.0, k, &it, &rr, s, hh);
  cudaStreamSynchronize(s);
  cudaFree(x);
  if (st != MPSPMV_OK && st != MPSPMV_ENOCONV) return st;
  for (int i = 0; i < k; i++) hist[i] = hh[i];
  return MPSPMV_OK;
}

extern "C" int mpspmv_select_precision(const mpspmv_h* hs, const float* params, int C, const double* b,
                                       int* prec, float* feat_out, void* stream) {
  int64_t n;
  if (!hs || !hs[0] || !params || !b || !prec || !ladder_ok(hs, &n)) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  // features: matrix statistics + 8 binary64 CG residual ratios (b as given)
  double hist[16];
  int st = mpspmv_cg_history(hs[0], b, 8, hist, stream);
  float feat[32];
  if (!st) st = mps_features(hs[0], hist, feat, s);
  int cls = 0;
  if (!st) st = mps_mlp_classify(params, C, feat, &cls, s);
  if (st) return st;
  if (feat_out)
    for (int i = 0; i < 32; i++) feat_out[i] = feat[i];
  *prec = std::min(cls + 1, 4);  // classes: binary64, DD, TD, QD, (none -> QD)
  return MPSPMV_OK;
}

extern "C" int mpspmv_solve_auto(const mpspmv_h* hs, const float* params, int C, const double* b, double* x,
                                 double rtol, double atol, int maxit, int* chosen_L, int* final_L, int* iters,
                                 double* relres, void* stream) {
  int p = 1;
  int st = mpspmv_select_precision(hs, params, C, b, &p, nullptr, stream);
  if (st) return st;
  if (chosen_L) *chosen_L = p;
  return mpspmv_ladder_solve(hs, p, b, x, rtol, atol, maxit, final_L, iters, relres, stream);
}
