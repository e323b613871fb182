// exact_prod.cuh -- error-free products of MP operands fed to the exact
// fixed-point accumulator (fixacc.cuh).  Shared by the SpMV / SpMM run
// kernels and the Krylov vector kernels of handles created with
// MPSPMV_EXACT_ACC (GB300-specific alternative to the MP multiply-add of
// arXiv 2412.17510, Section 2).
#pragma once
#include "fixacc.cuh"
#include "mp_arith.cuh"

namespace mpk {

// ---------------------------------------------------------------------------
// Only the error-free products run on the binary64 pipe; their terms are
// added exactly on the integer pipe (fixacc.cuh).  Product of a . x:
//   P mode, L = 2: TwoProd(a0, x0) + fma(a0, x1, a1 x0)           4 binary64 ops, 3 terms
//           L = 3: TwoProd for i+j <= 1, FMA chain for i+j = 2    9 ops, 7 terms
//           L = 4: TwoProd for i+j <= 2, FMA chain for i+j = 3   16 ops, 13 terms
//   binary64 a: TwoProd(a, x_j) for j < L-1, a x_{L-1}             2L-1 ops, 2L-1 terms
// Products of order below the format's unit roundoff are dropped or rounded
// once; the sum is then exact up to the window and cut to L components.
// ---------------------------------------------------------------------------

template <int L>
struct AccDigits {
  static constexpr int D = L == 1 ? 4 : (L == 2 ? 6 : (L == 3 ? 8 : 10));
};

template <int D, int T>
__device__ __forceinline__ void acc_add(FixAccS<D, T>& a, double v, bool neg) {
  fas_add<D, T>(a, v, neg);
}

template <class Acc, int L>
__device__ __forceinline__ void add_prod(Acc& acc, const mp<L>& a, const mp<L>& x, bool negate) {
  if constexpr (L == 1) {
    double p, e;
    two_prod(a.v[0], x.v[0], p, e);
    acc_add(acc, p, negate);
    acc_add(acc, e, negate);
  } else if constexpr (L == 2) {
    double p, e;
    two_prod(a.v[0], x.v[0], p, e);
    const double c = __fma_rn(a.v[0], x.v[1], __dmul_rn(a.v[1], x.v[0]));
    acc_add(acc, p, negate);
    acc_add(acc, e, negate);
    acc_add(acc, c, negate);
  } else if constexpr (L == 3) {
    const int ij[3][2] = {{0, 0}, {0, 1}, {1, 0}};
#pragma unroll
    for (int t = 0; t < 3; t++) {
      double ai = a.v[ij[t][0]], xj = x.v[ij[t][1]], p, e;
      // keep the products in step with the accumulation (the compiler would
      // otherwise form every product first and run out of registers)
      asm volatile("" : "+d"(ai), "+d"(xj)::"memory");
      two_prod(ai, xj, p, e);
      acc_add(acc, p, negate);
      acc_add(acc, e, negate);
    }
    const double c = __fma_rn(a.v[0], x.v[2], __fma_rn(a.v[1], x.v[1], __dmul_rn(a.v[2], x.v[0])));
    acc_add(acc, c, negate);
  } else {
#pragma unroll
    for (int i = 0; i < 3; i++) {
#pragma unroll
      for (int j = 0; j < 3 - i; j++) {
        double ai = a.v[i], xj = x.v[j], p, e;
        asm volatile("" : "+d"(ai), "+d"(xj)::"memory");
        two_prod(ai, xj, p, e);
        acc_add(acc, p, negate);
        acc_add(acc, e, negate);
      }
    }
    const double c =
        __fma_rn(a.v[0], x.v[3], __fma_rn(a.v[1], x.v[2], __fma_rn(a.v[2], x.v[1], __dmul_rn(a.v[3], x.v[0]))));
    acc_add(acc, c, negate);
  }
}

// binary64 matrix value (M mode)
template <class Acc, int L>
__device__ __forceinline__ void add_prod_d(Acc& acc, double a, const mp<L>& x, bool negate) {
#pragma unroll
  for (int j = 0; j < L - 1; j++) {
    double p, e;
    two_prod(a, x.v[j], p, e);
    acc_add(acc, p, negate);
    acc_add(acc, e, negate);
  }
  acc_add(acc, __dmul_rn(a, x.v[L - 1]), negate);
}

}  // namespace mpk
