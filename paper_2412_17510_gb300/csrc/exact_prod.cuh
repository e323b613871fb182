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
// The products of an entry, a . x, go into the exact accumulator
// (fixacc.cuh) as:
//   P mode, L = 2: a0 x0 exactly, plus fma(a0, x1, a1 x0)
//           L = 3: a_i x_j exactly for i+j <= 1, plus one FMA chain for i+j = 2
//           L = 4: a_i x_j exactly for i+j <= 2, plus one FMA chain for i+j = 3
//   binary64 a: a x_j exactly for j < L-1, plus a x_{L-1} rounded
// An exact product is formed on the integer pipe as one 106-bit integer
// (fas_add_prod) when the window has at least 6 digits (DD, TD, QD); the
// binary64 pipe then only runs the FMA chain (2, 3, 4 instructions per entry
// in P mode, 1 for binary64 a).  Binary64 sums (4 digits) keep TwoProd by
// FMA, two binary64 terms per product.  Products below the format's unit
// roundoff are dropped or rounded once; the sum is exact up to the window
// and cut to L components.
// ---------------------------------------------------------------------------

template <int L>
struct AccDigits {
  static constexpr int D = L == 1 ? 4 : (L == 2 ? 6 : (L == 3 ? 8 : 10));
};

template <int D, int T>
__device__ __forceinline__ void acc_add(FixAccS<D, T>& a, double v, bool neg) {
  fas_add<D, T>(a, v, neg);
}

// acc += x y exactly: on the integer pipe when the window (D digits) holds a
// 106-bit product with room for its offset (D >= 6), else TwoProd by FMA.
template <int D, int T>
__device__ __forceinline__ void acc_add_prod(FixAccS<D, T>& a, double x, double y, bool neg) {
  if constexpr (D >= 6) {
    fas_add_prod<D, T>(a, x, y, neg);
  } else {
    double p, e;
    two_prod(x, y, p, e);
    fas_add<D, T>(a, p, neg);
    fas_add<D, T>(a, e, neg);
  }
}

template <class Acc, int L>
__device__ __forceinline__ void add_prod(Acc& acc, const mp<L>& a, const mp<L>& x, bool negate) {
  if constexpr (L == 1) {
    double p, e;
    two_prod(a.v[0], x.v[0], p, e);
    acc_add(acc, p, negate);
    acc_add(acc, e, negate);
  } else if constexpr (L == 2) {
    const double c = __fma_rn(a.v[0], x.v[1], __dmul_rn(a.v[1], x.v[0]));
    acc_add_prod(acc, a.v[0], x.v[0], negate);
    acc_add(acc, c, negate);
  } else if constexpr (L == 3) {
    const int ij[3][2] = {{0, 0}, {0, 1}, {1, 0}};
#pragma unroll
    for (int t = 0; t < 3; t++) {
      double ai = a.v[ij[t][0]], xj = x.v[ij[t][1]];
      // keep the products in step with the accumulation (the compiler would
      // otherwise form every product first and run out of registers)
      asm volatile("" : "+d"(ai), "+d"(xj)::"memory");
      acc_add_prod(acc, ai, xj, negate);
    }
    const double c = __fma_rn(a.v[0], x.v[2], __fma_rn(a.v[1], x.v[1], __dmul_rn(a.v[2], x.v[0])));
    acc_add(acc, c, negate);
  } else {
#pragma unroll
    for (int i = 0; i < 3; i++) {
#pragma unroll
      for (int j = 0; j < 3 - i; j++) {
        double ai = a.v[i], xj = x.v[j];
        asm volatile("" : "+d"(ai), "+d"(xj)::"memory");
        acc_add_prod(acc, ai, xj, negate);
      }
    }
    const double c =
        __fma_rn(a.v[0], x.v[3], __fma_rn(a.v[1], x.v[2], __fma_rn(a.v[2], x.v[1], __dmul_rn(a.v[3], x.v[0]))));
    acc_add(acc, c, negate);
  }
}

// acc += u u (neg: -=) for an MP u: the same exact sum as add_prod(acc, u,
// u, neg) with fewer products -- each symmetric pair u_i u_j + u_j u_i
// (i != j, i + j < L - 1) is added once at twice the weight, which is exact,
// and the FMA chain over i + j = L - 1 is add_prod's own.  QD: 4 exact
// products instead of 6; TD: 2 instead of 3.
template <class Acc, int L>
__device__ __forceinline__ void add_prod_self(Acc& acc, const mp<L>& u, bool negate) {
  if constexpr (L < 3) {
    add_prod<Acc, L>(acc, u, u, negate);
  } else if constexpr (L == 3) {
    acc_add_prod(acc, u.v[0], u.v[0], negate);
    double u0 = u.v[0], u1 = u.v[1];
    asm volatile("" : "+d"(u0), "+d"(u1)::"memory");
    fas_add_prod(acc, u0, u1, negate, 1);
    const double c = __fma_rn(u.v[0], u.v[2], __fma_rn(u.v[1], u.v[1], __dmul_rn(u.v[2], u.v[0])));
    acc_add(acc, c, negate);
  } else {
    const int ij[4][3] = {{0, 0, 0}, {0, 1, 1}, {0, 2, 1}, {1, 1, 0}};
#pragma unroll
    for (int t = 0; t < 4; t++) {
      double ui = u.v[ij[t][0]], uj = u.v[ij[t][1]];
      asm volatile("" : "+d"(ui), "+d"(uj)::"memory");
      fas_add_prod(acc, ui, uj, negate, ij[t][2]);
    }
    const double c =
        __fma_rn(u.v[0], u.v[3], __fma_rn(u.v[1], u.v[2], __fma_rn(u.v[2], u.v[1], __dmul_rn(u.v[3], u.v[0]))));
    acc_add(acc, c, negate);
  }
}

// binary64 matrix value (M mode)
template <class Acc, int L>
__device__ __forceinline__ void add_prod_d(Acc& acc, double a, const mp<L>& x, bool negate) {
#pragma unroll
  for (int j = 0; j < L - 1; j++) acc_add_prod(acc, a, x.v[j], negate);
  acc_add(acc, __dmul_rn(a, x.v[L - 1]), negate);
}

}  // namespace mpk
