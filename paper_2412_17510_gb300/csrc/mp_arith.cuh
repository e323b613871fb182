// mp_arith.cuh -- multi-component (DD / TD / QD) arithmetic on the binary64
// pipe of sm_103a, built from error-free transformations (arXiv 2412.17510,
// Section 2).
//
// Every binary64 operation is an explicit round-to-nearest intrinsic
// (__dadd_rn, __dsub_rn, __dmul_rn, __fma_rn) so that the compiler can neither
// contract a*b+c into an FMA nor reassociate: TwoSum and QuickTwoSum are only
// error-free when each step is rounded on its own.
//
// A number with L components is mp<L>: v[0] + v[1] + ... + v[L-1], v[0] the
// leading component.  L = 1 is plain binary64 (used by the precision ladder).
//
// Operation sequences (the order matters for reproducibility):
//   add  L=2  Algorithm 1 (DDadd, sloppy)              11 binary64 ops
//   mul  L=2  Algorithm 2 (DDmul, cross terms by mul)    9
//   add  L=4  QD sloppy add (TwoSum per component,
//             ThreeSum / ThreeSum2 by magnitude class,
//             Renorm of five terms)                      87
//   mul  L=4  QD sloppy mul (TwoProd for i+j <= 2,
//             plain products for i+j = 3, Renorm)       123
//   L=3       the QD operations with zero fourth components, the fourth
//             result component folded into the third (one addition)
//   mul_d     Algorithms 3, 5, 4 (MP x binary64, "M" mode)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mpk {

// ---------------------------------------------------------------------------
// Error-free transformations
// ---------------------------------------------------------------------------
__device__ __forceinline__ void quick_two_sum(double a, double b, double& s, double& e) {
  double t = __dadd_rn(a, b);
  e = __dsub_rn(b, __dsub_rn(t, a));
  s = t;
}

__device__ __forceinline__ void two_sum(double a, double b, double& s, double& e) {
  double t = __dadd_rn(a, b);
  double bv = __dsub_rn(t, a);
  double av = __dsub_rn(t, bv);
  e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
  s = t;
}

__device__ __forceinline__ void two_prod(double a, double b, double& p, double& e) {
  double t = __dmul_rn(a, b);
  e = __fma_rn(a, b, -t);
  p = t;
}

// (a, b, c) -> leading, middle, tail with the same exact sum.
__device__ __forceinline__ void three_sum(double& a, double& b, double& c) {
  double t1, t2, t3;
  two_sum(a, b, t1, t2);
  two_sum(c, t1, a, t3);
  two_sum(t2, t3, b, c);
}

// (a, b, c) -> leading term and a rounded tail.
__device__ __forceinline__ void three_sum2(double& a, double& b, double c) {
  double t1, t2, t3;
  two_sum(a, b, t1, t2);
  two_sum(c, t1, a, t3);
  b = __dadd_rn(t2, t3);
}

// ---------------------------------------------------------------------------
// Renormalisation.  Bottom-up QuickTwoSum sweep, then a top-down sweep that
// starts a new output component each time the rounding error is non-zero.
// The slot selection uses predicated moves, so all lanes of a warp issue the
// same binary64 instruction stream.
// ---------------------------------------------------------------------------
template <int NOUT>
__device__ __forceinline__ void place(double* b, int k, double s) {
#pragma unroll
  for (int i = 0; i < NOUT; i++)
    if (k == i) b[i] = s;
}

__device__ __forceinline__ void renorm5to4(double c0, double c1, double c2, double c3, double c4,
                                           double* r) {
  if (isinf(c0)) {
    r[0] = c0; r[1] = r[2] = r[3] = 0.0;
    return;
  }
  double s, t[4];
  quick_two_sum(c3, c4, s, t[3]);
  quick_two_sum(c2, s, s, t[2]);
  quick_two_sum(c1, s, s, t[1]);
  quick_two_sum(c0, s, s, t[0]);
  double b[4] = {0.0, 0.0, 0.0, 0.0};
  int k = 0;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    double e;
    double ss;
    quick_two_sum(s, t[i], ss, e);
    // the oracle stops feeding once four components are out; the binary64
    // work is identical, only the stores are suppressed
    if (k < 4) {
      s = ss;
      if (e != 0.0) {
        place<4>(b, k, s);
        k++;
        s = e;
      }
    }
  }
  if (k < 4) place<4>(b, k, s);
  r[0] = b[0]; r[1] = b[1]; r[2] = b[2]; r[3] = b[3];
}

__device__ __forceinline__ void renorm4to3(double c0, double c1, double c2, double c3, double* r) {
  if (isinf(c0)) {
    r[0] = c0; r[1] = r[2] = 0.0;
    return;
  }
  double s, t[3];
  quick_two_sum(c2, c3, s, t[2]);
  quick_two_sum(c1, s, s, t[1]);
  quick_two_sum(c0, s, s, t[0]);
  double b[3] = {0.0, 0.0, 0.0};
  int k = 0;
#pragma unroll
  for (int i = 0; i < 3; i++) {
    double e, ss;
    quick_two_sum(s, t[i], ss, e);
    if (k < 3) {
      s = ss;
      if (e != 0.0) {
        place<3>(b, k, s);
        k++;
        s = e;
      }
    }
  }
  if (k < 3) place<3>(b, k, s);
  r[0] = b[0]; r[1] = b[1]; r[2] = b[2];
}

// ---------------------------------------------------------------------------
// The number type
// ---------------------------------------------------------------------------
template <int L>
struct mp {
  double v[L];
};

template <int L>
__device__ __forceinline__ mp<L> mp_zero() {
  mp<L> r;
#pragma unroll
  for (int i = 0; i < L; i++) r.v[i] = 0.0;
  return r;
}

template <int L>
__device__ __forceinline__ mp<L> mp_neg(const mp<L>& a) {
  mp<L> r;
#pragma unroll
  for (int i = 0; i < L; i++) r.v[i] = -a.v[i];
  return r;
}

// ---- QD kernels on raw arrays (also used for TD with zero fourth parts) ----
__device__ __forceinline__ void qd_add_raw(const double* a, const double* b, double* r) {
  double s0, s1, s2, s3, t0, t1, t2, t3;
  two_sum(a[0], b[0], s0, t0);
  two_sum(a[1], b[1], s1, t1);
  two_sum(a[2], b[2], s2, t2);
  two_sum(a[3], b[3], s3, t3);
  two_sum(s1, t0, s1, t0);          // eps^1 class
  three_sum(s2, t0, t1);            // eps^2 class
  three_sum2(s3, t0, t2);           // eps^3 class
  t0 = __dadd_rn(__dadd_rn(t0, t1), t3);
  renorm5to4(s0, s1, s2, s3, t0, r);
}

__device__ __forceinline__ void qd_mul_raw(const double* a, const double* b, double* r) {
  double p0, p1, p2, p3, p4, p5, q0, q1, q2, q3, q4, q5;
  two_prod(a[0], b[0], p0, q0);
  two_prod(a[0], b[1], p1, q1);
  two_prod(a[1], b[0], p2, q2);
  two_prod(a[0], b[2], p3, q3);
  two_prod(a[1], b[1], p4, q4);
  two_prod(a[2], b[0], p5, q5);
  three_sum(p1, p2, q0);            // eps^1 terms
  three_sum(p2, q1, q2);            // eps^2 terms, first triple
  three_sum(p3, p4, p5);            // eps^2 terms, second triple
  double s0, s1, s2, t0, t1;
  two_sum(p2, p3, s0, t0);
  two_sum(q1, p4, s1, t1);
  s2 = __dadd_rn(q2, p5);
  two_sum(s1, t0, s1, t0);
  s2 = __dadd_rn(s2, __dadd_rn(t0, t1));
  double w = __dmul_rn(a[0], b[3]);  // eps^3 terms, plain binary64
  w = __dadd_rn(w, __dmul_rn(a[1], b[2]));
  w = __dadd_rn(w, __dmul_rn(a[2], b[1]));
  w = __dadd_rn(w, __dmul_rn(a[3], b[0]));
  w = __dadd_rn(w, q0);
  w = __dadd_rn(w, q3);
  w = __dadd_rn(w, q4);
  w = __dadd_rn(w, q5);
  s1 = __dadd_rn(s1, w);
  renorm5to4(p0, p1, s0, s1, s2, r);
}

// ---- generic add / mul ----
template <int L>
__device__ __forceinline__ mp<L> mp_add(const mp<L>& x, const mp<L>& y);
template <int L>
__device__ __forceinline__ mp<L> mp_mul(const mp<L>& x, const mp<L>& y);

template <>
__device__ __forceinline__ mp<1> mp_add<1>(const mp<1>& x, const mp<1>& y) {
  mp<1> r;
  r.v[0] = __dadd_rn(x.v[0], y.v[0]);
  return r;
}
template <>
__device__ __forceinline__ mp<1> mp_mul<1>(const mp<1>& x, const mp<1>& y) {
  mp<1> r;
  r.v[0] = __dmul_rn(x.v[0], y.v[0]);
  return r;
}

// Algorithm 1
template <>
__device__ __forceinline__ mp<2> mp_add<2>(const mp<2>& x, const mp<2>& y) {
  double s, e;
  two_sum(x.v[0], y.v[0], s, e);
  double w = __dadd_rn(x.v[1], y.v[1]);
  e = __dadd_rn(e, w);
  mp<2> r;
  quick_two_sum(s, e, r.v[0], r.v[1]);
  return r;
}

// Algorithm 2
template <>
__device__ __forceinline__ mp<2> mp_mul<2>(const mp<2>& x, const mp<2>& y) {
  double p1, p2;
  two_prod(x.v[0], y.v[0], p1, p2);
  double w1 = __dmul_rn(x.v[0], y.v[1]);
  double w2 = __dmul_rn(x.v[1], y.v[0]);
  double w3 = __dadd_rn(w1, w2);
  p2 = __dadd_rn(p2, w3);
  mp<2> r;
  quick_two_sum(p1, p2, r.v[0], r.v[1]);
  return r;
}

template <>
__device__ __forceinline__ mp<4> mp_add<4>(const mp<4>& x, const mp<4>& y) {
  mp<4> r;
  qd_add_raw(x.v, y.v, r.v);
  return r;
}
template <>
__device__ __forceinline__ mp<4> mp_mul<4>(const mp<4>& x, const mp<4>& y) {
  mp<4> r;
  qd_mul_raw(x.v, y.v, r.v);
  return r;
}

// TD: QD operation with zero fourth components, fourth result folded in.
template <>
__device__ __forceinline__ mp<3> mp_add<3>(const mp<3>& x, const mp<3>& y) {
  double a[4] = {x.v[0], x.v[1], x.v[2], 0.0}, b[4] = {y.v[0], y.v[1], y.v[2], 0.0}, q[4];
  qd_add_raw(a, b, q);
  mp<3> r;
  r.v[0] = q[0]; r.v[1] = q[1]; r.v[2] = __dadd_rn(q[2], q[3]);
  return r;
}
template <>
__device__ __forceinline__ mp<3> mp_mul<3>(const mp<3>& x, const mp<3>& y) {
  double a[4] = {x.v[0], x.v[1], x.v[2], 0.0}, b[4] = {y.v[0], y.v[1], y.v[2], 0.0}, q[4];
  qd_mul_raw(a, b, q);
  mp<3> r;
  r.v[0] = q[0]; r.v[1] = q[1]; r.v[2] = __dadd_rn(q[2], q[3]);
  return r;
}

// ---- MP x binary64 (Algorithms 3, 4, 5; "M" mode) ----
template <int L>
__device__ __forceinline__ mp<L> mp_mul_d(const mp<L>& x, double y);

template <>
__device__ __forceinline__ mp<1> mp_mul_d<1>(const mp<1>& x, double y) {
  mp<1> r;
  r.v[0] = __dmul_rn(x.v[0], y);
  return r;
}
template <>
__device__ __forceinline__ mp<2> mp_mul_d<2>(const mp<2>& x, double y) {
  double p1, p2;
  two_prod(x.v[0], y, p1, p2);
  p2 = __fma_rn(x.v[1], y, p2);      // x[1]*y enters through an FMA
  mp<2> r;
  quick_two_sum(p1, p2, r.v[0], r.v[1]);
  return r;
}
template <>
__device__ __forceinline__ mp<4> mp_mul_d<4>(const mp<4>& x, double y) {
  double p0, p1, p2, q0, q1, q2;
  two_prod(x.v[0], y, p0, q0);
  two_prod(x.v[1], y, p1, q1);
  two_prod(x.v[2], y, p2, q2);
  double p3 = __dmul_rn(x.v[3], y);
  double s1, s2;
  two_sum(q0, p1, s1, s2);
  three_sum(s2, q1, p2);
  three_sum2(q1, q2, p3);
  double s4 = __dadd_rn(q2, p2);
  mp<4> r;
  renorm5to4(p0, s1, s2, q1, s4, r.v);
  return r;
}
template <>
__device__ __forceinline__ mp<3> mp_mul_d<3>(const mp<3>& x, double y) {
  double p0, p1, p2, q0, q1, q2;
  two_prod(x.v[0], y, p0, q0);
  two_prod(x.v[1], y, p1, q1);
  two_prod(x.v[2], y, p2, q2);
  double s1, s2;
  two_sum(q0, p1, s1, s2);
  three_sum(s2, q1, p2);
  double s3 = __dadd_rn(q1, __dadd_rn(q2, p2));
  mp<3> r;
  renorm4to3(p0, s1, s2, s3, r.v);
  return r;
}

// ---- division (long division with L+1 binary64 quotient digits) ----
template <int L>
__device__ __forceinline__ mp<L> mp_sub(const mp<L>& a, const mp<L>& b) {
  return mp_add<L>(a, mp_neg<L>(b));
}

template <int L>
__device__ __forceinline__ mp<L> mp_div(const mp<L>& a, const mp<L>& b) {
  mp<L> r;
  if constexpr (L == 1) {
    r.v[0] = __ddiv_rn(a.v[0], b.v[0]);
    return r;
  }
  double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  mp<L> rem = a;
#pragma unroll
  for (int k = 0; k <= L; k++) {
    q[k] = __ddiv_rn(rem.v[0], b.v[0]);
    if (k < L) rem = mp_sub<L>(rem, mp_mul_d<L>(b, q[k]));
  }
  if constexpr (L == 2) {
    double s, e;
    quick_two_sum(q[0], q[1], s, e);
    e = __dadd_rn(e, q[2]);
    quick_two_sum(s, e, r.v[0], r.v[1]);
  } else if constexpr (L == 3) {
    renorm4to3(q[0], q[1], q[2], q[3], r.v);
  } else {
    renorm5to4(q[0], q[1], q[2], q[3], q[4], r.v);
  }
  return r;
}

// binary64 value (sum of the components, smallest first)
template <int L>
__device__ __forceinline__ double mp_to_double(const mp<L>& a) {
  double t = 0.0;
#pragma unroll
  for (int i = L - 1; i >= 0; i--) t = __dadd_rn(t, a.v[i]);
  return t;
}

}  // namespace mpk
