// Host stand-in for <cuda_runtime.h>, used only by the host build of the
// device arithmetic headers in tests/host_build/harness.cpp.  It maps the
// CUDA function qualifiers to plain C++ and gives the few device intrinsics
// those headers call their IEEE 754 meaning on the host: correctly rounded
// binary64 add, subtract, multiply, divide and fused multiply-add, bit casts,
// the high half of a 64 x 64-bit product, count of leading zeros, and the
// classification functions the device code calls unqualified.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#define __device__
#define __host__
#define __forceinline__ inline __attribute__((always_inline))
#define __noinline__ __attribute__((noinline))

inline double __dadd_rn(double a, double b) { return a + b; }
inline double __dsub_rn(double a, double b) { return a - b; }
inline double __dmul_rn(double a, double b) { return a * b; }
inline double __ddiv_rn(double a, double b) { return a / b; }
inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
inline long long __double_as_longlong(double d) {
  long long r;
  std::memcpy(&r, &d, sizeof r);
  return r;
}
inline double __longlong_as_double(long long v) {
  double r;
  std::memcpy(&r, &v, sizeof r);
  return r;
}
inline unsigned long long __umul64hi(unsigned long long a, unsigned long long b) {
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
inline int __clz(int x) { return x == 0 ? 32 : __builtin_clz((unsigned)x); }
inline int __clzll(long long x) { return x == 0 ? 64 : __builtin_clzll((unsigned long long)x); }
using std::isinf;
using std::isnan;
using std::isfinite;
using std::scalbn;
using std::max;
using std::min;
