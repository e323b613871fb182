// fixacc.cuh -- exact fixed-point accumulation of binary64 terms on the
// integer pipe (GB300-specific alternative to the MP additions of Section 2).
//
// GB300 issues binary64 instructions at about 2 per clock per SM and 32-bit
// integer instructions at 64-128 per clock per SM.  The MP additions of a row
// sum (Algorithm 1: 11 binary64 operations; the QD sloppy add: 87) are the
// larger part of the binary64 work, so this path adds every term exactly into
// a fixed-point accumulator on the integer pipe, and the error-free products
// themselves are formed there too (fas_add_prod: the 106-bit product of two
// mantissas); the binary64 pipe keeps one FMA chain per entry (exact_prod.cuh).
//
// Register form (FixAcc, below): D signed 64-bit digits, digit j worth
// 2^(32 j + base); a term (53-bit mantissa at an arbitrary exponent) is split
// into at most three 32-bit chunks added to three consecutive digits without
// carry propagation (a digit absorbs 2^31 chunks before it could overflow).
// The shared-memory form (FixAccS, further down) keeps two non-negative digit
// arrays, one per sign, with the same window rules.  The top digit is
// head-room: terms are placed so that their top bit lies below digit D-1; a
// larger term moves the window up by whole digits (carries of the dropped
// digits are propagated first; what falls below the window is below the
// format's unit roundoff relative to the largest term).  At the end of a row
// the carries are propagated once and the value is cut into L binary64
// components by truncation (value = sum of components to 53 L bits).
#pragma once
#include <climits>
#include <stdint.h>

namespace mpk {

template <int D>
struct FixAcc {
  long long d[D];
  int base;   // binary exponent of the unit of digit 0
  bool live;  // a non-zero term has been added
  bool bad;   // a non-finite term was seen (the result is NaN)
};

template <int D>
__device__ __forceinline__ void fa_reset(FixAcc<D>& a) {
#pragma unroll
  for (int j = 0; j < D; j++) a.d[j] = 0;
  a.base = 0;
  a.live = false;
  a.bad = false;
}

// Move the window up by s digits (rare): carries of the dropped digits go up
// first, the dropped remainders are below the new window.
template <int D>
__device__ __forceinline__ void fa_shift_digits(FixAcc<D>& a, int s) {
  if (s >= D) {
#pragma unroll
    for (int j = 0; j < D; j++) a.d[j] = 0;
    a.base += 32 * s;
    return;
  }
  for (int t = 0; t < s; t++) {
    const long long c = a.d[0] >> 32;  // floor(d0 / 2^32)
#pragma unroll
    for (int j = 0; j < D - 1; j++) a.d[j] = a.d[j + 1];
    a.d[D - 1] = 0;
    a.d[0] += c;
    a.base += 32;
  }
}

// a += v exactly (up to the window's lower end)
template <int D>
__device__ __forceinline__ void fa_add(FixAcc<D>& a, double v) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int ef = (int)((bits >> 52) & 0x7ff);
  unsigned long long m = bits & 0xfffffffffffffULL;
  if (ef == 0x7ff) {
    a.bad = true;
    return;
  }
  if (ef) m |= 1ULL << 52;
  if (m == 0) return;
  const int e0 = (ef ? ef : 1) - 1075;  // v = +-m * 2^e0
  if (!a.live) {
    // place the top bit (at most e0 + 52) in the last bit of digit D-2
    a.base = e0 + 52 - (32 * (D - 1) - 1);
    a.live = true;
  }
  int pos = e0 - a.base;
  if (pos + 52 >= 32 * (D - 1)) {
    fa_shift_digits<D>(a, (pos + 52 - (32 * (D - 1) - 1) + 31) >> 5);
    pos = e0 - a.base;
  }
  if (pos < 0) {
    if (pos <= -53) return;  // entirely below the window
    m >>= -pos;              // truncate the part below the window
    pos = 0;
  }
  const int w = pos >> 5, r = pos & 31;
  const unsigned long long lo = m << r;
  const unsigned long long hi = r ? (m >> (64 - r)) : 0ULL;
  long long c0 = (long long)(lo & 0xffffffffULL), c1 = (long long)(lo >> 32), c2 = (long long)hi;
  if (bits >> 63) {
    c0 = -c0;
    c1 = -c1;
    c2 = -c2;
  }
#pragma unroll
  for (int j = 0; j < D; j++) a.d[j] += (j == w) ? c0 : ((j == w + 1) ? c1 : ((j == w + 2) ? c2 : 0LL));
}

// bits pos .. pos+63 of the non-negative multi-digit value dig (32-bit digits)
template <int D>
__device__ __forceinline__ unsigned long long fa_bits(const unsigned int (&dig)[D], int pos) {
  unsigned long long r = 0;
#pragma unroll
  for (int j = 0; j < D; j++) {
    const int sh = 32 * j - pos;
    const unsigned long long v = dig[j];
    if (sh >= 0 && sh < 64) r |= v << sh;
    else if (sh < 0 && sh > -32) r |= v >> (-sh);
  }
  return r;
}

// chunk * 2^e with the sign neg, exact for 0 <= chunk < 2^53.  A normal
// result is assembled from its fields on the integer pipe (sign, biased
// exponent of the top bit, the 52 bits below it); the rest goes through
// scalbn.  GB300 runs conversions and binary64 scaling on the slow binary64
// pipe, which the per-row flush would otherwise occupy.
__device__ __forceinline__ double chunk_to_double(unsigned long long chunk, int e, bool neg) {
  if (chunk == 0) return neg ? -0.0 : 0.0;
  const int k = 63 - __clzll((long long)chunk);  // top bit, 0 .. 52
  const int E = k + e;                           // chunk * 2^e lies in [2^E, 2^(E+1))
  if (E >= -1022 && E <= 1023) {
    const unsigned long long frac = (chunk << (52 - k)) & ((1ULL << 52) - 1);
    return __longlong_as_double((long long)(((neg ? 1ULL : 0ULL) << 63) |
                                            ((unsigned long long)(E + 1023) << 52) | frac));
  }
  const double c = scalbn((double)chunk, e);
  return neg ? -c : c;
}

// Cut the accumulated value into L binary64 components (truncation).
template <int L, int D>
__device__ __forceinline__ void fa_to_mp(const FixAcc<D>& a, double* out) {
#pragma unroll
  for (int l = 0; l < L; l++) out[l] = 0.0;
  if (a.bad) {
    out[0] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  if (!a.live) return;
  long long d[D];
#pragma unroll
  for (int j = 0; j < D; j++) d[j] = a.d[j];
#pragma unroll
  for (int j = 0; j < D - 1; j++) {
    const long long c = d[j] >> 32;
    d[j] -= c << 32;
    d[j + 1] += c;
  }
  const bool neg = d[D - 1] < 0;
  if (neg) {
#pragma unroll
    for (int j = 0; j < D; j++) d[j] = -d[j];
#pragma unroll
    for (int j = 0; j < D - 1; j++) {
      const long long c = d[j] >> 32;
      d[j] -= c << 32;
      d[j + 1] += c;
    }
  }
  unsigned int dig[D];
  int top = -1;
#pragma unroll
  for (int j = 0; j < D; j++) {
    dig[j] = (unsigned int)d[j];  // every digit is now in [0, 2^32)
    if (dig[j]) top = 32 * j + 31 - __clz(dig[j]);
  }
  if (top < 0) return;
#pragma unroll
  for (int l = 0; l < L; l++) {
    const int lsb = top - 52 - 53 * l;  // component l holds bits lsb .. lsb + 52
    if (lsb + 52 < 0) break;
    unsigned long long chunk;
    if (lsb >= 0) {
      chunk = fa_bits<D>(dig, lsb) & ((1ULL << 53) - 1);
    } else {
      chunk = (fa_bits<D>(dig, 0) << (-lsb)) & ((1ULL << 53) - 1);
    }
    out[l] = chunk_to_double(chunk, lsb + a.base, neg);  // exact: chunk < 2^53
  }
}

}  // namespace mpk

// ---------------------------------------------------------------------------
// Shared-memory digit storage.  Registers cannot be indexed by a run-time
// digit number, so the register accumulator above updates every digit with
// selects (about 8 D integer instructions per term).  Here the digits of the
// thread live in shared memory, digit j of thread t at d[j * T + t] (a
// warp's lanes hit consecutive addresses for any digit numbers), and a term
// costs three read-modify-writes of the digits it touches.  Positive and
// negative terms go to separate non-negative digit arrays (the sign selects
// the array instead of negating three chunks); the flush subtracts them.
// ---------------------------------------------------------------------------
namespace mpk {

// Base of an accumulator that has not received a term yet: every term then
// lands far above the window and takes the out-of-line window path, which
// anchors the window at that term.  (e0 - kNotLive stays below 2^31.)
constexpr int kNotLive = -(1 << 30);

template <int D, int T>
struct FixAccS {
  unsigned long long* dp;  // this thread's digit 0 of the positive terms; digit j at dp[j * T]
  unsigned long long* dn;  // ... of the negative terms
  int base;                // kNotLive until the first non-zero term
  bool bad;
};

template <int D, int T>
__device__ __forceinline__ void fas_reset(FixAccS<D, T>& a) {
#pragma unroll
  for (int j = 0; j < D; j++) {
    a.dp[j * T] = 0;
    a.dn[j * T] = 0;
  }
  a.base = kNotLive;
  a.bad = false;
}

// Move the window up by s digits (rare; out of line so that the per-term
// path stays small): carries of the dropped digits go up first.
template <int D, int T>
__device__ __noinline__ void fas_shift_smem(unsigned long long* d, int s) {
  if (s >= D) {
#pragma unroll
    for (int j = 0; j < D; j++) d[j * T] = 0;
    return;
  }
  for (int t = 0; t < s; t++) {
    const unsigned long long c = d[0] >> 32;
#pragma unroll
    for (int j = 0; j < D - 1; j++) d[j * T] = d[(j + 1) * T];
    d[(D - 1) * T] = 0;
    d[0] += c;
  }
}

// The window for a term whose top bit (at 2^top) lies at or above digit
// D - 1: the first term anchors it (top bit in the last bit of digit D - 2),
// a later one moves it up by whole digits.  Returns the new base.
template <int D, int T>
__device__ __noinline__ int fas_window(unsigned long long* dp, unsigned long long* dn, int base, int top) {
  if (base == kNotLive) return top - (32 * (D - 1) - 1);
  const int sd = (top - base - (32 * (D - 1) - 1) + 31) >> 5;
  fas_shift_smem<D, T>(dp, sd);
  fas_shift_smem<D, T>(dn, sd);
  return base + 32 * sd;
}

// a += m 2^e0 (m < 2^53; neg: a -= ...), any e0: the general path, also
// taken by subnormal terms.  Returns the new base.
template <int D, int T>
__device__ __noinline__ int fas_add_general(unsigned long long* dp, unsigned long long* dn, int base,
                                            unsigned long long m, int e0, bool negative) {
  if (m == 0) return base;
  int pos = e0 - base;
  if (pos + 52 >= 32 * (D - 1)) {
    base = fas_window<D, T>(dp, dn, base, e0 + 52);
    pos = e0 - base;
  }
  if (pos < 0) {
    if (pos <= -53) return base;
    m >>= -pos;
    pos = 0;
  }
  const int w = pos >> 5, r = pos & 31;
  const unsigned long long lo = m << r;
  const unsigned long long hi = (m >> 1) >> (63 - r);
  unsigned long long* p = (negative ? dn : dp) + w * T;
  p[0] += lo & 0xffffffffULL;
  p[T] += lo >> 32;
  p[2 * T] += hi;
  return base;
}

// a += v (neg: a -= v).  The common case, a normal binary64 term inside the
// window, takes one test on the exponent field, one on the window and one
// on the window's lower end; the rest is out of line.  Three digits receive
// the term's 32-bit chunks: with the top bit below digit D - 1 the third one
// is at most digit D - 1, so no digit index needs a bounds test.
template <int D, int T>
__device__ __forceinline__ void fas_add(FixAccS<D, T>& a, double v, bool neg) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int ef = (int)((bits >> 52) & 0x7ff);
  const bool negative = ((bits >> 63) != 0) != neg;
  if ((unsigned)(ef - 1) >= 0x7feu) {  // zero, subnormal, infinity or NaN
    if (ef == 0x7ff) {
      a.bad = true;
    } else if ((bits << 1) != 0) {
      a.base = fas_add_general<D, T>(a.dp, a.dn, a.base, bits & 0xfffffffffffffULL, -1074, negative);
    }
    return;
  }
  unsigned long long m = (bits & 0xfffffffffffffULL) | (1ULL << 52);
  const int e0 = ef - 1075;  // v = +-m 2^e0
  int pos = e0 - a.base;
  if (pos > 32 * (D - 1) - 53) {  // first term, or the window has to move up
    a.base = fas_window<D, T>(a.dp, a.dn, a.base, e0 + 52);
    pos = e0 - a.base;
  }
  if (pos < 0) {
    if (pos <= -53) return;  // entirely below the window
    m >>= -pos;              // truncate the part below the window
    pos = 0;
  }
  const int w = pos >> 5, r = pos & 31;
  const unsigned long long lo = m << r;
  const unsigned long long hi = (m >> 1) >> (63 - r);  // m >> (64 - r), and 0 for r = 0
  unsigned long long* p = (negative ? a.dn : a.dp) + w * T;
  p[0] += lo & 0xffffffffULL;
  p[T] += lo >> 32;
  p[2 * T] += hi;
}

// a += x y exactly (neg: a -= x y) for binary64 x, y: the two 53-bit
// mantissas are multiplied on the integer pipe into one exact 106-bit
// integer, added as five 32-bit chunks (with the top bit below digit D - 1
// the fifth chunk is at most digit D - 1).  This replaces TwoProd by FMA
// (two binary64 instructions) and the two separate additions of its terms:
// p + e of TwoProd is the same exact product.  Zero, subnormal and
// non-finite operands take the binary64 path.
// With twice = 1 the product is added at twice its weight (2 x y, exact: one
// more in the exponent of its chunks).
template <int D, int T>
__device__ __forceinline__ void fas_add_prod(FixAccS<D, T>& a, double x, double y, bool neg, int twice = 0) {
  const unsigned long long bx = (unsigned long long)__double_as_longlong(x);
  const unsigned long long by = (unsigned long long)__double_as_longlong(y);
  const int ex = (int)((bx >> 52) & 0x7ff), ey = (int)((by >> 52) & 0x7ff);
  if ((unsigned)(ex - 1) >= 0x7feu || (unsigned)(ey - 1) >= 0x7feu) {
    const double p = __dmul_rn(x, y);
    const double e = __fma_rn(x, y, -p);
    for (int k = 0; k <= twice; k++) {
      fas_add<D, T>(a, p, neg);
      fas_add<D, T>(a, e, neg);
    }
    return;
  }
  const bool negative = (((bx ^ by) >> 63) != 0) != neg;
  const unsigned long long mx = (bx & 0xfffffffffffffULL) | (1ULL << 52);
  const unsigned long long my = (by & 0xfffffffffffffULL) | (1ULL << 52);
  unsigned long long lo = mx * my;            // the product mx my < 2^106 as hi 2^64 + lo
  unsigned long long hi = __umul64hi(mx, my);
  const int e0 = ex + ey - 2150 + twice;      // x y = mx my 2^e0 (times 2 with twice)
  int pos = e0 - a.base;
  if (pos > 32 * (D - 1) - 106) {             // top bit (at most e0 + 105) at or above digit D - 1
    a.base = fas_window<D, T>(a.dp, a.dn, a.base, e0 + 105);
    pos = e0 - a.base;
  }
  if (pos < 0) {                              // truncate the part below the window
    if (pos <= -106) return;
    const int sh = -pos;
    if (sh >= 64) {
      lo = hi >> (sh - 64);
      hi = 0;
    } else {
      lo = (lo >> sh) | ((hi << 1) << (63 - sh));  // hi << (64 - sh), 0 for sh = 0
      hi >>= sh;
    }
    pos = 0;
  }
  const int w = pos >> 5, r = pos & 31;
  const unsigned long long w0 = lo << r;
  const unsigned long long w1 = (hi << r) | ((lo >> 1) >> (63 - r));  // lo >> (64 - r), 0 for r = 0
  const unsigned long long w2 = (hi >> 1) >> (63 - r);
  unsigned long long* p = (negative ? a.dn : a.dp) + w * T;
  p[0] += w0 & 0xffffffffULL;
  p[T] += w0 >> 32;
  p[2 * T] += w1 & 0xffffffffULL;
  p[3 * T] += w1 >> 32;
  p[4 * T] += w2;
}

// Row flush, kept out of line: it runs once per row and its many temporaries
// would otherwise raise the register count of the whole per-entry loop.  In
// a warp the rows of different threads end at different steps, so the flush
// mostly runs in a divergent branch: it is kept short.  One signed carry pass
// leaves 32-bit magnitude digits in dp (dn is left as it is; callers reset
// the accumulator afterwards), a negative sum is negated in two's complement,
// and each component's 53 bits come from three digits read at a computed
// index, cut by truncation.  Kernels in which every thread flushes at the
// same step (the vector kernels) take the inline form fas_flush_body, which
// keeps out[] in registers.
template <int L, int D, int T>
__device__ __forceinline__ void fas_flush_body(unsigned long long* dp, const unsigned long long* dn, int base,
                                               int flags, double* out) {
#pragma unroll
  for (int l = 0; l < L; l++) out[l] = 0.0;
  if (flags & 2) {
    out[0] = __longlong_as_double(0x7ff8000000000000LL);
    return;
  }
  if (!(flags & 1)) return;
  // value = sum_j (dp_j - dn_j) 2^(32 j); every digit is below 2^63
  long long c = 0;
#pragma unroll
  for (int j = 0; j < D; j++) {
    const long long v = (long long)dp[j * T] - (long long)dn[j * T] + c;
    c = v >> 32;  // floor(v / 2^32)
    dp[j * T] = (unsigned long long)(v & 0xffffffffLL);
  }
  // value = sum_j dp_j 2^(32 j) + c 2^(32 D); the head-room digit keeps
  // |value| below 2^(32 D), so c is 0 or -1
  const bool neg = c < 0;
  if (neg) {  // magnitude = (2^(32 D) - sum) in two's complement over D digits
    unsigned long long carry = 1;
#pragma unroll
    for (int j = 0; j < D; j++) {
      const unsigned long long t = (unsigned long long)(~(unsigned int)dp[j * T]) + carry;
      dp[j * T] = t & 0xffffffffULL;
      carry = t >> 32;
    }
  }
  int top = -1;
  for (int j = D - 1; j >= 0; j--) {
    const unsigned int dj = (unsigned int)dp[j * T];
    if (dj) {
      top = 32 * j + 31 - __clz(dj);
      break;
    }
  }
  if (top < 0) return;
  constexpr unsigned long long kMask = (1ULL << 53) - 1;
#pragma unroll
  for (int l = 0; l < L; l++) {
    const int lsb = top - 52 - 53 * l;  // component l holds bits lsb .. lsb + 52
    if (lsb + 52 < 0) break;
    unsigned long long chunk;
    if (lsb >= 0) {
      const int w = lsb >> 5, r = lsb & 31;  // w + 1 <= D - 1 since lsb + 52 <= top < 32 D
      const unsigned long long lo = dp[w * T] | (dp[(w + 1) * T] << 32);
      const unsigned long long hi = (w + 2 < D) ? dp[(w + 2) * T] : 0ULL;
      chunk = ((lo >> r) | ((hi << 1) << (63 - r))) & kMask;  // hi << (64 - r), and 0 for r = 0
    } else {
      chunk = ((dp[0] | (dp[T] << 32)) << (-lsb)) & kMask;
    }
    out[l] = chunk_to_double(chunk, lsb + base, neg);
  }
}

// The out-of-line flush returns its components by value, so they come back
// in registers instead of through a stack array whose address the call takes.
template <int L>
struct FlushOut {
  double v[L];
};

template <int L, int D, int T>
__device__ __noinline__ FlushOut<L> fas_flush(unsigned long long* dp, const unsigned long long* dn, int base,
                                              int flags) {
  FlushOut<L> r;
  fas_flush_body<L, D, T>(dp, dn, base, flags, r.v);
  return r;
}

template <int L, int D, int T>
__device__ __forceinline__ void fas_to_mp(const FixAccS<D, T>& a, double* out) {
  const FlushOut<L> r = fas_flush<L, D, T>(a.dp, a.dn, a.base, (a.base != kNotLive ? 1 : 0) | (a.bad ? 2 : 0));
#pragma unroll
  for (int l = 0; l < L; l++) out[l] = r.v[l];
}

// The same flush with the components written through a pointer.  The run
// kernel's per-entry loop sits at its register cap; there the by-value
// return costs more spills than the stack array it saves, so that kernel
// takes this form.
template <int L, int D, int T>
__device__ __noinline__ void fas_flush_to(unsigned long long* dp, const unsigned long long* dn, int base, int flags,
                                          double* out) {
  fas_flush_body<L, D, T>(dp, dn, base, flags, out);
}

template <int L, int D, int T>
__device__ __forceinline__ void fas_to_mp_to(const FixAccS<D, T>& a, double* out) {
  fas_flush_to<L, D, T>(a.dp, a.dn, a.base, (a.base != kNotLive ? 1 : 0) | (a.bad ? 2 : 0), out);
}

template <int L, int D, int T>
__device__ __forceinline__ void fas_to_mp_inline(const FixAccS<D, T>& a, double* out) {
  fas_flush_body<L, D, T>(a.dp, a.dn, a.base, (a.base != kNotLive ? 1 : 0) | (a.bad ? 2 : 0), out);
}

// ---------------------------------------------------------------------------
// Sums over many threads: every thread places its terms in register digits at
// one common base, taken from the largest term of the group (so no term moves
// the window), and the digits are then added as integers.
// ---------------------------------------------------------------------------
// position of the top mantissa bit the accumulator assumes (e0 + 52);
// INT_MIN for zero and non-finite values
__device__ __forceinline__ int top_exp(double v) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int ef = (int)((bits >> 52) & 0x7ff);
  if (ef == 0x7ff || (bits << 1) == 0) return INT_MIN;
  return (ef ? ef : 1) - 1075 + 52;
}

// digits of every thread at the base for block top exponent t
template <int D>
__device__ __forceinline__ void fa_at_top(FixAcc<D>& f, int t) {
  fa_reset<D>(f);
  if (t != INT_MIN) {
    f.base = t - (32 * (D - 1) - 1);
    f.live = true;
  }
}

}  // namespace mpk
