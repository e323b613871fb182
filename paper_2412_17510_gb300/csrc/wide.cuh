// wide.cuh -- the wide-x form of the exact-accumulation SpMV (MPSPMV_EXACT_ACC
// handles whose matrix values are binary64, single-vector products).
//
// The exact form of exact_prod.cuh forms, per stored entry, L - 1 exact
// 106-bit products a x_j and one rounded product a x_{L-1}, each decoded,
// placed and added on its own (QD: 18 digit updates per entry).  Here x is
// turned once per product, per column, into one fixed-point number
// X = s M 2^E with a W-word mantissa (W = 4 / 5 / 7 words of 32 bits for
// DD / TD / QD): x truncated toward zero to 32 W bits below its top bit, so
// |a X - a x| < 2^(1-32W) |a x|, below the unit roundoff of each format.  An
// entry is then one 53 x 32W-bit integer product a X (its lowest 32-bit word
// dropped), added to the row's exact sum as W + 2 aligned 32-bit chunks:
// 6 / 7 / 9 digit updates per entry instead of 8 / 13 / 18, one decode of a,
// one window test, and no binary64 instruction.  The row sum and its cut to
// L components are those of fixacc.cuh, in an accumulator one digit wider
// (a margin above the products, so that the window rarely moves).
//
// Record of one column part (real or imaginary): 8 words of 32 bits, words
// 0 .. W-1 the mantissa M (least significant first, top bit of word W-1 set
// unless X = 0; unused words zero), word 7 the exponent E of M's last bit
// shifted left by 2, with the sign in bit 1 and "a component is not finite"
// in bit 0.  (QD uses words 0 .. 6 for M.)
#pragma once
#include <climits>
#include <stdint.h>

#include "fixacc.cuh"

namespace mpk {

template <int L>
struct Wide {
  static constexpr int W = L == 2 ? 4 : (L == 3 ? 5 : 7);   // mantissa words
  static constexpr int DX = W + 2;                          // digits of the record's construction
  static constexpr int D = L == 2 ? 8 : (L == 3 ? 9 : 11);  // digits of the row accumulator
};

// Bits the row window keeps above a product when it is placed (the row's
// first product) or moved: later products up to 2^32 larger than the one
// that placed it do not move it again.  The extra digit of Wide<L>::D holds
// this margin, so the window's lower end is where it would be without it.
constexpr int kWideMargin = 32;

constexpr int kWideRecWords = 8;

// Build the record of one column part from its L binary64 components: the
// components are added exactly (each truncated below the base of a DX-digit
// register accumulator anchored at the largest component's top bit), the
// sum is cut to the 32 W bits below its top bit.
template <int L>
__device__ __forceinline__ void wide_build(const double* c, uint32_t* rec) {
  constexpr int W = Wide<L>::W, DX = Wide<L>::DX;
  for (int i = 0; i < kWideRecWords; i++) rec[i] = 0u;
  int t0 = INT_MIN;
  bool bad = false;
#pragma unroll
  for (int k = 0; k < L; k++) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(c[k]);
    if (((bits >> 52) & 0x7ff) == 0x7ff) bad = true;
    t0 = max(t0, top_exp(c[k]));
  }
  if (bad) {
    rec[7] = 1u;
    return;
  }
  if (t0 == INT_MIN) return;  // every component zero
  FixAcc<DX> f;
  fa_at_top<DX>(f, t0);
#pragma unroll
  for (int k = 0; k < L; k++) fa_add<DX>(f, c[k]);
  // carries, sign and magnitude of the sum (as in fa_to_mp)
  long long d[DX];
#pragma unroll
  for (int j = 0; j < DX; j++) d[j] = f.d[j];
#pragma unroll
  for (int j = 0; j < DX - 1; j++) {
    const long long cc = d[j] >> 32;
    d[j] -= cc << 32;
    d[j + 1] += cc;
  }
  const bool neg = d[DX - 1] < 0;
  if (neg) {
#pragma unroll
    for (int j = 0; j < DX; j++) d[j] = -d[j];
#pragma unroll
    for (int j = 0; j < DX - 1; j++) {
      const long long cc = d[j] >> 32;
      d[j] -= cc << 32;
      d[j + 1] += cc;
    }
  }
  unsigned int dig[DX];
  int top = -1;
#pragma unroll
  for (int j = 0; j < DX; j++) {
    dig[j] = (unsigned int)d[j];
    if (dig[j]) top = 32 * j + 31 - __clz((int)dig[j]);
  }
  if (top < 0) return;  // the components cancel
  const int lsb = top - 32 * W + 1;  // bit of the sum that becomes M's last bit
#pragma unroll
  for (int i = 0; i < W; i++) {
    // word i of M: bits lsb + 32 i .. lsb + 32 i + 31 of the digits (zero below bit 0)
    const int p = lsb + 32 * i;
    unsigned int w = 0u;
#pragma unroll
    for (int j = 0; j < DX; j++) {
      const int sh = 32 * j - p;  // position of digit j's bit 0 within the word
      if (sh >= 0 && sh < 32) w |= dig[j] << sh;
      else if (sh < 0 && sh > -32) w |= dig[j] >> (-sh);
    }
    rec[i] = w;
  }
  const int E = f.base + lsb;
  rec[7] = ((uint32_t)E << 2) | (neg ? 2u : 0u);
}

// The product a X without its lowest 32-bit word, as W + 1 words (least
// significant first), for a binary64 mantissa ma < 2^53.
template <int W>
__device__ __forceinline__ void wide_mul(unsigned long long ma, const uint32_t* M, uint32_t* P) {
  const uint32_t alo = (uint32_t)ma, ahi = (uint32_t)(ma >> 32);
  uint32_t q[W + 2];
  unsigned long long t = 0;
#pragma unroll
  for (int i = 0; i < W; i++) {
    t = (unsigned long long)alo * M[i] + (t >> 32);
    q[i] = (uint32_t)t;
  }
  q[W] = (uint32_t)(t >> 32);
  t = 0;
#pragma unroll
  for (int i = 0; i < W; i++) {
    t = (unsigned long long)ahi * M[i] + q[i + 1] + (t >> 32);
    q[i + 1] = (uint32_t)t;
  }
  q[W + 1] = (uint32_t)(t >> 32);
#pragma unroll
  for (int i = 0; i < W + 1; i++) P[i] = q[i + 1];
}

// A product whose last bit lies below the window (pos < 0): shift it right
// by -pos (truncating the magnitude) and add it at digit 0.  Kept out of
// line: it only runs for terms far smaller than the row's largest.
template <int W, int T>
__device__ __noinline__ void wide_add_low(unsigned long long* p, const uint32_t* P, int pos) {
  const int sh = -pos;
  const int ws = sh >> 5, bs = sh & 31;
  for (int i = 0; i < W + 1; i++) {
    const int s0 = i + ws;
    if (s0 > W) break;
    const unsigned long long lo = P[s0];
    const unsigned long long hi = (s0 + 1 <= W) ? P[s0 + 1] : 0ull;
    p[i * T] += (uint32_t)(((hi << 32) | lo) >> bs);
  }
}

// acc += a X (neg: acc -= a X) for a binary64 a and the record rec of X.
template <int L, int D, int T>
__device__ __forceinline__ void fas_add_wide(FixAccS<D, T>& acc, double a, const uint32_t* rec, bool neg) {
  constexpr int W = Wide<L>::W;
  const uint32_t meta = rec[7];
  if (meta & 1u) {  // a component of x is not finite
    acc.bad = true;
    return;
  }
  if (rec[W - 1] == 0u) return;  // X = 0
  const unsigned long long bits = (unsigned long long)__double_as_longlong(a);
  const int ef = (int)((bits >> 52) & 0x7ff);
  unsigned long long ma = bits & 0xfffffffffffffULL;
  if (ef) ma |= 1ULL << 52;
  if (ma == 0) return;  // a = 0
  const int ea = (ef ? ef : 1) - 1075;
  const int E = (int)meta >> 2;
  const bool negative = (((bits >> 63) != 0) != ((meta & 2u) != 0)) != neg;
  uint32_t P[W + 1];
  wide_mul<W>(ma, rec, P);
  const int e0 = ea + E + 32;  // weight of P's last bit
  int pos = e0 - acc.base;
  // P has at most 53 + 32 W - 32 bits: its top bit lies at most at pos + 20 + 32 W
  if (pos > 32 * (D - 1) - 21 - 32 * W) {
    acc.base = fas_window<D, T>(acc.dp, acc.dn, acc.base, e0 + 20 + 32 * W + kWideMargin);
    pos = e0 - acc.base;
  }
  unsigned long long* p = negative ? acc.dn : acc.dp;
  if (pos < 0) {
    if (pos > -(21 + 32 * W)) wide_add_low<W, T>(p, P, pos);
    return;
  }
  const int w = pos >> 5, r = pos & 31;
  p += w * T;
  // the W + 1 words shifted left by r: W + 2 chunks (funnel shifts)
  p[0] += (uint32_t)((unsigned long long)P[0] << r);
#pragma unroll
  for (int i = 1; i < W + 1; i++)
    p[i * T] += (uint32_t)(((((unsigned long long)P[i]) << 32) | P[i - 1]) >> (32 - r));
  p[(W + 1) * T] += (uint32_t)(((unsigned long long)P[W]) >> (32 - r));
}

}  // namespace mpk
