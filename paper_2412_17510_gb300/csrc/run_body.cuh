// run_body.cuh -- per-run summation shared by the single-matrix SpMV/SpMM
// kernels and the batched persistent kernel (arXiv 2412.17510, Section 3;
// complex by Eq. complex_spmv).
#pragma once
#include "internal.h"
#include "mp_arith.cuh"

namespace mpk {

__device__ __forceinline__ int64_t tile_pos(int64_t c, int j, int K) {
  return (c >> 5) * (32 * (int64_t)K) + (int64_t)j * 32 + (c & 31);
}

// ---------------------------------------------------------------------------
// Per-entry contribution: (sr, si) += a * x[col]  (Eq. complex_spmv order:
// re += a_re x_re; re += -(a_im x_im); im += a_re x_im; im += a_im x_re).
// ---------------------------------------------------------------------------
template <int L, bool CPLX, bool MIXED>
__device__ __forceinline__ void accumulate(const DevMat& m, int64_t pos, const double* __restrict__ x,
                                           int64_t xs, int64_t xcol_off, mp<L>& sr, mp<L>& si) {
  const int64_t col = __ldg(m.cols + pos);
  mp<L> xr, xi;
#pragma unroll
  for (int l = 0; l < L; l++) xr.v[l] = __ldg(x + (int64_t)l * xs + col * xcol_off);
  if (CPLX) {
#pragma unroll
    for (int l = 0; l < L; l++) xi.v[l] = __ldg(x + (int64_t)(L + l) * xs + col * xcol_off);
  }
  if (MIXED) {
    const double ar = __ldg(m.vals + pos);
    sr = mp_add<L>(sr, mp_mul_d<L>(xr, ar));
    if (CPLX) {
      const double ai = __ldg(m.vals + m.tlen + pos);
      sr = mp_add<L>(sr, mp_neg<L>(mp_mul_d<L>(xi, ai)));
      si = mp_add<L>(si, mp_mul_d<L>(xi, ar));
      si = mp_add<L>(si, mp_mul_d<L>(xr, ai));
    }
  } else {
    mp<L> ar;
#pragma unroll
    for (int l = 0; l < L; l++) ar.v[l] = __ldg(m.vals + (int64_t)l * m.tlen + pos);
    sr = mp_add<L>(sr, mp_mul<L>(ar, xr));
    if (CPLX) {
      mp<L> ai;
#pragma unroll
      for (int l = 0; l < L; l++) ai.v[l] = __ldg(m.vals + (int64_t)(L + l) * m.tlen + pos);
      sr = mp_add<L>(sr, mp_neg<L>(mp_mul<L>(ai, xi)));
      si = mp_add<L>(si, mp_mul<L>(ar, xi));
      si = mp_add<L>(si, mp_mul<L>(ai, xr));
    }
  }
}

template <int L, bool CPLX>
__device__ __forceinline__ void store_mp(double* __restrict__ out, int64_t ps, int64_t idx, const mp<L>& sr,
                                         const mp<L>& si) {
#pragma unroll
  for (int l = 0; l < L; l++) out[(int64_t)l * ps + idx] = sr.v[l];
  if (CPLX) {
#pragma unroll
    for (int l = 0; l < L; l++) out[(int64_t)(L + l) * ps + idx] = si.v[l];
  }
}

// One thread sums run c (entries c*K .. c*K+K-1, left to right) for the
// right-hand side rhs: a row that ends inside the run is written to y, the
// partial sum of a row cut by a run boundary goes to the carry buffer (slot
// w = 0 when the row started before the run, w = 1 when it continues past it).
// Carry layout: carry[((w*P + p)*nchunks + c)*kc + rhs].
template <int L, bool CPLX, bool MIXED>
__device__ __forceinline__ void process_run(const DevMat& m, int64_t c, int rhs, const double* __restrict__ x,
                                            int64_t xs, int64_t xoff, double* __restrict__ y, int64_t ys,
                                            int64_t yoff, double* __restrict__ carry, int kc) {
  constexpr int P = CPLX ? 2 * L : L;
  const double* xr = x + rhs;
  double* yr = y + rhs;
  const int64_t k0 = c * m.K;
  const int64_t k1 = min(k0 + (int64_t)m.K, m.nnz);
  int64_t row = __ldg(m.chunk_row + c);
  const int64_t first_row = row;
  const bool first_partial = __ldg(m.indptr + row) < k0;
  int64_t rend = __ldg(m.indptr + row + 1);
  const mp<L> z = mp_zero<L>();
  if (c == 0) {  // rows before the first stored entry are empty
    for (int64_t r = 0; r < row; r++) store_mp<L, CPLX>(yr, ys, r * yoff, z, z);
  }
  mp<L> sr = z, si = z;
  bool have = false;
  const int n = (int)(k1 - k0);
  const int64_t chunk_base = tile_pos(c, 0, m.K);
  for (int j = 0; j < n; j++) {
    accumulate<L, CPLX, MIXED>(m, chunk_base + (int64_t)j * 32, xr, xs, xoff, sr, si);
    have = true;
    const int64_t kk = k0 + j + 1;
    if (kk == rend) {
      if (row == first_row && first_partial) {
#pragma unroll
        for (int p = 0; p < P; p++)
          carry[((int64_t)(0 * P + p) * m.nchunks + c) * kc + rhs] = p < L ? sr.v[p % L] : si.v[p % L];
      } else {
        store_mp<L, CPLX>(yr, ys, row * yoff, sr, si);
      }
      sr = z;
      si = z;
      have = false;
      row++;
      while (row < m.nrows && __ldg(m.indptr + row + 1) == kk) {  // empty rows at this position
        store_mp<L, CPLX>(yr, ys, row * yoff, z, z);
        row++;
      }
      rend = row < m.nrows ? __ldg(m.indptr + row + 1) : INT64_MAX;
    }
  }
  if (have) {
    const int w = (row == first_row && first_partial) ? 0 : 1;
#pragma unroll
    for (int p = 0; p < P; p++)
      carry[((int64_t)(w * P + p) * m.nchunks + c) * kc + rhs] = p < L ? sr.v[p % L] : si.v[p % L];
  }
}


// ---------------------------------------------------------------------------
// Exact-accumulation variant (handles created with MPSPMV_EXACT_ACC): per
// entry only the error-free products run on the binary64 pipe, their terms
// are added exactly on the integer pipe (fixacc.cuh).
//   P mode, L = 2: TwoProd(a0, x0) + fma(a0, x1, a1 x0)           4 binary64 ops, 3 terms
//           L = 3: TwoProd for i+j <= 1, FMA chain for i+j = 2    9 ops, 7 terms
//           L = 4: TwoProd for i+j <= 2, FMA chain for i+j = 3   16 ops, 13 terms
//   M mode: TwoProd(a, x_j) for j < L-1, a x_{L-1}                 2L-1 ops, 2L-1 terms
// Products of order below the format's unit roundoff are dropped or rounded
// once; the row value is then exact up to the window and cut to L components.
// ---------------------------------------------------------------------------
}  // namespace mpk
#include "fixacc.cuh"
namespace mpk {

template <int L>
struct AccDigits {
  static constexpr int D = L == 1 ? 4 : (L == 2 ? 6 : (L == 3 ? 8 : 10));
};

template <int L, int D>
__device__ __forceinline__ void add_prod(FixAcc<D>& acc, const mp<L>& a, const mp<L>& x, bool negate) {
  const double sg = negate ? -1.0 : 1.0;  // exact sign flip of every term
  if constexpr (L == 1) {
    double p, e;
    two_prod(a.v[0], x.v[0], p, e);
    fa_add<D>(acc, sg * p);
    fa_add<D>(acc, sg * e);
  } else if constexpr (L == 2) {
    double p, e;
    two_prod(a.v[0], x.v[0], p, e);
    const double c = __fma_rn(a.v[0], x.v[1], __dmul_rn(a.v[1], x.v[0]));
    fa_add<D>(acc, sg * p);
    fa_add<D>(acc, sg * e);
    fa_add<D>(acc, sg * c);
  } else if constexpr (L == 3) {
    double p, e;
    two_prod(a.v[0], x.v[0], p, e);
    fa_add<D>(acc, sg * p);
    fa_add<D>(acc, sg * e);
    two_prod(a.v[0], x.v[1], p, e);
    fa_add<D>(acc, sg * p);
    fa_add<D>(acc, sg * e);
    two_prod(a.v[1], x.v[0], p, e);
    fa_add<D>(acc, sg * p);
    fa_add<D>(acc, sg * e);
    const double c = __fma_rn(a.v[0], x.v[2], __fma_rn(a.v[1], x.v[1], __dmul_rn(a.v[2], x.v[0])));
    fa_add<D>(acc, sg * c);
  } else {
#pragma unroll
    for (int i = 0; i < 3; i++) {
#pragma unroll
      for (int j = 0; j < 3 - i; j++) {
        double p, e;
        two_prod(a.v[i], x.v[j], p, e);
        fa_add<D>(acc, sg * p);
        fa_add<D>(acc, sg * e);
      }
    }
    const double c =
        __fma_rn(a.v[0], x.v[3], __fma_rn(a.v[1], x.v[2], __fma_rn(a.v[2], x.v[1], __dmul_rn(a.v[3], x.v[0]))));
    fa_add<D>(acc, sg * c);
  }
}

// binary64 matrix value (M mode)
template <int L, int D>
__device__ __forceinline__ void add_prod_d(FixAcc<D>& acc, double a, const mp<L>& x, bool negate) {
  const double sg = negate ? -1.0 : 1.0;
#pragma unroll
  for (int j = 0; j < L - 1; j++) {
    double p, e;
    two_prod(a, x.v[j], p, e);
    fa_add<D>(acc, sg * p);
    fa_add<D>(acc, sg * e);
  }
  fa_add<D>(acc, sg * __dmul_rn(a, x.v[L - 1]));
}

template <int L, bool CPLX, bool MIXED, int D>
__device__ __forceinline__ void accumulate_exact(const DevMat& m, int64_t pos, const double* __restrict__ x,
                                                 int64_t xs, int64_t xcol_off, FixAcc<D>& sr, FixAcc<D>& si) {
  const int64_t col = __ldg(m.cols + pos);
  mp<L> xr, xi;
#pragma unroll
  for (int l = 0; l < L; l++) xr.v[l] = __ldg(x + (int64_t)l * xs + col * xcol_off);
  if (CPLX) {
#pragma unroll
    for (int l = 0; l < L; l++) xi.v[l] = __ldg(x + (int64_t)(L + l) * xs + col * xcol_off);
  }
  if (MIXED) {
    const double ar = __ldg(m.vals + pos);
    add_prod_d<L, D>(sr, ar, xr, false);
    if (CPLX) {
      const double ai = __ldg(m.vals + m.tlen + pos);
      add_prod_d<L, D>(sr, ai, xi, true);
      add_prod_d<L, D>(si, ar, xi, false);
      add_prod_d<L, D>(si, ai, xr, false);
    }
  } else {
    mp<L> ar;
#pragma unroll
    for (int l = 0; l < L; l++) ar.v[l] = __ldg(m.vals + (int64_t)l * m.tlen + pos);
    add_prod<L, D>(sr, ar, xr, false);
    if (CPLX) {
      mp<L> ai;
#pragma unroll
      for (int l = 0; l < L; l++) ai.v[l] = __ldg(m.vals + (int64_t)(L + l) * m.tlen + pos);
      add_prod<L, D>(sr, ai, xi, true);
      add_prod<L, D>(si, ar, xi, false);
      add_prod<L, D>(si, ai, xr, false);
    }
  }
}

template <int L, bool CPLX, int D>
__device__ __forceinline__ void flush_exact(const FixAcc<D>& sr, const FixAcc<D>& si, mp<L>& r, mp<L>& i) {
  fa_to_mp<L, D>(sr, r.v);
  if (CPLX) fa_to_mp<L, D>(si, i.v);
}

// Same run structure, carries and empty-row handling as process_run.
template <int L, bool CPLX, bool MIXED>
__device__ __forceinline__ void process_run_exact(const DevMat& m, int64_t c, int rhs, const double* __restrict__ x,
                                                  int64_t xs, int64_t xoff, double* __restrict__ y, int64_t ys,
                                                  int64_t yoff, double* __restrict__ carry, int kc) {
  constexpr int P = CPLX ? 2 * L : L;
  constexpr int D = AccDigits<L>::D;
  const double* xr = x + rhs;
  double* yr = y + rhs;
  const int64_t k0 = c * m.K;
  const int64_t k1 = min(k0 + (int64_t)m.K, m.nnz);
  int64_t row = __ldg(m.chunk_row + c);
  const int64_t first_row = row;
  const bool first_partial = __ldg(m.indptr + row) < k0;
  int64_t rend = __ldg(m.indptr + row + 1);
  const mp<L> z = mp_zero<L>();
  if (c == 0) {
    for (int64_t r = 0; r < row; r++) store_mp<L, CPLX>(yr, ys, r * yoff, z, z);
  }
  FixAcc<D> sr, si;
  fa_reset<D>(sr);
  fa_reset<D>(si);
  bool have = false;
  const int n = (int)(k1 - k0);
  const int64_t chunk_base = tile_pos(c, 0, m.K);
  for (int j = 0; j < n; j++) {
    accumulate_exact<L, CPLX, MIXED, D>(m, chunk_base + (int64_t)j * 32, xr, xs, xoff, sr, si);
    have = true;
    const int64_t kk = k0 + j + 1;
    if (kk == rend) {
      mp<L> vr, vi;
      flush_exact<L, CPLX, D>(sr, si, vr, vi);
      if (row == first_row && first_partial) {
#pragma unroll
        for (int p = 0; p < P; p++)
          carry[((int64_t)(0 * P + p) * m.nchunks + c) * kc + rhs] = p < L ? vr.v[p % L] : vi.v[p % L];
      } else {
        store_mp<L, CPLX>(yr, ys, row * yoff, vr, vi);
      }
      fa_reset<D>(sr);
      fa_reset<D>(si);
      have = false;
      row++;
      while (row < m.nrows && __ldg(m.indptr + row + 1) == kk) {
        store_mp<L, CPLX>(yr, ys, row * yoff, z, z);
        row++;
      }
      rend = row < m.nrows ? __ldg(m.indptr + row + 1) : INT64_MAX;
    }
  }
  if (have) {
    mp<L> vr, vi;
    flush_exact<L, CPLX, D>(sr, si, vr, vi);
    const int w = (row == first_row && first_partial) ? 0 : 1;
#pragma unroll
    for (int p = 0; p < P; p++)
      carry[((int64_t)(w * P + p) * m.nchunks + c) * kc + rhs] = p < L ? vr.v[p % L] : vi.v[p % L];
  }
}

}  // namespace mpk
