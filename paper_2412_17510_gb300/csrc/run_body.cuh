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


}  // namespace mpk
#include "exact_prod.cuh"
#include "wide.cuh"
namespace mpk {

// Operands of one stored entry, loaded ahead of their use.
template <int L, bool CPLX, bool MIXED>
struct EntryIn {
  mp<L> xr, xi;  // x[col] (real / imaginary components)
  mp<L> ar, ai;  // matrix value (MIXED: binary64 in ar.v[0], ai.v[0])
};

template <int L, bool CPLX, bool MIXED>
__device__ __forceinline__ void load_entry(const DevMat& m, int64_t pos, int64_t col, const double* __restrict__ x,
                                           int64_t xs, int64_t xcol_off, EntryIn<L, CPLX, MIXED>& e) {
#pragma unroll
  for (int l = 0; l < L; l++) e.xr.v[l] = __ldg(x + (int64_t)l * xs + col * xcol_off);
  if (CPLX) {
#pragma unroll
    for (int l = 0; l < L; l++) e.xi.v[l] = __ldg(x + (int64_t)(L + l) * xs + col * xcol_off);
  }
  if (MIXED) {
    e.ar.v[0] = __ldg(m.vals + pos);
    if (CPLX) e.ai.v[0] = __ldg(m.vals + m.tlen + pos);
  } else {
#pragma unroll
    for (int l = 0; l < L; l++) e.ar.v[l] = __ldg(m.vals + (int64_t)l * m.tlen + pos);
    if (CPLX) {
#pragma unroll
      for (int l = 0; l < L; l++) e.ai.v[l] = __ldg(m.vals + (int64_t)(L + l) * m.tlen + pos);
    }
  }
}

template <int L, bool CPLX, bool MIXED, class Acc>
__device__ __forceinline__ void compute_entry(const EntryIn<L, CPLX, MIXED>& e, Acc& sr, Acc& si) {
  if (MIXED) {
    add_prod_d<Acc, L>(sr, e.ar.v[0], e.xr, false);
    if (CPLX) {
      add_prod_d<Acc, L>(sr, e.ai.v[0], e.xi, true);
      add_prod_d<Acc, L>(si, e.ar.v[0], e.xi, false);
      add_prod_d<Acc, L>(si, e.ai.v[0], e.xr, false);
    }
  } else {
    add_prod<Acc, L>(sr, e.ar, e.xr, false);
    if (CPLX) {
      add_prod<Acc, L>(sr, e.ai, e.xi, true);
      add_prod<Acc, L>(si, e.ar, e.xi, false);
      add_prod<Acc, L>(si, e.ai, e.xr, false);
    }
  }
}

// Same run structure, carries and empty-row handling as process_run.  T is
// the block size (the accumulator digits of the block live in shared memory).
template <int L, bool CPLX, bool MIXED, int T>
__device__ __forceinline__ void process_run_exact(const DevMat& m, int64_t c, int rhs, const double* __restrict__ x,
                                                  int64_t xs, int64_t xoff, double* __restrict__ y, int64_t ys,
                                                  int64_t yoff, double* __restrict__ carry, int kc) {
  constexpr int P = CPLX ? 2 * L : L;
  constexpr int D = AccDigits<L>::D;
  __shared__ unsigned long long s_digits[(CPLX ? 4 : 2) * D * T];
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
  FixAccS<D, T> sr, si;
  sr.dp = s_digits + threadIdx.x;
  sr.dn = s_digits + D * T + threadIdx.x;
  si.dp = s_digits + (CPLX ? 2 * D * T : 0) + threadIdx.x;
  si.dn = s_digits + (CPLX ? 3 * D * T : D * T) + threadIdx.x;
  fas_reset<D, T>(sr);
  if (CPLX) fas_reset<D, T>(si);
  bool have = false;
  const int n = (int)(k1 - k0);
  const int64_t chunk_base = tile_pos(c, 0, m.K);
  // Entries are loaded in the step that uses them: the resident warps (6 to
  // 8 blocks of 128 threads) hide the gathers' latency, and holding the next
  // entry's operands in registers cost more (spills, fewer blocks) than it
  // saved.
#pragma unroll 1
  for (int j = 0; j < n; j++) {
    EntryIn<L, CPLX, MIXED> cur;
    const int64_t pos = chunk_base + (int64_t)j * 32;
    load_entry<L, CPLX, MIXED>(m, pos, __ldg(m.cols + pos), xr, xs, xoff, cur);
    compute_entry<L, CPLX, MIXED>(cur, sr, si);
    have = true;
    const int64_t kk = k0 + j + 1;
    if (kk == rend) {
      mp<L> vr, vi = z;
      fas_to_mp_to<L, D, T>(sr, vr.v);
      if (CPLX) fas_to_mp_to<L, D, T>(si, vi.v);
      if (row == first_row && first_partial) {
#pragma unroll
        for (int p = 0; p < P; p++)
          carry[((int64_t)(0 * P + p) * m.nchunks + c) * kc + rhs] = p < L ? vr.v[p % L] : vi.v[p % L];
      } else {
        store_mp<L, CPLX>(yr, ys, row * yoff, vr, vi);
      }
      fas_reset<D, T>(sr);
      if (CPLX) fas_reset<D, T>(si);
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
    mp<L> vr, vi = z;
    fas_to_mp_to<L, D, T>(sr, vr.v);
    if (CPLX) fas_to_mp_to<L, D, T>(si, vi.v);
    const int w = (row == first_row && first_partial) ? 0 : 1;
#pragma unroll
    for (int p = 0; p < P; p++)
      carry[((int64_t)(w * P + p) * m.nchunks + c) * kc + rhs] = p < L ? vr.v[p % L] : vi.v[p % L];
  }
}

// One whole row per thread from the sliced-ELL copy (exact accumulation):
// entry q of row r at base + 32 q + r % 32, so the 32 threads of a warp read
// 32 consecutive slots per step, and all of them flush at the end of the
// loop instead of whenever one of their rows ends.  T is the block size.
template <int L, bool CPLX, bool MIXED, int T>
__device__ __forceinline__ void process_row_exact(const DevMat& m, int64_t base, int64_t r,
                                                  const double* __restrict__ x, int64_t xs, int64_t xoff,
                                                  double* __restrict__ y, int64_t ys, int64_t yoff) {
  constexpr int D = AccDigits<L>::D;
  __shared__ unsigned long long s_digits[(CPLX ? 4 : 2) * D * T];
  FixAccS<D, T> sr, si;
  sr.dp = s_digits + threadIdx.x;
  sr.dn = s_digits + D * T + threadIdx.x;
  si.dp = s_digits + (CPLX ? 2 * D * T : 0) + threadIdx.x;
  si.dn = s_digits + (CPLX ? 3 * D * T : D * T) + threadIdx.x;
  fas_reset<D, T>(sr);
  if (CPLX) fas_reset<D, T>(si);
  const int64_t len = __ldg(m.indptr + r + 1) - __ldg(m.indptr + r);
  const int64_t slot0 = base + (r & 31);
#pragma unroll 1
  for (int64_t q = 0; q < len; q++) {
    EntryIn<L, CPLX, MIXED> e;
    const int64_t pos = slot0 + 32 * q;
    load_entry<L, CPLX, MIXED>(m, pos, __ldg(m.cols + pos), x, xs, xoff, e);
    compute_entry<L, CPLX, MIXED>(e, sr, si);
  }
  mp<L> vr, vi = mp_zero<L>();
  fas_to_mp<L, D, T>(sr, vr.v);
  if (CPLX) fas_to_mp<L, D, T>(si, vi.v);
  store_mp<L, CPLX>(y, ys, r * yoff, vr, vi);
}

// ---------------------------------------------------------------------------
// Wide-x form (wide.cuh): single-vector products of exact handles with one
// stored value plane.  xr points at the column records (8 words per column
// part; complex: the real part's record, then the imaginary part's).
// ---------------------------------------------------------------------------
template <bool CPLX>
__device__ __forceinline__ void load_rec(const uint32_t* __restrict__ xr, int64_t col, int part, uint32_t* rec) {
  const uint4* q = reinterpret_cast<const uint4*>(xr + (col * (CPLX ? 2 : 1) + part) * kWideRecWords);
  const uint4 u0 = __ldg(q), u1 = __ldg(q + 1);
  rec[0] = u0.x; rec[1] = u0.y; rec[2] = u0.z; rec[3] = u0.w;
  rec[4] = u1.x; rec[5] = u1.y; rec[6] = u1.z; rec[7] = u1.w;
}

// Software pipeline of an entry stream (entry q at pos0 + 32 q).  Before
// entry q is summed the pipe holds the records and values of entries
// q .. q + kWideRecAhead - 1 (their gathers issued) and the columns and values
// of entries q + kWideRecAhead .. q + kWideColAhead - 1 (loads issued).  Each
// step takes entry q, issues the gather of entry q + kWideRecAhead from the
// column that arrived and loads the column and value of entry
// q + kWideColAhead.  Depths chosen by timing the benchmark's matrices: one
// record and one column ahead is fastest (columns 2 or 3 entries ahead, or
// two records ahead, cost registers and time; power-law TD 2.85 -> 3.07 ms
// with columns 2 ahead).  Holding the column as 32 bits instead of 64 took
// power-law QD from 3.67 to 3.31 ms and the stencil from 0.638 to 0.574 ms.
constexpr int kWideRecAhead = 1;
constexpr int kWideColAhead = 2;
constexpr int kWideColSlots = kWideColAhead - kWideRecAhead;
static_assert(kWideRecAhead >= 1 && kWideColSlots >= 1, "pipeline depths");

// V = 1 (real) or 2 (complex: the real part's record and value, then the
// imaginary part's)
template <int V>
struct WidePipe {
  uint32_t rec[kWideRecAhead][V][kWideRecWords];  // gathered records
  double a[kWideRecAhead][V];                     // their values
  int32_t col[kWideColSlots];                     // columns of the entries after them
  double av[kWideColSlots][V];                    // their values
};

template <int V>
__device__ __forceinline__ void wide_load_vals(const DevMat& m, int64_t pos, double* a) {
  a[0] = __ldg(m.vals + pos);
  if (V == 2) a[1] = __ldg(m.vals + m.tlen + pos);
}

template <int V>
__device__ __forceinline__ void wide_load_recs(const uint32_t* __restrict__ xr, int64_t col,
                                               uint32_t (&rec)[V][kWideRecWords]) {
#pragma unroll
  for (int p = 0; p < V; p++) load_rec<V == 2>(xr, col, p, rec[p]);
}

template <int V>
__device__ __forceinline__ void wide_pipe_start(const DevMat& m, int64_t pos0, int n, const uint32_t* __restrict__ xr,
                                                WidePipe<V>& pp) {
#pragma unroll
  for (int i = 0; i < kWideRecAhead; i++) {
    if (i < n) {
      const int64_t pos = pos0 + 32 * (int64_t)i;
      wide_load_vals<V>(m, pos, pp.a[i]);
      wide_load_recs<V>(xr, __ldg(m.cols + pos), pp.rec[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < kWideColSlots; i++) {
    if (kWideRecAhead + i < n) {
      const int64_t pos = pos0 + 32 * (int64_t)(kWideRecAhead + i);
      pp.col[i] = __ldg(m.cols + pos);
      wide_load_vals<V>(m, pos, pp.av[i]);
    }
  }
}

template <int V>
__device__ __forceinline__ void wide_pipe_step(const DevMat& m, int64_t pos0, int q, int n,
                                               const uint32_t* __restrict__ xr, WidePipe<V>& pp, double (&a)[V],
                                               uint32_t (&rec)[V][kWideRecWords]) {
#pragma unroll
  for (int p = 0; p < V; p++) {
    a[p] = pp.a[0][p];
#pragma unroll
    for (int w = 0; w < kWideRecWords; w++) rec[p][w] = pp.rec[0][p][w];
  }
#pragma unroll
  for (int i = 0; i + 1 < kWideRecAhead; i++)
#pragma unroll
    for (int p = 0; p < V; p++) {
      pp.a[i][p] = pp.a[i + 1][p];
#pragma unroll
      for (int w = 0; w < kWideRecWords; w++) pp.rec[i][p][w] = pp.rec[i + 1][p][w];
    }
  if (q + kWideRecAhead < n) {
#pragma unroll
    for (int p = 0; p < V; p++) pp.a[kWideRecAhead - 1][p] = pp.av[0][p];
    wide_load_recs<V>(xr, pp.col[0], pp.rec[kWideRecAhead - 1]);
  }
#pragma unroll
  for (int i = 0; i + 1 < kWideColSlots; i++) {
    pp.col[i] = pp.col[i + 1];
#pragma unroll
    for (int p = 0; p < V; p++) pp.av[i][p] = pp.av[i + 1][p];
  }
  if (q + kWideColAhead < n) {
    const int64_t pos = pos0 + 32 * (int64_t)(q + kWideColAhead);
    pp.col[kWideColSlots - 1] = __ldg(m.cols + pos);
    wide_load_vals<V>(m, pos, pp.av[kWideColSlots - 1]);
  }
}

// One entry's products into the row sums (complex in the order re += a_re
// X_re, im += a_im X_re, re -= a_im X_im, im += a_re X_im).
template <int L, bool CPLX, int D, int T>
__device__ __forceinline__ void wide_sum_entry(const double (&a)[CPLX ? 2 : 1],
                                               const uint32_t (&rec)[CPLX ? 2 : 1][kWideRecWords],
                                               FixAccS<D, T>& sr, FixAccS<D, T>& si) {
  fas_add_wide<L, D, T>(sr, a[0], rec[0], false);
  if constexpr (CPLX) {
    fas_add_wide<L, D, T>(si, a[1], rec[0], false);
    fas_add_wide<L, D, T>(sr, a[1], rec[1], true);
    fas_add_wide<L, D, T>(si, a[0], rec[1], false);
  }
}

// One complex entry loaded in the step that sums it (the imaginary part's
// record after the real part's two products).  Complex QD takes this form:
// with two records in flight its registers cost more than the pipeline
// saved (A/B on the complex band: 10.8 against 9.8 Gnnz/s), while complex DD
// and TD gain from the pipeline (DD 18.6 -> 21.9).
template <int L, int D, int T>
__device__ __forceinline__ void wide_entry_cplx(const DevMat& m, int64_t pos, const uint32_t* __restrict__ xr,
                                                FixAccS<D, T>& sr, FixAccS<D, T>& si) {
  const int64_t col = __ldg(m.cols + pos);
  const double ar = __ldg(m.vals + pos), ai = __ldg(m.vals + m.tlen + pos);
  uint32_t rec[kWideRecWords];
  load_rec<true>(xr, col, 0, rec);
  fas_add_wide<L, D, T>(sr, ar, rec, false);   // a_re X_re
  fas_add_wide<L, D, T>(si, ai, rec, false);   // a_im X_re
  load_rec<true>(xr, col, 1, rec);
  fas_add_wide<L, D, T>(sr, ai, rec, true);    // - a_im X_im
  fas_add_wide<L, D, T>(si, ar, rec, false);   // a_re X_im
}

template <int L, bool CPLX>
struct WidePipelined {
  static constexpr bool value = !(CPLX && L == 4);
};

// One row per thread from the sliced-ELL copy, wide-x form.
template <int L, bool CPLX, int T>
__device__ __forceinline__ void process_row_wide(const DevMat& m, int64_t base, int64_t r,
                                                 const uint32_t* __restrict__ xr, double* __restrict__ y, int64_t ys) {
  constexpr int D = Wide<L>::D;
  __shared__ unsigned long long s_digits[(CPLX ? 4 : 2) * D * T];
  FixAccS<D, T> sr, si;
  sr.dp = s_digits + threadIdx.x;
  sr.dn = s_digits + D * T + threadIdx.x;
  si.dp = s_digits + (CPLX ? 2 * D * T : 0) + threadIdx.x;
  si.dn = s_digits + (CPLX ? 3 * D * T : D * T) + threadIdx.x;
  fas_reset<D, T>(sr);
  if (CPLX) fas_reset<D, T>(si);
  const int64_t len = __ldg(m.indptr + r + 1) - __ldg(m.indptr + r);
  const int64_t slot0 = base + (r & 31);
  if constexpr (WidePipelined<L, CPLX>::value) {
    constexpr int V = CPLX ? 2 : 1;
    WidePipe<V> pp;
    wide_pipe_start<V>(m, slot0, (int)len, xr, pp);
#pragma unroll 1
    for (int q = 0; q < (int)len; q++) {
      double a[V];
      uint32_t rec[V][kWideRecWords];
      wide_pipe_step<V>(m, slot0, q, (int)len, xr, pp, a, rec);
      wide_sum_entry<L, CPLX, D, T>(a, rec, sr, si);
    }
  } else {
#pragma unroll 1
    for (int64_t q = 0; q < len; q++) wide_entry_cplx<L, D, T>(m, slot0 + 32 * q, xr, sr, si);
  }
  mp<L> vr, vi = mp_zero<L>();
  fas_to_mp_inline<L, D, T>(sr, vr.v);
  if (CPLX) fas_to_mp_inline<L, D, T>(si, vi.v);
  store_mp<L, CPLX>(y, ys, r, vr, vi);
}

// A finished row of a real wide-x run, staged for the finishing pass: the
// accumulator's D signed digit differences dp_j - dn_j (each digit is below
// 2^63, so the difference fits) and one word with the window base and the
// flags the flush takes.  The finishing pass runs the flush on these digits,
// so the components are those of the inline flush; the run kernel's part is
// about a quarter of the flush's instructions, and the divergent lanes (only
// those whose row ends at this entry) wait that much less.
template <int D, int T>
__device__ __forceinline__ void fas_stage(const FixAccS<D, T>& a, int64_t* __restrict__ out) {
  static_assert(D + 1 <= kRowDigWords, "row buffer words");
#pragma unroll
  for (int j = 0; j < D; j++) out[j] = (long long)a.dp[j * T] - (long long)a.dn[j * T];
  const int flags = (a.base != kNotLive ? 1 : 0) | (a.bad ? 2 : 0);
  out[D] = (int64_t)(uint32_t)a.base | ((int64_t)flags << 32);
}

// One run per thread, wide-x form: the run structure, carries and empty-row
// handling of process_run_exact (single right-hand side).  The row flushes
// are inline here (fas_to_mp_inline): the wide kernels hold fewer registers
// per entry than the decomposed ones, and the call cost more than it saved
// (power-law QD 3.90 -> 3.67 ms).
template <int L, bool CPLX, int T>
__device__ __forceinline__ void process_run_wide(const DevMat& m, int64_t c, const uint32_t* __restrict__ xr,
                                                 double* __restrict__ y, int64_t ys, double* __restrict__ carry,
                                                 int kc, int64_t* __restrict__ rowdig) {
  constexpr int P = CPLX ? 2 * L : L;
  constexpr int D = Wide<L>::D;
  __shared__ unsigned long long s_digits[(CPLX ? 4 : 2) * D * T];
  const int64_t k0 = c * m.K;
  const int64_t k1 = min(k0 + (int64_t)m.K, m.nnz);
  int64_t row = __ldg(m.chunk_row + c);
  const int64_t first_row = row;
  const bool first_partial = __ldg(m.indptr + row) < k0;
  int64_t rend = __ldg(m.indptr + row + 1);
  const mp<L> z = mp_zero<L>();
  if (c == 0) {
    for (int64_t r = 0; r < row; r++) store_mp<L, CPLX>(y, ys, r, z, z);
  }
  FixAccS<D, T> sr, si;
  sr.dp = s_digits + threadIdx.x;
  sr.dn = s_digits + D * T + threadIdx.x;
  si.dp = s_digits + (CPLX ? 2 * D * T : 0) + threadIdx.x;
  si.dn = s_digits + (CPLX ? 3 * D * T : D * T) + threadIdx.x;
  fas_reset<D, T>(sr);
  if (CPLX) fas_reset<D, T>(si);
  bool have = false;
  const int n = (int)(k1 - k0);
  const int64_t chunk_base = tile_pos(c, 0, m.K);
  constexpr int V = CPLX ? 2 : 1;
  WidePipe<V> pp;
  if constexpr (WidePipelined<L, CPLX>::value) wide_pipe_start<V>(m, chunk_base, n, xr, pp);
#pragma unroll 1
  for (int j = 0; j < n; j++) {
    if constexpr (WidePipelined<L, CPLX>::value) {
      double a[V];
      uint32_t rec[V][kWideRecWords];
      wide_pipe_step<V>(m, chunk_base, j, n, xr, pp, a, rec);
      wide_sum_entry<L, CPLX, D, T>(a, rec, sr, si);
    } else {
      wide_entry_cplx<L, D, T>(m, chunk_base + (int64_t)j * 32, xr, sr, si);
    }
    have = true;
    const int64_t kk = k0 + j + 1;
    if (kk == rend) {
      if constexpr (CPLX) {
        mp<L> vr, vi;
        fas_to_mp_inline<L, D, T>(sr, vr.v);
        fas_to_mp_inline<L, D, T>(si, vi.v);
        if (row == first_row && first_partial) {
#pragma unroll
          for (int p = 0; p < P; p++) carry[((int64_t)p * m.nchunks + c) * kc] = p < L ? vr.v[p % L] : vi.v[p % L];
        } else {
          store_mp<L, CPLX>(y, ys, row, vr, vi);
        }
      } else {
        // the finishing pass writes y, or for a row begun in an earlier run
        // this run's partial into the carry buffer
        fas_stage<D, T>(sr, rowdig + row * kRowDigWords);
      }
      fas_reset<D, T>(sr);
      if (CPLX) fas_reset<D, T>(si);
      have = false;
      row++;
      while (row < m.nrows && __ldg(m.indptr + row + 1) == kk) {
        store_mp<L, CPLX>(y, ys, row, z, z);
        row++;
      }
      rend = row < m.nrows ? __ldg(m.indptr + row + 1) : INT64_MAX;
    }
  }
  if (have) {
    mp<L> vr, vi = z;
    fas_to_mp_inline<L, D, T>(sr, vr.v);
    if (CPLX) fas_to_mp_inline<L, D, T>(si, vi.v);
    const int w = (row == first_row && first_partial) ? 0 : 1;
#pragma unroll
    for (int p = 0; p < P; p++)
      carry[((int64_t)(w * P + p) * m.nchunks + c) * kc] = p < L ? vr.v[p % L] : vi.v[p % L];
  }
}

// Exact sum of the run partials of a row cut by run boundaries (exact-
// accumulation handles): the starting run's partial (slot 1 of run c0) and
// the partials of runs c0+1 .. c1 (slot 0), components off .. off+L-1 of the
// carry buffer.  All components go into register digits at the base of the
// largest one and are cut to L components once.  The result depends only on
// the set of components, so every kernel that combines a row this way (one
// thread or one warp per row) gives the same bits.
template <int L>
__device__ __forceinline__ mp<L> combine_exact(const double* __restrict__ carry, int64_t nchunks, int kc, int rhs,
                                               int P, int off, int64_t c0, int64_t c1) {
  constexpr int D = AccDigits<L>::D;
  auto ld = [&](int w, int l, int64_t c) { return carry[((int64_t)(w * P + off + l) * nchunks + c) * kc + rhs]; };
  int t = INT_MIN;
#pragma unroll
  for (int l = 0; l < L; l++) t = max(t, top_exp(ld(1, l, c0)));
  for (int64_t c = c0 + 1; c <= c1; c++)
#pragma unroll
    for (int l = 0; l < L; l++) t = max(t, top_exp(ld(0, l, c)));
  FixAcc<D> f;
  fa_at_top<D>(f, t);
#pragma unroll
  for (int l = 0; l < L; l++) fa_add<D>(f, ld(1, l, c0));
  for (int64_t c = c0 + 1; c <= c1; c++)
#pragma unroll
    for (int l = 0; l < L; l++) fa_add<D>(f, ld(0, l, c));
  mp<L> r;
  fa_to_mp<L, D>(f, r.v);
  return r;
}

// The same sum by one warp: lane j takes runs c0+1+j, c0+1+j+32, ... (lane 0
// also the starting partial); the base comes from a warp-wide maximum and
// the digits are added by integer shuffles.  Valid in lane 0.
template <int L>
__device__ __forceinline__ mp<L> combine_exact_warp(const double* __restrict__ carry, int64_t nchunks, int kc,
                                                    int rhs, int P, int off, int64_t c0, int64_t c1, int lane) {
  constexpr int D = AccDigits<L>::D;
  auto ld = [&](int w, int l, int64_t c) { return carry[((int64_t)(w * P + off + l) * nchunks + c) * kc + rhs]; };
  int t = INT_MIN;
  if (lane == 0)
#pragma unroll
    for (int l = 0; l < L; l++) t = max(t, top_exp(ld(1, l, c0)));
  for (int64_t c = c0 + 1 + lane; c <= c1; c += 32)
#pragma unroll
    for (int l = 0; l < L; l++) t = max(t, top_exp(ld(0, l, c)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t = max(t, __shfl_xor_sync(0xffffffffu, t, o));
  FixAcc<D> f;
  fa_at_top<D>(f, t);
  if (lane == 0)
#pragma unroll
    for (int l = 0; l < L; l++) fa_add<D>(f, ld(1, l, c0));
  for (int64_t c = c0 + 1 + lane; c <= c1; c += 32)
#pragma unroll
    for (int l = 0; l < L; l++) fa_add<D>(f, ld(0, l, c));
  f.bad = __any_sync(0xffffffffu, f.bad);
#pragma unroll
  for (int j = 0; j < D; j++)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f.d[j] += __shfl_down_sync(0xffffffffu, f.d[j], o);
  mp<L> r;
  fa_to_mp<L, D>(f, r.v);
  return r;
}

}  // namespace mpk
