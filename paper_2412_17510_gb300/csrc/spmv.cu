// spmv.cu -- multiple-precision CSR SpMV / SpMM on the binary64 pipe
// (arXiv 2412.17510, Section 3; complex by Eq. complex_spmv).
//
// Work decomposition (GB300 design, not the paper's AVX2 one): the stored
// entries are cut into runs of K consecutive entries and each thread sums one
// run, left to right, with one MP multiply and one MP add per entry -- the
// same operation sequence as a sequential row sweep.  Every thread therefore
// issues the same binary64 instruction stream (K products and K additions),
// whatever the row lengths: short rows, 27-entry stencil rows and
// 20,000-entry power-law rows all keep the FP64 pipe equally busy.  A row
// that ends inside a run is written directly; a row cut by a run boundary
// leaves a partial sum per run in a carry buffer, and a second kernel adds
// the partials of each such row in run order.
//
// Rows that lie inside one run are therefore computed exactly as a
// sequential sweep computes them (bit-identical), and rows cut by run
// boundaries differ only in the association of the partial sums.
#include <algorithm>

#include "internal.h"
#include "mp_arith.cuh"
#include "run_body.cuh"

using namespace mpk;

namespace {

constexpr int kThreads = 128;

// ---------------------------------------------------------------------------
// Build: sorted triplets (duplicates adjacent) -> tiled column / value arrays.
// ---------------------------------------------------------------------------
template <int L, bool CPLX, bool MIXED>
__global__ void build_tiles_kernel(DevMat m, int32_t* __restrict__ cols_out, double* __restrict__ vals_out,
                                   const double* __restrict__ vin, int64_t nin, int vin_limbs,
                                   const int64_t* __restrict__ run_start, const int64_t* __restrict__ col_src) {
  int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= m.nnz) return;
  const int64_t t0 = run_start ? run_start[u] : u;
  const int64_t t1 = run_start ? run_start[u + 1] : u + 1;
  const int64_t c = u / m.K;
  const int j = (int)(u - c * m.K);
  const int64_t pos = tile_pos(c, j, m.K);
  cols_out[pos] = (int32_t)col_src[t0];
  constexpr int NC = CPLX ? 2 : 1;
#pragma unroll
  for (int part = 0; part < NC; part++) {
    if (MIXED) {
      double acc = vin[(int64_t)part * nin + t0];
      for (int64_t t = t0 + 1; t < t1; t++) acc = __dadd_rn(acc, vin[(int64_t)part * nin + t]);
      vals_out[(int64_t)part * m.tlen + pos] = acc;
    } else {
      mp<L> acc;
#pragma unroll
      for (int l = 0; l < L; l++) acc.v[l] = l < vin_limbs ? vin[(int64_t)(part * vin_limbs + l) * nin + t0] : 0.0;
      for (int64_t t = t0 + 1; t < t1; t++) {
        mp<L> v;
#pragma unroll
        for (int l = 0; l < L; l++) v.v[l] = l < vin_limbs ? vin[(int64_t)(part * vin_limbs + l) * nin + t] : 0.0;
        acc = mp_add<L>(acc, v);
      }
#pragma unroll
      for (int l = 0; l < L; l++) vals_out[(int64_t)(part * L + l) * m.tlen + pos] = acc.v[l];
    }
  }
}

// Sliced-ELL copy of the tiled arrays: entry u (CSR order) of row r at
// offset q goes to slice_ptr[r / 32] + 32 q + r % 32.
__global__ void build_sell_kernel(DevMat m, const int64_t* __restrict__ slice_ptr, int32_t* __restrict__ cols_out,
                                  double* __restrict__ vals_out, int64_t sell_len, int Pv) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= m.nnz) return;
  int64_t lo = 0, hi = m.nrows - 1;  // the row holding entry u: last r with indptr[r] <= u
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (__ldg(m.indptr + mid) <= u) lo = mid;
    else hi = mid - 1;
  }
  const int64_t r = lo, q = u - __ldg(m.indptr + r);
  const int64_t ps = __ldg(slice_ptr + (r >> 5)) + 32 * q + (r & 31);
  const int64_t c = u / m.K;
  const int64_t pt = tile_pos(c, (int)(u - c * m.K), m.K);
  cols_out[ps] = m.cols[pt];
  for (int p = 0; p < Pv; p++) vals_out[(int64_t)p * sell_len + ps] = m.vals[(int64_t)p * m.tlen + pt];
}

// One thread per row of the sliced-ELL copy (exact accumulation, single
// vector).  It holds fewer registers than the run kernel: timed over 5..8
// resident blocks, QD runs best with 7 and DD/TD with 8.
template <int L, bool CPLX, bool MIXED>
__global__ void __launch_bounds__(kThreads, CPLX ? 3 : (L == 4 ? 7 : 8))
    sell_exact_kernel(DevMat m, const int64_t* __restrict__ slice_ptr, const double* __restrict__ x, int64_t xs,
                      int64_t xoff, double* __restrict__ y, int64_t ys, int64_t yoff, const int* __restrict__ gate) {
  if (gate && *gate != 0) return;
  const int64_t r = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (r >= m.nrows) return;
  process_row_exact<L, CPLX, MIXED, kThreads>(m, __ldg(slice_ptr + (r >> 5)), r, x, xs, xoff, y, ys, yoff);
}

// ---------------------------------------------------------------------------
// Run kernel.  Vectors: x plane stride xs, entry j at x[j*xoff] within a plane
// (xoff = ldx for SpMM, 1 for SpMV); y likewise.  rhs selects the column of a
// multi-right-hand-side product (0 for SpMV); `kp` threads share a run.
// Carry layout: carry[((w*P + p)*nchunks + c)*kc + rhs], w = 0 first-row
// partial, w = 1 last-row partial.
// The exact variant is bound by integer issue and latency, so it asks for
// more resident blocks (fewer registers): timed on the stencil and
// power-law steps over 5..8 blocks, DD and TD run best with 8 and QD with
// 7; the complex variant's shared memory allows only 5 blocks and more
// register pressure spills.
// ---------------------------------------------------------------------------
template <int L>
constexpr int exact_min_blocks() {
  return L == 4 ? 7 : 8;
}

template <int L, bool CPLX, bool MIXED, bool EXACT>
__global__ void __launch_bounds__(kThreads, EXACT ? (CPLX ? 3 : exact_min_blocks<L>()) : 1) spmv_runs_kernel(DevMat m, const double* __restrict__ x, int64_t xs,
                                                             int64_t xoff, double* __restrict__ y, int64_t ys,
                                                             int64_t yoff, double* __restrict__ carry, int kc,
                                                             int kp, int k, const int* __restrict__ gate) {
  if (gate && *gate != 0) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t c = t / kp;
  const int rhs = (int)(t - c * kp);
  if (c >= m.nchunks || rhs >= k) return;
  if (EXACT) process_run_exact<L, CPLX, MIXED, kThreads>(m, c, rhs, x, xs, xoff, y, ys, yoff, carry, kc);
  else process_run<L, CPLX, MIXED>(m, c, rhs, x, xs, xoff, y, ys, yoff, carry, kc);
}

// Rows cut by run boundaries: partial of the run where the row starts (slot
// w = 1), then the partials of the following runs (slot w = 0) in order.
// One thread per (row, right-hand side) for rows spanning few runs.
template <int L, bool CPLX, bool EXACT>
__global__ void __launch_bounds__(kThreads) combine_kernel(DevMat m, double* __restrict__ y, int64_t ys,
                                                           int64_t yoff, const double* __restrict__ carry,
                                                           int kc, int k, const int* __restrict__ gate) {
  constexpr int P = CPLX ? 2 * L : L;
  if (gate && *gate != 0) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t s = t / k;
  const int rhs = (int)(t - s * k);
  if (s >= m.nshort) return;
  const int64_t r = __ldg(m.split_rows + s);
  const int64_t c0 = __ldg(m.indptr + r) / m.K;
  const int64_t c1 = (__ldg(m.indptr + r + 1) - 1) / m.K;
  if (EXACT) {
    const mp<L> er = combine_exact<L>(carry, m.nchunks, kc, rhs, P, 0, c0, c1);
    const mp<L> ei = CPLX ? combine_exact<L>(carry, m.nchunks, kc, rhs, P, L, c0, c1) : mp_zero<L>();
    store_mp<L, CPLX>(y + rhs, ys, r * yoff, er, ei);
    return;
  }
  auto ld = [&](int w, int p, int64_t c) { return carry[((int64_t)(w * P + p) * m.nchunks + c) * kc + rhs]; };
  mp<L> sr, si;
#pragma unroll
  for (int l = 0; l < L; l++) sr.v[l] = ld(1, l, c0);
  if (CPLX) {
#pragma unroll
    for (int l = 0; l < L; l++) si.v[l] = ld(1, L + l, c0);
  }
  for (int64_t c = c0 + 1; c <= c1; c++) {
    mp<L> ar, ai;
#pragma unroll
    for (int l = 0; l < L; l++) ar.v[l] = ld(0, l, c);
    sr = mp_add<L>(sr, ar);
    if (CPLX) {
#pragma unroll
      for (int l = 0; l < L; l++) ai.v[l] = ld(0, L + l, c);
      si = mp_add<L>(si, ai);
    }
  }
  store_mp<L, CPLX>(y + rhs, ys, r * yoff, sr, si);
}

template <int L>
__device__ __forceinline__ mp<L> shfl_down_mp(const mp<L>& a, int off) {
  mp<L> r;
#pragma unroll
  for (int l = 0; l < L; l++) r.v[l] = __shfl_down_sync(0xffffffffu, a.v[l], off);
  return r;
}

// Rows spanning many runs (power-law rows): one warp per (row, right-hand
// side).  Lane l sums the following-run partials c0+1+l, c0+1+l+32, ... in
// order, a shuffle tree adds the 32 lane sums, and the starting run's partial
// goes in front.
template <int L, bool CPLX, bool EXACT>
__global__ void __launch_bounds__(kThreads) combine_long_kernel(DevMat m, double* __restrict__ y, int64_t ys,
                                                                int64_t yoff, const double* __restrict__ carry,
                                                                int kc, int k, const int* __restrict__ gate) {
  constexpr int P = CPLX ? 2 * L : L;
  if (gate && *gate != 0) return;
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t s = wid / k;
  const int rhs = (int)(wid - s * k);
  if (s >= m.nsplit - m.nshort) return;  // whole warp leaves together
  const int64_t r = __ldg(m.split_rows + m.nshort + s);
  const int64_t c0 = __ldg(m.indptr + r) / m.K;
  const int64_t c1 = (__ldg(m.indptr + r + 1) - 1) / m.K;
  if (EXACT) {
    const mp<L> er = combine_exact_warp<L>(carry, m.nchunks, kc, rhs, P, 0, c0, c1, lane);
    const mp<L> ei = CPLX ? combine_exact_warp<L>(carry, m.nchunks, kc, rhs, P, L, c0, c1, lane) : mp_zero<L>();
    if (lane == 0) store_mp<L, CPLX>(y + rhs, ys, r * yoff, er, ei);
    return;
  }
  auto ld = [&](int w, int p, int64_t c) { return carry[((int64_t)(w * P + p) * m.nchunks + c) * kc + rhs]; };
  mp<L> sr = mp_zero<L>(), si = mp_zero<L>();
  for (int64_t c = c0 + 1 + lane; c <= c1; c += 32) {
    mp<L> ar, ai;
#pragma unroll
    for (int l = 0; l < L; l++) ar.v[l] = ld(0, l, c);
    sr = mp_add<L>(sr, ar);
    if (CPLX) {
#pragma unroll
      for (int l = 0; l < L; l++) ai.v[l] = ld(0, L + l, c);
      si = mp_add<L>(si, ai);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    mp<L> o = shfl_down_mp<L>(sr, off);
    if (lane < off) sr = mp_add<L>(sr, o);
    if (CPLX) {
      o = shfl_down_mp<L>(si, off);
      if (lane < off) si = mp_add<L>(si, o);
    }
  }
  if (lane == 0) {
    mp<L> fr, fi;
#pragma unroll
    for (int l = 0; l < L; l++) fr.v[l] = ld(1, l, c0);
    fr = mp_add<L>(fr, sr);
    if (CPLX) {
#pragma unroll
      for (int l = 0; l < L; l++) fi.v[l] = ld(1, L + l, c0);
      fi = mp_add<L>(fi, si);
    }
    store_mp<L, CPLX>(y + rhs, ys, r * yoff, fr, fi);
  }
}

// xi[col * P + p] = x[p * n + col]: the components of one column adjacent,
// so an exact run kernel gathers them from one 32-byte sector (real QD)
// instead of P sectors of P planes.  Gated like the run kernel.
__global__ void interleave_kernel(const double* __restrict__ x, int64_t n, int P, double* __restrict__ xi,
                                  const int* gate) {
  if (gate && *gate != 0) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * P) return;
  const int64_t col = t / P;
  const int p = (int)(t - col * P);
  xi[t] = x[(int64_t)p * n + col];
}

// Records of the wide-x form (wide.cuh): one thread per column part, the
// real part's record then the imaginary part's.  Gated like the run kernel.
template <int L, bool CPLX>
__global__ void widen_kernel(const double* __restrict__ x, int64_t n, uint32_t* __restrict__ out, const int* gate) {
  if (gate && *gate != 0) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  constexpr int parts = CPLX ? 2 : 1;
  if (t >= n * parts) return;
  const int64_t col = t / parts;
  const int part = (int)(t - col * parts);
  double c[L];
#pragma unroll
  for (int l = 0; l < L; l++) c[l] = x[(int64_t)(part * L + l) * n + col];
  uint32_t rec[kWideRecWords];
  wide_build<L>(c, rec);
  uint4* o = reinterpret_cast<uint4*>(out + t * kWideRecWords);
  o[0] = make_uint4(rec[0], rec[1], rec[2], rec[3]);
  o[1] = make_uint4(rec[4], rec[5], rec[6], rec[7]);
}

// Wide-x form, one row per thread (sliced-ELL copy) and one run per thread.
// The real kernels keep a second gather in flight per thread (software
// pipeline, run_body.cuh) and hold more registers.  Resident blocks, timed
// on the stencil and power-law steps: the row kernel 6; the real run kernel,
// whose loop stages finished rows instead of flushing them (82 / 88 / 96
// registers for DD / TD / QD), 6 for DD (power-law DD 2.21 -> 2.15 ms
// against 5; at 7 it spills), 5 for TD and 4 for QD.  The QD kernel then
// takes 96 registers and runs 5 blocks per SM all the same; a bound of 5
// compiles to a slightly slower kernel (2.89 against 2.87 ms).
constexpr int kWideRowBlocks = 6;

template <int L>
constexpr int wide_run_blocks() {
  return L == 2 ? 6 : (L == 3 ? 5 : 4);
}

template <int L, bool CPLX>
__global__ void __launch_bounds__(kThreads, CPLX ? 3 : kWideRowBlocks)
    sell_wide_kernel(DevMat m, const int64_t* __restrict__ slice_ptr, const uint32_t* __restrict__ xw,
                     double* __restrict__ y, int64_t ys, const int* __restrict__ gate) {
  if (gate && *gate != 0) return;
  const int64_t r = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (r >= m.nrows) return;
  process_row_wide<L, CPLX, kThreads>(m, __ldg(slice_ptr + (r >> 5)), r, xw, y, ys);
}

template <int L, bool CPLX>
__global__ void __launch_bounds__(kThreads, CPLX ? 3 : wide_run_blocks<L>())
    spmv_runs_wide_kernel(DevMat m, const uint32_t* __restrict__ xw, double* __restrict__ y, int64_t ys,
                          double* __restrict__ carry, int kc, int64_t* __restrict__ rowdig,
                          const int* __restrict__ gate) {
  if (gate && *gate != 0) return;
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= m.nchunks) return;
  process_run_wide<L, CPLX, kThreads>(m, c, xw, y, ys, carry, kc, rowdig);
}

// The finishing pass of real wide-x products over runs, one row per thread.
// The run kernel staged (fas_stage) the sum of every non-empty row over the
// run that holds its last entry; it is flushed here, with the flush
// arithmetic of the run kernels.  A row whose entries all lie in that run
// goes to y; a row begun in an earlier run is that run's first partial and
// goes to the carry buffer (slot 0 of the run), which the combine kernels
// read after this pass.  Empty rows are written by the run kernel.
template <int L>
__global__ void __launch_bounds__(kThreads) rowdig_finish_kernel(DevMat m, const int64_t* __restrict__ rowdig,
                                                                 double* __restrict__ y, int64_t ys,
                                                                 double* __restrict__ carry, int kc,
                                                                 const int* __restrict__ gate) {
  if (gate && *gate != 0) return;
  const int64_t r = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (r >= m.nrows) return;
  const int64_t k0 = __ldg(m.indptr + r), k1 = __ldg(m.indptr + r + 1);
  if (k1 == k0) return;
  const int64_t c1 = (k1 - 1) / m.K;
  constexpr int D = Wide<L>::D;
  __shared__ unsigned long long s_digits[2 * D * kThreads];
  unsigned long long* dp = s_digits + threadIdx.x;
  unsigned long long* dn = s_digits + D * kThreads + threadIdx.x;
  const int64_t* q = rowdig + r * kRowDigWords;
#pragma unroll
  for (int j = 0; j < D; j++) {
    dp[j * kThreads] = (unsigned long long)__ldg(q + j);  // dp - dn is the staged difference
    dn[j * kThreads] = 0ull;
  }
  const int64_t meta = __ldg(q + D);
  double v[L];
  fas_flush_body<L, D, kThreads>(dp, dn, (int)(uint32_t)meta, (int)(meta >> 32), v);
  if (k0 / m.K == c1) {
#pragma unroll
    for (int l = 0; l < L; l++) y[(int64_t)l * ys + r] = v[l];
  } else {
#pragma unroll
    for (int l = 0; l < L; l++) carry[((int64_t)l * m.nchunks + c1) * kc] = v[l];
  }
}

// y = 0 (single right-hand side), gated
__global__ void zero_kernel(double* y, int64_t ys, int64_t yoff, int64_t nrows, int P, const int* gate) {
  if (gate && *gate != 0) return;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nrows * P) return;
  const int64_t p = t / nrows, r = t - p * nrows;
  y[p * ys + r * yoff] = 0.0;
}

template <int L, bool CPLX>
int launch_combine(const mpspmv_mat* h, const DevMat& m, double* y, int64_t ys, int64_t yoff, int k, const int* gate,
                   cudaStream_t s);

template <int L, bool CPLX, bool MIXED>
int launch_all(const mpspmv_mat* h, const double* x, int64_t xs, int64_t xoff, double* y, int64_t ys,
               int64_t yoff, int k, const int* gate, cudaStream_t s) {
  const DevMat m = h->view();
  if (h->nnz == 0 && gate) {
    zero_kernel<<<(unsigned)((h->nrows * h->P + kThreads - 1) / kThreads + 1), kThreads, 0, s>>>(y, ys, yoff, h->nrows,
                                                                                          h->P, gate);
    MPS_CUDA(cudaGetLastError());
    return MPSPMV_OK;
  }
  if (h->nnz == 0) {
    // no stored entry: y = 0
    for (int p = 0; p < h->P; p++)
      for (int c = 0; c < k; c++) {
        if (yoff == 1) {
          MPS_CUDA(cudaMemsetAsync(y + (int64_t)p * ys, 0, sizeof(double) * h->nrows, s));
          break;
        }
        MPS_CUDA(cudaMemset2DAsync(y + (int64_t)p * ys + c, sizeof(double) * yoff, 0, sizeof(double), h->nrows, s));
      }
    return MPSPMV_OK;
  }
  int kp = 1;
  while (kp < k) kp <<= 1;
  if constexpr (MIXED && L > 1) {
    if (h->d_xwide && k == 1 && xoff == 1 && yoff == 1) {  // single vector, wide-x form
      const int64_t tot = (int64_t)(CPLX ? 2 : 1) * h->ncols;
      if (tot > 0) {
        widen_kernel<L, CPLX><<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(x, xs, h->d_xwide,
                                                                                          gate);
        MPS_CUDA(cudaGetLastError());
      }
      if (h->sell_len > 0) {
        DevMat ms = m;
        ms.cols = h->d_sell_cols;
        ms.vals = h->d_sell_vals;
        ms.tlen = h->sell_len;
        sell_wide_kernel<L, CPLX><<<(unsigned)((h->nrows + kThreads - 1) / kThreads), kThreads, 0, s>>>(
            ms, h->d_slice_ptr, h->d_xwide, y, ys, gate);
        MPS_CUDA(cudaGetLastError());
        return MPSPMV_OK;
      }
      if (!CPLX && !h->d_rowdig) return MPSPMV_EINVAL;  // allocated with the records for real handles
      spmv_runs_wide_kernel<L, CPLX><<<(unsigned)((h->nchunks + kThreads - 1) / kThreads), kThreads, 0, s>>>(
          m, h->d_xwide, y, ys, h->d_carry, h->carry_k, h->d_rowdig, gate);
      MPS_CUDA(cudaGetLastError());
      if constexpr (!CPLX) {
        rowdig_finish_kernel<L><<<(unsigned)((h->nrows + kThreads - 1) / kThreads), kThreads, 0, s>>>(
            m, h->d_rowdig, y, ys, h->d_carry, h->carry_k, gate);
        MPS_CUDA(cudaGetLastError());
      }
      return launch_combine<L, CPLX>(h, m, y, ys, yoff, k, gate, s);
    }
  }
  if (h->exact && k == 1 && h->d_xint) {  // single vector: gather from the interleaved copy
    const int64_t tot = (int64_t)h->P * h->ncols;
    interleave_kernel<<<(unsigned)((tot + kThreads - 1) / kThreads), kThreads, 0, s>>>(x, h->ncols, h->P, h->d_xint,
                                                                                     gate);
    MPS_CUDA(cudaGetLastError());
    x = h->d_xint;
    xs = 1;
    xoff = h->P;
  }
  if (h->exact && k == 1 && h->sell_len > 0) {  // short, even rows: whole rows per thread
    DevMat ms = m;
    ms.cols = h->d_sell_cols;
    ms.vals = h->d_sell_vals;
    ms.tlen = h->sell_len;
    sell_exact_kernel<L, CPLX, MIXED><<<(unsigned)((h->nrows + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        ms, h->d_slice_ptr, x, xs, xoff, y, ys, yoff, gate);
    MPS_CUDA(cudaGetLastError());
    return MPSPMV_OK;
  }
  const int64_t threads = h->nchunks * kp;
  const int64_t blocks = (threads + kThreads - 1) / kThreads;
  if (h->exact)
    spmv_runs_kernel<L, CPLX, MIXED, true><<<(unsigned)blocks, kThreads, 0, s>>>(m, x, xs, xoff, y, ys, yoff,
                                                                              h->d_carry, h->carry_k, kp, k, gate);
  else
    spmv_runs_kernel<L, CPLX, MIXED, false><<<(unsigned)blocks, kThreads, 0, s>>>(m, x, xs, xoff, y, ys, yoff,
                                                                               h->d_carry, h->carry_k, kp, k, gate);
  MPS_CUDA(cudaGetLastError());
  return launch_combine<L, CPLX>(h, m, y, ys, yoff, k, gate, s);
}

// Rows cut by run boundaries: the combine kernels over the carry buffer.
template <int L, bool CPLX>
int launch_combine(const mpspmv_mat* h, const DevMat& m, double* y, int64_t ys, int64_t yoff, int k, const int* gate,
                   cudaStream_t s) {
  if (h->nshort > 0) {
    const int64_t ct = h->nshort * k;
    const unsigned nb = (unsigned)((ct + kThreads - 1) / kThreads);
    if (h->exact)
      combine_kernel<L, CPLX, true><<<nb, kThreads, 0, s>>>(m, y, ys, yoff, h->d_carry, h->carry_k, k, gate);
    else
      combine_kernel<L, CPLX, false><<<nb, kThreads, 0, s>>>(m, y, ys, yoff, h->d_carry, h->carry_k, k, gate);
    MPS_CUDA(cudaGetLastError());
  }
  if (h->nsplit > h->nshort) {
    const int64_t ct = (h->nsplit - h->nshort) * k * 32;
    const unsigned nb = (unsigned)((ct + kThreads - 1) / kThreads);
    if (h->exact)
      combine_long_kernel<L, CPLX, true><<<nb, kThreads, 0, s>>>(m, y, ys, yoff, h->d_carry, h->carry_k, k, gate);
    else
      combine_long_kernel<L, CPLX, false><<<nb, kThreads, 0, s>>>(m, y, ys, yoff, h->d_carry, h->carry_k, k, gate);
    MPS_CUDA(cudaGetLastError());
  }
  return MPSPMV_OK;
}

template <int L, bool CPLX, bool MIXED>
int build_one(mpspmv_mat* h, const double* vin, int64_t nin, int vin_limbs, const int64_t* run_start,
              const int64_t* col_src, cudaStream_t s) {
  if (h->nnz == 0) return MPSPMV_OK;
  const int64_t blocks = (h->nnz + kThreads - 1) / kThreads;
  build_tiles_kernel<L, CPLX, MIXED><<<(unsigned)blocks, kThreads, 0, s>>>(h->view(), h->d_cols, h->d_vals, vin, nin,
                                                                          vin_limbs, run_start, col_src);
  MPS_CUDA(cudaGetLastError());
  return MPSPMV_OK;
}

}  // namespace

// Precision / complex / mode dispatch.
#define MPS_DISPATCH(FN, h, ...)                                                   \
  do {                                                                            \
    switch ((h)->L * 4 + ((h)->cplx ? 2 : 0) + (((h)->mixed || (h)->dstore) ? 1 : 0)) { \
      case 1 * 4 + 0: return FN<1, false, false>(__VA_ARGS__);                    \
      case 1 * 4 + 2: return FN<1, true, false>(__VA_ARGS__);                     \
      case 2 * 4 + 0: return FN<2, false, false>(__VA_ARGS__);                    \
      case 2 * 4 + 1: return FN<2, false, true>(__VA_ARGS__);                     \
      case 2 * 4 + 2: return FN<2, true, false>(__VA_ARGS__);                     \
      case 2 * 4 + 3: return FN<2, true, true>(__VA_ARGS__);                      \
      case 3 * 4 + 0: return FN<3, false, false>(__VA_ARGS__);                    \
      case 3 * 4 + 1: return FN<3, false, true>(__VA_ARGS__);                     \
      case 3 * 4 + 2: return FN<3, true, false>(__VA_ARGS__);                     \
      case 3 * 4 + 3: return FN<3, true, true>(__VA_ARGS__);                      \
      case 4 * 4 + 0: return FN<4, false, false>(__VA_ARGS__);                    \
      case 4 * 4 + 1: return FN<4, false, true>(__VA_ARGS__);                     \
      case 4 * 4 + 2: return FN<4, true, false>(__VA_ARGS__);                     \
      case 4 * 4 + 3: return FN<4, true, true>(__VA_ARGS__);                      \
      default: return MPSPMV_ENOTSUP;                                             \
    }                                                                             \
  } while (0)

int mps_build_tiles(mpspmv_mat* h, const double* d_sorted_vals, int64_t nin, int vin_limbs,
                    const int64_t* d_run_start, const int64_t* d_col_src, cudaStream_t s) {
  MPS_DISPATCH(build_one, h, h, d_sorted_vals, nin, vin_limbs, d_run_start, d_col_src, s);
}

int mps_build_sell(mpspmv_mat* h, cudaStream_t s) {
  // rows qualify when short and evenly sized: the slices pad at most 25 %
  if (h->nnz == 0 || h->max_row_nnz > 128) return MPSPMV_OK;
  const int64_t nsl = (h->nrows + 31) / 32;
  std::vector<int64_t> sp(nsl + 1, 0);
  for (int64_t sl = 0; sl < nsl; sl++) {
    int64_t w = 0;
    for (int64_t r = sl * 32; r < std::min<int64_t>(h->nrows, sl * 32 + 32); r++)
      w = std::max<int64_t>(w, h->h_indptr[r + 1] - h->h_indptr[r]);
    sp[sl + 1] = sp[sl] + 32 * w;
  }
  const int64_t len = sp[nsl];
  if (len * 4 > h->nnz * 5) return MPSPMV_OK;
  const size_t bsp = sizeof(int64_t) * (nsl + 1), bc = sizeof(int32_t) * len, bv = sizeof(double) * h->Pv * len;
  if (cudaMalloc(&h->d_slice_ptr, bsp) != cudaSuccess || cudaMalloc(&h->d_sell_cols, bc) != cudaSuccess ||
      cudaMalloc(&h->d_sell_vals, bv) != cudaSuccess) {
    cudaGetLastError();
    return MPSPMV_ENOMEM;  // the handle's teardown frees what was allocated
  }
  h->device_bytes += (int64_t)(bsp + bc + bv);
  MPS_CUDA(cudaMemcpyAsync(h->d_slice_ptr, sp.data(), bsp, cudaMemcpyHostToDevice, s));
  MPS_CUDA(cudaMemsetAsync(h->d_sell_cols, 0, bc, s));
  MPS_CUDA(cudaMemsetAsync(h->d_sell_vals, 0, bv, s));
  build_sell_kernel<<<(unsigned)((h->nnz + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      h->view(), h->d_slice_ptr, h->d_sell_cols, h->d_sell_vals, len, h->Pv);
  MPS_CUDA(cudaGetLastError());
  h->sell_len = len;
  return MPSPMV_OK;
}

int mps_ensure_carry(mpspmv_mat* h, int k) {
  if (h->carry_k >= k) return MPSPMV_OK;
  int want = k <= 1 ? 1 : 32;
  if (h->d_carry) {
    MPS_CUDA(cudaFree(h->d_carry));
    h->device_bytes -= (int64_t)sizeof(double) * 2 * h->P * h->nchunks * h->carry_k;
    h->d_carry = nullptr;
    h->carry_k = 0;
  }
  const int64_t n = 2 * (int64_t)h->P * std::max<int64_t>(h->nchunks, 1) * want;
  if (cudaMalloc(&h->d_carry, sizeof(double) * n) != cudaSuccess) return MPSPMV_ENOMEM;
  h->device_bytes += (int64_t)sizeof(double) * n;
  h->carry_k = want;
  return MPSPMV_OK;
}

int mps_launch_spmv(const mpspmv_mat* h, const double* x, double* y, cudaStream_t s) {
  MPS_DISPATCH(launch_all, h, h, x, h->ncols, 1, y, h->nrows, 1, 1, nullptr, s);
}

int mps_launch_spmv_if_running(const mpspmv_mat* h, const double* x, double* y, const void* gate,
                               cudaStream_t s) {
  const int* g = static_cast<const int*>(gate);
  MPS_DISPATCH(launch_all, h, h, x, h->ncols, 1, y, h->nrows, 1, 1, g, s);
}

int mps_launch_spmm(mpspmv_mat* h, int k, const double* X, int64_t ldx, double* Y, int64_t ldy, cudaStream_t s) {
  int st = mps_ensure_carry(h, k);
  if (st != MPSPMV_OK) return st;
  MPS_DISPATCH(launch_all, h, h, X, h->ncols * ldx, ldx, Y, h->nrows * ldy, ldy, k, nullptr, s);
}

// ---------------------------------------------------------------------------
// Re-cut the stored entries into runs of a different length (used by the
// batched autotuner): entry u moves from its tiled position for the old run
// length to its tiled position for the new one.
// ---------------------------------------------------------------------------
namespace {
__global__ void retile_kernel(int64_t nnz, int32_t Kold, int32_t Knew, const int32_t* __restrict__ cols_old,
                              const double* __restrict__ vals_old, int64_t tlen_old, int32_t* __restrict__ cols_new,
                              double* __restrict__ vals_new, int64_t tlen_new, int Pv) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= nnz) return;
  const int64_t co = u / Kold, cn = u / Knew;
  const int64_t po = tile_pos(co, (int)(u - co * Kold), Kold);
  const int64_t pn = tile_pos(cn, (int)(u - cn * Knew), Knew);
  cols_new[pn] = cols_old[po];
  for (int p = 0; p < Pv; p++) vals_new[(int64_t)p * tlen_new + pn] = vals_old[(int64_t)p * tlen_old + po];
}
}  // namespace

int mps_retile(mpspmv_mat* h, int32_t K, cudaStream_t s) {
  if (K == h->K) return MPSPMV_OK;
  if (K < 1 || K > 1024) return MPSPMV_EINVAL;
  const int64_t nchunks = (h->nnz + K - 1) / K;
  const int64_t ntiles = (nchunks + 31) / 32;
  const int64_t tlen = ntiles * 32 * (int64_t)K;
  std::vector<int64_t> chunk_row, split;
  int64_t nshort = 0;
  mps_plan(h->h_indptr.data(), h->nrows, h->nnz, K, chunk_row, split, nshort);
  int32_t* cols = nullptr;
  double* vals = nullptr;
  int64_t* crow = nullptr;
  int64_t* spl = nullptr;
  double* carry = nullptr;
  const int kc = std::max(h->carry_k, 1);
  auto fail = [&](int st) {
    cudaFree(cols); cudaFree(vals); cudaFree(crow); cudaFree(spl); cudaFree(carry);
    cudaGetLastError();
    return st;
  };
  if (cudaMalloc(&cols, sizeof(int32_t) * std::max<int64_t>(tlen, 1)) != cudaSuccess ||
      cudaMalloc(&vals, sizeof(double) * h->Pv * std::max<int64_t>(tlen, 1)) != cudaSuccess ||
      cudaMalloc(&crow, sizeof(int64_t) * std::max<int64_t>(nchunks, 1)) != cudaSuccess ||
      cudaMalloc(&spl, sizeof(int64_t) * std::max<size_t>(split.size(), 1)) != cudaSuccess ||
      cudaMalloc(&carry, sizeof(double) * 2 * h->P * std::max<int64_t>(nchunks, 1) * kc) != cudaSuccess)
    return fail(MPSPMV_ENOMEM);
  if (cudaMemsetAsync(cols, 0, sizeof(int32_t) * tlen, s) != cudaSuccess ||
      cudaMemsetAsync(vals, 0, sizeof(double) * h->Pv * tlen, s) != cudaSuccess ||
      (nchunks && cudaMemcpyAsync(crow, chunk_row.data(), sizeof(int64_t) * nchunks, cudaMemcpyHostToDevice, s) !=
                      cudaSuccess) ||
      (!split.empty() && cudaMemcpyAsync(spl, split.data(), sizeof(int64_t) * split.size(), cudaMemcpyHostToDevice,
                                         s) != cudaSuccess))
    return fail(MPSPMV_ECUDA);
  if (h->nnz > 0) {
    retile_kernel<<<(unsigned)((h->nnz + kThreads - 1) / kThreads), kThreads, 0, s>>>(
        h->nnz, h->K, K, h->d_cols, h->d_vals, h->tlen, cols, vals, tlen, h->Pv);
    if (cudaGetLastError() != cudaSuccess) return fail(MPSPMV_ECUDA);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(MPSPMV_ECUDA);
  h->device_bytes += (int64_t)(sizeof(int32_t) + sizeof(double) * h->Pv) * (tlen - h->tlen) +
                     (int64_t)sizeof(int64_t) * ((nchunks - h->nchunks) + ((int64_t)split.size() - h->nsplit)) +
                     (int64_t)sizeof(double) * 2 * h->P * kc * (nchunks - h->nchunks);
  cudaFree(h->d_cols);
  cudaFree(h->d_vals);
  cudaFree(h->d_chunk_row);
  cudaFree(h->d_split);
  cudaFree(h->d_carry);
  h->d_cols = cols;
  h->d_vals = vals;
  h->d_chunk_row = crow;
  h->d_split = spl;
  h->d_carry = carry;
  h->carry_k = kc;
  h->K = K;
  h->nchunks = nchunks;
  h->ntiles = ntiles;
  h->tlen = tlen;
  h->nsplit = (int64_t)split.size();
  h->nshort = nshort;
  return MPSPMV_OK;
}
