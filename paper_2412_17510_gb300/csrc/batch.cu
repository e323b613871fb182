// batch.cu -- many independent matrices in one persistent launch: batched
// multiple-precision SpMM Y_m = A_m X_m and batched CG on every (matrix,
// right-hand side) system, with a per-matrix autotuner for the run length K
// and the number of right-hand sides sharing a run (arXiv 2412.17510,
// Section 3 products and Section 4.2 CG, grown to many small problems).
//
// Persistent execution: a grid of (SM count x resident blocks) warps pulls
// work items from a device queue (one atomic counter).  An item is (matrix,
// group of 32/w consecutive runs, block of w right-hand sides); lane l of the
// warp sums run l / w of the group for right-hand side l % w with exactly the
// operation sequence of the single-matrix kernel (run_body.cuh).  Items of
// one run group are consecutive in the queue, so the group's matrix entries
// come from DRAM once and from L2 for the other right-hand side blocks.
// Rows cut by run boundaries are finished by a second kernel in the same
// CUDA graph; one graph launch does the whole batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"
#include "mp_arith.cuh"
#include "run_body.cuh"

using namespace mpk;

namespace {

constexpr int kBT = 256;  // threads per block (run kernel and vector kernels)
// Rows per vector block of the batched Krylov kernels: the paper-order
// kernels use long blocks; the exact ones do more integer work per element
// in 128-thread blocks, and the small systems of a batch then need shorter
// blocks to fill the GPU.
constexpr int kRB = 2048;
constexpr int kRBX = 512;
constexpr int kCgItersPerGraph = 8;

struct BatchEntry {
  DevMat m;
  double* carry;
  int kc;        // right-hand sides the carry buffer is laid out for
  int k, w, kp;  // right-hand sides, lanes per run, next power of two >= k
  const double* X;
  int64_t ldx;
  double* Y;
  int64_t ldy;
  int64_t sys0;  // first system index (batched CG)
  int64_t vb0;   // first vector block (batched CG)
  int64_t rb;    // rows per vector block (batched CG)
};

struct CgSys {  // per-system solver state (structure of arrays)
  int* status;  // 0 running, 1 converged, MPSPMV_E* otherwise
  int* iter;
  double* tol;
  double* bnorm;
  double* relres;
  double* rho;    // [sys][4]
  double* alpha;  // [sys][4]
  double* beta;   // [sys][4]
};

__device__ __forceinline__ int find_entry(const int64_t* __restrict__ start, int nm, int64_t item) {
  int lo = 0, hi = nm - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int L, bool EXACT, bool DSTORE>
__global__ void __launch_bounds__(kBT) batch_runs_kernel(const BatchEntry* __restrict__ E,
                                                         const int64_t* __restrict__ istart, int nm, int64_t total,
                                                         unsigned long long* __restrict__ head,
                                                         const int* __restrict__ sys_status) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(head, 1ULL);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned long long)total) return;
    const int64_t item = (int64_t)it;
    const int e = find_entry(istart, nm, item);
    const BatchEntry* be = E + e;
    const int w = be->w, k = be->k;
    const int64_t local = item - __ldg(istart + e);
    const int nrb = (k + w - 1) / w;
    const int64_t g = local / nrb;
    const int b = (int)(local - g * nrb);
    const int64_t c = g * (32 / w) + lane / w;
    const int rhs = b * w + (lane & (w - 1));
    if (c < be->m.nchunks && rhs < k && (!sys_status || sys_status[be->sys0 + rhs] == 0)) {
      if (EXACT)
        process_run_exact<L, false, DSTORE, kBT>(be->m, c, rhs, be->X, be->m.ncols * be->ldx, be->ldx, be->Y,
                                           be->m.nrows * be->ldy, be->ldy, be->carry, be->kc);
      else
        process_run<L, false, false>(be->m, c, rhs, be->X, be->m.ncols * be->ldx, be->ldx, be->Y,
                                     be->m.nrows * be->ldy, be->ldy, be->carry, be->kc);
    }
  }
}

// One thread per (split row, right-hand side) of every matrix.
template <int L, bool EXACT>
__global__ void __launch_bounds__(kBT) batch_combine_kernel(const BatchEntry* __restrict__ E,
                                                            const int64_t* __restrict__ cstart, int nm,
                                                            int64_t total, const int* __restrict__ sys_status) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int e = find_entry(cstart, nm, t);
  const BatchEntry* be = E + e;
  const int k = be->k;
  const int64_t local = t - __ldg(cstart + e);
  const int64_t s = local / k;
  const int rhs = (int)(local - s * k);
  if (sys_status && sys_status[be->sys0 + rhs] != 0) return;
  const DevMat& m = be->m;
  const int64_t r = __ldg(m.split_rows + s);
  const int64_t c0 = __ldg(m.indptr + r) / m.K;
  const int64_t c1 = (__ldg(m.indptr + r + 1) - 1) / m.K;
  const int kc = be->kc;
  if (EXACT) {  // the same bits as the single-matrix combine kernels
    const mp<L> a = combine_exact<L>(be->carry, m.nchunks, kc, rhs, L, 0, c0, c1);
#pragma unroll
    for (int l = 0; l < L; l++) be->Y[(int64_t)l * m.nrows * be->ldy + r * be->ldy + rhs] = a.v[l];
    return;
  }
  mp<L> acc;
#pragma unroll
  for (int l = 0; l < L; l++) acc.v[l] = be->carry[((int64_t)(L + l) * m.nchunks + c0) * kc + rhs];
  for (int64_t c = c0 + 1; c <= c1; c++) {
    mp<L> a;
#pragma unroll
    for (int l = 0; l < L; l++) a.v[l] = be->carry[((int64_t)l * m.nchunks + c) * kc + rhs];
    acc = mp_add<L>(acc, a);
  }
#pragma unroll
  for (int l = 0; l < L; l++) be->Y[(int64_t)l * m.nrows * be->ldy + r * be->ldy + rhs] = acc.v[l];
}

__global__ void fill_kernel(double* p, int64_t n, double seed) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) p[t] = sin(seed + 0.37 * (double)(t % 100003));
}

// ---------------------------------------------------------------------------
// batched CG vector kernels: block = (matrix, rb rows), thread = (row
// stripe, right-hand side); right-hand sides are contiguous in the n x ld
// row-major planes.
// ---------------------------------------------------------------------------
template <int L>
__device__ __forceinline__ mp<L> ldv(const double* __restrict__ v, int64_t plane, int64_t idx) {
  mp<L> r;
#pragma unroll
  for (int l = 0; l < L; l++) r.v[l] = v[(int64_t)l * plane + idx];
  return r;
}
template <int L>
__device__ __forceinline__ void stv(double* __restrict__ v, int64_t plane, int64_t idx, const mp<L>& a) {
#pragma unroll
  for (int l = 0; l < L; l++) v[(int64_t)l * plane + idx] = a.v[l];
}
template <int L>
__device__ __forceinline__ mp<L> lds(const double* __restrict__ s, int64_t sys) {
  mp<L> r;
#pragma unroll
  for (int l = 0; l < L; l++) r.v[l] = s[sys * 4 + l];
  return r;
}
template <int L>
__device__ __forceinline__ void sts(double* __restrict__ s, int64_t sys, const mp<L>& a) {
#pragma unroll
  for (int l = 0; l < L; l++) s[sys * 4 + l] = a.v[l];
}

// Reduce the per-thread MP sums of threads sharing a right-hand side and
// write one partial per (block, rhs): part[(vb * 32 + rhs) * L + l].
template <int L>
__device__ __forceinline__ void block_rhs_reduce(mp<L> acc, int kp, double* __restrict__ part, int64_t vb) {
  __shared__ double sm[kBT / 32][32][L];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off >= kp; off >>= 1) {
    mp<L> o;
#pragma unroll
    for (int l = 0; l < L; l++) o.v[l] = __shfl_down_sync(0xffffffffu, acc.v[l], off);
    if (lane < off) acc = mp_add<L>(acc, o);
  }
  if (lane < kp) {
#pragma unroll
    for (int l = 0; l < L; l++) sm[warp][lane][l] = acc.v[l];
  }
  __syncthreads();
  if (threadIdx.x < kp) {
    mp<L> s;
#pragma unroll
    for (int l = 0; l < L; l++) s.v[l] = sm[0][threadIdx.x][l];
    for (int wv = 1; wv < kBT / 32; wv++) {
      mp<L> o;
#pragma unroll
      for (int l = 0; l < L; l++) o.v[l] = sm[wv][threadIdx.x][l];
      s = mp_add<L>(s, o);
    }
#pragma unroll
    for (int l = 0; l < L; l++) part[(vb * 32 + threadIdx.x) * L + l] = s.v[l];
  }
}

enum VecOp { V_RESID = 0, V_DOT = 1, V_XR = 2, V_P = 3 };

// V_RESID: r = b - q, p = r (if p), partial (r, r); also partial (b, b) in part2
// V_DOT:   partial (u, v)
// V_XR:    x += alpha p, r -= alpha q, partial (r, r)
// V_P:     p = r + beta p
template <int L, int OP>
__global__ void __launch_bounds__(kBT) batch_vec_kernel(const BatchEntry* __restrict__ E,
                                                        const int64_t* __restrict__ vstart, int nm, CgSys S,
                                                        double* const* __restrict__ vec, int i0, int i1, int i2,
                                                        int i3, double* __restrict__ part,
                                                        double* __restrict__ part2, bool gate) {
  const int64_t vb = blockIdx.x;
  const int e = find_entry(vstart, nm, vb);
  const BatchEntry* be = E + e;
  const int kp = be->kp, k = be->k;
  const int64_t n = be->m.nrows, ld = be->ldx;
  const int64_t plane = n * ld;
  const int64_t r0 = (vb - __ldg(vstart + e)) * be->rb;
  const int rhs = threadIdx.x & (kp - 1);
  const int stripe = threadIdx.x / kp, nstripe = kBT / kp;
  const int64_t sys = be->sys0 + rhs;
  const bool live = rhs < k && (!gate || S.status[sys] == 0);
  double* v0 = vec[(int64_t)e * 8 + i0];
  double* v1 = vec[(int64_t)e * 8 + i1];
  double* v2 = vec[(int64_t)e * 8 + i2];
  double* v3 = vec[(int64_t)e * 8 + i3];
  mp<L> acc = mp_zero<L>(), acc2 = mp_zero<L>();
  mp<L> al, nal, be_;
  if (live && OP == V_XR) {
    al = lds<L>(S.alpha, sys);
    nal = mp_neg<L>(al);
  }
  if (live && OP == V_P) be_ = lds<L>(S.beta, sys);
  if (live) {
    const int64_t rend = min(r0 + be->rb, n);
    for (int64_t r = r0 + stripe; r < rend; r += nstripe) {
      const int64_t idx = r * ld + rhs;
      if (OP == V_RESID) {  // v0 = b, v1 = q (A x), v2 = r, v3 = p
        const mp<L> b = ldv<L>(v0, plane, idx);
        mp<L> m1 = mp_zero<L>();
        m1.v[0] = -1.0;
        const mp<L> ri = mp_add<L>(b, mp_mul<L>(m1, ldv<L>(v1, plane, idx)));
        stv<L>(v2, plane, idx, ri);
        if (v3) stv<L>(v3, plane, idx, ri);
        acc = mp_add<L>(acc, mp_mul<L>(ri, ri));
        acc2 = mp_add<L>(acc2, mp_mul<L>(b, b));
      } else if (OP == V_DOT) {  // (v0, v1)
        acc = mp_add<L>(acc, mp_mul<L>(ldv<L>(v0, plane, idx), ldv<L>(v1, plane, idx)));
      } else if (OP == V_XR) {  // v0 = x, v1 = r, v2 = p, v3 = q
        stv<L>(v0, plane, idx, mp_add<L>(ldv<L>(v0, plane, idx), mp_mul<L>(al, ldv<L>(v2, plane, idx))));
        const mp<L> ri = mp_add<L>(ldv<L>(v1, plane, idx), mp_mul<L>(nal, ldv<L>(v3, plane, idx)));
        stv<L>(v1, plane, idx, ri);
        acc = mp_add<L>(acc, mp_mul<L>(ri, ri));
      } else {  // V_P: v0 = r, v1 = p
        stv<L>(v1, plane, idx, mp_add<L>(ldv<L>(v0, plane, idx), mp_mul<L>(be_, ldv<L>(v1, plane, idx))));
      }
    }
  }
  if (OP != V_P) {
    block_rhs_reduce<L>(acc, kp, part, vb);
    if (OP == V_RESID) {
      __syncthreads();
      block_rhs_reduce<L>(acc2, kp, part2, vb);
    }
  }
}

// ---------------------------------------------------------------------------
// Exact-accumulation variant of the batched CG vector kernels (batches of
// handles created with MPSPMV_EXACT_ACC): each updated element is formed from
// its terms' components and error-free products in one exact accumulator and
// cut once; each thread sums its share of an inner product exactly; the
// threads of one right-hand side are then added on fixed-point digits at
// their common base, and the finishing step adds the block partials exactly.
// Blocks of kBTX threads; accumulator a of a thread uses 2 D digits of the
// block's dynamic shared memory (digit j of thread t at j kBTX + t).
// ---------------------------------------------------------------------------
constexpr int kBTX = 128;

template <int L>
using BAcc = FixAccS<AccDigits<L>::D, kBTX>;

template <int L>
constexpr size_t bx_smem(int nacc) {
  return (size_t)nacc * 2 * AccDigits<L>::D * kBTX * sizeof(unsigned long long);
}

template <int L>
__device__ __forceinline__ BAcc<L> bx_acc(unsigned long long* digits, int a) {
  constexpr int D = AccDigits<L>::D;
  BAcc<L> r;
  r.dp = digits + (size_t)a * 2 * D * kBTX + threadIdx.x;
  r.dn = r.dp + D * kBTX;
  fas_reset<D, kBTX>(r);
  return r;
}

template <int L>
__device__ __forceinline__ mp<L> bx_flush(BAcc<L>& a) {
  mp<L> r;
  fas_to_mp<L, AccDigits<L>::D, kBTX>(a, r.v);
  fas_reset<AccDigits<L>::D, kBTX>(a);
  return r;
}

template <int L>
__device__ __forceinline__ void bx_add(BAcc<L>& a, const mp<L>& u, bool neg) {
#pragma unroll
  for (int l = 0; l < L; l++) acc_add(a, u.v[l], neg);
}

// Exact sum over the threads of each right-hand side (threads rhs, rhs + kp,
// ...) of one MP value per thread; thread rhs < kp writes the partial of
// block vb: part[(vb * 32 + rhs) * L + l].
template <int L>
__device__ __forceinline__ void block_rhs_reduce_x(const mp<L>& v, int kp, double* __restrict__ part, int64_t vb) {
  constexpr int D = AccDigits<L>::D, NW = kBTX / 32;
  __shared__ int s_top[NW][32];
  __shared__ int s_bad[NW][32];
  __shared__ long long s_d[NW][32][D];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int t = INT_MIN, bad = 0;
#pragma unroll
  for (int l = 0; l < L; l++) {
    t = max(t, top_exp(v.v[l]));
    bad |= isfinite(v.v[l]) ? 0 : 1;
  }
  // lanes with the same right-hand side differ by multiples of kp
  for (int off = 16; off >= kp; off >>= 1) {
    t = max(t, __shfl_xor_sync(0xffffffffu, t, off));
    bad |= __shfl_xor_sync(0xffffffffu, bad, off);
  }
  if (lane < kp) {
    s_top[warp][lane] = t;
    s_bad[warp][lane] = bad;
  }
  __syncthreads();
  const int rhs = lane & (kp - 1);
  t = s_top[0][rhs];
  for (int w = 1; w < NW; w++) t = max(t, s_top[w][rhs]);
  FixAcc<D> f;
  fa_at_top<D>(f, t);
#pragma unroll
  for (int l = 0; l < L; l++) fa_add<D>(f, v.v[l]);
#pragma unroll
  for (int j = 0; j < D; j++)
    for (int off = 16; off >= kp; off >>= 1) f.d[j] += __shfl_down_sync(0xffffffffu, f.d[j], off);
  if (lane < kp) {
#pragma unroll
    for (int j = 0; j < D; j++) s_d[warp][lane][j] = f.d[j];
  }
  __syncthreads();
  if (threadIdx.x < kp) {
    FixAcc<D> r;
    fa_at_top<D>(r, t);
    for (int w = 0; w < NW; w++) {
#pragma unroll
      for (int j = 0; j < D; j++) r.d[j] += s_d[w][threadIdx.x][j];
      r.bad |= s_bad[w][threadIdx.x] != 0;
    }
    double out[L];
    fa_to_mp<L, D>(r, out);
#pragma unroll
    for (int l = 0; l < L; l++) part[(vb * 32 + threadIdx.x) * L + l] = out[l];
  }
  __syncthreads();
}

// Same operations and vector roles as batch_vec_kernel.
template <int L, int OP>
__global__ void __launch_bounds__(kBTX) batch_vec_kernel_x(const BatchEntry* __restrict__ E,
                                                           const int64_t* __restrict__ vstart, int nm, CgSys S,
                                                           double* const* __restrict__ vec, int i0, int i1, int i2,
                                                           int i3, double* __restrict__ part,
                                                           double* __restrict__ part2, bool gate) {
  extern __shared__ unsigned long long bx_digits[];
  const int64_t vb = blockIdx.x;
  const int e = find_entry(vstart, nm, vb);
  const BatchEntry* be = E + e;
  const int kp = be->kp, k = be->k;
  const int64_t n = be->m.nrows, ld = be->ldx;
  const int64_t plane = n * ld;
  const int64_t r0 = (vb - __ldg(vstart + e)) * be->rb;
  const int rhs = threadIdx.x & (kp - 1);
  const int stripe = threadIdx.x / kp, nstripe = kBTX / kp;
  const int64_t sys = be->sys0 + rhs;
  const bool live = rhs < k && (!gate || S.status[sys] == 0);
  double* v0 = vec[(int64_t)e * 8 + i0];
  double* v1 = vec[(int64_t)e * 8 + i1];
  double* v2 = vec[(int64_t)e * 8 + i2];
  double* v3 = vec[(int64_t)e * 8 + i3];
  // accumulators: 0 element, 1 first inner product, 2 second (V_RESID)
  BAcc<L> el, d1, d2;
  if (OP != V_DOT) el = bx_acc<L>(bx_digits, 0);
  if (OP != V_P) d1 = bx_acc<L>(bx_digits, OP == V_DOT ? 0 : 1);
  if (OP == V_RESID) d2 = bx_acc<L>(bx_digits, 2);
  mp<L> al, be_;
  if (live && OP == V_XR) al = lds<L>(S.alpha, sys);
  if (live && OP == V_P) be_ = lds<L>(S.beta, sys);
  if (live) {
    const int64_t rend = min(r0 + be->rb, n);
    for (int64_t r = r0 + stripe; r < rend; r += nstripe) {
      const int64_t idx = r * ld + rhs;
      if (OP == V_RESID) {  // v0 = b, v1 = q (A x), v2 = r, v3 = p
        const mp<L> b = ldv<L>(v0, plane, idx);
        bx_add<L>(el, b, false);
        bx_add<L>(el, ldv<L>(v1, plane, idx), true);
        const mp<L> ri = bx_flush<L>(el);
        stv<L>(v2, plane, idx, ri);
        if (v3) stv<L>(v3, plane, idx, ri);
        add_prod<BAcc<L>, L>(d1, ri, ri, false);
        add_prod<BAcc<L>, L>(d2, b, b, false);
      } else if (OP == V_DOT) {  // (v0, v1)
        add_prod<BAcc<L>, L>(d1, ldv<L>(v0, plane, idx), ldv<L>(v1, plane, idx), false);
      } else if (OP == V_XR) {  // v0 = x, v1 = r, v2 = p, v3 = q
        bx_add<L>(el, ldv<L>(v0, plane, idx), false);
        add_prod<BAcc<L>, L>(el, al, ldv<L>(v2, plane, idx), false);
        stv<L>(v0, plane, idx, bx_flush<L>(el));
        bx_add<L>(el, ldv<L>(v1, plane, idx), false);
        add_prod<BAcc<L>, L>(el, al, ldv<L>(v3, plane, idx), true);
        const mp<L> ri = bx_flush<L>(el);
        stv<L>(v1, plane, idx, ri);
        add_prod<BAcc<L>, L>(d1, ri, ri, false);
      } else {  // V_P: v0 = r, v1 = p
        bx_add<L>(el, ldv<L>(v0, plane, idx), false);
        add_prod<BAcc<L>, L>(el, be_, ldv<L>(v1, plane, idx), false);
        stv<L>(v1, plane, idx, bx_flush<L>(el));
      }
    }
  }
  if (OP != V_P) {
    block_rhs_reduce_x<L>(bx_flush<L>(d1), kp, part, vb);
    if (OP == V_RESID) block_rhs_reduce_x<L>(bx_flush<L>(d2), kp, part2, vb);
  }
}

// exact sum of the nb block partials of one system (thread per system)
template <int L>
__device__ __forceinline__ mp<L> sum_partials_x(const double* __restrict__ part, int64_t vb0, int64_t nb, int rhs) {
  constexpr int D = AccDigits<L>::D;
  int t = INT_MIN;
  for (int64_t j = 0; j < nb; j++)
#pragma unroll
    for (int l = 0; l < L; l++) t = max(t, top_exp(part[((vb0 + j) * 32 + rhs) * L + l]));
  FixAcc<D> f;
  fa_at_top<D>(f, t);
  for (int64_t j = 0; j < nb; j++)
#pragma unroll
    for (int l = 0; l < L; l++) fa_add<D>(f, part[((vb0 + j) * 32 + rhs) * L + l]);
  mp<L> r;
  fa_to_mp<L, D>(f, r.v);
  return r;
}

// Per-system finishing steps (thread per system).
enum FinOp { F_START = 0, F_ALPHA = 1, F_BETA = 2, F_RELRES = 3 };

template <int L, int OP, bool EX = false>
__global__ void batch_finish_kernel(const BatchEntry* __restrict__ E, const int64_t* __restrict__ sstart, int nm,
                                    int64_t nsys, CgSys S, const double* __restrict__ part,
                                    const double* __restrict__ part2, double rtol, double atol, int maxit) {
  const int64_t sys = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (sys >= nsys) return;
  if (OP != F_START && OP != F_RELRES && S.status[sys] != 0) return;
  const int e = find_entry(sstart, nm, sys);
  const BatchEntry* be = E + e;
  const int rhs = (int)(sys - be->sys0);
  const int64_t nb = (be->m.nrows + be->rb - 1) / be->rb;
  mp<L> a = mp_zero<L>(), b = mp_zero<L>();
  if (EX) {
    a = sum_partials_x<L>(part, be->vb0, nb, rhs);
    if (OP == F_START) b = sum_partials_x<L>(part2, be->vb0, nb, rhs);
  } else {
    for (int64_t j = 0; j < nb; j++) {
      a = mp_add<L>(a, ldv<L>(part, 1, ((be->vb0 + j) * 32 + rhs) * L));
      if (OP == F_START) b = mp_add<L>(b, ldv<L>(part2, 1, ((be->vb0 + j) * 32 + rhs) * L));
    }
  }
  if (OP == F_START) {  // a = (r, r), b = (b, b)
    const double bb = mp_to_double<L>(b), rr = mp_to_double<L>(a);
    const double bn = sqrt(bb > 0.0 ? bb : 0.0);
    S.bnorm[sys] = bn;
    S.tol[sys] = rtol * bn + atol;
    sts<L>(S.rho, sys, a);
    S.iter[sys] = 0;
    int st = sqrt(rr > 0.0 ? rr : 0.0) <= S.tol[sys] ? 1 : 0;
    if (st == 0 && maxit <= 0) st = MPSPMV_ENOCONV;
    S.status[sys] = st;
  } else if (OP == F_ALPHA) {  // a = (p, q)
    if (a.v[0] == 0.0 || !isfinite(a.v[0])) {
      S.status[sys] = MPSPMV_EBREAKDOWN;
      return;
    }
    sts<L>(S.alpha, sys, mp_div<L>(lds<L>(S.rho, sys), a));
  } else if (OP == F_BETA) {  // a = (r, r)
    const int it = ++S.iter[sys];
    const double t = mp_to_double<L>(a);
    if (!isfinite(t)) {
      S.status[sys] = MPSPMV_EBREAKDOWN;
      return;
    }
    if (sqrt(t > 0.0 ? t : 0.0) <= S.tol[sys]) {
      S.status[sys] = 1;
      return;
    }
    const mp<L> rho = lds<L>(S.rho, sys);
    if (rho.v[0] == 0.0) {
      S.status[sys] = MPSPMV_EBREAKDOWN;
      return;
    }
    sts<L>(S.beta, sys, mp_div<L>(a, rho));
    sts<L>(S.rho, sys, a);
    if (it >= maxit) S.status[sys] = MPSPMV_ENOCONV;
  } else {  // F_RELRES: a = (r_true, r_true)
    const double t = mp_to_double<L>(a);
    const double rn = sqrt(t > 0.0 ? t : 0.0);
    S.relres[sys] = S.bnorm[sys] > 0.0 ? rn / S.bnorm[sys] : rn;
  }
}

int pow2_at_least(int k) {
  int p = 1;
  while (p < k) p <<= 1;
  return p;
}

}  // namespace

struct mpspmv_batch {
  int device = 0, count = 0, L = 2;
  std::vector<mpspmv_mat*> mats;
  std::vector<int> k, w;
  std::vector<int64_t> item_start, comb_start, sys_start, vec_start;
  int64_t total_items = 0, total_comb = 0, nsys = 0, nvb = 0;
  int grid_runs = 0;
  BatchEntry* d_entries = nullptr;
  int64_t* d_item_start = nullptr;
  int64_t* d_comb_start = nullptr;
  int64_t* d_sys_start = nullptr;
  int64_t* d_vec_start = nullptr;
  unsigned long long* d_head = nullptr;
  std::vector<BatchEntry> h_entries;
  // cached SpMM graph for one set of X / Y pointers
  cudaGraphExec_t spmm_exec = nullptr;
  std::vector<const void*> spmm_key;
  // batched CG workspace
  double* d_cg = nullptr;
  int64_t cg_len = 0;
  double** d_vecs = nullptr;
  CgSys sys{};
  void* d_sysmem = nullptr;
};

namespace {

void free_batch(mpspmv_batch* b) {
  if (!b) return;
  if (b->spmm_exec) cudaGraphExecDestroy(b->spmm_exec);
  cudaFree(b->d_entries);
  cudaFree(b->d_item_start);
  cudaFree(b->d_comb_start);
  cudaFree(b->d_sys_start);
  cudaFree(b->d_vec_start);
  cudaFree(b->d_head);
  cudaFree(b->d_cg);
  cudaFree(b->d_vecs);
  cudaFree(b->d_sysmem);
  delete b;
}

// Recompute the work-item layout after (K, w) choices and upload it.
int layout(mpspmv_batch* b, cudaStream_t s) {
  const int n = b->count;
  b->item_start.assign(n + 1, 0);
  b->comb_start.assign(n + 1, 0);
  b->sys_start.assign(n + 1, 0);
  b->vec_start.assign(n + 1, 0);
  b->h_entries.resize(n);
  for (int i = 0; i < n; i++) {
    mpspmv_mat* h = b->mats[i];
    int st = mps_ensure_carry(h, b->k[i]);
    if (st) return st;
    const int w = b->w[i], k = b->k[i];
    const int64_t groups = (h->nchunks + (32 / w) - 1) / (32 / w);
    b->item_start[i + 1] = b->item_start[i] + groups * ((k + w - 1) / w);
    b->comb_start[i + 1] = b->comb_start[i] + h->nsplit * k;
    b->sys_start[i + 1] = b->sys_start[i] + k;
    const int64_t rb = h->exact ? kRBX : kRB;
    b->vec_start[i + 1] = b->vec_start[i] + (h->nrows + rb - 1) / rb;
    BatchEntry& e = b->h_entries[i];
    e.m = h->view();
    e.carry = h->d_carry;
    e.kc = h->carry_k;
    e.k = k;
    e.w = w;
    e.kp = pow2_at_least(k);
    e.X = nullptr;
    e.Y = nullptr;
    e.ldx = e.ldy = k;
    e.sys0 = b->sys_start[i];
    e.vb0 = b->vec_start[i];
    e.rb = rb;
  }
  b->total_items = b->item_start[n];
  b->total_comb = b->comb_start[n];
  b->nsys = b->sys_start[n];
  b->nvb = b->vec_start[n];
  auto up = [&](int64_t* d, const std::vector<int64_t>& v) {
    return cudaMemcpyAsync(d, v.data(), sizeof(int64_t) * v.size(), cudaMemcpyHostToDevice, s);
  };
  MPS_CUDA(up(b->d_item_start, b->item_start));
  MPS_CUDA(up(b->d_comb_start, b->comb_start));
  MPS_CUDA(up(b->d_sys_start, b->sys_start));
  MPS_CUDA(up(b->d_vec_start, b->vec_start));
  MPS_CUDA(cudaMemcpyAsync(b->d_entries, b->h_entries.data(), sizeof(BatchEntry) * n, cudaMemcpyHostToDevice, s));
  MPS_CUDA(cudaStreamSynchronize(s));
  if (b->spmm_exec) {
    cudaGraphExecDestroy(b->spmm_exec);
    b->spmm_exec = nullptr;
    b->spmm_key.clear();
  }
  return MPSPMV_OK;
}

template <int L>
int enqueue_spmm(mpspmv_batch* b, const int* sys_status, cudaStream_t s) {
  MPS_CUDA(cudaMemsetAsync(b->d_head, 0, sizeof(unsigned long long), s));
  if (b->mats[0]->exact && b->mats[0]->dstore)
    batch_runs_kernel<L, true, true><<<b->grid_runs, kBT, 0, s>>>(b->d_entries, b->d_item_start, b->count,
                                                                  b->total_items, b->d_head, sys_status);
  else if (b->mats[0]->exact)
    batch_runs_kernel<L, true, false><<<b->grid_runs, kBT, 0, s>>>(b->d_entries, b->d_item_start, b->count,
                                                                   b->total_items, b->d_head, sys_status);
  else
    batch_runs_kernel<L, false, false><<<b->grid_runs, kBT, 0, s>>>(b->d_entries, b->d_item_start, b->count,
                                                                    b->total_items, b->d_head, sys_status);
  MPS_CUDA(cudaGetLastError());
  if (b->total_comb > 0) {
    const unsigned nb = (unsigned)((b->total_comb + kBT - 1) / kBT);
    if (b->mats[0]->exact)
      batch_combine_kernel<L, true><<<nb, kBT, 0, s>>>(b->d_entries, b->d_comb_start, b->count, b->total_comb,
                                                       sys_status);
    else
      batch_combine_kernel<L, false><<<nb, kBT, 0, s>>>(b->d_entries, b->d_comb_start, b->count, b->total_comb,
                                                        sys_status);
    MPS_CUDA(cudaGetLastError());
  }
  return MPSPMV_OK;
}

int enqueue_spmm_any(mpspmv_batch* b, const int* sys_status, cudaStream_t s) {
  switch (b->L) {
    case 1: return enqueue_spmm<1>(b, sys_status, s);
    case 2: return enqueue_spmm<2>(b, sys_status, s);
    case 3: return enqueue_spmm<3>(b, sys_status, s);
    case 4: return enqueue_spmm<4>(b, sys_status, s);
  }
  return MPSPMV_ENOTSUP;
}

// point the entries at (X, Y) arrays and upload the table
int set_vectors(mpspmv_batch* b, const double* const* X, const int64_t* ldx, double* const* Y, const int64_t* ldy,
                cudaStream_t s) {
  for (int i = 0; i < b->count; i++) {
    BatchEntry& e = b->h_entries[i];
    e.X = X[i];
    e.Y = Y[i];
    e.ldx = ldx ? ldx[i] : b->k[i];
    e.ldy = ldy ? ldy[i] : b->k[i];
    if (!e.X || !e.Y || e.ldx < e.k || e.ldy < e.k) return MPSPMV_EINVAL;
  }
  MPS_CUDA(cudaMemcpyAsync(b->d_entries, b->h_entries.data(), sizeof(BatchEntry) * b->count, cudaMemcpyHostToDevice,
                           s));
  return MPSPMV_OK;
}

// time one matrix alone with the current (K, w): best of three graph-free runs
int time_one(mpspmv_batch* b, int i, const double* X, double* Y, cudaStream_t s, float* ms) {
  mpspmv_batch one;
  one.device = b->device;
  one.count = 1;
  one.L = b->L;
  one.mats = {b->mats[i]};
  one.k = {b->k[i]};
  one.w = {b->w[i]};
  one.grid_runs = b->grid_runs;
  one.d_entries = b->d_entries;  // borrow the device tables (rewritten below)
  one.d_item_start = b->d_item_start;
  one.d_comb_start = b->d_comb_start;
  one.d_sys_start = b->d_sys_start;
  one.d_vec_start = b->d_vec_start;
  one.d_head = b->d_head;
  int st = layout(&one, s);
  const double* xs[1] = {X};
  double* ys[1] = {Y};
  if (!st) st = set_vectors(&one, xs, nullptr, ys, nullptr, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 3 && !st; rep++) {
    cudaEventRecord(e0, s);
    st = enqueue_spmm_any(&one, nullptr, s);
    cudaEventRecord(e1, s);
    if (!st && cudaEventSynchronize(e1) != cudaSuccess) st = MPSPMV_ECUDA;
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0) best = std::min(best, t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the borrowed device pointers stay owned by b
  one.d_entries = nullptr;
  one.d_item_start = one.d_comb_start = one.d_sys_start = one.d_vec_start = nullptr;
  one.d_head = nullptr;
  *ms = best;
  return st;
}

// Per-matrix autotuner: run length K from {8, 16, 32, 64} (with one lane per
// run), then lanes per run w from {1, 2, 4, 8} (capped by k), each timed on
// the device; the matrix keeps the fastest pair.
int autotune(mpspmv_batch* b, cudaStream_t s) {
  int64_t xmax = 1, ymax = 1;
  for (int i = 0; i < b->count; i++) {
    xmax = std::max(xmax, b->mats[i]->ncols * (int64_t)b->k[i] * b->L);
    ymax = std::max(ymax, b->mats[i]->nrows * (int64_t)b->k[i] * b->L);
  }
  double *X = nullptr, *Y = nullptr;
  if (cudaMalloc(&X, sizeof(double) * xmax) != cudaSuccess || cudaMalloc(&Y, sizeof(double) * ymax) != cudaSuccess) {
    cudaFree(X);
    cudaGetLastError();
    return MPSPMV_ENOMEM;
  }
  fill_kernel<<<(unsigned)((xmax + 255) / 256), 256, 0, s>>>(X, xmax, 0.5);
  int st = MPSPMV_OK;
  for (int i = 0; i < b->count && !st; i++) {
    mpspmv_mat* h = b->mats[i];
    int bestK = h->K, bestw = 1;
    float best = 1e30f, t = 0.0f;
    b->w[i] = 1;
    for (int K : {8, 16, 32, 64}) {
      if ((st = mps_retile(h, K, s))) break;
      if ((st = time_one(b, i, X, Y, s, &t))) break;
      if (t < best) {
        best = t;
        bestK = K;
      }
    }
    if (st) break;
    if ((st = mps_retile(h, bestK, s))) break;
    const int kp = pow2_at_least(b->k[i]);
    for (int w : {2, 4, 8}) {
      if (w > kp) break;
      b->w[i] = w;
      if ((st = time_one(b, i, X, Y, s, &t))) break;
      if (t < best) {
        best = t;
        bestw = w;
      }
    }
    b->w[i] = bestw;
  }
  cudaStreamSynchronize(s);
  cudaFree(X);
  cudaFree(Y);
  return st;
}

// Launch the paper-order or the exact batched vector kernel.
template <int L, int OP>
int launch_vec(bool ex, unsigned nvb, cudaStream_t s, const mpspmv_batch* b, int n, const CgSys& S, int i0, int i1,
               int i2, int i3, double* part, double* part2, bool gate) {
  if (!ex) {
    batch_vec_kernel<L, OP><<<nvb, kBT, 0, s>>>(b->d_entries, b->d_vec_start, n, S, b->d_vecs, i0, i1, i2, i3, part,
                                                part2, gate);
    return MPSPMV_OK;
  }
  constexpr int nacc = OP == V_RESID ? 3 : (OP == V_XR ? 2 : 1);
  static bool attr = false;  // the residual kernel's three accumulators exceed the default 48 KB
  if (!attr) {
    if (cudaFuncSetAttribute(batch_vec_kernel_x<L, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)bx_smem<L>(nacc)) != cudaSuccess) {
      cudaGetLastError();
      return MPSPMV_ECUDA;
    }
    attr = true;
  }
  batch_vec_kernel_x<L, OP><<<nvb, kBTX, bx_smem<L>(nacc), s>>>(b->d_entries, b->d_vec_start, n, S, b->d_vecs, i0, i1,
                                                               i2, i3, part, part2, gate);
  return MPSPMV_OK;
}

template <int L, int OP>
void launch_fin(bool ex, unsigned fin, cudaStream_t s, const mpspmv_batch* b, int n, const CgSys& S,
                const double* part, const double* part2, double rtol, double atol, int maxit) {
  if (ex)
    batch_finish_kernel<L, OP, true><<<fin, 128, 0, s>>>(b->d_entries, b->d_sys_start, n, b->nsys, S, part, part2,
                                                         rtol, atol, maxit);
  else
    batch_finish_kernel<L, OP, false><<<fin, 128, 0, s>>>(b->d_entries, b->d_sys_start, n, b->nsys, S, part, part2,
                                                          rtol, atol, maxit);
}

template <int L>
int batch_cg_impl(mpspmv_batch* b, const double* const* B, const int64_t* ldb, double* const* X,
                  const int64_t* ldx, double rtol, double atol, int maxit, int* iters, double* relres,
                  int* status_out, cudaStream_t s) {
  const int n = b->count;
  // every matrix's vectors share one leading dimension per matrix (ld = k)
  for (int i = 0; i < n; i++) {
    if ((ldb && ldb[i] != b->k[i]) || (ldx && ldx[i] != b->k[i])) return MPSPMV_ENOTSUP;
    if (!B[i] || !X[i]) return MPSPMV_EINVAL;
  }
  // workspace: r, p, q, t per matrix (L planes of n x k)
  int64_t need = 0;
  std::vector<int64_t> off(n);
  for (int i = 0; i < n; i++) {
    off[i] = need;
    need += 4 * (int64_t)L * b->mats[i]->nrows * b->k[i];
  }
  const int64_t npart = b->nvb * 32 * L;
  need += 2 * npart;
  if (b->cg_len < need) {
    cudaFree(b->d_cg);
    b->d_cg = nullptr;
    if (cudaMalloc(&b->d_cg, sizeof(double) * need) != cudaSuccess) {
      cudaGetLastError();
      b->cg_len = 0;
      return MPSPMV_ENOMEM;
    }
    b->cg_len = need;
  }
  if (!b->d_vecs) {
    if (cudaMalloc(&b->d_vecs, sizeof(double*) * 8 * n) != cudaSuccess) return MPSPMV_ENOMEM;
  }
  if (!b->d_sysmem) {
    const size_t bytes = (sizeof(int) * 2 + sizeof(double) * 3 + sizeof(double) * 12) * (size_t)b->nsys + 256;
    if (cudaMalloc(&b->d_sysmem, bytes) != cudaSuccess) return MPSPMV_ENOMEM;
    char* p = static_cast<char*>(b->d_sysmem);
    const int64_t ns = b->nsys;
    b->sys.status = reinterpret_cast<int*>(p);
    b->sys.iter = b->sys.status + ns;
    double* d = reinterpret_cast<double*>(p + ((sizeof(int) * 2 * ns + 63) / 64) * 64);
    b->sys.tol = d;
    b->sys.bnorm = d + ns;
    b->sys.relres = d + 2 * ns;
    b->sys.rho = d + 3 * ns;
    b->sys.alpha = d + 7 * ns;
    b->sys.beta = d + 11 * ns;
  }
  double* part = b->d_cg + need - 2 * npart;
  double* part2 = part + npart;
  // vector table: [i*8 + 0] b, 1 x, 2 r, 3 p, 4 q, 5 t
  std::vector<double*> vt(8 * (size_t)n, nullptr);
  for (int i = 0; i < n; i++) {
    const int64_t len = (int64_t)L * b->mats[i]->nrows * b->k[i];
    vt[i * 8 + 0] = const_cast<double*>(B[i]);
    vt[i * 8 + 1] = X[i];
    vt[i * 8 + 2] = b->d_cg + off[i];
    vt[i * 8 + 3] = b->d_cg + off[i] + len;
    vt[i * 8 + 4] = b->d_cg + off[i] + 2 * len;
    vt[i * 8 + 5] = b->d_cg + off[i] + 3 * len;
  }
  MPS_CUDA(cudaMemcpyAsync(b->d_vecs, vt.data(), sizeof(double*) * vt.size(), cudaMemcpyHostToDevice, s));
  // q = A x
  std::vector<const double*> xin(n);
  std::vector<double*> qout(n), pin(n);
  for (int i = 0; i < n; i++) {
    xin[i] = X[i];
    qout[i] = vt[i * 8 + 4];
  }
  int st = set_vectors(b, xin.data(), nullptr, qout.data(), nullptr, s);
  if (st) return st;
  if ((st = enqueue_spmm<L>(b, nullptr, s))) return st;
  const unsigned nvb = (unsigned)b->nvb;
  const unsigned fin = (unsigned)((b->nsys + 127) / 128);
  const bool ex = b->mats[0]->exact;  // the batch's handles share the arithmetic
  CgSys S = b->sys;
  // r = b - q, p = r, (r, r), (b, b), per-system start
  if ((st = launch_vec<L, V_RESID>(ex, nvb, s, b, n, S, 0, 4, 2, 3, part, part2, false))) return st;
  launch_fin<L, F_START>(ex, fin, s, b, n, S, part, part2, rtol, atol, maxit);
  MPS_CUDA(cudaGetLastError());
  // iterations: SpMM now reads p and writes q
  for (int i = 0; i < n; i++) pin[i] = vt[i * 8 + 3];
  std::vector<const double*> pc(pin.begin(), pin.end());
  if ((st = set_vectors(b, pc.data(), nullptr, qout.data(), nullptr, s))) return st;
  cudaStream_t cs;
  MPS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, s);
  cudaStreamWaitEvent(cs, ev, 0);
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = MPSPMV_ECUDA;
  for (int it = 0; it < kCgItersPerGraph && !st; it++) {
    st = enqueue_spmm<L>(b, S.status, cs);
    if (!st) st = launch_vec<L, V_DOT>(ex, nvb, cs, b, n, S, 3, 4, 0, 0, part, nullptr, true);
    launch_fin<L, F_ALPHA>(ex, fin, cs, b, n, S, part, nullptr, rtol, atol, maxit);
    if (!st) st = launch_vec<L, V_XR>(ex, nvb, cs, b, n, S, 1, 2, 3, 4, part, nullptr, true);
    launch_fin<L, F_BETA>(ex, fin, cs, b, n, S, part, nullptr, rtol, atol, maxit);
    if (!st) st = launch_vec<L, V_P>(ex, nvb, cs, b, n, S, 2, 3, 0, 0, part, nullptr, true);
    if (cudaGetLastError() != cudaSuccess) st = MPSPMV_ECUDA;
  }
  cudaError_t ee = cudaStreamEndCapture(cs, &g);
  if (!st && ee != cudaSuccess) st = MPSPMV_ECUDA;
  if (!st && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) st = MPSPMV_ECUDA;
  std::vector<int> hs(b->nsys);
  while (!st) {
    if (cudaGraphLaunch(ge, cs) != cudaSuccess ||
        cudaMemcpyAsync(hs.data(), S.status, sizeof(int) * b->nsys, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess) {
      st = MPSPMV_ECUDA;
      break;
    }
    if (std::none_of(hs.begin(), hs.end(), [](int v) { return v == 0; })) break;
  }
  cudaEventRecord(ev, cs);
  cudaStreamWaitEvent(s, ev, 0);
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  cudaStreamSynchronize(cs);
  cudaStreamDestroy(cs);
  cudaEventDestroy(ev);
  if (st) return st;
  // true residual: t = b - A x, relres
  std::vector<double*> tout(n);
  for (int i = 0; i < n; i++) tout[i] = vt[i * 8 + 5];
  if ((st = set_vectors(b, xin.data(), nullptr, qout.data(), nullptr, s))) return st;
  if ((st = enqueue_spmm<L>(b, nullptr, s))) return st;
  if ((st = launch_vec<L, V_RESID>(ex, nvb, s, b, n, S, 0, 4, 5, 7, part, part2, false))) return st;
  launch_fin<L, F_RELRES>(ex, fin, s, b, n, S, part, part2, rtol, atol, maxit);
  MPS_CUDA(cudaGetLastError());
  std::vector<int> hit(b->nsys);
  std::vector<double> hrr(b->nsys);
  MPS_CUDA(cudaMemcpyAsync(hs.data(), S.status, sizeof(int) * b->nsys, cudaMemcpyDeviceToHost, s));
  MPS_CUDA(cudaMemcpyAsync(hit.data(), S.iter, sizeof(int) * b->nsys, cudaMemcpyDeviceToHost, s));
  MPS_CUDA(cudaMemcpyAsync(hrr.data(), S.relres, sizeof(double) * b->nsys, cudaMemcpyDeviceToHost, s));
  MPS_CUDA(cudaStreamSynchronize(s));
  int worst = MPSPMV_OK;
  for (int64_t q = 0; q < b->nsys; q++) {
    if (iters) iters[q] = hit[q];
    if (relres) relres[q] = hrr[q];
    if (status_out) status_out[q] = hs[q] == 1 ? MPSPMV_OK : hs[q];
    if (hs[q] == MPSPMV_EBREAKDOWN) worst = MPSPMV_EBREAKDOWN;
    else if (hs[q] == MPSPMV_ENOCONV && worst == MPSPMV_OK) worst = MPSPMV_ENOCONV;
  }
  return worst;
}

}  // namespace

extern "C" {

int mpspmv_batch_create(const mpspmv_h* mats, const int* k, int count, unsigned flags, mpspmv_batch_h* out,
                        void* stream) {
  if (!out || !mats || !k || count < 1 || (flags & ~MPSPMV_BATCH_AUTOTUNE)) return MPSPMV_EINVAL;
  *out = nullptr;
  const int L = mats[0] ? mats[0]->L : 0;
  for (int i = 0; i < count; i++) {
    const mpspmv_mat* h = mats[i];
    if (!h || h->L != L || h->cplx || h->mixed || h->nnz == 0 || k[i] < 1 || k[i] > 32 ||
        h->exact != mats[0]->exact || h->dstore != mats[0]->dstore)
      return MPSPMV_EINVAL;
  }
  cudaStream_t s = mps_stream(stream);
  mpspmv_batch* b = new mpspmv_batch();
  cudaGetDevice(&b->device);
  b->count = count;
  b->L = L;
  b->mats.assign(mats, mats + count);
  b->k.assign(k, k + count);
  b->w.assign(count, 1);
  int st = MPSPMV_OK;
  if (cudaMalloc(&b->d_entries, sizeof(BatchEntry) * count) != cudaSuccess ||
      cudaMalloc(&b->d_item_start, sizeof(int64_t) * (count + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_comb_start, sizeof(int64_t) * (count + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_sys_start, sizeof(int64_t) * (count + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_vec_start, sizeof(int64_t) * (count + 1)) != cudaSuccess ||
      cudaMalloc(&b->d_head, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return MPSPMV_ENOMEM;
  }
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
  const bool ex = mats[0]->exact, ds = mats[0]->dstore;
  auto occ = [&](auto kern) { cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kBT, 0); };
  switch (L) {
    case 1: ex ? (ds ? occ(batch_runs_kernel<1, true, true>) : occ(batch_runs_kernel<1, true, false>))
               : occ(batch_runs_kernel<1, false, false>); break;
    case 2: ex ? (ds ? occ(batch_runs_kernel<2, true, true>) : occ(batch_runs_kernel<2, true, false>))
               : occ(batch_runs_kernel<2, false, false>); break;
    case 3: ex ? (ds ? occ(batch_runs_kernel<3, true, true>) : occ(batch_runs_kernel<3, true, false>))
               : occ(batch_runs_kernel<3, false, false>); break;
    default: ex ? (ds ? occ(batch_runs_kernel<4, true, true>) : occ(batch_runs_kernel<4, true, false>))
                : occ(batch_runs_kernel<4, false, false>); break;
  }
  b->grid_runs = std::max(1, sms * std::max(per, 1));
  if ((flags & MPSPMV_BATCH_AUTOTUNE) && (st = autotune(b, s))) {
    free_batch(b);
    return st;
  }
  if ((st = layout(b, s))) {
    free_batch(b);
    return st;
  }
  *out = b;
  return MPSPMV_OK;
}

int mpspmv_batch_destroy(mpspmv_batch_h b) {
  if (!b) return MPSPMV_EINVAL;
  cudaDeviceSynchronize();
  free_batch(b);
  return MPSPMV_OK;
}

int mpspmv_batch_get_plan(mpspmv_batch_h b, int* K, int* w) {
  if (!b) return MPSPMV_EINVAL;
  for (int i = 0; i < b->count; i++) {
    if (K) K[i] = b->mats[i]->K;
    if (w) w[i] = b->w[i];
  }
  return MPSPMV_OK;
}

int mpspmv_batch_spmm(mpspmv_batch_h b, const double* const* X, const int64_t* ldx, double* const* Y,
                      const int64_t* ldy, void* stream) {
  if (!b || !X || !Y) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  std::vector<const void*> key;
  key.reserve(4 * b->count);
  for (int i = 0; i < b->count; i++) {
    key.push_back(X[i]);
    key.push_back(Y[i]);
    key.push_back(reinterpret_cast<const void*>(ldx ? ldx[i] : b->k[i]));
    key.push_back(reinterpret_cast<const void*>(ldy ? ldy[i] : b->k[i]));
  }
  if (!b->spmm_exec || key != b->spmm_key) {
    if (b->spmm_exec) {
      cudaGraphExecDestroy(b->spmm_exec);
      b->spmm_exec = nullptr;
    }
    int st = set_vectors(b, X, ldx, Y, ldy, s);
    if (st) return st;
    MPS_CUDA(cudaStreamSynchronize(s));
    // capture the batched product (queue reset, persistent run kernel,
    // combine) as one graph
    cudaStream_t cs;
    MPS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    st = MPSPMV_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = MPSPMV_ECUDA;
    if (!st) st = enqueue_spmm_any(b, nullptr, cs);
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess && !st) st = MPSPMV_ECUDA;
    if (!st && cudaGraphInstantiate(&b->spmm_exec, g, 0) != cudaSuccess) st = MPSPMV_ECUDA;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (st) return st;
    b->spmm_key = key;
  }
  MPS_CUDA(cudaGraphLaunch(b->spmm_exec, s));
  return MPSPMV_OK;
}

int mpspmv_batch_cg(mpspmv_batch_h b, const double* const* B, const int64_t* ldb, double* const* X,
                    const int64_t* ldx, double rtol, double atol, int maxit, int* iters, double* relres,
                    int* status, void* stream) {
  if (!b || !B || !X || !(rtol >= 0.0) || !(atol >= 0.0) || maxit < 0) return MPSPMV_EINVAL;
  for (int i = 0; i < b->count; i++)
    if (b->mats[i]->nrows != b->mats[i]->ncols) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  int st;
  switch (b->L) {
    case 1: st = batch_cg_impl<1>(b, B, ldb, X, ldx, rtol, atol, maxit, iters, relres, status, s); break;
    case 2: st = batch_cg_impl<2>(b, B, ldb, X, ldx, rtol, atol, maxit, iters, relres, status, s); break;
    case 3: st = batch_cg_impl<3>(b, B, ldb, X, ldx, rtol, atol, maxit, iters, relres, status, s); break;
    default: st = batch_cg_impl<4>(b, B, ldb, X, ldx, rtol, atol, maxit, iters, relres, status, s); break;
  }
  // the SpMM graph was built for other vectors
  if (b->spmm_exec) {
    cudaGraphExecDestroy(b->spmm_exec);
    b->spmm_exec = nullptr;
    b->spmm_key.clear();
  }
  return st;
}

}  // extern "C"
