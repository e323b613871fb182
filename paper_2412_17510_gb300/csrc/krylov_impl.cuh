// krylov_impl.cuh -- Krylov solvers with every vector and scalar in DD / TD / QD
// (arXiv 2412.17510, Section 4.2: x0 given (0 in the paper), stop when
// ||r_k||_2 <= rtol ||b||_2 + atol).
//
// Formulations: unpreconditioned CG (Hestenes-Stiefel) for real symmetric
// positive definite A; BiCGSTAB (van der Vorst) with r_hat = r_0 for real or
// complex A, inner products (u, v) = sum conj(u_i) v_i.
//
// GB300 design: the whole iteration stays on the device.  Dot products are
// two-stage deterministic reductions (fixed grid; per-thread sequential MP
// sums, an MP shuffle tree per warp, a tree across warps, then one block over
// the per-block partials) and the scalar recurrences (alpha, beta, omega,
// the stopping test) run in the single-block finishing kernel, so there is no
// host round trip per iteration.  The axpy updates are fused with the dot
// product that follows them.  Each kernel returns at once when the solver
// state is no longer "running", so a CUDA graph holding several iterations
// can be replayed until the host sees a final state.
//
// Handles created with MPSPMV_EXACT_ACC use the exact-accumulation vector
// kernels below (kx_*) instead: each updated element is rounded once and each
// thread's share of a dot product is summed exactly.
#pragma once
#include <algorithm>
#include <climits>
#include <cmath>

#include "internal.h"
#include "krylov.h"
#include "krylov_ops.h"
#include "exact_prod.cuh"
#include "mp_arith.cuh"

using namespace mpk;

// digits of the exact accumulators of a block (dynamic shared memory)
extern __shared__ unsigned long long x_digits[];

namespace mpkry {
// Kernels and helpers have internal linkage: each translation unit that
// instantiates them launches (and configures) its own copies.
namespace {

constexpr int kT = 256;           // threads per block
constexpr int kMaxBlocks = 1024;  // partials per dot (paper-order kernels)
constexpr int kTX = 128;          // threads per block of the exact kernels
constexpr int kMaxPart = 2048;    // partials buffer length (either kind)
constexpr int kItersPerGraph = 8;

enum : int { RUNNING = 0, CONVERGED = 1, PENDING_X = 2 };

// ---------------------------------------------------------------------------
// complex MP helpers (re, im pairs)
// ---------------------------------------------------------------------------
template <int L>
struct cmp {
  mp<L> re, im;
};

template <int L>
__device__ __forceinline__ cmp<L> c_mul(const cmp<L>& a, const cmp<L>& b) {
  mp<L> t1 = mp_mul<L>(a.re, b.re), t2 = mp_mul<L>(a.im, b.im);
  mp<L> t3 = mp_mul<L>(a.re, b.im), t4 = mp_mul<L>(a.im, b.re);
  cmp<L> r;
  r.re = mp_sub<L>(t1, t2);
  r.im = mp_add<L>(t3, t4);
  return r;
}

// a / b = a conj(b) / |b|^2, with a and b first scaled by the same power of
// two (exact, component by component) so that the larger part of b is near
// 1: |b|^2 then stays in range when b is tiny or huge (the scalars of a
// converged iteration reach 1e-200 and below).
template <int L>
__device__ __forceinline__ cmp<L> c_div(const cmp<L>& a, const cmp<L>& b) {
  const double m = fmax(fabs(b.re.v[0]), fabs(b.im.v[0]));
  const int e = (m > 0.0 && isfinite(m)) ? ilogb(m) : 0;
  cmp<L> as, bs;
#pragma unroll
  for (int l = 0; l < L; l++) {
    as.re.v[l] = scalbn(a.re.v[l], -e);
    as.im.v[l] = scalbn(a.im.v[l], -e);
    bs.re.v[l] = scalbn(b.re.v[l], -e);
    bs.im.v[l] = scalbn(b.im.v[l], -e);
  }
  cmp<L> nb;
  nb.re = bs.re;
  nb.im = mp_neg<L>(bs.im);
  cmp<L> num = c_mul<L>(as, nb);
  mp<L> d = mp_add<L>(mp_mul<L>(bs.re, bs.re), mp_mul<L>(bs.im, bs.im));
  cmp<L> r;
  r.re = mp_div<L>(num.re, d);
  r.im = mp_div<L>(num.im, d);
  return r;
}

template <int L, bool CPLX>
__device__ __forceinline__ cmp<L> load_v(const double* __restrict__ v, int64_t n, int64_t i) {
  cmp<L> r;
#pragma unroll
  for (int l = 0; l < L; l++) r.re.v[l] = v[(int64_t)l * n + i];
  if (CPLX) {
#pragma unroll
    for (int l = 0; l < L; l++) r.im.v[l] = v[(int64_t)(L + l) * n + i];
  } else {
    r.im = mp_zero<L>();
  }
  return r;
}

template <int L, bool CPLX>
__device__ __forceinline__ void store_v(double* __restrict__ v, int64_t n, int64_t i, const cmp<L>& a) {
#pragma unroll
  for (int l = 0; l < L; l++) v[(int64_t)l * n + i] = a.re.v[l];
  if (CPLX) {
#pragma unroll
    for (int l = 0; l < L; l++) v[(int64_t)(L + l) * n + i] = a.im.v[l];
  }
}

// w = u + a * v   (the real case multiplies only the real parts)
template <int L, bool CPLX>
__device__ __forceinline__ cmp<L> axpy1(const cmp<L>& a, const cmp<L>& u, const cmp<L>& v) {
  cmp<L> r;
  if (CPLX) {
    cmp<L> t = c_mul<L>(a, v);
    r.re = mp_add<L>(u.re, t.re);
    r.im = mp_add<L>(u.im, t.im);
  } else {
    r.re = mp_add<L>(u.re, mp_mul<L>(a.re, v.re));
    r.im = u.im;
  }
  return r;
}

// acc += conj(u) v   (order: re += ur vr; re += ui vi; im += ur vi; im -= ui vr)
template <int L, bool CPLX>
__device__ __forceinline__ void dot_acc(mp<L>& dr, mp<L>& di, const cmp<L>& u, const cmp<L>& v) {
  dr = mp_add<L>(dr, mp_mul<L>(u.re, v.re));
  if (CPLX) {
    dr = mp_add<L>(dr, mp_mul<L>(u.im, v.im));
    di = mp_add<L>(di, mp_mul<L>(u.re, v.im));
    di = mp_add<L>(di, mp_neg<L>(mp_mul<L>(u.im, v.re)));
  }
}

template <int L>
__device__ __forceinline__ mp<L> shfl_down(const mp<L>& a, int off) {
  mp<L> r;
#pragma unroll
  for (int l = 0; l < L; l++) r.v[l] = __shfl_down_sync(0xffffffffu, a.v[l], off);
  return r;
}

// Reduce NA MP accumulators over the block of TB threads (result valid in
// thread 0).
// Accumulators come in (real part, imaginary part) pairs; RE_ONLY (real
// data) skips the imaginary ones, which are zero.
template <bool RE_ONLY>
__device__ __forceinline__ constexpr bool live_acc(int a) {
  return !RE_ONLY || (a % 2) == 0;
}

template <int L, int NA, int TB = kT, bool RE_ONLY = false>
__device__ __forceinline__ void block_reduce(mp<L> (&acc)[NA]) {
  __shared__ double sm[TB / 32][NA][L];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int a = 0; a < NA; a++) {
      if (!live_acc<RE_ONLY>(a)) continue;
      mp<L> o = shfl_down<L>(acc[a], off);
      if (lane < off) acc[a] = mp_add<L>(acc[a], o);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < NA; a++)
#pragma unroll
      for (int l = 0; l < L; l++) sm[warp][a][l] = acc[a].v[l];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int a = 0; a < NA; a++) {
      if (lane < TB / 32) {
#pragma unroll
        for (int l = 0; l < L; l++) acc[a].v[l] = sm[lane][a][l];
      } else {
        acc[a] = mp_zero<L>();
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
      for (int a = 0; a < NA; a++) {
        if (!live_acc<RE_ONLY>(a)) continue;
        mp<L> o = shfl_down<L>(acc[a], off);
        if (lane < off) acc[a] = mp_add<L>(acc[a], o);
      }
    }
  }
}

template <int L, int NA, int TB = kT, bool RE_ONLY = false>
__device__ __forceinline__ void write_partials(double* __restrict__ part, int G, mp<L> (&acc)[NA]) {
  block_reduce<L, NA, TB, RE_ONLY>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NA; a++)
      if (live_acc<RE_ONLY>(a))
#pragma unroll
        for (int l = 0; l < L; l++) part[((int64_t)a * L + l) * G + blockIdx.x] = acc[a].v[l];
  }
}

// Finishing step: reduce the G block partials of NA accumulators (one block).
template <int L, int NA, bool RE_ONLY = false>
__device__ __forceinline__ void reduce_partials(const double* __restrict__ part, int G, mp<L> (&acc)[NA]) {
#pragma unroll
  for (int a = 0; a < NA; a++) acc[a] = mp_zero<L>();
  for (int g = threadIdx.x; g < G; g += kT) {
#pragma unroll
    for (int a = 0; a < NA; a++) {
      if (!live_acc<RE_ONLY>(a)) continue;
      mp<L> v;
#pragma unroll
      for (int l = 0; l < L; l++) v.v[l] = part[((int64_t)a * L + l) * G + g];
      acc[a] = mp_add<L>(acc[a], v);
    }
  }
  block_reduce<L, NA, kT, RE_ONLY>(acc);
}

// ---------------------------------------------------------------------------
// Exact block sums (MPSPMV_EXACT_ACC handles).  Every component entering the
// sum is placed in signed 64-bit digits of 32 bits each (FixAcc) at one
// common base, chosen from the largest component in the block so that no
// term moves the window; the digits are then added as integers across the
// warp (shuffles) and the block, and the total is cut to L components once.
// A sum of up to 2^13 terms of magnitude below 2^(top+1) stays inside the
// head-room digit.  Components far below the largest one lose the bits below
// the window (32 (D - 1) - 1 bits under the top), far below u_L relative to
// it.
// ---------------------------------------------------------------------------
template <int TB>
__device__ __forceinline__ int block_max_int(int v) {
  __shared__ int s[TB / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  v = s[0];
#pragma unroll
  for (int w = 1; w < TB / 32; w++) v = max(v, s[w]);
  __syncthreads();
  return v;
}

// Sum the digit arrays f[a] over the block; thread 0 gets the totals cut to
// L components in out[a] (zero for accumulators that are not live).
template <int L, int D, int NA, int TB, bool RE_ONLY>
__device__ __forceinline__ void block_digit_sum(FixAcc<D> (&f)[NA], mp<L> (&out)[NA]) {
  __shared__ long long s_d[TB / 32][NA][D];
  __shared__ int s_bad[TB / 32][NA];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int a = 0; a < NA; a++) {
    if (!live_acc<RE_ONLY>(a)) continue;
    const bool bad = __any_sync(0xffffffffu, f[a].bad);
    if (f[a].live) {  // uniform over the block (set from the block's top exponent)
#pragma unroll
      for (int j = 0; j < D; j++) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) f[a].d[j] += __shfl_down_sync(0xffffffffu, f[a].d[j], off);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < D; j++) s_d[warp][a][j] = f[a].d[j];
      s_bad[warp][a] = bad;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NA; a++) {
      out[a] = mp_zero<L>();
      if (!live_acc<RE_ONLY>(a)) continue;
      FixAcc<D> r = f[a];  // base and live of the block
      r.bad = false;
#pragma unroll
      for (int j = 0; j < D; j++) r.d[j] = 0;
      for (int w = 0; w < TB / 32; w++) {
#pragma unroll
        for (int j = 0; j < D; j++) r.d[j] += s_d[w][a][j];
        r.bad |= s_bad[w][a] != 0;
      }
      fa_to_mp<L, D>(r, out[a].v);
    }
  }
  __syncthreads();
}

// exact counterpart of write_partials (one MP value per thread and accumulator)
template <int L, int NA, int TB, bool RE_ONLY>
__device__ __forceinline__ void write_partials_x(double* __restrict__ part, int G, mp<L> (&acc)[NA]) {
  constexpr int D = AccDigits<L>::D;
  FixAcc<D> f[NA];
#pragma unroll
  for (int a = 0; a < NA; a++) {
    if (!live_acc<RE_ONLY>(a)) continue;
    int t = INT_MIN;
    bool bad = false;
#pragma unroll
    for (int l = 0; l < L; l++) {
      t = max(t, top_exp(acc[a].v[l]));
      bad |= !isfinite(acc[a].v[l]);
    }
    t = block_max_int<TB>(t);
    fa_at_top<D>(f[a], t);
#pragma unroll
    for (int l = 0; l < L; l++) fa_add<D>(f[a], acc[a].v[l]);
    f[a].bad = bad;
  }
  mp<L> out[NA];
  block_digit_sum<L, D, NA, TB, RE_ONLY>(f, out);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NA; a++)
      if (live_acc<RE_ONLY>(a))
#pragma unroll
        for (int l = 0; l < L; l++) part[((int64_t)a * L + l) * G + blockIdx.x] = out[a].v[l];
  }
}

// exact counterpart of reduce_partials (block of kT threads)
template <int L, int NA, bool RE_ONLY>
__device__ __forceinline__ void reduce_partials_x(const double* __restrict__ part, int G, mp<L> (&acc)[NA]) {
  constexpr int D = AccDigits<L>::D;
  FixAcc<D> f[NA];
#pragma unroll
  for (int a = 0; a < NA; a++) {
    if (!live_acc<RE_ONLY>(a)) continue;
    int t = INT_MIN;
    for (int g = threadIdx.x; g < G; g += kT)
#pragma unroll
      for (int l = 0; l < L; l++) t = max(t, top_exp(part[((int64_t)a * L + l) * G + g]));
    t = block_max_int<kT>(t);
    fa_at_top<D>(f[a], t);
    for (int g = threadIdx.x; g < G; g += kT)
#pragma unroll
      for (int l = 0; l < L; l++) fa_add<D>(f[a], part[((int64_t)a * L + l) * G + g]);
  }
  block_digit_sum<L, D, NA, kT, RE_ONLY>(f, acc);
}

// the finishing kernels' reduction: exact for exact handles
template <int L, int NA, bool RE_ONLY>
__device__ __forceinline__ void reduce_any(const KrylovState* st, const double* __restrict__ part, int G,
                                           mp<L> (&acc)[NA]) {
  if (st->exact)
    reduce_partials_x<L, NA, RE_ONLY>(part, G, acc);
  else
    reduce_partials<L, NA, RE_ONLY>(part, G, acc);
}

template <int L>
__device__ __forceinline__ double to_d(const mp<L>& a) {
  return mp_to_double<L>(a);
}

template <int L>
__device__ __forceinline__ bool is_zero(const mp<L>& a) {
  return a.v[0] == 0.0;
}

// scalar slots in the state
template <int L>
__device__ __forceinline__ cmp<L> get_s(const KrylovState* st, int i) {
  cmp<L> r;
#pragma unroll
  for (int l = 0; l < L; l++) {
    r.re.v[l] = st->sc[i][l];
    r.im.v[l] = st->sc[i][4 + l];
  }
  return r;
}
template <int L>
__device__ __forceinline__ void put_s(KrylovState* st, int i, const cmp<L>& a) {
#pragma unroll
  for (int l = 0; l < L; l++) {
    st->sc[i][l] = a.re.v[l];
    st->sc[i][4 + l] = a.im.v[l];
  }
}
template <int L>
__device__ __forceinline__ cmp<L> neg_c(const cmp<L>& a) {
  cmp<L> r;
  r.re = mp_neg<L>(a.re);
  r.im = mp_neg<L>(a.im);
  return r;
}

enum Slot : int { S_RHO = 0, S_ALPHA, S_BETA, S_OMEGA, S_RHO1, S_TMP, S_BETA_OMEGA };

#define ACTIVE(st) if (st->status != RUNNING) return

// ---------------------------------------------------------------------------
// Dot kernels: NDOT inner products conj(u_d) v_d -> partials
// ---------------------------------------------------------------------------
template <int L, bool CPLX, int NDOT>
__global__ void __launch_bounds__(kT) k_dot(const KrylovState* st, int64_t n, const double* u0, const double* v0,
                                            const double* u1, const double* v1, double* part, int G,
                                            bool ignore_state) {
  if (!ignore_state) {
    ACTIVE(st);
  }
  constexpr int NA = 2 * NDOT;
  mp<L> acc[NA];
#pragma unroll
  for (int a = 0; a < NA; a++) acc[a] = mp_zero<L>();
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)G * kT) {
    dot_acc<L, CPLX>(acc[0], acc[1], load_v<L, CPLX>(u0, n, i), load_v<L, CPLX>(v0, n, i));
    if (NDOT > 1) dot_acc<L, CPLX>(acc[2], acc[3], load_v<L, CPLX>(u1, n, i), load_v<L, CPLX>(v1, n, i));
  }
  write_partials<L, NA, kT, !CPLX>(part, G, acc);
}

// r = b - q (q = A x); optionally p = r and rh = r; partial (r, r)
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_residual(int64_t n, const double* b, const double* q, double* r, double* p,
                                                 double* rh, double* part, int G) {
  mp<L> acc[2] = {mp_zero<L>(), mp_zero<L>()};
  cmp<L> m1;
  m1.re = mp_zero<L>();
  m1.re.v[0] = -1.0;
  m1.im = mp_zero<L>();
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)G * kT) {
    cmp<L> ri = axpy1<L, CPLX>(m1, load_v<L, CPLX>(b, n, i), load_v<L, CPLX>(q, n, i));
    store_v<L, CPLX>(r, n, i, ri);
    if (p) store_v<L, CPLX>(p, n, i, ri);
    if (rh) store_v<L, CPLX>(rh, n, i, ri);
    dot_acc<L, CPLX>(acc[0], acc[1], ri, ri);
  }
  write_partials<L, 2, kT, true>(part, G, acc);
}

// ---------------------------------------------------------------------------
// CG
// ---------------------------------------------------------------------------
// start: part0 = (r, r), part1 = (b, b)
template <int L>
__global__ void __launch_bounds__(kT) k_cg_start(KrylovState* st, const double* part_r, const double* part_b, int G,
                                                 double rtol, double atol) {
  mp<L> a[2], b[2];
  reduce_any<L, 2, true>(st, part_r, G, a);
  __syncthreads();
  reduce_any<L, 2, true>(st, part_b, G, b);
  if (threadIdx.x == 0) {
    const double bb = to_d<L>(b[0]);
    const double bnorm = sqrt(bb > 0.0 ? bb : 0.0);
    const double tol = rtol * bnorm + atol;
    st->bnorm = bnorm;
    st->tol = tol;
    cmp<L> rho;
    rho.re = a[0];
    rho.im = mp_zero<L>();
    put_s<L>(st, S_RHO, rho);
    const double rr = to_d<L>(a[0]);
    st->iter = 0;
    st->status = (sqrt(rr > 0.0 ? rr : 0.0) <= tol) ? CONVERGED : RUNNING;
    if (st->status == RUNNING && st->maxit <= 0) st->status = MPSPMV_ENOCONV;
  }
}

// alpha = rho / (p, q)
template <int L>
__global__ void __launch_bounds__(kT) k_cg_alpha(KrylovState* st, const double* part, int G) {
  ACTIVE(st);
  mp<L> a[2];
  reduce_any<L, 2, true>(st, part, G, a);
  if (threadIdx.x == 0) {
    if (is_zero<L>(a[0]) || !isfinite(a[0].v[0])) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    cmp<L> al;
    al.re = mp_div<L>(get_s<L>(st, S_RHO).re, a[0]);
    al.im = mp_zero<L>();
    put_s<L>(st, S_ALPHA, al);
  }
}

// x += alpha p; r += (-alpha) q; partial (r, r)
template <int L>
__global__ void __launch_bounds__(kT) k_cg_xr(const KrylovState* st, int64_t n, double* x, double* r,
                                              const double* p, const double* q, double* part, int G) {
  ACTIVE(st);
  const cmp<L> al = get_s<L>(st, S_ALPHA);
  const cmp<L> nal = neg_c<L>(al);
  mp<L> acc[2] = {mp_zero<L>(), mp_zero<L>()};
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)G * kT) {
    cmp<L> xi = axpy1<L, false>(al, load_v<L, false>(x, n, i), load_v<L, false>(p, n, i));
    store_v<L, false>(x, n, i, xi);
    cmp<L> ri = axpy1<L, false>(nal, load_v<L, false>(r, n, i), load_v<L, false>(q, n, i));
    store_v<L, false>(r, n, i, ri);
    dot_acc<L, false>(acc[0], acc[1], ri, ri);
  }
  write_partials<L, 2, kT, true>(part, G, acc);
}

// rho1 = (r, r); k++; stopping test; beta = rho1 / rho; rho = rho1
template <int L>
__global__ void __launch_bounds__(kT) k_cg_beta(KrylovState* st, const double* part, int G) {
  ACTIVE(st);
  mp<L> a[2];
  reduce_any<L, 2, true>(st, part, G, a);
  if (threadIdx.x == 0) {
    st->iter++;
    const double t = to_d<L>(a[0]);
    if (st->iter <= 16) st->hist[st->iter - 1] = st->bnorm > 0.0 ? sqrt(t > 0.0 ? t : 0.0) / st->bnorm : 0.0;
    if (!isfinite(t)) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    if (sqrt(t > 0.0 ? t : 0.0) <= st->tol) {
      st->status = CONVERGED;
      return;
    }
    const cmp<L> rho = get_s<L>(st, S_RHO);
    if (is_zero<L>(rho.re)) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    cmp<L> be;
    be.re = mp_div<L>(a[0], rho.re);
    be.im = mp_zero<L>();
    put_s<L>(st, S_BETA, be);
    cmp<L> r1;
    r1.re = a[0];
    r1.im = mp_zero<L>();
    put_s<L>(st, S_RHO, r1);
    if (st->iter >= st->maxit) st->status = MPSPMV_ENOCONV;
  }
}

// p = r + beta p
template <int L>
__global__ void __launch_bounds__(kT) k_cg_p(const KrylovState* st, int64_t n, const double* r, double* p, int G) {
  ACTIVE(st);
  const cmp<L> be = get_s<L>(st, S_BETA);
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)G * kT)
    store_v<L, false>(p, n, i, axpy1<L, false>(be, load_v<L, false>(r, n, i), load_v<L, false>(p, n, i)));
}

// ---------------------------------------------------------------------------
// BiCGSTAB
// ---------------------------------------------------------------------------
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_start(KrylovState* st, const double* part_r, const double* part_b, int G,
                                                 double rtol, double atol) {
  mp<L> a[2], b[2];
  reduce_any<L, 2, true>(st, part_r, G, a);
  __syncthreads();
  reduce_any<L, 2, true>(st, part_b, G, b);
  if (threadIdx.x == 0) {
    const double bb = to_d<L>(b[0]);
    const double bnorm = sqrt(bb > 0.0 ? bb : 0.0);
    const double tol = rtol * bnorm + atol;
    st->bnorm = bnorm;
    st->tol = tol;
    cmp<L> one;
    one.re = mp_zero<L>();
    one.re.v[0] = 1.0;
    one.im = mp_zero<L>();
    put_s<L>(st, S_RHO, one);
    put_s<L>(st, S_ALPHA, one);
    put_s<L>(st, S_OMEGA, one);
    const double rr = to_d<L>(a[0]);
    st->iter = 0;
    st->status = (sqrt(rr > 0.0 ? rr : 0.0) <= tol) ? CONVERGED : RUNNING;
    if (st->status == RUNNING && st->maxit <= 0) st->status = MPSPMV_ENOCONV;
  }
}

// rho1 = (rh, r); beta = (rho1 / rho) (alpha / omega)
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_beta(KrylovState* st, const double* part, int G) {
  ACTIVE(st);
  mp<L> a[2];
  reduce_any<L, 2, !CPLX>(st, part, G, a);
  if (threadIdx.x == 0) {
    if (is_zero<L>(a[0]) && (!CPLX || is_zero<L>(a[1]))) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    cmp<L> r1;
    r1.re = a[0];
    r1.im = CPLX ? a[1] : mp_zero<L>();
    const cmp<L> rho = get_s<L>(st, S_RHO), al = get_s<L>(st, S_ALPHA), om = get_s<L>(st, S_OMEGA);
    cmp<L> be;
    if (CPLX) {
      be = c_mul<L>(c_div<L>(r1, rho), c_div<L>(al, om));
    } else {
      be.re = mp_mul<L>(mp_div<L>(r1.re, rho.re), mp_div<L>(al.re, om.re));
      be.im = mp_zero<L>();
    }
    put_s<L>(st, S_BETA, be);
    put_s<L>(st, S_RHO1, r1);
    // the exact p update uses r + beta p - (beta omega) v
    if (CPLX) {
      put_s<L>(st, S_BETA_OMEGA, c_mul<L>(be, om));
    } else {
      cmp<L> bw;
      bw.re = mp_mul<L>(be.re, om.re);
      bw.im = mp_zero<L>();
      put_s<L>(st, S_BETA_OMEGA, bw);
    }
  }
}

// p = r + beta (p - omega v)
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_p(const KrylovState* st, int64_t n, const double* r, double* p,
                                             const double* v, int G) {
  ACTIVE(st);
  const cmp<L> be = get_s<L>(st, S_BETA), nom = neg_c<L>(get_s<L>(st, S_OMEGA));
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)G * kT) {
    cmp<L> t = axpy1<L, CPLX>(nom, load_v<L, CPLX>(p, n, i), load_v<L, CPLX>(v, n, i));
    store_v<L, CPLX>(p, n, i, axpy1<L, CPLX>(be, load_v<L, CPLX>(r, n, i), t));
  }
}

// alpha = rho1 / (rh, v)
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_alpha(KrylovState* st, const double* part, int G) {
  ACTIVE(st);
  mp<L> a[2];
  reduce_any<L, 2, !CPLX>(st, part, G, a);
  if (threadIdx.x == 0) {
    if (is_zero<L>(a[0]) && (!CPLX || is_zero<L>(a[1]))) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    cmp<L> d;
    d.re = a[0];
    d.im = CPLX ? a[1] : mp_zero<L>();
    const cmp<L> r1 = get_s<L>(st, S_RHO1);
    cmp<L> al;
    if (CPLX) {
      al = c_div<L>(r1, d);
    } else {
      al.re = mp_div<L>(r1.re, d.re);
      al.im = mp_zero<L>();
    }
    put_s<L>(st, S_ALPHA, al);
  }
}

// s = r - alpha v; partial (s, s)
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_s(const KrylovState* st, int64_t n, const double* r, const double* v,
                                             double* s, double* part, int G) {
  ACTIVE(st);
  const cmp<L> nal = neg_c<L>(get_s<L>(st, S_ALPHA));
  mp<L> acc[2] = {mp_zero<L>(), mp_zero<L>()};
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)G * kT) {
    cmp<L> si = axpy1<L, CPLX>(nal, load_v<L, CPLX>(r, n, i), load_v<L, CPLX>(v, n, i));
    store_v<L, CPLX>(s, n, i, si);
    dot_acc<L, CPLX>(acc[0], acc[1], si, si);
  }
  write_partials<L, 2, kT, true>(part, G, acc);
}

// k++; if ||s|| <= tol: converge after x += alpha p
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_scheck(KrylovState* st, const double* part, int G) {
  ACTIVE(st);
  mp<L> a[2];
  reduce_any<L, 2, true>(st, part, G, a);
  if (threadIdx.x == 0) {
    st->iter++;
    const double t = to_d<L>(a[0]);
    if (!isfinite(t)) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    if (sqrt(t > 0.0 ? t : 0.0) <= st->tol) st->status = PENDING_X;
  }
}

// the early exit: x += alpha p
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_xfix(KrylovState* st, int64_t n, double* x, const double* p, int G,
                                                int* done_counter) {
  if (st->status != PENDING_X) return;
  const cmp<L> al = get_s<L>(st, S_ALPHA);
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)G * kT)
    store_v<L, CPLX>(x, n, i, axpy1<L, CPLX>(al, load_v<L, CPLX>(x, n, i), load_v<L, CPLX>(p, n, i)));
  // the last block to finish publishes the final state
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(done_counter, 1) == G - 1) {
      *done_counter = 0;
      st->status = CONVERGED;
    }
  }
}

// omega = (t, s) / (t, t)   (parts: [0..1] (t,s), [2..3] (t,t))
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_omega(KrylovState* st, const double* part, int G) {
  ACTIVE(st);
  mp<L> a[4];
  reduce_any<L, 4, !CPLX>(st, part, G, a);
  if (threadIdx.x == 0) {
    if (is_zero<L>(a[2])) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    cmp<L> ts, tt, om;
    ts.re = a[0];
    ts.im = CPLX ? a[1] : mp_zero<L>();
    tt.re = a[2];
    tt.im = CPLX ? a[3] : mp_zero<L>();
    if (CPLX) {
      om = c_div<L>(ts, tt);
    } else {
      om.re = mp_div<L>(ts.re, tt.re);
      om.im = mp_zero<L>();
    }
    put_s<L>(st, S_OMEGA, om);
  }
}

// x += alpha p; x += omega s; r = s - omega t; partial (r, r)
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_xr(const KrylovState* st, int64_t n, double* x, double* r,
                                              const double* p, const double* s, const double* t, double* part,
                                              int G) {
  ACTIVE(st);
  const cmp<L> al = get_s<L>(st, S_ALPHA), om = get_s<L>(st, S_OMEGA), nom = neg_c<L>(om);
  mp<L> acc[2] = {mp_zero<L>(), mp_zero<L>()};
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)G * kT) {
    const cmp<L> si = load_v<L, CPLX>(s, n, i);
    cmp<L> xi = axpy1<L, CPLX>(al, load_v<L, CPLX>(x, n, i), load_v<L, CPLX>(p, n, i));
    xi = axpy1<L, CPLX>(om, xi, si);
    store_v<L, CPLX>(x, n, i, xi);
    cmp<L> ri = axpy1<L, CPLX>(nom, si, load_v<L, CPLX>(t, n, i));
    store_v<L, CPLX>(r, n, i, ri);
    dot_acc<L, CPLX>(acc[0], acc[1], ri, ri);
  }
  write_partials<L, 2, kT, true>(part, G, acc);
}

// ||r|| test; omega == 0 breakdown; rho = rho1; maxit
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_rcheck(KrylovState* st, const double* part, int G) {
  ACTIVE(st);
  mp<L> a[2];
  reduce_any<L, 2, true>(st, part, G, a);
  if (threadIdx.x == 0) {
    const double t = to_d<L>(a[0]);
    if (!isfinite(t)) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    if (sqrt(t > 0.0 ? t : 0.0) <= st->tol) {
      st->status = CONVERGED;
      return;
    }
    const cmp<L> om = get_s<L>(st, S_OMEGA);
    if (is_zero<L>(om.re) && (!CPLX || is_zero<L>(om.im))) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    put_s<L>(st, S_RHO, get_s<L>(st, S_RHO1));
    if (st->iter >= st->maxit) st->status = MPSPMV_ENOCONV;
  }
}

// relres = sqrt((r,r)) / bnorm   (r = true residual)
template <int L>
__global__ void __launch_bounds__(kT) k_relres(KrylovState* st, const double* part, int G) {
  mp<L> a[2];
  reduce_any<L, 2, true>(st, part, G, a);
  if (threadIdx.x == 0) {
    const double t = to_d<L>(a[0]);
    const double rn = sqrt(t > 0.0 ? t : 0.0);
    st->relres = st->bnorm > 0.0 ? rn / st->bnorm : rn;
  }
}

// ---------------------------------------------------------------------------
// Exact-accumulation vector kernels (handles created with MPSPMV_EXACT_ACC).
// An updated element u + sum_k c_k v_k is formed from the components of u and
// the error-free products c_k v_k (exact_prod.cuh) in one exact fixed-point
// accumulator and cut to L components once (the real and imaginary parts one
// after the other in the same accumulator).  Each thread sums its share of a
// dot product in a second accumulator, flushed once; only the block tree and
// the finishing kernel add in MP arithmetic.  Accumulator k of a thread uses
// 2 D digits at x_digits[k * 2 D kTX ...] (digit j of thread t at j kTX + t).
// ---------------------------------------------------------------------------
template <int L>
using XAcc = FixAccS<AccDigits<L>::D, kTX>;

// dynamic shared memory of a kernel holding nacc accumulators per thread
template <int L>
constexpr size_t x_smem(int nacc) {
  return (size_t)nacc * 2 * AccDigits<L>::D * kTX * sizeof(unsigned long long);
}

template <int L>
__device__ __forceinline__ XAcc<L> x_acc(int k) {
  constexpr int D = AccDigits<L>::D;
  XAcc<L> a;
  a.dp = x_digits + (size_t)k * 2 * D * kTX + threadIdx.x;
  a.dn = a.dp + D * kTX;
  fas_reset<D, kTX>(a);
  return a;
}

template <int L>
__device__ __forceinline__ void x_add_mp(XAcc<L>& a, const mp<L>& u, bool neg) {
#pragma unroll
  for (int l = 0; l < L; l++) acc_add(a, u.v[l], neg);
}

// the accumulated value cut to L components; the accumulator is cleared
template <int L>
__device__ __forceinline__ mp<L> x_flush(XAcc<L>& a) {
  mp<L> r;
  fas_to_mp_inline<L, AccDigits<L>::D, kTX>(a, r.v);
  fas_reset<AccDigits<L>::D, kTX>(a);
  return r;
}

// u + sum_k c_k v_k, each part rounded once
template <int L, bool CPLX, int NT>
__device__ __forceinline__ cmp<L> x_lin(XAcc<L>& e, const cmp<L>& u, const cmp<L> (&c)[NT], const cmp<L> (&v)[NT]) {
  cmp<L> r;
  x_add_mp<L>(e, u.re, false);
#pragma unroll
  for (int k = 0; k < NT; k++) {
    add_prod<XAcc<L>, L>(e, c[k].re, v[k].re, false);
    if (CPLX) add_prod<XAcc<L>, L>(e, c[k].im, v[k].im, true);
  }
  r.re = x_flush<L>(e);
  if (CPLX) {
    x_add_mp<L>(e, u.im, false);
#pragma unroll
    for (int k = 0; k < NT; k++) {
      add_prod<XAcc<L>, L>(e, c[k].re, v[k].im, false);
      add_prod<XAcc<L>, L>(e, c[k].im, v[k].re, false);
    }
    r.im = x_flush<L>(e);
  } else {
    r.im = mp_zero<L>();
  }
  return r;
}

// u - v, rounded once per part
template <int L, bool CPLX>
__device__ __forceinline__ cmp<L> x_sub(XAcc<L>& e, const cmp<L>& u, const cmp<L>& v) {
  cmp<L> r;
  x_add_mp<L>(e, u.re, false);
  x_add_mp<L>(e, v.re, true);
  r.re = x_flush<L>(e);
  if (CPLX) {
    x_add_mp<L>(e, u.im, false);
    x_add_mp<L>(e, v.im, true);
    r.im = x_flush<L>(e);
  } else {
    r.im = mp_zero<L>();
  }
  return r;
}

// (dr, di) += conj(u) v; self (u == v): the imaginary part is exactly zero
// and di is not touched
template <int L, bool CPLX>
__device__ __forceinline__ void x_dot(XAcc<L>& dr, XAcc<L>& di, const cmp<L>& u, const cmp<L>& v, bool self) {
  if (self) {  // (u, u): the symmetric products once, doubled
    add_prod_self<XAcc<L>, L>(dr, u.re, false);
    if (CPLX) add_prod_self<XAcc<L>, L>(dr, u.im, false);
    return;
  }
  add_prod<XAcc<L>, L>(dr, u.re, v.re, false);
  if (CPLX) {
    add_prod<XAcc<L>, L>(dr, u.im, v.im, false);
    {
      add_prod<XAcc<L>, L>(di, u.re, v.im, false);
      add_prod<XAcc<L>, L>(di, u.im, v.re, true);
    }
  }
}

// NDOT inner products; with NDOT = 2 the second one must be a self product
// (t, t).  Accumulators: (u0, v0) re [, im], (u1, u1) re.
template <int L, bool CPLX, int NDOT>
__global__ void __launch_bounds__(kTX) kx_dot(const KrylovState* st, int64_t n, const double* u0, const double* v0,
                                              const double* u1, double* part, int G, bool ignore_state) {
  if (!ignore_state) {
    ACTIVE(st);
  }
  constexpr int NA = 2 * NDOT;
  const bool self0 = u0 == v0;
  XAcc<L> d[NA];
  d[0] = x_acc<L>(0);
  if (CPLX) d[1] = x_acc<L>(1);
  if (NDOT > 1) d[2] = x_acc<L>(CPLX ? 2 : 1);
  for (int64_t i = blockIdx.x * (int64_t)kTX + threadIdx.x; i < n; i += (int64_t)G * kTX) {
    x_dot<L, CPLX>(d[0], d[1], load_v<L, CPLX>(u0, n, i), load_v<L, CPLX>(v0, n, i), self0);
    if (NDOT > 1) {
      const cmp<L> t = load_v<L, CPLX>(u1, n, i);
      x_dot<L, CPLX>(d[2], d[2], t, t, true);
    }
  }
  mp<L> acc[NA];
#pragma unroll
  for (int a = 0; a < NA; a++) acc[a] = mp_zero<L>();
  acc[0] = x_flush<L>(d[0]);
  if (CPLX && !self0) acc[1] = x_flush<L>(d[1]);
  if (NDOT > 1) acc[2] = x_flush<L>(d[2]);
  write_partials_x<L, NA, kTX, !CPLX>(part, G, acc);
}

template <int L>
__device__ __forceinline__ void x_write_rr(double* part, int G, XAcc<L>& dr) {
  mp<L> acc[2] = {x_flush<L>(dr), mp_zero<L>()};
  write_partials_x<L, 2, kTX, true>(part, G, acc);
}

// r = b - q; optionally p = r and rh = r; partial (r, r)
template <int L, bool CPLX>
__global__ void __launch_bounds__(kTX) kx_residual(int64_t n, const double* b, const double* q, double* r, double* p,
                                                   double* rh, double* part, int G) {
  XAcc<L> e = x_acc<L>(0), dr = x_acc<L>(1);
  for (int64_t i = blockIdx.x * (int64_t)kTX + threadIdx.x; i < n; i += (int64_t)G * kTX) {
    const cmp<L> ri = x_sub<L, CPLX>(e, load_v<L, CPLX>(b, n, i), load_v<L, CPLX>(q, n, i));
    store_v<L, CPLX>(r, n, i, ri);
    if (p) store_v<L, CPLX>(p, n, i, ri);
    if (rh) store_v<L, CPLX>(rh, n, i, ri);
    x_dot<L, CPLX>(dr, dr, ri, ri, true);
  }
  x_write_rr<L>(part, G, dr);
}

// CG: x += alpha p; r -= alpha q; partial (r, r)
template <int L>
__global__ void __launch_bounds__(kTX) kx_cg_xr(const KrylovState* st, int64_t n, double* x, double* r,
                                                const double* p, const double* q, double* part, int G) {
  ACTIVE(st);
  const cmp<L> al[1] = {get_s<L>(st, S_ALPHA)};
  const cmp<L> nal[1] = {neg_c<L>(al[0])};
  XAcc<L> e = x_acc<L>(0), dr = x_acc<L>(1);
  for (int64_t i = blockIdx.x * (int64_t)kTX + threadIdx.x; i < n; i += (int64_t)G * kTX) {
    const cmp<L> pi[1] = {load_v<L, false>(p, n, i)};
    store_v<L, false>(x, n, i, x_lin<L, false, 1>(e, load_v<L, false>(x, n, i), al, pi));
    const cmp<L> qi[1] = {load_v<L, false>(q, n, i)};
    const cmp<L> ri = x_lin<L, false, 1>(e, load_v<L, false>(r, n, i), nal, qi);
    store_v<L, false>(r, n, i, ri);
    x_dot<L, false>(dr, dr, ri, ri, true);
  }
  x_write_rr<L>(part, G, dr);
}

// CG: p = r + beta p
template <int L>
__global__ void __launch_bounds__(kTX) kx_cg_p(const KrylovState* st, int64_t n, const double* r, double* p, int G) {
  ACTIVE(st);
  const cmp<L> be[1] = {get_s<L>(st, S_BETA)};
  XAcc<L> e = x_acc<L>(0);
  for (int64_t i = blockIdx.x * (int64_t)kTX + threadIdx.x; i < n; i += (int64_t)G * kTX) {
    const cmp<L> pi[1] = {load_v<L, false>(p, n, i)};
    store_v<L, false>(p, n, i, x_lin<L, false, 1>(e, load_v<L, false>(r, n, i), be, pi));
  }
}

// BiCGSTAB: p = r + beta p - (beta omega) v
template <int L, bool CPLX>
__global__ void __launch_bounds__(kTX) kx_bi_p(const KrylovState* st, int64_t n, const double* r, double* p,
                                               const double* v, int G) {
  ACTIVE(st);
  const cmp<L> c[2] = {get_s<L>(st, S_BETA), neg_c<L>(get_s<L>(st, S_BETA_OMEGA))};
  XAcc<L> e = x_acc<L>(0);
  for (int64_t i = blockIdx.x * (int64_t)kTX + threadIdx.x; i < n; i += (int64_t)G * kTX) {
    const cmp<L> w[2] = {load_v<L, CPLX>(p, n, i), load_v<L, CPLX>(v, n, i)};
    store_v<L, CPLX>(p, n, i, x_lin<L, CPLX, 2>(e, load_v<L, CPLX>(r, n, i), c, w));
  }
}

// BiCGSTAB: s = r - alpha v; partial (s, s)
template <int L, bool CPLX>
__global__ void __launch_bounds__(kTX) kx_bi_s(const KrylovState* st, int64_t n, const double* r, const double* v,
                                               double* s, double* part, int G) {
  ACTIVE(st);
  const cmp<L> nal[1] = {neg_c<L>(get_s<L>(st, S_ALPHA))};
  XAcc<L> e = x_acc<L>(0), dr = x_acc<L>(1);
  for (int64_t i = blockIdx.x * (int64_t)kTX + threadIdx.x; i < n; i += (int64_t)G * kTX) {
    const cmp<L> vi[1] = {load_v<L, CPLX>(v, n, i)};
    const cmp<L> si = x_lin<L, CPLX, 1>(e, load_v<L, CPLX>(r, n, i), nal, vi);
    store_v<L, CPLX>(s, n, i, si);
    x_dot<L, CPLX>(dr, dr, si, si, true);
  }
  x_write_rr<L>(part, G, dr);
}

// BiCGSTAB early exit: x += alpha p
template <int L, bool CPLX>
__global__ void __launch_bounds__(kTX) kx_bi_xfix(KrylovState* st, int64_t n, double* x, const double* p, int G,
                                                  int* done_counter) {
  if (st->status != PENDING_X) return;
  const cmp<L> al[1] = {get_s<L>(st, S_ALPHA)};
  XAcc<L> e = x_acc<L>(0);
  for (int64_t i = blockIdx.x * (int64_t)kTX + threadIdx.x; i < n; i += (int64_t)G * kTX) {
    const cmp<L> pi[1] = {load_v<L, CPLX>(p, n, i)};
    store_v<L, CPLX>(x, n, i, x_lin<L, CPLX, 1>(e, load_v<L, CPLX>(x, n, i), al, pi));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(done_counter, 1) == G - 1) {
      *done_counter = 0;
      st->status = CONVERGED;
    }
  }
}

// BiCGSTAB: x += alpha p + omega s (one rounding); r = s - omega t; partial (r, r)
template <int L, bool CPLX>
__global__ void __launch_bounds__(kTX) kx_bi_xr(const KrylovState* st, int64_t n, double* x, double* r,
                                                const double* p, const double* s, const double* t, double* part,
                                                int G) {
  ACTIVE(st);
  const cmp<L> ao[2] = {get_s<L>(st, S_ALPHA), get_s<L>(st, S_OMEGA)};
  const cmp<L> nom[1] = {neg_c<L>(ao[1])};
  XAcc<L> e = x_acc<L>(0), dr = x_acc<L>(1);
  for (int64_t i = blockIdx.x * (int64_t)kTX + threadIdx.x; i < n; i += (int64_t)G * kTX) {
    const cmp<L> si = load_v<L, CPLX>(s, n, i);
    const cmp<L> ps[2] = {load_v<L, CPLX>(p, n, i), si};
    store_v<L, CPLX>(x, n, i, x_lin<L, CPLX, 2>(e, load_v<L, CPLX>(x, n, i), ao, ps));
    const cmp<L> ti[1] = {load_v<L, CPLX>(t, n, i)};
    const cmp<L> ri = x_lin<L, CPLX, 1>(e, si, nom, ti);
    store_v<L, CPLX>(r, n, i, ri);
    x_dot<L, CPLX>(dr, dr, ri, ri, true);
  }
  x_write_rr<L>(part, G, dr);
}

// ---------------------------------------------------------------------------
// Stand-alone vector operations (mpspmv_dot / mpspmv_axpy)
// ---------------------------------------------------------------------------
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_vaxpy(int64_t n, const double* alpha, const double* u, const double* v,
                                              double* w) {
  cmp<L> a;
#pragma unroll
  for (int l = 0; l < L; l++) {
    a.re.v[l] = alpha[l];
    a.im.v[l] = CPLX ? alpha[L + l] : 0.0;
  }
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT)
    store_v<L, CPLX>(w, n, i, axpy1<L, CPLX>(a, load_v<L, CPLX>(u, n, i), load_v<L, CPLX>(v, n, i)));
}

template <int L, bool CPLX>
__global__ void __launch_bounds__(kTX) kx_vaxpy(int64_t n, const double* alpha, const double* u, const double* v,
                                                double* w) {
  cmp<L> a[1];
#pragma unroll
  for (int l = 0; l < L; l++) {
    a[0].re.v[l] = alpha[l];
    a[0].im.v[l] = CPLX ? alpha[L + l] : 0.0;
  }
  XAcc<L> e = x_acc<L>(0);
  for (int64_t i = blockIdx.x * (int64_t)kTX + threadIdx.x; i < n; i += (int64_t)gridDim.x * kTX) {
    const cmp<L> vi[1] = {load_v<L, CPLX>(v, n, i)};
    store_v<L, CPLX>(w, n, i, x_lin<L, CPLX, 1>(e, load_v<L, CPLX>(u, n, i), a, vi));
  }
}

// out[0..L) = real part, out[L..2L) = imaginary part of the reduced partials
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_dot_finish(const double* part, int G, double* out, bool ex) {
  mp<L> a[2];
  if (ex)
    reduce_partials_x<L, 2, !CPLX>(part, G, a);
  else
    reduce_partials<L, 2, !CPLX>(part, G, a);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int l = 0; l < L; l++) {
      out[l] = a[0].v[l];
      out[L + l] = a[1].v[l];
    }
  }
}

// ---------------------------------------------------------------------------
// Generic vector kernels for BiCG, CGS and GPBiCG: linear combinations
// out = base + sum_k c_k v_k with coefficients read from the state's scalar
// slots (or +-1), optionally with the partial of (out, out), and single
// inner products, conjugated ((u, v) = sum conj(u_i) v_i) or bilinear
// (sum u_i v_i, for BiCG's conjugated shadow vectors).  Paper order: the
// terms are added one at a time in MP arithmetic (Algorithms 1-5).  Exact
// (kx_*): each part of an element is summed exactly and rounded once.
// ---------------------------------------------------------------------------
struct Term {
  const double* v;
  int slot;  // scalar slot of the coefficient; -1: the coefficient is 1
  int neg;   // subtract the term
};
template <int NT>
struct Terms {
  Term t[NT];
};

template <int L, int NT>
__device__ __forceinline__ void comb_coeffs(const KrylovState* st, const Terms<NT>& tm, cmp<L> (&c)[NT]) {
#pragma unroll
  for (int k = 0; k < NT; k++) {
    if (tm.t[k].slot >= 0) {
      c[k] = get_s<L>(st, tm.t[k].slot);
      if (tm.t[k].neg) c[k] = neg_c<L>(c[k]);
    } else {
      c[k].re = mp_zero<L>();
      c[k].im = mp_zero<L>();
    }
  }
}

template <int L, bool CPLX, int NT>
__global__ void __launch_bounds__(kT) k_comb(const KrylovState* st, int64_t n, double* out, const double* base,
                                             Terms<NT> tm, double* part, int G) {
  ACTIVE(st);
  cmp<L> c[NT];
  comb_coeffs<L, NT>(st, tm, c);
  mp<L> acc[2] = {mp_zero<L>(), mp_zero<L>()};
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)G * kT) {
    cmp<L> w;
    if (base) {
      w = load_v<L, CPLX>(base, n, i);
    } else {
      w.re = mp_zero<L>();
      w.im = mp_zero<L>();
    }
    // one copy of the term body (NT copies of a complex QD multiply-add
    // would multiply the kernel's size and compile time)
#pragma unroll 1
    for (int k = 0; k < NT; k++) {
      const cmp<L> v = load_v<L, CPLX>(tm.t[k].v, n, i);
      if (tm.t[k].slot >= 0) {
        w = axpy1<L, CPLX>(c[k], w, v);
      } else if (tm.t[k].neg) {
        w.re = mp_sub<L>(w.re, v.re);
        if (CPLX) w.im = mp_sub<L>(w.im, v.im);
      } else {
        w.re = mp_add<L>(w.re, v.re);
        if (CPLX) w.im = mp_add<L>(w.im, v.im);
      }
    }
    store_v<L, CPLX>(out, n, i, w);
    if (part) dot_acc<L, CPLX>(acc[0], acc[1], w, w);
  }
  if (part) write_partials<L, 2, kT, true>(part, G, acc);  // part is uniform over the grid
}

template <int L, bool CPLX, int NT>
__global__ void __launch_bounds__(kTX) kx_comb(const KrylovState* st, int64_t n, double* out, const double* base,
                                               Terms<NT> tm, double* part, int G) {
  ACTIVE(st);
  cmp<L> c[NT];
  comb_coeffs<L, NT>(st, tm, c);
  XAcc<L> e = x_acc<L>(0), dr = x_acc<L>(1);
  for (int64_t i = blockIdx.x * (int64_t)kTX + threadIdx.x; i < n; i += (int64_t)G * kTX) {
    cmp<L> w;
#pragma unroll
    for (int part_im = 0; part_im < (CPLX ? 2 : 1); part_im++) {
      if (base) {
        const cmp<L> b0 = load_v<L, CPLX>(base, n, i);
        x_add_mp<L>(e, part_im ? b0.im : b0.re, false);
      }
#pragma unroll 1
      for (int k = 0; k < NT; k++) {
        const cmp<L> v = load_v<L, CPLX>(tm.t[k].v, n, i);
        if (tm.t[k].slot < 0) {
          x_add_mp<L>(e, part_im ? v.im : v.re, tm.t[k].neg != 0);
        } else if (!part_im) {  // re: c_re v_re - c_im v_im
          add_prod<XAcc<L>, L>(e, c[k].re, v.re, false);
          if (CPLX) add_prod<XAcc<L>, L>(e, c[k].im, v.im, true);
        } else {  // im: c_re v_im + c_im v_re
          add_prod<XAcc<L>, L>(e, c[k].re, v.im, false);
          add_prod<XAcc<L>, L>(e, c[k].im, v.re, false);
        }
      }
      if (part_im)
        w.im = x_flush<L>(e);
      else
        w.re = x_flush<L>(e);
    }
    if (!CPLX) w.im = mp_zero<L>();
    store_v<L, CPLX>(out, n, i, w);
    if (part) x_dot<L, CPLX>(dr, dr, w, w, true);
  }
  if (part) x_write_rr<L>(part, G, dr);
}

// (dr, di) += conj(u) v (conj) or u v (bilinear)
template <int L, bool CPLX>
__device__ __forceinline__ void dot_acc_b(mp<L>& dr, mp<L>& di, const cmp<L>& u, const cmp<L>& v, bool conj) {
  dr = mp_add<L>(dr, mp_mul<L>(u.re, v.re));
  if (CPLX) {
    const mp<L> t1 = mp_mul<L>(u.im, v.im);
    dr = mp_add<L>(dr, conj ? t1 : mp_neg<L>(t1));
    di = mp_add<L>(di, mp_mul<L>(u.re, v.im));
    const mp<L> t2 = mp_mul<L>(u.im, v.re);
    di = mp_add<L>(di, conj ? mp_neg<L>(t2) : t2);
  }
}

template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_dotg(const KrylovState* st, int64_t n, const double* u, const double* v,
                                             bool conj, double* part, int G, bool ignore_state) {
  if (!ignore_state) {
    ACTIVE(st);
  }
  mp<L> acc[2] = {mp_zero<L>(), mp_zero<L>()};
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)G * kT)
    dot_acc_b<L, CPLX>(acc[0], acc[1], load_v<L, CPLX>(u, n, i), load_v<L, CPLX>(v, n, i), conj);
  write_partials<L, 2, kT, !CPLX>(part, G, acc);
}

template <int L, bool CPLX>
__global__ void __launch_bounds__(kTX) kx_dotg(const KrylovState* st, int64_t n, const double* u, const double* v,
                                               bool conj, double* part, int G, bool ignore_state) {
  if (!ignore_state) {
    ACTIVE(st);
  }
  const bool self = conj && u == v;  // the imaginary part is exactly zero
  XAcc<L> dr = x_acc<L>(0);
  XAcc<L> di;
  if (CPLX) di = x_acc<L>(1);
  for (int64_t i = blockIdx.x * (int64_t)kTX + threadIdx.x; i < n; i += (int64_t)G * kTX) {
    const cmp<L> a = load_v<L, CPLX>(u, n, i), b = load_v<L, CPLX>(v, n, i);
    add_prod<XAcc<L>, L>(dr, a.re, b.re, false);
    if (CPLX) {
      add_prod<XAcc<L>, L>(dr, a.im, b.im, !conj);
      if (!self) {
        add_prod<XAcc<L>, L>(di, a.re, b.im, false);
        add_prod<XAcc<L>, L>(di, a.im, b.re, conj);
      }
    }
  }
  mp<L> acc[2] = {x_flush<L>(dr), mp_zero<L>()};
  if (CPLX && !self) acc[1] = x_flush<L>(di);
  write_partials_x<L, 2, kTX, !CPLX>(part, G, acc);
}

// dst1 = dst2 = conj(src) (exact: a copy with the imaginary planes negated)
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_conj_copy(int64_t n, const double* src, double* dst1, double* dst2) {
  for (int64_t i = blockIdx.x * (int64_t)kT + threadIdx.x; i < n; i += (int64_t)gridDim.x * kT) {
    cmp<L> a = load_v<L, CPLX>(src, n, i);
    a.im = mp_neg<L>(a.im);
    store_v<L, CPLX>(dst1, n, i, a);
    store_v<L, CPLX>(dst2, n, i, a);
  }
}

// ---------------------------------------------------------------------------
// Finishing kernels shared by BiCG and CGS (and GPBiCG's start and alpha).
// ---------------------------------------------------------------------------
enum PtSlot : int { P_RHO = 0, P_ALPHA = 1, P_BETA = 2, P_ZETA = 3, P_ETA = 4, P_ETA_BETA = 5 };

template <int L, bool CPLX>
__device__ __forceinline__ bool c_is_zero(const cmp<L>& a) {
  return is_zero<L>(a.re) && (!CPLX || is_zero<L>(a.im));
}

template <int L, bool CPLX>
__device__ __forceinline__ cmp<L> c_div_any(const cmp<L>& a, const cmp<L>& b) {
  if (CPLX) return c_div<L>(a, b);
  cmp<L> r;
  r.re = mp_div<L>(a.re, b.re);
  r.im = mp_zero<L>();
  return r;
}

template <int L, bool CPLX>
__device__ __forceinline__ cmp<L> c_mul_any(const cmp<L>& a, const cmp<L>& b) {
  if (CPLX) return c_mul<L>(a, b);
  cmp<L> r;
  r.re = mp_mul<L>(a.re, b.re);
  r.im = mp_zero<L>();
  return r;
}

template <int L>
__device__ __forceinline__ cmp<L> c_of(const mp<L> (&a)[2]) {
  cmp<L> r;
  r.re = a[0];
  r.im = a[1];
  return r;
}

// start: (r, r), (b, b), rho = (r~, r); beta = 0; stopping test on r_0
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_pt_start(KrylovState* st, const double* part_rr, const double* part_bb,
                                                 const double* part_rho, int G, double rtol, double atol) {
  mp<L> a[2], b[2], c[2];
  reduce_any<L, 2, true>(st, part_rr, G, a);
  __syncthreads();
  reduce_any<L, 2, true>(st, part_bb, G, b);
  __syncthreads();
  reduce_any<L, 2, !CPLX>(st, part_rho, G, c);
  if (threadIdx.x == 0) {
    const double bb = to_d<L>(b[0]);
    const double bnorm = sqrt(bb > 0.0 ? bb : 0.0);
    const double tol = rtol * bnorm + atol;
    st->bnorm = bnorm;
    st->tol = tol;
    cmp<L> rho = c_of<L>(c), zero;
    if (!CPLX) rho.im = mp_zero<L>();
    zero.re = mp_zero<L>();
    zero.im = mp_zero<L>();
    put_s<L>(st, P_RHO, rho);
    put_s<L>(st, P_BETA, zero);
    const double rr = to_d<L>(a[0]);
    st->iter = 0;
    st->status = (sqrt(rr > 0.0 ? rr : 0.0) <= tol) ? CONVERGED : RUNNING;
    if (st->status == RUNNING && st->maxit <= 0) st->status = MPSPMV_ENOCONV;
  }
}

// alpha = rho / sigma (sigma from the partials); breakdown on a zero rho or sigma
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_pt_alpha(KrylovState* st, const double* part, int G) {
  ACTIVE(st);
  mp<L> a[2];
  reduce_any<L, 2, !CPLX>(st, part, G, a);
  if (threadIdx.x == 0) {
    cmp<L> sigma = c_of<L>(a);
    if (!CPLX) sigma.im = mp_zero<L>();
    const cmp<L> rho = get_s<L>(st, P_RHO);
    if (c_is_zero<L, CPLX>(rho) || c_is_zero<L, CPLX>(sigma) || !isfinite(sigma.re.v[0])) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    put_s<L>(st, P_ALPHA, c_div_any<L, CPLX>(rho, sigma));
  }
}

// shared stopping test on the (r, r) partials; returns false when the
// iteration ends here (thread 0 only)
template <int L>
__device__ __forceinline__ bool pt_test(KrylovState* st, const mp<L>& rr) {
  const double t = to_d<L>(rr);
  if (!isfinite(t)) {
    st->status = MPSPMV_EBREAKDOWN;
    return false;
  }
  if (sqrt(t > 0.0 ? t : 0.0) <= st->tol) {
    st->status = CONVERGED;
    return false;
  }
  return true;
}

// k++; test; rho' from the partials; beta = rho' / rho; rho = rho'
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_pt_beta(KrylovState* st, const double* part_rr, const double* part_rho,
                                                int G) {
  ACTIVE(st);
  mp<L> a[2], c[2];
  reduce_any<L, 2, true>(st, part_rr, G, a);
  __syncthreads();
  reduce_any<L, 2, !CPLX>(st, part_rho, G, c);
  if (threadIdx.x == 0) {
    st->iter++;
    if (!pt_test<L>(st, a[0])) return;
    cmp<L> rho1 = c_of<L>(c);
    if (!CPLX) rho1.im = mp_zero<L>();
    put_s<L>(st, P_BETA, c_div_any<L, CPLX>(rho1, get_s<L>(st, P_RHO)));
    put_s<L>(st, P_RHO, rho1);
    if (st->iter >= st->maxit) st->status = MPSPMV_ENOCONV;
  }
}

// GPBiCG: ||t|| meets the test -> finish with x += alpha p (PENDING_X)
template <int L>
__global__ void __launch_bounds__(kT) k_gp_tcheck(KrylovState* st, const double* part_tt, int G) {
  ACTIVE(st);
  mp<L> a[2];
  reduce_any<L, 2, true>(st, part_tt, G, a);
  if (threadIdx.x == 0) {
    const double t = to_d<L>(a[0]);
    if (!isfinite(t)) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    if (sqrt(t > 0.0 ? t : 0.0) <= st->tol) {
      st->iter++;
      st->status = PENDING_X;
    }
  }
}

// GPBiCG: zeta, eta from a = (At, At), b = (y, y), c = (At, y), d = (At, t),
// e = (y, t) (first iteration: zeta = d / a, eta = 0); also eta * beta
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_gp_zeta(KrylovState* st, const double* pa, const double* pb,
                                                const double* pc, const double* pd, const double* pe, int G) {
  ACTIVE(st);
  mp<L> a[2], b[2], c[2], d[2], e[2];
  reduce_any<L, 2, !CPLX>(st, pa, G, a);
  __syncthreads();
  reduce_any<L, 2, !CPLX>(st, pd, G, d);
  __syncthreads();
  const bool first = st->iter == 0;
  if (!first) {
    reduce_any<L, 2, !CPLX>(st, pb, G, b);
    __syncthreads();
    reduce_any<L, 2, !CPLX>(st, pc, G, c);
    __syncthreads();
    reduce_any<L, 2, !CPLX>(st, pe, G, e);
  }
  if (threadIdx.x == 0) {
    cmp<L> A = c_of<L>(a), D = c_of<L>(d), zeta, eta;
    if (!CPLX) {
      A.im = mp_zero<L>();
      D.im = mp_zero<L>();
    }
    if (first) {
      if (c_is_zero<L, CPLX>(A)) {
        st->status = MPSPMV_EBREAKDOWN;
        return;
      }
      zeta = c_div_any<L, CPLX>(D, A);
      eta.re = mp_zero<L>();
      eta.im = mp_zero<L>();
    } else {
      cmp<L> B = c_of<L>(b), C = c_of<L>(c), E = c_of<L>(e);
      if (!CPLX) {
        B.im = mp_zero<L>();
        C.im = mp_zero<L>();
        E.im = mp_zero<L>();
      }
      cmp<L> Cc;
      Cc.re = C.re;
      Cc.im = mp_neg<L>(C.im);
      const cmp<L> ab = c_mul_any<L, CPLX>(A, B), c2 = c_mul_any<L, CPLX>(C, Cc);
      cmp<L> det;
      det.re = mp_sub<L>(ab.re, c2.re);
      det.im = mp_sub<L>(ab.im, c2.im);
      if (c_is_zero<L, CPLX>(det)) {
        st->status = MPSPMV_EBREAKDOWN;
        return;
      }
      const cmp<L> bd = c_mul_any<L, CPLX>(B, D), ce = c_mul_any<L, CPLX>(C, E);
      const cmp<L> ae = c_mul_any<L, CPLX>(A, E), cd = c_mul_any<L, CPLX>(Cc, D);
      cmp<L> zn, en;
      zn.re = mp_sub<L>(bd.re, ce.re);
      zn.im = mp_sub<L>(bd.im, ce.im);
      en.re = mp_sub<L>(ae.re, cd.re);
      en.im = mp_sub<L>(ae.im, cd.im);
      zeta = c_div_any<L, CPLX>(zn, det);
      eta = c_div_any<L, CPLX>(en, det);
    }
    if (c_is_zero<L, CPLX>(zeta)) {
      st->status = MPSPMV_EBREAKDOWN;
      return;
    }
    put_s<L>(st, P_ZETA, zeta);
    put_s<L>(st, P_ETA, eta);
    put_s<L>(st, P_ETA_BETA, c_mul_any<L, CPLX>(eta, get_s<L>(st, P_BETA)));
  }
}

// GPBiCG: k++; test; beta = (alpha / zeta) (rho' / rho); rho = rho'
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_gp_beta(KrylovState* st, const double* part_rr, const double* part_rho,
                                                int G) {
  ACTIVE(st);
  mp<L> a[2], c[2];
  reduce_any<L, 2, true>(st, part_rr, G, a);
  __syncthreads();
  reduce_any<L, 2, !CPLX>(st, part_rho, G, c);
  if (threadIdx.x == 0) {
    st->iter++;
    if (!pt_test<L>(st, a[0])) return;
    cmp<L> rho1 = c_of<L>(c);
    if (!CPLX) rho1.im = mp_zero<L>();
    const cmp<L> az = c_div_any<L, CPLX>(get_s<L>(st, P_ALPHA), get_s<L>(st, P_ZETA));
    const cmp<L> rr = c_div_any<L, CPLX>(rho1, get_s<L>(st, P_RHO));
    put_s<L>(st, P_BETA, c_mul_any<L, CPLX>(az, rr));
    put_s<L>(st, P_RHO, rho1);
    if (st->iter >= st->maxit) st->status = MPSPMV_ENOCONV;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
inline int grid_for(int64_t n) {
  int64_t g = (n + kT - 1) / kT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, kMaxBlocks));
}

// Grid of the exact kernels: at most as many blocks as are resident on the
// device at once (so that a grid-stride loop gives every block the same
// share), at most kMaxPart.  The dot kernel holding three accumulators per
// thread needs more than the default 48 KB of dynamic shared memory.
template <int L, bool CPLX>
int x_grid(int64_t n, int* G) {
  static int cap = 0;
  if (!cap) {
    int dev = 0, sms = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kx_bi_xr<L, CPLX>, kTX, x_smem<L>(2)) != cudaSuccess ||
        cudaFuncSetAttribute(kx_dot<L, CPLX, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)x_smem<L>(CPLX ? 3 : 2)) != cudaSuccess) {
      cudaGetLastError();
      return MPSPMV_ECUDA;
    }
    cap = std::max(1, std::min(kMaxPart, sms * std::max(nb, 1)));
  }
  const int64_t g = (n + kTX - 1) / kTX;
  *G = (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
  return MPSPMV_OK;
}

// Launch helpers choosing the paper-order (k_*) or exact (kx_*) kernel.
template <int L, bool CPLX>
void launch_residual(bool ex, int G, cudaStream_t s, int64_t n, const double* b, const double* q, double* r,
                     double* p, double* rh, double* part) {
  if (ex)
    kx_residual<L, CPLX><<<G, kTX, x_smem<L>(2), s>>>(n, b, q, r, p, rh, part, G);
  else
    k_residual<L, CPLX><<<G, kT, 0, s>>>(n, b, q, r, p, rh, part, G);
}

// one inner product (u, v)
template <int L, bool CPLX>
void launch_dot1(bool ex, int G, cudaStream_t s, const KrylovState* st, int64_t n, const double* u, const double* v,
                 double* part, bool ignore_state) {
  if (ex)
    kx_dot<L, CPLX, 1><<<G, kTX, x_smem<L>(CPLX ? 2 : 1), s>>>(st, n, u, v, nullptr, part, G, ignore_state);
  else
    k_dot<L, CPLX, 1><<<G, kT, 0, s>>>(st, n, u, v, nullptr, nullptr, part, G, ignore_state);
}

constexpr int kNumVec = 12;  // workspace vectors (GPBiCG uses 11, the true residual v[6], v[7])
constexpr int kNumPart = 8;  // reduction partial buffers

struct Work {
  double* v[kNumVec];
  double* part[kNumPart];
  KrylovState* st;
  int* counter;
};

inline int ensure_ws(mpspmv_mat* h, Work& w) {
  const int64_t vec = (int64_t)h->P * std::max(h->nrows, h->ncols);
  const int64_t part = 4 * 4 * (int64_t)kMaxPart;
  const int64_t need = kNumVec * vec + kNumPart * part;
  if (!h->d_kws || h->kws_len < need) {
    if (h->d_kws) {
      cudaFree(h->d_kws);
      h->device_bytes -= (int64_t)sizeof(double) * h->kws_len;
      h->d_kws = nullptr;
    }
    if (cudaMalloc(&h->d_kws, sizeof(double) * need) != cudaSuccess) {
      cudaGetLastError();
      return MPSPMV_ENOMEM;
    }
    h->kws_len = need;
    h->device_bytes += (int64_t)sizeof(double) * need;
  }
  if (!h->d_kstate) {
    if (cudaMalloc(&h->d_kstate, sizeof(KrylovState) + 64) != cudaSuccess) {
      cudaGetLastError();
      return MPSPMV_ENOMEM;
    }
    cudaMemset(h->d_kstate, 0, sizeof(KrylovState) + 64);
  }
  for (int i = 0; i < kNumVec; i++) w.v[i] = h->d_kws + i * vec;
  for (int i = 0; i < kNumPart; i++) w.part[i] = h->d_kws + kNumVec * vec + i * part;
  w.st = h->d_kstate;
  w.counter = reinterpret_cast<int*>(reinterpret_cast<char*>(h->d_kstate) + sizeof(KrylovState));
  return MPSPMV_OK;
}

// Run `body` (which enqueues kItersPerGraph iterations) as a captured graph
// until the device state leaves RUNNING.
template <typename F>
int iterate(cudaStream_t s, KrylovState* d_st, F&& body, KrylovState* host_st) {
  cudaStream_t cs;
  MPS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  int st = MPSPMV_OK;
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  // order the capture stream after the caller's stream
  cudaEventRecord(ev, s);
  cudaStreamWaitEvent(cs, ev, 0);
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = MPSPMV_ECUDA;
  if (st == MPSPMV_OK) {
    for (int k = 0; k < kItersPerGraph && st == MPSPMV_OK; k++) st = body(cs);
    cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (st == MPSPMV_OK && e != cudaSuccess) st = MPSPMV_ECUDA;
  }
  if (st == MPSPMV_OK && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) st = MPSPMV_ECUDA;
  while (st == MPSPMV_OK) {
    if (cudaGraphLaunch(ge, cs) != cudaSuccess ||
        cudaMemcpyAsync(host_st, d_st, sizeof(KrylovState), cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess) {
      st = MPSPMV_ECUDA;
      break;
    }
    if (host_st->status != RUNNING) break;
  }
  // later work on the caller's stream follows the solve
  cudaEventRecord(ev, cs);
  cudaStreamWaitEvent(s, ev, 0);
  if (ge) cudaGraphExecDestroy(ge);
  if (g) cudaGraphDestroy(g);
  cudaStreamSynchronize(cs);
  cudaStreamDestroy(cs);
  cudaEventDestroy(ev);
  return st;
}

template <int L, bool CPLX>
int vec_grid(const mpspmv_mat* h, int64_t n, int* G) {
  if (h->exact) return x_grid<L, CPLX>(n, G);
  *G = grid_for(n);
  return MPSPMV_OK;
}

template <int L, bool CPLX>
int true_residual(mpspmv_mat* h, Work& w, const double* b, const double* x, cudaStream_t s) {
  const int64_t n = h->nrows;
  int G;
  int st = vec_grid<L, CPLX>(h, n, &G);
  if (st) return st;
  if ((st = mps_launch_spmv(h, x, w.v[7], s))) return st;
  launch_residual<L, CPLX>(h->exact, G, s, n, b, w.v[7], w.v[6], nullptr, nullptr, w.part[0]);
  k_relres<L><<<1, kT, 0, s>>>(w.st, w.part[0], G);
  MPS_CUDA(cudaGetLastError());
  return MPSPMV_OK;
}

template <int L>
int cg_impl(mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
            double* relres, cudaStream_t s, double* hist = nullptr) {
  Work w;
  int st = ensure_ws(h, w);
  if (st) return st;
  const int64_t n = h->nrows;
  const bool ex = h->exact;
  int G;
  if ((st = vec_grid<L, false>(h, n, &G))) return st;
  double *r = w.v[0], *p = w.v[1], *q = w.v[2];
  KrylovState init{};
  init.maxit = maxit;
  init.exact = h->exact ? 1 : 0;
  MPS_CUDA(cudaMemcpyAsync(w.st, &init, sizeof(KrylovState), cudaMemcpyHostToDevice, s));
  // r = b - A x; p = r; rho = (r, r); (b, b)
  if ((st = mps_launch_spmv(h, x, q, s))) return st;
  launch_residual<L, false>(ex, G, s, n, b, q, r, p, nullptr, w.part[0]);
  launch_dot1<L, false>(ex, G, s, w.st, n, b, b, w.part[1], true);
  k_cg_start<L><<<1, kT, 0, s>>>(w.st, w.part[0], w.part[1], G, rtol, atol);
  MPS_CUDA(cudaGetLastError());
  KrylovState hs{};
  auto body = [&](cudaStream_t cs) -> int {
    int e = mps_launch_spmv_if_running(h, p, q, &w.st->status, cs);
    if (e) return e;
    launch_dot1<L, false>(ex, G, cs, w.st, n, p, q, w.part[0], false);
    k_cg_alpha<L><<<1, kT, 0, cs>>>(w.st, w.part[0], G);
    if (ex)
      kx_cg_xr<L><<<G, kTX, x_smem<L>(2), cs>>>(w.st, n, x, r, p, q, w.part[1], G);
    else
      k_cg_xr<L><<<G, kT, 0, cs>>>(w.st, n, x, r, p, q, w.part[1], G);
    k_cg_beta<L><<<1, kT, 0, cs>>>(w.st, w.part[1], G);
    if (ex)
      kx_cg_p<L><<<G, kTX, x_smem<L>(1), cs>>>(w.st, n, r, p, G);
    else
      k_cg_p<L><<<G, kT, 0, cs>>>(w.st, n, r, p, G);
    return cudaGetLastError() == cudaSuccess ? MPSPMV_OK : MPSPMV_ECUDA;
  };
  MPS_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
  MPS_CUDA(cudaStreamSynchronize(s));
  if (hs.status == RUNNING) {
    st = iterate(s, w.st, body, &hs);
    if (st) return st;
  }
  if ((st = true_residual<L, false>(h, w, b, x, s))) return st;
  MPS_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
  MPS_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = hs.iter;
  if (relres) *relres = hs.relres;
  if (hist)
    for (int k = 0; k < 16; k++) hist[k] = k < hs.iter ? hs.hist[k] : 0.0;
  return hs.status == CONVERGED ? MPSPMV_OK : hs.status;
}

template <int L, bool CPLX>
int bicgstab_impl(mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                  double* relres, cudaStream_t s) {
  Work w;
  int st = ensure_ws(h, w);
  if (st) return st;
  const int64_t n = h->nrows;
  const bool ex = h->exact;
  int G;
  if ((st = vec_grid<L, CPLX>(h, n, &G))) return st;
  double *r = w.v[0], *rh = w.v[1], *p = w.v[2], *v = w.v[3], *sv = w.v[4], *t = w.v[5];
  KrylovState init{};
  init.maxit = maxit;
  init.exact = h->exact ? 1 : 0;
  MPS_CUDA(cudaMemcpyAsync(w.st, &init, sizeof(KrylovState), cudaMemcpyHostToDevice, s));
  MPS_CUDA(cudaMemsetAsync(p, 0, sizeof(double) * h->P * n, s));
  MPS_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * h->P * n, s));
  MPS_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(int), s));
  if ((st = mps_launch_spmv(h, x, t, s))) return st;
  launch_residual<L, CPLX>(ex, G, s, n, b, t, r, nullptr, rh, w.part[0]);
  launch_dot1<L, CPLX>(ex, G, s, w.st, n, b, b, w.part[1], true);
  k_bi_start<L, CPLX><<<1, kT, 0, s>>>(w.st, w.part[0], w.part[1], G, rtol, atol);
  MPS_CUDA(cudaGetLastError());
  KrylovState hs{};
  auto body = [&](cudaStream_t cs) -> int {
    launch_dot1<L, CPLX>(ex, G, cs, w.st, n, rh, r, w.part[0], false);
    k_bi_beta<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[0], G);
    if (ex)
      kx_bi_p<L, CPLX><<<G, kTX, x_smem<L>(1), cs>>>(w.st, n, r, p, v, G);
    else
      k_bi_p<L, CPLX><<<G, kT, 0, cs>>>(w.st, n, r, p, v, G);
    int e = mps_launch_spmv_if_running(h, p, v, &w.st->status, cs);
    if (e) return e;
    launch_dot1<L, CPLX>(ex, G, cs, w.st, n, rh, v, w.part[0], false);
    k_bi_alpha<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[0], G);
    if (ex)
      kx_bi_s<L, CPLX><<<G, kTX, x_smem<L>(2), cs>>>(w.st, n, r, v, sv, w.part[1], G);
    else
      k_bi_s<L, CPLX><<<G, kT, 0, cs>>>(w.st, n, r, v, sv, w.part[1], G);
    k_bi_scheck<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[1], G);
    if (ex)
      kx_bi_xfix<L, CPLX><<<G, kTX, x_smem<L>(1), cs>>>(w.st, n, x, p, G, w.counter);
    else
      k_bi_xfix<L, CPLX><<<G, kT, 0, cs>>>(w.st, n, x, p, G, w.counter);
    if ((e = mps_launch_spmv_if_running(h, sv, t, &w.st->status, cs))) return e;
    if (ex)
      kx_dot<L, CPLX, 2><<<G, kTX, x_smem<L>(CPLX ? 3 : 2), cs>>>(w.st, n, t, sv, t, w.part[2], G, false);
    else
      k_dot<L, CPLX, 2><<<G, kT, 0, cs>>>(w.st, n, t, sv, t, t, w.part[2], G, false);
    k_bi_omega<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[2], G);
    if (ex)
      kx_bi_xr<L, CPLX><<<G, kTX, x_smem<L>(2), cs>>>(w.st, n, x, r, p, sv, t, w.part[1], G);
    else
      k_bi_xr<L, CPLX><<<G, kT, 0, cs>>>(w.st, n, x, r, p, sv, t, w.part[1], G);
    k_bi_rcheck<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[1], G);
    return cudaGetLastError() == cudaSuccess ? MPSPMV_OK : MPSPMV_ECUDA;
  };
  MPS_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
  MPS_CUDA(cudaStreamSynchronize(s));
  if (hs.status == RUNNING) {
    st = iterate(s, w.st, body, &hs);
    if (st) return st;
  }
  if ((st = true_residual<L, CPLX>(h, w, b, x, s))) return st;
  MPS_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
  MPS_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = hs.iter;
  if (relres) *relres = hs.relres;
  return hs.status == CONVERGED ? MPSPMV_OK : hs.status;
}


template <int L, bool CPLX>
int dot_impl(mpspmv_mat* h, int64_t n, const double* u, const double* v, double* out, cudaStream_t s) {
  Work w;
  int st = ensure_ws(h, w);
  if (st) return st;
  int G;
  if ((st = vec_grid<L, CPLX>(h, n, &G))) return st;
  launch_dot1<L, CPLX>(h->exact, G, s, w.st, n, u, v, w.part[0], true);
  k_dot_finish<L, CPLX><<<1, kT, 0, s>>>(w.part[0], G, w.part[1], h->exact);
  MPS_CUDA(cudaGetLastError());
  double r[8];
  MPS_CUDA(cudaMemcpyAsync(r, w.part[1], sizeof(double) * 2 * L, cudaMemcpyDeviceToHost, s));
  MPS_CUDA(cudaStreamSynchronize(s));
  for (int l = 0; l < L; l++) {
    out[l] = r[l];
    out[L + l] = CPLX ? r[L + l] : 0.0;
  }
  return MPSPMV_OK;
}

template <int L, bool CPLX>
int axpy_impl(mpspmv_mat* h, int64_t n, const double* alpha, const double* u, const double* v, double* w,
              cudaStream_t s) {
  if (n == 0) return MPSPMV_OK;
  // alpha travels in a device buffer of the handle's workspace
  Work ws;
  int st = ensure_ws(h, ws);
  if (st) return st;
  double a[8];
  for (int l = 0; l < L; l++) {
    a[l] = alpha[l];
    a[L + l] = CPLX ? alpha[L + l] : 0.0;
  }
  double* da = ws.part[2];
  MPS_CUDA(cudaMemcpyAsync(da, a, sizeof(double) * 2 * L, cudaMemcpyHostToDevice, s));
  int G;
  if ((st = vec_grid<L, CPLX>(h, n, &G))) return st;
  if (h->exact)
    kx_vaxpy<L, CPLX><<<G, kTX, x_smem<L>(1), s>>>(n, da, u, v, w);
  else
    k_vaxpy<L, CPLX><<<G, kT, 0, s>>>(n, da, u, v, w);
  MPS_CUDA(cudaGetLastError());
  // the host copy of alpha must stay valid until the copy has run
  MPS_CUDA(cudaStreamSynchronize(s));
  return MPSPMV_OK;
}


// ---------------------------------------------------------------------------
// MP scalars of a distributed solve: the inner-product partials of several
// row blocks summed in block order, and the quotients of the solver's
// scalars (one thread each; the work is a handful of MP operations).
// ---------------------------------------------------------------------------
constexpr int kMaxScalarParts = 4096;

// out = parts[0] + parts[1] + ... + parts[count-1], real and imaginary parts
// separately.  Paper order: MP additions from left to right.  Exact
// (MPSPMV_EXACT_ACC): every component in register digits at the base of the
// largest one, cut to L components once (independent of the order).
template <int L, bool CPLX>
__global__ void k_scalar_sum(const double* __restrict__ parts, int count, double* __restrict__ out, bool ex) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
#pragma unroll 1
  for (int c = 0; c < (CPLX ? 2 : 1); c++) {
    mp<L> r;
    if (ex) {
      constexpr int D = AccDigits<L>::D;
      int t = INT_MIN;
      for (int i = 0; i < count; i++)
#pragma unroll
        for (int l = 0; l < L; l++) t = max(t, top_exp(parts[(int64_t)i * 2 * L + c * L + l]));
      FixAcc<D> f;
      fa_at_top<D>(f, t);
      for (int i = 0; i < count; i++)
#pragma unroll
        for (int l = 0; l < L; l++) fa_add<D>(f, parts[(int64_t)i * 2 * L + c * L + l]);
      fa_to_mp<L, D>(f, r.v);
    } else {
#pragma unroll
      for (int l = 0; l < L; l++) r.v[l] = parts[c * L + l];
      for (int i = 1; i < count; i++) {
        mp<L> a;
#pragma unroll
        for (int l = 0; l < L; l++) a.v[l] = parts[(int64_t)i * 2 * L + c * L + l];
        r = mp_add<L>(r, a);
      }
    }
#pragma unroll
    for (int l = 0; l < L; l++) out[c * L + l] = r.v[l];
  }
  if (!CPLX)
#pragma unroll
    for (int l = 0; l < L; l++) out[L + l] = 0.0;
}

// out = a / b (ab = a, then b, each 2L components)
template <int L, bool CPLX>
__global__ void k_scalar_div(const double* __restrict__ ab, double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  cmp<L> a, b;
#pragma unroll
  for (int l = 0; l < L; l++) {
    a.re.v[l] = ab[l];
    a.im.v[l] = ab[L + l];
    b.re.v[l] = ab[2 * L + l];
    b.im.v[l] = ab[3 * L + l];
  }
  const cmp<L> q = c_div_any<L, CPLX>(a, b);
#pragma unroll
  for (int l = 0; l < L; l++) {
    out[l] = q.re.v[l];
    out[L + l] = CPLX ? q.im.v[l] : 0.0;
  }
}

template <int L, bool CPLX>
int scalar_sum_impl(mpspmv_mat* h, int count, const double* parts, double* out, cudaStream_t s) {
  Work w;
  int st = ensure_ws(h, w);
  if (st) return st;
  double* din = w.part[3];
  double* dout = w.part[4];
  MPS_CUDA(cudaMemcpyAsync(din, parts, sizeof(double) * 2 * L * count, cudaMemcpyHostToDevice, s));
  k_scalar_sum<L, CPLX><<<1, 32, 0, s>>>(din, count, dout, h->exact);
  MPS_CUDA(cudaGetLastError());
  MPS_CUDA(cudaMemcpyAsync(out, dout, sizeof(double) * 2 * L, cudaMemcpyDeviceToHost, s));
  MPS_CUDA(cudaStreamSynchronize(s));
  return MPSPMV_OK;
}

template <int L, bool CPLX>
int scalar_div_impl(mpspmv_mat* h, const double* a, const double* b, double* out, cudaStream_t s) {
  bool zero = true;
  for (int l = 0; l < L; l++) zero = zero && b[l] == 0.0 && (!CPLX || b[L + l] == 0.0);
  if (zero) return MPSPMV_EBREAKDOWN;
  Work w;
  int st = ensure_ws(h, w);
  if (st) return st;
  double ab[16];
  for (int l = 0; l < L; l++) {
    ab[l] = a[l];
    ab[L + l] = CPLX ? a[L + l] : 0.0;
    ab[2 * L + l] = b[l];
    ab[3 * L + l] = CPLX ? b[L + l] : 0.0;
  }
  double* din = w.part[3];
  double* dout = w.part[4];
  MPS_CUDA(cudaMemcpyAsync(din, ab, sizeof(double) * 4 * L, cudaMemcpyHostToDevice, s));
  k_scalar_div<L, CPLX><<<1, 32, 0, s>>>(din, dout);
  MPS_CUDA(cudaGetLastError());
  MPS_CUDA(cudaMemcpyAsync(out, dout, sizeof(double) * 2 * L, cudaMemcpyDeviceToHost, s));
  // ab is host stack memory: the copy must have run before returning
  MPS_CUDA(cudaStreamSynchronize(s));
  return MPSPMV_OK;
}

// ---------------------------------------------------------------------------
// BiCG, CGS, GPBiCG (host side).  Same structure as bicgstab_impl: a setup on
// the caller's stream, then graph-captured iterations gated by the state.
// ---------------------------------------------------------------------------
inline Term term(const double* v, int slot, bool neg = false) {
  Term t;
  t.v = v;
  t.slot = slot;
  t.neg = neg ? 1 : 0;
  return t;
}

template <int L, bool CPLX, int NT>
void launch_comb(bool ex, int G, cudaStream_t s, const KrylovState* st, int64_t n, double* out, const double* base,
                 const Terms<NT>& tm, double* part) {
  if (ex)
    kx_comb<L, CPLX, NT><<<G, kTX, x_smem<L>(2), s>>>(st, n, out, base, tm, part, G);
  else
    k_comb<L, CPLX, NT><<<G, kT, 0, s>>>(st, n, out, base, tm, part, G);
}

template <int L, bool CPLX>
void launch_dotg(bool ex, int G, cudaStream_t s, const KrylovState* st, int64_t n, const double* u, const double* v,
                 bool conj, double* part, bool ignore_state = false) {
  if (ex)
    kx_dotg<L, CPLX><<<G, kTX, x_smem<L>(CPLX ? 2 : 1), s>>>(st, n, u, v, conj, part, G, ignore_state);
  else
    k_dotg<L, CPLX><<<G, kT, 0, s>>>(st, n, u, v, conj, part, G, ignore_state);
}

// common start: r = b - A x (also into p and rh when given), (r, r), (b, b);
// the caller adds rho and launches k_pt_start
template <int L, bool CPLX>
int pt_setup(mpspmv_mat* h, Work& w, const double* b, const double* x, double* r, double* p, double* rh, int maxit,
             int G, cudaStream_t s) {
  const int64_t n = h->nrows;
  KrylovState init{};
  init.maxit = maxit;
  init.exact = h->exact ? 1 : 0;
  MPS_CUDA(cudaMemcpyAsync(w.st, &init, sizeof(KrylovState), cudaMemcpyHostToDevice, s));
  MPS_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(int), s));
  int st = mps_launch_spmv(h, x, w.v[7], s);
  if (st) return st;
  launch_residual<L, CPLX>(h->exact, G, s, n, b, w.v[7], r, p, rh, w.part[0]);
  launch_dotg<L, CPLX>(h->exact, G, s, w.st, n, b, b, true, w.part[1], true);
  MPS_CUDA(cudaGetLastError());
  return MPSPMV_OK;
}

// iterate and report, as the other solvers
template <int L, bool CPLX, class F>
int pt_run(mpspmv_mat* h, Work& w, const double* b, double* x, int* iters, double* relres, cudaStream_t s,
           F&& body) {
  KrylovState hs{};
  MPS_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
  MPS_CUDA(cudaStreamSynchronize(s));
  if (hs.status == RUNNING) {
    int st = iterate(s, w.st, body, &hs);
    if (st) return st;
  }
  int st = true_residual<L, CPLX>(h, w, b, x, s);
  if (st) return st;
  MPS_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
  MPS_CUDA(cudaStreamSynchronize(s));
  if (iters) *iters = hs.iter;
  if (relres) *relres = hs.relres;
  return hs.status == CONVERGED ? MPSPMV_OK : hs.status;
}

// BiCG with conjugated shadow vectors rt = conj(r~), pt = conj(p~): then
// A^H p~ = conj(A^T pt), the shadow updates keep alpha and beta unconjugated
// and (p~, q), (r~, r) become the bilinear sums of pt q and rt r.
template <int L, bool CPLX>
int bicg_impl(mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
              double* relres, cudaStream_t s) {
  if (!h->tr) return MPSPMV_ENOTSUP;
  Work w;
  int st = ensure_ws(h, w);
  if (st) return st;
  const int64_t n = h->nrows;
  const bool ex = h->exact;
  int G;
  if ((st = vec_grid<L, CPLX>(h, n, &G))) return st;
  double *r = w.v[0], *rt = w.v[1], *p = w.v[2], *pt = w.v[3], *q = w.v[4], *qt = w.v[5];
  if ((st = pt_setup<L, CPLX>(h, w, b, x, r, p, nullptr, maxit, G, s))) return st;
  k_conj_copy<L, CPLX><<<G, kT, 0, s>>>(n, r, rt, pt);
  launch_dotg<L, CPLX>(ex, G, s, w.st, n, rt, r, false, w.part[2], true);
  k_pt_start<L, CPLX><<<1, kT, 0, s>>>(w.st, w.part[0], w.part[1], w.part[2], G, rtol, atol);
  MPS_CUDA(cudaGetLastError());
  auto body = [&](cudaStream_t cs) -> int {
    int e = mps_launch_spmv_if_running(h, p, q, &w.st->status, cs);
    if (!e) e = mps_launch_spmv_if_running(h->tr, pt, qt, &w.st->status, cs);
    if (e) return e;
    launch_dotg<L, CPLX>(ex, G, cs, w.st, n, pt, q, false, w.part[0]);
    k_pt_alpha<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[0], G);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, x, x, Terms<1>{{term(p, P_ALPHA)}}, nullptr);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, r, r, Terms<1>{{term(q, P_ALPHA, true)}}, w.part[1]);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, rt, rt, Terms<1>{{term(qt, P_ALPHA, true)}}, nullptr);
    launch_dotg<L, CPLX>(ex, G, cs, w.st, n, rt, r, false, w.part[2]);
    k_pt_beta<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[1], w.part[2], G);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, p, r, Terms<1>{{term(p, P_BETA)}}, nullptr);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, pt, rt, Terms<1>{{term(pt, P_BETA)}}, nullptr);
    return cudaGetLastError() == cudaSuccess ? MPSPMV_OK : MPSPMV_ECUDA;
  };
  return pt_run<L, CPLX>(h, w, b, x, iters, relres, s, body);
}

// CGS (Sonneveld), r^ = r_0.
template <int L, bool CPLX>
int cgs_impl(mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
             double* relres, cudaStream_t s) {
  Work w;
  int st = ensure_ws(h, w);
  if (st) return st;
  const int64_t n = h->nrows;
  const bool ex = h->exact;
  int G;
  if ((st = vec_grid<L, CPLX>(h, n, &G))) return st;
  double *r = w.v[0], *rh = w.v[1], *p = w.v[2], *u = w.v[3], *v = w.v[4], *q = w.v[5], *wv = w.v[8],
         *t = w.v[9];
  if ((st = pt_setup<L, CPLX>(h, w, b, x, r, p, rh, maxit, G, s))) return st;
  MPS_CUDA(cudaMemcpyAsync(u, r, sizeof(double) * h->P * n, cudaMemcpyDeviceToDevice, s));
  launch_dotg<L, CPLX>(ex, G, s, w.st, n, rh, r, true, w.part[2], true);
  k_pt_start<L, CPLX><<<1, kT, 0, s>>>(w.st, w.part[0], w.part[1], w.part[2], G, rtol, atol);
  MPS_CUDA(cudaGetLastError());
  auto body = [&](cudaStream_t cs) -> int {
    int e = mps_launch_spmv_if_running(h, p, v, &w.st->status, cs);
    if (e) return e;
    launch_dotg<L, CPLX>(ex, G, cs, w.st, n, rh, v, true, w.part[0]);
    k_pt_alpha<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[0], G);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, q, u, Terms<1>{{term(v, P_ALPHA, true)}}, nullptr);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, wv, u, Terms<1>{{term(q, -1)}}, nullptr);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, x, x, Terms<1>{{term(wv, P_ALPHA)}}, nullptr);
    if ((e = mps_launch_spmv_if_running(h, wv, t, &w.st->status, cs))) return e;
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, r, r, Terms<1>{{term(t, P_ALPHA, true)}}, w.part[1]);
    launch_dotg<L, CPLX>(ex, G, cs, w.st, n, rh, r, true, w.part[2]);
    k_pt_beta<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[1], w.part[2], G);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, u, r, Terms<1>{{term(q, P_BETA)}}, nullptr);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, p, q, Terms<1>{{term(p, P_BETA)}}, nullptr);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, p, u, Terms<1>{{term(p, P_BETA)}}, nullptr);
    return cudaGetLastError() == cudaSuccess ? MPSPMV_OK : MPSPMV_ECUDA;
  };
  return pt_run<L, CPLX>(h, w, b, x, iters, relres, s, body);
}

// GPBiCG (Zhang), r^ = r_0, with the exit on ||t|| (x += alpha p).
template <int L, bool CPLX>
int gpbicg_impl(mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                double* relres, cudaStream_t s) {
  Work w;
  int st = ensure_ws(h, w);
  if (st) return st;
  const int64_t n = h->nrows;
  const bool ex = h->exact;
  int G;
  if ((st = vec_grid<L, CPLX>(h, n, &G))) return st;
  double *r = w.v[0], *rh = w.v[1], *p = w.v[2], *u = w.v[3], *z = w.v[4], *wv = w.v[5], *y = w.v[6];
  double *tp = w.v[8], *t = w.v[9], *ap = w.v[10], *at = w.v[11];
  const size_t vb = sizeof(double) * h->P * n;
  for (double* zv : {p, u, z, wv, tp}) MPS_CUDA(cudaMemsetAsync(zv, 0, vb, s));
  if ((st = pt_setup<L, CPLX>(h, w, b, x, r, nullptr, rh, maxit, G, s))) return st;
  launch_dotg<L, CPLX>(ex, G, s, w.st, n, rh, r, true, w.part[2], true);
  k_pt_start<L, CPLX><<<1, kT, 0, s>>>(w.st, w.part[0], w.part[1], w.part[2], G, rtol, atol);
  MPS_CUDA(cudaGetLastError());
  auto body = [&](cudaStream_t cs) -> int {
    // p = r + beta (p - u)
    launch_comb<L, CPLX, 2>(ex, G, cs, w.st, n, p, r, Terms<2>{{term(p, P_BETA), term(u, P_BETA, true)}}, nullptr);
    int e = mps_launch_spmv_if_running(h, p, ap, &w.st->status, cs);
    if (e) return e;
    launch_dotg<L, CPLX>(ex, G, cs, w.st, n, rh, ap, true, w.part[0]);
    k_pt_alpha<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[0], G);
    // y = t_prev - r - alpha w + alpha A p ; t = r - alpha A p
    launch_comb<L, CPLX, 3>(ex, G, cs, w.st, n, y, tp,
                            Terms<3>{{term(r, -1, true), term(wv, P_ALPHA, true), term(ap, P_ALPHA)}}, nullptr);
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, t, r, Terms<1>{{term(ap, P_ALPHA, true)}}, w.part[1]);
    k_gp_tcheck<L><<<1, kT, 0, cs>>>(w.st, w.part[1], G);
    if (ex)
      kx_bi_xfix<L, CPLX><<<G, kTX, x_smem<L>(1), cs>>>(w.st, n, x, p, G, w.counter);
    else
      k_bi_xfix<L, CPLX><<<G, kT, 0, cs>>>(w.st, n, x, p, G, w.counter);
    if ((e = mps_launch_spmv_if_running(h, t, at, &w.st->status, cs))) return e;
    launch_dotg<L, CPLX>(ex, G, cs, w.st, n, at, at, true, w.part[2]);
    launch_dotg<L, CPLX>(ex, G, cs, w.st, n, y, y, true, w.part[3]);
    launch_dotg<L, CPLX>(ex, G, cs, w.st, n, at, y, true, w.part[4]);
    launch_dotg<L, CPLX>(ex, G, cs, w.st, n, at, t, true, w.part[5]);
    launch_dotg<L, CPLX>(ex, G, cs, w.st, n, y, t, true, w.part[6]);
    k_gp_zeta<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[2], w.part[3], w.part[4], w.part[5], w.part[6], G);
    // u = zeta A p + eta t_prev - eta r + (eta beta) u ; z = eta z + zeta r - alpha u
    launch_comb<L, CPLX, 4>(ex, G, cs, w.st, n, u, nullptr,
                            Terms<4>{{term(ap, P_ZETA), term(tp, P_ETA), term(r, P_ETA, true), term(u, P_ETA_BETA)}},
                            nullptr);
    launch_comb<L, CPLX, 3>(ex, G, cs, w.st, n, z, nullptr,
                            Terms<3>{{term(z, P_ETA), term(r, P_ZETA), term(u, P_ALPHA, true)}}, nullptr);
    // x += alpha p + z ; r = t - eta y - zeta A t
    launch_comb<L, CPLX, 2>(ex, G, cs, w.st, n, x, x, Terms<2>{{term(p, P_ALPHA), term(z, -1)}}, nullptr);
    launch_comb<L, CPLX, 2>(ex, G, cs, w.st, n, r, t, Terms<2>{{term(y, P_ETA, true), term(at, P_ZETA, true)}},
                            w.part[1]);
    launch_dotg<L, CPLX>(ex, G, cs, w.st, n, rh, r, true, w.part[7]);
    k_gp_beta<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[1], w.part[7], G);
    // w = A t + beta A p ; t_prev = t
    launch_comb<L, CPLX, 1>(ex, G, cs, w.st, n, wv, at, Terms<1>{{term(ap, P_BETA)}}, nullptr);
    if (cudaMemcpyAsync(tp, t, vb, cudaMemcpyDeviceToDevice, cs) != cudaSuccess) return MPSPMV_ECUDA;
    return cudaGetLastError() == cudaSuccess ? MPSPMV_OK : MPSPMV_ECUDA;
  };
  return pt_run<L, CPLX>(h, w, b, x, iters, relres, s, body);
}

}  // namespace

// ---------------------------------------------------------------------------
// The per-precision interface (krylov_ops.h), instantiated once per L in
// krylov_L<L>.cu.
// ---------------------------------------------------------------------------
template <int L>
int KrylovOps<L>::cg(mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                     double* relres, cudaStream_t s, double* hist) {
  return cg_impl<L>(h, b, x, rtol, atol, maxit, iters, relres, s, hist);
}

template <int L, bool CPLX, int M>
int KrylovSolve<L, CPLX, M>::run(mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit,
                                 int* iters, double* relres, cudaStream_t s) {
  if constexpr (M == KRY_BICGSTAB) return bicgstab_impl<L, CPLX>(h, b, x, rtol, atol, maxit, iters, relres, s);
  if constexpr (M == KRY_BICG) return bicg_impl<L, CPLX>(h, b, x, rtol, atol, maxit, iters, relres, s);
  if constexpr (M == KRY_CGS) return cgs_impl<L, CPLX>(h, b, x, rtol, atol, maxit, iters, relres, s);
  if constexpr (M == KRY_GPBICG) return gpbicg_impl<L, CPLX>(h, b, x, rtol, atol, maxit, iters, relres, s);
  return MPSPMV_ENOTSUP;
}

template <int L>
int KrylovOps<L>::dot(mpspmv_mat* h, int64_t n, const double* u, const double* v, double* out, cudaStream_t s) {
  return h->cplx ? dot_impl<L, true>(h, n, u, v, out, s) : dot_impl<L, false>(h, n, u, v, out, s);
}

template <int L>
int KrylovOps<L>::axpy(mpspmv_mat* h, int64_t n, const double* alpha, const double* u, const double* v, double* w,
                       cudaStream_t s) {
  return h->cplx ? axpy_impl<L, true>(h, n, alpha, u, v, w, s) : axpy_impl<L, false>(h, n, alpha, u, v, w, s);
}

template <int L>
int KrylovOps<L>::scalar_sum(mpspmv_mat* h, int count, const double* parts, double* out, cudaStream_t s) {
  if (count < 1 || count > kMaxScalarParts) return MPSPMV_EINVAL;
  return h->cplx ? scalar_sum_impl<L, true>(h, count, parts, out, s)
                 : scalar_sum_impl<L, false>(h, count, parts, out, s);
}

template <int L>
int KrylovOps<L>::scalar_div(mpspmv_mat* h, const double* a, const double* b, double* out, cudaStream_t s) {
  return h->cplx ? scalar_div_impl<L, true>(h, a, b, out, s) : scalar_div_impl<L, false>(h, a, b, out, s);
}

}  // namespace mpkry
