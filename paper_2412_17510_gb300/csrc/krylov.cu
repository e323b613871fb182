// krylov.cu -- CG and BiCGSTAB with every vector and scalar in DD / TD / QD
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
#include <algorithm>
#include <cmath>

#include "internal.h"
#include "krylov.h"
#include "mp_arith.cuh"

using namespace mpk;

namespace {

constexpr int kT = 256;           // threads per block
constexpr int kMaxBlocks = 1024;  // partials per dot
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

template <int L>
__device__ __forceinline__ cmp<L> c_div(const cmp<L>& a, const cmp<L>& b) {
  cmp<L> nb;
  nb.re = b.re;
  nb.im = mp_neg<L>(b.im);
  cmp<L> num = c_mul<L>(a, nb);
  mp<L> d = mp_add<L>(mp_mul<L>(b.re, b.re), mp_mul<L>(b.im, b.im));
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

// Reduce NA MP accumulators over the block (result valid in thread 0).
template <int L, int NA>
__device__ __forceinline__ void block_reduce(mp<L> (&acc)[NA]) {
  __shared__ double sm[kT / 32][NA][L];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
    for (int a = 0; a < NA; a++) {
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
      if (lane < kT / 32) {
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
        mp<L> o = shfl_down<L>(acc[a], off);
        if (lane < off) acc[a] = mp_add<L>(acc[a], o);
      }
    }
  }
}

template <int L, int NA>
__device__ __forceinline__ void write_partials(double* __restrict__ part, int G, mp<L> (&acc)[NA]) {
  block_reduce<L, NA>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NA; a++)
#pragma unroll
      for (int l = 0; l < L; l++) part[((int64_t)a * L + l) * G + blockIdx.x] = acc[a].v[l];
  }
}

// Finishing step: reduce the G block partials of NA accumulators (one block).
template <int L, int NA>
__device__ __forceinline__ void reduce_partials(const double* __restrict__ part, int G, mp<L> (&acc)[NA]) {
#pragma unroll
  for (int a = 0; a < NA; a++) acc[a] = mp_zero<L>();
  for (int g = threadIdx.x; g < G; g += kT) {
#pragma unroll
    for (int a = 0; a < NA; a++) {
      mp<L> v;
#pragma unroll
      for (int l = 0; l < L; l++) v.v[l] = part[((int64_t)a * L + l) * G + g];
      acc[a] = mp_add<L>(acc[a], v);
    }
  }
  block_reduce<L, NA>(acc);
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

enum Slot : int { S_RHO = 0, S_ALPHA, S_BETA, S_OMEGA, S_RHO1, S_TMP };

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
  write_partials<L, NA>(part, G, acc);
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
  write_partials<L, 2>(part, G, acc);
}

// ---------------------------------------------------------------------------
// CG
// ---------------------------------------------------------------------------
// start: part0 = (r, r), part1 = (b, b)
template <int L>
__global__ void __launch_bounds__(kT) k_cg_start(KrylovState* st, const double* part_r, const double* part_b, int G,
                                                 double rtol, double atol) {
  mp<L> a[2], b[2];
  reduce_partials<L, 2>(part_r, G, a);
  __syncthreads();
  reduce_partials<L, 2>(part_b, G, b);
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
  reduce_partials<L, 2>(part, G, a);
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
  write_partials<L, 2>(part, G, acc);
}

// rho1 = (r, r); k++; stopping test; beta = rho1 / rho; rho = rho1
template <int L>
__global__ void __launch_bounds__(kT) k_cg_beta(KrylovState* st, const double* part, int G) {
  ACTIVE(st);
  mp<L> a[2];
  reduce_partials<L, 2>(part, G, a);
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
  reduce_partials<L, 2>(part_r, G, a);
  __syncthreads();
  reduce_partials<L, 2>(part_b, G, b);
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
  reduce_partials<L, 2>(part, G, a);
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
  reduce_partials<L, 2>(part, G, a);
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
  write_partials<L, 2>(part, G, acc);
}

// k++; if ||s|| <= tol: converge after x += alpha p
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_scheck(KrylovState* st, const double* part, int G) {
  ACTIVE(st);
  mp<L> a[2];
  reduce_partials<L, 2>(part, G, a);
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
  reduce_partials<L, 4>(part, G, a);
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
  write_partials<L, 2>(part, G, acc);
}

// ||r|| test; omega == 0 breakdown; rho = rho1; maxit
template <int L, bool CPLX>
__global__ void __launch_bounds__(kT) k_bi_rcheck(KrylovState* st, const double* part, int G) {
  ACTIVE(st);
  mp<L> a[2];
  reduce_partials<L, 2>(part, G, a);
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
  reduce_partials<L, 2>(part, G, a);
  if (threadIdx.x == 0) {
    const double t = to_d<L>(a[0]);
    const double rn = sqrt(t > 0.0 ? t : 0.0);
    st->relres = st->bnorm > 0.0 ? rn / st->bnorm : rn;
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int grid_for(int64_t n) {
  int64_t g = (n + kT - 1) / kT;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, kMaxBlocks));
}

struct Work {
  double* v[8];
  double* part[3];
  KrylovState* st;
  int* counter;
};

int ensure_ws(mpspmv_mat* h, Work& w) {
  const int64_t vec = (int64_t)h->P * std::max(h->nrows, h->ncols);
  const int64_t part = 4 * 4 * (int64_t)kMaxBlocks;
  const int64_t need = 8 * vec + 3 * part;
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
  for (int i = 0; i < 8; i++) w.v[i] = h->d_kws + i * vec;
  for (int i = 0; i < 3; i++) w.part[i] = h->d_kws + 8 * vec + i * part;
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
int true_residual(mpspmv_mat* h, Work& w, const double* b, const double* x, cudaStream_t s) {
  const int64_t n = h->nrows;
  const int G = grid_for(n);
  int st = mps_launch_spmv(h, x, w.v[7], s);
  if (st) return st;
  k_residual<L, CPLX><<<G, kT, 0, s>>>(n, b, w.v[7], w.v[6], nullptr, nullptr, w.part[0], G);
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
  const int G = grid_for(n);
  double *r = w.v[0], *p = w.v[1], *q = w.v[2];
  KrylovState init{};
  init.maxit = maxit;
  MPS_CUDA(cudaMemcpyAsync(w.st, &init, sizeof(KrylovState), cudaMemcpyHostToDevice, s));
  // r = b - A x; p = r; rho = (r, r); (b, b)
  if ((st = mps_launch_spmv(h, x, q, s))) return st;
  k_residual<L, false><<<G, kT, 0, s>>>(n, b, q, r, p, nullptr, w.part[0], G);
  k_dot<L, false, 1><<<G, kT, 0, s>>>(w.st, n, b, b, nullptr, nullptr, w.part[1], G, true);
  k_cg_start<L><<<1, kT, 0, s>>>(w.st, w.part[0], w.part[1], G, rtol, atol);
  MPS_CUDA(cudaGetLastError());
  KrylovState hs{};
  auto body = [&](cudaStream_t cs) -> int {
    int e = mps_launch_spmv_if_running(h, p, q, &w.st->status, cs);
    if (e) return e;
    k_dot<L, false, 1><<<G, kT, 0, cs>>>(w.st, n, p, q, nullptr, nullptr, w.part[0], G, false);
    k_cg_alpha<L><<<1, kT, 0, cs>>>(w.st, w.part[0], G);
    k_cg_xr<L><<<G, kT, 0, cs>>>(w.st, n, x, r, p, q, w.part[1], G);
    k_cg_beta<L><<<1, kT, 0, cs>>>(w.st, w.part[1], G);
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
  const int G = grid_for(n);
  double *r = w.v[0], *rh = w.v[1], *p = w.v[2], *v = w.v[3], *sv = w.v[4], *t = w.v[5];
  KrylovState init{};
  init.maxit = maxit;
  MPS_CUDA(cudaMemcpyAsync(w.st, &init, sizeof(KrylovState), cudaMemcpyHostToDevice, s));
  MPS_CUDA(cudaMemsetAsync(p, 0, sizeof(double) * h->P * n, s));
  MPS_CUDA(cudaMemsetAsync(v, 0, sizeof(double) * h->P * n, s));
  MPS_CUDA(cudaMemsetAsync(w.counter, 0, sizeof(int), s));
  if ((st = mps_launch_spmv(h, x, t, s))) return st;
  k_residual<L, CPLX><<<G, kT, 0, s>>>(n, b, t, r, nullptr, rh, w.part[0], G);
  k_dot<L, CPLX, 1><<<G, kT, 0, s>>>(w.st, n, b, b, nullptr, nullptr, w.part[1], G, true);
  k_bi_start<L, CPLX><<<1, kT, 0, s>>>(w.st, w.part[0], w.part[1], G, rtol, atol);
  MPS_CUDA(cudaGetLastError());
  KrylovState hs{};
  auto body = [&](cudaStream_t cs) -> int {
    k_dot<L, CPLX, 1><<<G, kT, 0, cs>>>(w.st, n, rh, r, nullptr, nullptr, w.part[0], G, false);
    k_bi_beta<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[0], G);
    k_bi_p<L, CPLX><<<G, kT, 0, cs>>>(w.st, n, r, p, v, G);
    int e = mps_launch_spmv_if_running(h, p, v, &w.st->status, cs);
    if (e) return e;
    k_dot<L, CPLX, 1><<<G, kT, 0, cs>>>(w.st, n, rh, v, nullptr, nullptr, w.part[0], G, false);
    k_bi_alpha<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[0], G);
    k_bi_s<L, CPLX><<<G, kT, 0, cs>>>(w.st, n, r, v, sv, w.part[1], G);
    k_bi_scheck<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[1], G);
    k_bi_xfix<L, CPLX><<<G, kT, 0, cs>>>(w.st, n, x, p, G, w.counter);
    if ((e = mps_launch_spmv_if_running(h, sv, t, &w.st->status, cs))) return e;
    k_dot<L, CPLX, 2><<<G, kT, 0, cs>>>(w.st, n, t, sv, t, t, w.part[2], G, false);
    k_bi_omega<L, CPLX><<<1, kT, 0, cs>>>(w.st, w.part[2], G);
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

bool args_ok(mpspmv_mat* h, const double* b, const double* x, double rtol, double atol, int maxit) {
  return h && b && x && h->nrows == h->ncols && rtol >= 0.0 && atol >= 0.0 && maxit >= 0 && !h->mixed &&
         std::isfinite(rtol) && std::isfinite(atol);
}

}  // namespace

extern "C" int mpspmv_cg(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                         double* relres, void* stream) {
  if (!args_ok(h, b, x, rtol, atol, maxit)) return MPSPMV_EINVAL;
  if (h->cplx) return MPSPMV_ENOTSUP;
  cudaStream_t s = mps_stream(stream);
  switch (h->L) {
    case 1: return cg_impl<1>(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 2: return cg_impl<2>(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 3: return cg_impl<3>(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 4: return cg_impl<4>(h, b, x, rtol, atol, maxit, iters, relres, s);
  }
  return MPSPMV_ENOTSUP;
}

extern "C" int mpspmv_bicgstab(mpspmv_h h, const double* b, double* x, double rtol, double atol, int maxit,
                               int* iters, double* relres, void* stream) {
  if (!args_ok(h, b, x, rtol, atol, maxit)) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  switch (h->L * 2 + (h->cplx ? 1 : 0)) {
    case 2: return bicgstab_impl<1, false>(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 3: return bicgstab_impl<1, true>(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 4: return bicgstab_impl<2, false>(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 5: return bicgstab_impl<2, true>(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 6: return bicgstab_impl<3, false>(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 7: return bicgstab_impl<3, true>(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 8: return bicgstab_impl<4, false>(h, b, x, rtol, atol, maxit, iters, relres, s);
    case 9: return bicgstab_impl<4, true>(h, b, x, rtol, atol, maxit, iters, relres, s);
  }
  return MPSPMV_ENOTSUP;
}

// ---------------------------------------------------------------------------
// Precision ladder and the learned selector's entry points.
// ---------------------------------------------------------------------------
namespace {

int cg_level(int L, mpspmv_mat* h, const double* b, double* x, double rtol, double atol, int maxit, int* it,
             double* rr, cudaStream_t s, double* hist = nullptr) {
  switch (L) {
    case 1: return cg_impl<1>(h, b, x, rtol, atol, maxit, it, rr, s, hist);
    case 2: return cg_impl<2>(h, b, x, rtol, atol, maxit, it, rr, s, hist);
    case 3: return cg_impl<3>(h, b, x, rtol, atol, maxit, it, rr, s, hist);
    case 4: return cg_impl<4>(h, b, x, rtol, atol, maxit, it, rr, s, hist);
  }
  return MPSPMV_ENOTSUP;
}

bool ladder_ok(const mpspmv_h* hs, int64_t* n) {
  *n = -1;
  for (int l = 0; l < 4; l++) {
    const mpspmv_mat* h = hs[l];
    if (!h) continue;
    if (h->L != l + 1 || h->cplx || h->mixed || h->nrows != h->ncols) return false;
    if (*n >= 0 && h->nrows != *n) return false;
    *n = h->nrows;
  }
  return *n >= 0;
}

// b (one binary64 plane) expanded to four planes with zero lower components
int expand_b(const double* b, int64_t n, double** out, cudaStream_t s) {
  if (cudaMalloc(out, sizeof(double) * 4 * std::max<int64_t>(n, 1)) != cudaSuccess) {
    cudaGetLastError();
    return MPSPMV_ENOMEM;
  }
  MPS_CUDA(cudaMemsetAsync(*out, 0, sizeof(double) * 4 * n, s));
  MPS_CUDA(cudaMemcpyAsync(*out, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  return MPSPMV_OK;
}

int ladder_run(const mpspmv_h* hs, int start, const double* b4, double* x, int64_t n, double rtol, double atol,
               int maxit, int* final_L, int* iters, double* relres, cudaStream_t s) {
  if (iters)
    for (int l = 0; l < 4; l++) iters[l] = 0;
  MPS_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * 4 * n, s));
  int st = MPSPMV_ENOCONV;
  double rr = INFINITY;
  int last = 0;
  for (int L = std::max(start, 1); L <= 4; L++) {
    mpspmv_mat* h = hs[L - 1];
    if (!h) continue;
    int it = 0;
    // continue from the current x: its components beyond the previous level
    // are zero, so the promotion is exact; r is recomputed at this level
    int e = cg_level(L, h, b4, x, rtol, atol, maxit, &it, &rr, s);
    last = L;
    if (iters) iters[L - 1] = it;
    if (e != MPSPMV_OK && e != MPSPMV_ENOCONV && e != MPSPMV_EBREAKDOWN) return e;
    // success means the residual recomputed at this level meets the target
    if (e == MPSPMV_OK && rr <= rtol + atol) {
      st = MPSPMV_OK;
      break;
    }
  }
  if (final_L) *final_L = last;
  if (relres) *relres = rr;
  return st;
}

}  // namespace

int mps_features(mpspmv_mat* h, const double* cg_hist, float* feat, cudaStream_t s);
int mps_mlp_classify(const float* params, int C, const float* feat, int* cls, cudaStream_t s);

extern "C" int mpspmv_ladder_solve(const mpspmv_h* hs, int start_L, const double* b, double* x, double rtol,
                                   double atol, int maxit, int* final_L, int* iters, double* relres,
                                   void* stream) {
  int64_t n;
  if (!hs || !b || !x || start_L < 1 || start_L > 4 || !ladder_ok(hs, &n) || !(rtol >= 0) || !(atol >= 0) ||
      maxit < 0)
    return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  double* b4 = nullptr;
  int st = expand_b(b, n, &b4, s);
  if (!st) st = ladder_run(hs, start_L, b4, x, n, rtol, atol, maxit, final_L, iters, relres, s);
  cudaStreamSynchronize(s);
  cudaFree(b4);
  return st;
}

extern "C" int mpspmv_cg_history(mpspmv_h h, const double* b, int k, double* hist, void* stream) {
  if (!h || !b || !hist || k < 1 || k > 16 || h->cplx || h->mixed || h->nrows != h->ncols) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  double* x = nullptr;
  if (cudaMalloc(&x, sizeof(double) * h->L * std::max<int64_t>(h->nrows, 1)) != cudaSuccess) return MPSPMV_ENOMEM;
  cudaMemsetAsync(x, 0, sizeof(double) * h->L * h->nrows, s);
  double hh[16];
  int it = 0;
  double rr;
  int st = cg_level(h->L, h, b, x, 0.0, 0.0, k, &it, &rr, s, hh);
  cudaStreamSynchronize(s);
  cudaFree(x);
  if (st != MPSPMV_OK && st != MPSPMV_ENOCONV) return st;
  for (int i = 0; i < k; i++) hist[i] = hh[i];
  return MPSPMV_OK;
}

extern "C" int mpspmv_select_precision(const mpspmv_h* hs, const float* params, int C, const double* b,
                                       int* prec, float* feat_out, void* stream) {
  int64_t n;
  if (!hs || !hs[0] || !params || !b || !prec || !ladder_ok(hs, &n)) return MPSPMV_EINVAL;
  cudaStream_t s = mps_stream(stream);
  // features: matrix statistics + 8 binary64 CG residual ratios (b as given)
  double hist[16];
  int st = mpspmv_cg_history(hs[0], b, 8, hist, stream);
  float feat[32];
  if (!st) st = mps_features(hs[0], hist, feat, s);
  int cls = 0;
  if (!st) st = mps_mlp_classify(params, C, feat, &cls, s);
  if (st) return st;
  if (feat_out)
    for (int i = 0; i < 32; i++) feat_out[i] = feat[i];
  *prec = std::min(cls + 1, 4);  // classes: binary64, DD, TD, QD, (none -> QD)
  return MPSPMV_OK;
}

extern "C" int mpspmv_solve_auto(const mpspmv_h* hs, const float* params, int C, const double* b, double* x,
                                 double rtol, double atol, int maxit, int* chosen_L, int* final_L, int* iters,
                                 double* relres, void* stream) {
  int p = 1;
  int st = mpspmv_select_precision(hs, params, C, b, &p, nullptr, stream);
  if (st) return st;
  if (chosen_L) *chosen_L = p;
  return mpspmv_ladder_solve(hs, p, b, x, rtol, atol, maxit, final_L, iters, relres, stream);
}
