// Host build of the device arithmetic (csrc/mp_arith.cuh, csrc/fixacc.cuh)
// for CPU tests: the same source the kernels compile, run on the host with
// IEEE 754 binary64 and -ffp-contract=off, exported through a C ABI.  The
// CUDA qualifiers and intrinsics come from the stand-in cuda_runtime.h next
// to this file.  Test infrastructure only.
#include "cuda_runtime.h"
#include "mp_arith.cuh"
#include "fixacc.cuh"
// exact_prod.cuh holds two empty PTX statements that only pin the order of
// the products for the device compiler ("+d" names a binary64 register
// there, an integer register on the host); for the host build they are
// preprocessed away.
#define asm
#define volatile(...)
#include "exact_prod.cuh"
#undef volatile
#undef asm
#include "wide.cuh"

namespace {

// digits of the exact accumulators per L
template <int L>
constexpr int kD = mpk::AccDigits<L>::D;

template <int L>
mpk::mp<L> load_mp(const double* p) {
  mpk::mp<L> r;
  for (int l = 0; l < L; l++) r.v[l] = p[l];
  return r;
}

template <int L>
void store_mp(const mpk::mp<L>& a, double* p) {
  for (int l = 0; l < L; l++) p[l] = a.v[l];
}

// op 0 add, 1 mul, 2 mul_d (b[0] is the binary64 factor), 3 div; operands
// and results are n consecutive groups of L components
template <int L>
void mp_ops(int op, int64_t n, const double* a, const double* b, double* r) {
  for (int64_t i = 0; i < n; i++) {
    const mpk::mp<L> x = load_mp<L>(a + i * L), y = load_mp<L>(b + i * L);
    mpk::mp<L> z;
    switch (op) {
      case 0: z = mpk::mp_add<L>(x, y); break;
      case 1: z = mpk::mp_mul<L>(x, y); break;
      case 2: z = mpk::mp_mul_d<L>(x, y.v[0]); break;
      default: z = mpk::mp_div<L>(x, y); break;
    }
    store_mp<L>(z, r + i * L);
  }
}

// Sum of n terms in the shared-memory-layout accumulator (stride 1): kind 0
// adds a[i], kind 1 adds the exact product a[i] b[i]; neg[i] negates the
// term.  The result is cut to L components by the kernels' flush.
template <int L>
int fas_sum(int n, const int* kind, const double* a, const double* b, const int* neg, double* out) {
  constexpr int D = kD<L>;
  unsigned long long dp[D], dn[D];
  mpk::FixAccS<D, 1> acc;
  acc.dp = dp;
  acc.dn = dn;
  mpk::fas_reset<D, 1>(acc);
  for (int i = 0; i < n; i++) {
    if (kind[i] == 1) {
      if constexpr (D >= 6) {
        mpk::fas_add_prod<D, 1>(acc, a[i], b[i], neg[i] != 0);
      } else {
        return -1;  // the kernels form binary64 products by TwoProd instead
      }
    } else {
      mpk::fas_add<D, 1>(acc, a[i], neg[i] != 0);
    }
  }
  mpk::fas_to_mp<L, D, 1>(acc, out);
  return 0;
}

// Sum of n binary64 terms in register digits at the base of the largest term
// (the combine kernels' and block sums' form), cut to L components.
template <int L>
void fa_sum(int n, const double* a, double* out) {
  constexpr int D = kD<L>;
  int t = INT_MIN;
  for (int i = 0; i < n; i++) t = t > mpk::top_exp(a[i]) ? t : mpk::top_exp(a[i]);
  mpk::FixAcc<D> f;
  mpk::fa_at_top<D>(f, t);
  for (int i = 0; i < n; i++) mpk::fa_add<D>(f, a[i]);
  mpk::fa_to_mp<L, D>(f, out);
}

// The terms of one stored entry a . x (exact_prod.cuh: add_prod for an MP
// value, add_prod_d for a binary64 value, the forms the exact run kernels
// use) summed into an empty accumulator and cut to L components.
template <int L>
int entry_sum(int mode, const double* a, const double* x, double* out) {
  constexpr int D = kD<L>;
  unsigned long long dp[D], dn[D];
  mpk::FixAccS<D, 1> acc;
  acc.dp = dp;
  acc.dn = dn;
  mpk::fas_reset<D, 1>(acc);
  const mpk::mp<L> xm = load_mp<L>(x);
  if (mode == 0)
    mpk::add_prod<mpk::FixAccS<D, 1>, L>(acc, load_mp<L>(a), xm, false);
  else
    mpk::add_prod_d<mpk::FixAccS<D, 1>, L>(acc, a[0], xm, false);
  mpk::fas_to_mp<L, D, 1>(acc, out);
  return 0;
}

// A whole row: the terms of n stored entries added in order into one
// accumulator (as the row-per-thread and run kernels do for a row that one
// thread sums), cut to L components.  A and X hold n groups of L components.
template <int L>
void row_sum(int mode, int n, const double* A, const double* X, double* out) {
  constexpr int D = kD<L>;
  unsigned long long dp[D], dn[D];
  mpk::FixAccS<D, 1> acc;
  acc.dp = dp;
  acc.dn = dn;
  mpk::fas_reset<D, 1>(acc);
  for (int k = 0; k < n; k++) {
    const mpk::mp<L> xm = load_mp<L>(X + (size_t)k * L);
    if (mode == 0)
      mpk::add_prod<mpk::FixAccS<D, 1>, L>(acc, load_mp<L>(A + (size_t)k * L), xm, false);
    else
      mpk::add_prod_d<mpk::FixAccS<D, 1>, L>(acc, A[(size_t)k * L], xm, false);
  }
  mpk::fas_to_mp<L, D, 1>(acc, out);
}

// A whole complex row, with the kernels' per-entry pattern for complex data
// (run_body.cuh, compute_entry): re += a_re x_re, re -= a_im x_im,
// im += a_re x_im, im += a_im x_re, each product in the decomposed form.
template <int L>
void row_sum_c(int mode, int n, const double* Ar, const double* Ai, const double* Xr, const double* Xi,
               double* out_re, double* out_im) {
  constexpr int D = kD<L>;
  using Acc = mpk::FixAccS<D, 1>;
  unsigned long long d[4][D];
  Acc sr, si;
  sr.dp = d[0];
  sr.dn = d[1];
  si.dp = d[2];
  si.dn = d[3];
  mpk::fas_reset<D, 1>(sr);
  mpk::fas_reset<D, 1>(si);
  for (int k = 0; k < n; k++) {
    const mpk::mp<L> xr = load_mp<L>(Xr + (size_t)k * L), xi = load_mp<L>(Xi + (size_t)k * L);
    if (mode == 0) {
      const mpk::mp<L> ar = load_mp<L>(Ar + (size_t)k * L), ai = load_mp<L>(Ai + (size_t)k * L);
      mpk::add_prod<Acc, L>(sr, ar, xr, false);
      mpk::add_prod<Acc, L>(sr, ai, xi, true);
      mpk::add_prod<Acc, L>(si, ar, xi, false);
      mpk::add_prod<Acc, L>(si, ai, xr, false);
    } else {
      const double ar = Ar[(size_t)k * L], ai = Ai[(size_t)k * L];
      mpk::add_prod_d<Acc, L>(sr, ar, xr, false);
      mpk::add_prod_d<Acc, L>(sr, ai, xi, true);
      mpk::add_prod_d<Acc, L>(si, ar, xi, false);
      mpk::add_prod_d<Acc, L>(si, ai, xr, false);
    }
  }
  mpk::fas_to_mp<L, D, 1>(sr, out_re);
  mpk::fas_to_mp<L, D, 1>(si, out_im);
}

// One element of w = u + alpha v in the vector kernels' form (x_lin in
// krylov_impl.cuh): u's components, then the decomposed products, one
// accumulator per part, each part cut once.  alpha, u, v, out: P components.
template <int L>
void axpy_elem(int cplx, const double* alpha, const double* u, const double* v, double* out) {
  constexpr int D = kD<L>;
  using Acc = mpk::FixAccS<D, 1>;
  unsigned long long dp[D], dn[D];
  Acc e;
  e.dp = dp;
  e.dn = dn;
  const mpk::mp<L> ar = load_mp<L>(alpha), vr = load_mp<L>(v);
  mpk::fas_reset<D, 1>(e);
  for (int l = 0; l < L; l++) mpk::acc_add(e, u[l], false);
  mpk::add_prod<Acc, L>(e, ar, vr, false);
  if (cplx) {
    const mpk::mp<L> ai = load_mp<L>(alpha + L), vi = load_mp<L>(v + L);
    mpk::add_prod<Acc, L>(e, ai, vi, true);
    mpk::fas_to_mp<L, D, 1>(e, out);
    mpk::fas_reset<D, 1>(e);
    for (int l = 0; l < L; l++) mpk::acc_add(e, u[L + l], false);
    mpk::add_prod<Acc, L>(e, ar, vi, false);
    mpk::add_prod<Acc, L>(e, ai, vr, false);
    mpk::fas_to_mp<L, D, 1>(e, out + L);
  } else {
    mpk::fas_to_mp<L, D, 1>(e, out);
  }
}

// The flush alone, on given digit arrays (D = the kernels' digit count for L).
template <int L>
void flush(const unsigned long long* dp_in, const unsigned long long* dn_in, int base, double* out) {
  constexpr int D = kD<L>;
  unsigned long long dp[D], dn[D];
  for (int j = 0; j < D; j++) {
    dp[j] = dp_in[j];
    dn[j] = dn_in[j];
  }
  mpk::FixAccS<D, 1> acc;
  acc.dp = dp;
  acc.dn = dn;
  acc.base = base;
  acc.bad = false;
  mpk::fas_to_mp<L, D, 1>(acc, out);
}

// The flush body on digit arrays of the wide-x row accumulator (D = its
// digit count for L), as the run kernels and the finishing pass of staged
// rows call it.
template <int L>
void flush_wide(const unsigned long long* dp_in, const unsigned long long* dn_in, int base, double* out) {
  constexpr int D = mpk::Wide<L>::D;
  unsigned long long dp[D], dn[D];
  for (int j = 0; j < D; j++) {
    dp[j] = dp_in[j];
    dn[j] = dn_in[j];
  }
  mpk::fas_flush_body<L, D, 1>(dp, dn, base, 1, out);
}

// wide-x form: the record of one column part, and a row of n entries (a[i]
// binary64, X + i L the components of the x it multiplies) summed in the
// row accumulator of that form and cut to L components
template <int L>
void wide_rec(const double* c, uint32_t* rec) {
  mpk::wide_build<L>(c, rec);
}

template <int L>
void wide_row(int n, const double* a, const double* X, double* out) {
  constexpr int D = mpk::Wide<L>::D;
  unsigned long long dp[D], dn[D];
  mpk::FixAccS<D, 1> acc;
  acc.dp = dp;
  acc.dn = dn;
  mpk::fas_reset<D, 1>(acc);
  for (int i = 0; i < n; i++) {
    uint32_t rec[mpk::kWideRecWords];
    mpk::wide_build<L>(X + (int64_t)i * L, rec);
    mpk::fas_add_wide<L, D, 1>(acc, a[i], rec, false);
  }
  mpk::fas_to_mp<L, D, 1>(acc, out);
}

// complex row in the kernels' order: re += a_re X_re, im += a_im X_re,
// re -= a_im X_im, im += a_re X_im
template <int L>
void wide_row_c(int n, const double* ar, const double* ai, const double* Xr, const double* Xi, double* out_re,
                double* out_im) {
  constexpr int D = mpk::Wide<L>::D;
  unsigned long long dp[2][D], dn[2][D];
  mpk::FixAccS<D, 1> sr, si;
  sr.dp = dp[0];
  sr.dn = dn[0];
  si.dp = dp[1];
  si.dn = dn[1];
  mpk::fas_reset<D, 1>(sr);
  mpk::fas_reset<D, 1>(si);
  for (int i = 0; i < n; i++) {
    uint32_t rr[mpk::kWideRecWords], ri[mpk::kWideRecWords];
    mpk::wide_build<L>(Xr + (int64_t)i * L, rr);
    mpk::wide_build<L>(Xi + (int64_t)i * L, ri);
    mpk::fas_add_wide<L, D, 1>(sr, ar[i], rr, false);
    mpk::fas_add_wide<L, D, 1>(si, ai[i], rr, false);
    mpk::fas_add_wide<L, D, 1>(sr, ai[i], ri, true);
    mpk::fas_add_wide<L, D, 1>(si, ar[i], ri, false);
  }
  mpk::fas_to_mp<L, D, 1>(sr, out_re);
  mpk::fas_to_mp<L, D, 1>(si, out_im);
}

// sum over n MP values u_i (L components each) of u_i u_i, formed with
// add_prod_self (self = 1) or add_prod(u, u) (self = 0), cut to L components
template <int L>
void self_sum(int self, int n, const double* U, double* out) {
  constexpr int D = kD<L>;
  unsigned long long dp[D], dn[D];
  mpk::FixAccS<D, 1> acc;
  acc.dp = dp;
  acc.dn = dn;
  mpk::fas_reset<D, 1>(acc);
  for (int i = 0; i < n; i++) {
    const mpk::mp<L> u = load_mp<L>(U + (int64_t)i * L);
    if (self) mpk::add_prod_self<mpk::FixAccS<D, 1>, L>(acc, u, false);
    else mpk::add_prod<mpk::FixAccS<D, 1>, L>(acc, u, u, false);
  }
  mpk::fas_to_mp<L, D, 1>(acc, out);
}

}  // namespace

extern "C" {

int host_self_sum(int L, int self, int n, const double* U, double* out) {
  switch (L) {
    case 2: self_sum<2>(self, n, U, out); return 0;
    case 3: self_sum<3>(self, n, U, out); return 0;
    case 4: self_sum<4>(self, n, U, out); return 0;
    default: return -1;
  }
}

int host_wide_rec(int L, const double* c, uint32_t* rec) {
  switch (L) {
    case 2: wide_rec<2>(c, rec); return 0;
    case 3: wide_rec<3>(c, rec); return 0;
    case 4: wide_rec<4>(c, rec); return 0;
    default: return -1;
  }
}

int host_wide_row(int L, int n, const double* a, const double* X, double* out) {
  switch (L) {
    case 2: wide_row<2>(n, a, X, out); return 0;
    case 3: wide_row<3>(n, a, X, out); return 0;
    case 4: wide_row<4>(n, a, X, out); return 0;
    default: return -1;
  }
}

int host_wide_row_c(int L, int n, const double* ar, const double* ai, const double* Xr, const double* Xi,
                    double* out_re, double* out_im) {
  switch (L) {
    case 2: wide_row_c<2>(n, ar, ai, Xr, Xi, out_re, out_im); return 0;
    case 3: wide_row_c<3>(n, ar, ai, Xr, Xi, out_re, out_im); return 0;
    case 4: wide_row_c<4>(n, ar, ai, Xr, Xi, out_re, out_im); return 0;
    default: return -1;
  }
}

int host_wide_digits(int L) {
  switch (L) {
    case 2: return mpk::Wide<2>::D;
    case 3: return mpk::Wide<3>::D;
    case 4: return mpk::Wide<4>::D;
    default: return -1;
  }
}

int host_wide_words(int L) {
  switch (L) {
    case 2: return mpk::Wide<2>::W;
    case 3: return mpk::Wide<3>::W;
    case 4: return mpk::Wide<4>::W;
    default: return -1;
  }
}


int host_row_sum(int L, int mode, int n, const double* A, const double* X, double* out) {
  switch (L) {
    case 1: row_sum<1>(mode, n, A, X, out); return 0;
    case 2: row_sum<2>(mode, n, A, X, out); return 0;
    case 3: row_sum<3>(mode, n, A, X, out); return 0;
    case 4: row_sum<4>(mode, n, A, X, out); return 0;
    default: return -1;
  }
}

int host_row_sum_c(int L, int mode, int n, const double* Ar, const double* Ai, const double* Xr, const double* Xi,
                   double* out_re, double* out_im) {
  switch (L) {
    case 1: row_sum_c<1>(mode, n, Ar, Ai, Xr, Xi, out_re, out_im); return 0;
    case 2: row_sum_c<2>(mode, n, Ar, Ai, Xr, Xi, out_re, out_im); return 0;
    case 3: row_sum_c<3>(mode, n, Ar, Ai, Xr, Xi, out_re, out_im); return 0;
    case 4: row_sum_c<4>(mode, n, Ar, Ai, Xr, Xi, out_re, out_im); return 0;
    default: return -1;
  }
}

int host_axpy_elem(int L, int cplx, const double* alpha, const double* u, const double* v, double* out) {
  switch (L) {
    case 1: axpy_elem<1>(cplx, alpha, u, v, out); return 0;
    case 2: axpy_elem<2>(cplx, alpha, u, v, out); return 0;
    case 3: axpy_elem<3>(cplx, alpha, u, v, out); return 0;
    case 4: axpy_elem<4>(cplx, alpha, u, v, out); return 0;
    default: return -1;
  }
}

int host_flush(int L, const unsigned long long* dp, const unsigned long long* dn, int base, double* out) {
  switch (L) {
    case 1: flush<1>(dp, dn, base, out); return 0;
    case 2: flush<2>(dp, dn, base, out); return 0;
    case 3: flush<3>(dp, dn, base, out); return 0;
    case 4: flush<4>(dp, dn, base, out); return 0;
    default: return -1;
  }
}

int host_flush_wide(int L, const unsigned long long* dp, const unsigned long long* dn, int base, double* out) {
  switch (L) {
    case 2: flush_wide<2>(dp, dn, base, out); return 0;
    case 3: flush_wide<3>(dp, dn, base, out); return 0;
    case 4: flush_wide<4>(dp, dn, base, out); return 0;
    default: return -1;
  }
}

int host_acc_digits(int L) {
  switch (L) {
    case 1: return kD<1>;
    case 2: return kD<2>;
    case 3: return kD<3>;
    case 4: return kD<4>;
    default: return -1;
  }
}

int host_entry_sum(int L, int mode, const double* a, const double* x, double* out) {
  switch (L) {
    case 1: return entry_sum<1>(mode, a, x, out);
    case 2: return entry_sum<2>(mode, a, x, out);
    case 3: return entry_sum<3>(mode, a, x, out);
    case 4: return entry_sum<4>(mode, a, x, out);
    default: return -1;
  }
}


int host_mp_ops(int L, int op, int64_t n, const double* a, const double* b, double* r) {
  switch (L) {
    case 1: mp_ops<1>(op, n, a, b, r); return 0;
    case 2: mp_ops<2>(op, n, a, b, r); return 0;
    case 3: mp_ops<3>(op, n, a, b, r); return 0;
    case 4: mp_ops<4>(op, n, a, b, r); return 0;
    default: return -1;
  }
}

int host_fas_sum(int L, int n, const int* kind, const double* a, const double* b, const int* neg, double* out) {
  switch (L) {
    case 1: return fas_sum<1>(n, kind, a, b, neg, out);
    case 2: return fas_sum<2>(n, kind, a, b, neg, out);
    case 3: return fas_sum<3>(n, kind, a, b, neg, out);
    case 4: return fas_sum<4>(n, kind, a, b, neg, out);
    default: return -1;
  }
}

int host_fa_sum(int L, int n, const double* a, double* out) {
  switch (L) {
    case 1: fa_sum<1>(n, a, out); return 0;
    case 2: fa_sum<2>(n, a, out); return 0;
    case 3: fa_sum<3>(n, a, out); return 0;
    case 4: fa_sum<4>(n, a, out); return 0;
    default: return -1;
  }
}

double host_chunk_to_double(unsigned long long chunk, int e, int neg) {
  return mpk::chunk_to_double(chunk, e, neg != 0);
}

}  // extern "C"
