/*
 * mporacle.c -- CPU oracle for multi-component multiple-precision CSR SpMV,
 * SpMM, CG and BiCGSTAB (arXiv 2412.17510, Kouya).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library and includes nothing
 * from it.
 *
 * Build with IEEE binary64 semantics and no contraction of a*b+c into an FMA
 * (gcc: -O2 -ffp-contract=off -fno-fast-math); every fused multiply-add below
 * is an explicit call to fma().  Compiled with -DORACLE_COUNT the four
 * primitive operations increment a global counter, which fixes the number of
 * binary64 operations each algorithm performs.
 *
 * Number formats (Section 2 of the paper): a DD/TD/QD number is an unevaluated
 * sum of L = 2/3/4 binary64 components x[0] + x[1] + ... ; L = 1 is plain
 * binary64.  Vectors and matrix values are stored structure-of-limbs: one
 * binary64 array per component (Section 3, "allocated independently ... for
 * each component").  A complex value is a real part and an imaginary part
 * with the same structure (Eq. complex_expression): planes 0..L-1 hold the real
 * limbs and planes L..2L-1 the imaginary limbs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Primitive binary64 operations, optionally counted.                        */
/* ------------------------------------------------------------------------- */
#ifdef ORACLE_COUNT
static long long g_ops = 0;
#define TICK (g_ops++)
#else
#define TICK ((void)0)
#endif

long long oracle_ops_get(void) {
#ifdef ORACLE_COUNT
  return g_ops;
#else
  return -1;
#endif
}
void oracle_ops_reset(void) {
#ifdef ORACLE_COUNT
  g_ops = 0;
#endif
}

static inline double fadd(double a, double b) { TICK; return a + b; }
static inline double fsub(double a, double b) { TICK; return a - b; }
static inline double fmul(double a, double b) { TICK; return a * b; }
static inline double ffma(double a, double b, double c) { TICK; return fma(a, b, c); }
static inline double fdiv(double a, double b) { TICK; return a / b; }

/* ------------------------------------------------------------------------- */
/* Error-free transformations (Section 2, QuickTwoSum / TwoSum / TwoProd-FMA) */
/* ------------------------------------------------------------------------- */

/* QuickTwoSum: s = fl(a+b), e = a+b-s exactly, valid when |a| >= |b| or a = 0. */
static inline void quick_two_sum(double a, double b, double* s, double* e) {
  double t = fadd(a, b);
  *e = fsub(b, fsub(t, a));
  *s = t;
}

/* TwoSum (Knuth): s = fl(a+b), e = a+b-s exactly, for any a, b. */
static inline void two_sum(double a, double b, double* s, double* e) {
  double t = fadd(a, b);
  double bb = fsub(t, a);
  double err = fadd(fsub(a, fsub(t, bb)), fsub(b, bb));
  *s = t;
  *e = err;
}

/* TwoProd-FMA: p = fl(a*b), e = a*b-p exactly (no underflow). */
static inline void two_prod(double a, double b, double* p, double* e) {
  double t = fmul(a, b);
  *e = ffma(a, b, -t);
  *p = t;
}

/* ThreeSum: (a,b,c) -> (a,b,c) with the same exact sum; a is the leading term,
 * b the next, c the rest (Hida, Li and Bailey 2001, used in Section 2 for QD). */
static inline void three_sum(double* a, double* b, double* c) {
  double t1, t2, t3;
  two_sum(*a, *b, &t1, &t2);
  two_sum(*c, t1, a, &t3);
  two_sum(t2, t3, b, c);
}

/* ThreeSum2: (a,b,c) -> (a,b): leading term and a rounded tail. */
static inline void three_sum2(double* a, double* b, double c) {
  double t1, t2, t3;
  two_sum(*a, *b, &t1, &t2);
  two_sum(c, t1, a, &t3);
  *b = fadd(t2, t3);
}

/* ------------------------------------------------------------------------- */
/* DD arithmetic: Algorithms 1, 2, 3.                                         */
/* ------------------------------------------------------------------------- */

/* Algorithm 1 (DDadd, the sloppy form). */
static void dd_add(const double* x, const double* y, double* r) {
  double s, e;
  two_sum(x[0], y[0], &s, &e);
  double w = fadd(x[1], y[1]);
  e = fadd(e, w);
  quick_two_sum(s, e, &r[0], &r[1]);
}

/* Algorithm 2 (DDmul). */
static void dd_mul(const double* x, const double* y, double* r) {
  double p1, p2;
  two_prod(x[0], y[0], &p1, &p2);
  double w1 = fmul(x[0], y[1]);
  double w2 = fmul(x[1], y[0]);
  double w3 = fadd(w1, w2);
  p2 = fadd(p2, w3);
  quick_two_sum(p1, p2, &r[0], &r[1]);
}

/* Algorithm 3 (DDmulD), DD times binary64.  The printed second step adds x[1]
 * to p2; the DD product needs the term x[1]*y there, so it is a fused
 * multiply-add of x[1] and y into p2. */
static void dd_mul_d(const double* x, double y, double* r) {
  double p1, p2;
  two_prod(x[0], y, &p1, &p2);
  p2 = ffma(x[1], y, p2);
  quick_two_sum(p1, p2, &r[0], &r[1]);
}

/* ------------------------------------------------------------------------- */
/* QD arithmetic (Section 2, "sloppy" add and multiply with ThreeSum,         */
/* ThreeSum2 and Renorm; Hida, Li and Bailey 2001).                           */
/* ------------------------------------------------------------------------- */

/* Renorm: five overlapping terms of decreasing magnitude -> four
 * non-overlapping components.  First a bottom-up pass of QuickTwoSum, then a
 * top-down pass that emits a component whenever the error is non-zero. */
static void renorm5(double c0, double c1, double c2, double c3, double c4, double* r) {
  double s, t0, t1, t2, t3;
  double b[4] = {0.0, 0.0, 0.0, 0.0};
  if (isinf(c0)) { r[0] = c0; r[1] = r[2] = r[3] = 0.0; return; }
  quick_two_sum(c3, c4, &s, &t3);
  quick_two_sum(c2, s, &s, &t2);
  quick_two_sum(c1, s, &s, &t1);
  quick_two_sum(c0, s, &c0, &t0);
  double t[4] = {t0, t1, t2, t3};
  s = c0;
  int k = 0;
  double e;
  for (int i = 0; i < 4 && k < 4; i++) {
    quick_two_sum(s, t[i], &s, &e);
    if (e != 0.0) {
      b[k++] = s;
      s = e;
    }
  }
  if (k < 4) b[k] = s;
  /* components left over when k reached 4 are below the last ulp kept */
  r[0] = b[0]; r[1] = b[1]; r[2] = b[2]; r[3] = b[3];
}

/* Renorm4: four overlapping terms -> three non-overlapping components. */
static void renorm4(double c0, double c1, double c2, double c3, double* r) {
  double s, t0, t1, t2;
  double b[3] = {0.0, 0.0, 0.0};
  if (isinf(c0)) { r[0] = c0; r[1] = r[2] = 0.0; return; }
  quick_two_sum(c2, c3, &s, &t2);
  quick_two_sum(c1, s, &s, &t1);
  quick_two_sum(c0, s, &c0, &t0);
  double t[3] = {t0, t1, t2};
  s = c0;
  int k = 0;
  double e;
  for (int i = 0; i < 3 && k < 3; i++) {
    quick_two_sum(s, t[i], &s, &e);
    if (e != 0.0) {
      b[k++] = s;
      s = e;
    }
  }
  if (k < 3) b[k] = s;
  r[0] = b[0]; r[1] = b[1]; r[2] = b[2];
}

/* QD sloppy addition: limb-wise TwoSum, then the errors are folded in by
 * magnitude class and the five terms renormalised. */
static void qd_add(const double* a, const double* b, double* r) {
  double s0, s1, s2, s3, t0, t1, t2, t3;
  two_sum(a[0], b[0], &s0, &t0);
  two_sum(a[1], b[1], &s1, &t1);
  two_sum(a[2], b[2], &s2, &t2);
  two_sum(a[3], b[3], &s3, &t3);
  two_sum(s1, t0, &s1, &t0);       /* O(eps) class: s1 and t0 */
  three_sum(&s2, &t0, &t1);        /* O(eps^2) class: s2, t0, t1 */
  three_sum2(&s3, &t0, t2);        /* O(eps^3) class: s3, t0, t2 */
  t0 = fadd(fadd(t0, t1), t3);     /* O(eps^4) remainder */
  renorm5(s0, s1, s2, s3, t0, r);
}

/* QD sloppy multiplication: the products a_i*b_j with i+j <= 2 are formed
 * exactly by TwoProd, the i+j = 3 products in plain binary64, and the terms
 * are summed by magnitude class before a final Renorm. */
static void qd_mul(const double* a, const double* b, double* r) {
  double p0, p1, p2, p3, p4, p5, q0, q1, q2, q3, q4, q5;
  two_prod(a[0], b[0], &p0, &q0);  /* O(1)     */
  two_prod(a[0], b[1], &p1, &q1);  /* O(eps)   */
  two_prod(a[1], b[0], &p2, &q2);
  two_prod(a[0], b[2], &p3, &q3);  /* O(eps^2) */
  two_prod(a[1], b[1], &p4, &q4);
  two_prod(a[2], b[0], &p5, &q5);

  /* O(eps) class: p1, p2, q0 */
  three_sum(&p1, &p2, &q0);

  /* O(eps^2) class: p2, q1, q2, p3, p4, p5 -> three terms s0, s1, s2 */
  three_sum(&p2, &q1, &q2);
  three_sum(&p3, &p4, &p5);
  double s0, s1, s2, t0, t1;
  two_sum(p2, p3, &s0, &t0);
  two_sum(q1, p4, &s1, &t1);
  s2 = fadd(q2, p5);
  two_sum(s1, t0, &s1, &t0);
  s2 = fadd(s2, fadd(t0, t1));

  /* O(eps^3) class */
  double w = fmul(a[0], b[3]);
  w = fadd(w, fmul(a[1], b[2]));
  w = fadd(w, fmul(a[2], b[1]));
  w = fadd(w, fmul(a[3], b[0]));
  w = fadd(w, q0);
  w = fadd(w, q3);
  w = fadd(w, q4);
  w = fadd(w, q5);
  s1 = fadd(s1, w);

  renorm5(p0, p1, s0, s1, s2, r);
}

/* Algorithm 4 (QDmulD), QD times binary64.  Readings of the printed steps:
 * the fourth product is x[3]*y (a multiply), the pair (s1,s2) is the TwoSum of
 * q0 and p1, and ThreeSum2 combines q1 with q2 and p3 (p2 is used afterwards
 * for s4). */
static void qd_mul_d(const double* x, double y, double* r) {
  double p0, p1, p2, q0, q1, q2;
  two_prod(x[0], y, &p0, &q0);
  two_prod(x[1], y, &p1, &q1);
  two_prod(x[2], y, &p2, &q2);
  double p3 = fmul(x[3], y);
  double s0 = p0, s1, s2;
  two_sum(q0, p1, &s1, &s2);
  three_sum(&s2, &q1, &p2);
  three_sum2(&q1, &q2, p3);
  double s3 = q1;
  double s4 = fadd(q2, p2);
  renorm5(s0, s1, s2, s3, s4, r);
}

/* ------------------------------------------------------------------------- */
/* TD arithmetic (Section 2): TDaddq / TDmulq are the QD operations with the  */
/* fourth components set to zero.  The four-component result is brought to   */
/* three components by folding the fourth into the third (one rounding).      */
/* ------------------------------------------------------------------------- */
static void td_add(const double* x, const double* y, double* r) {
  double a[4] = {x[0], x[1], x[2], 0.0}, b[4] = {y[0], y[1], y[2], 0.0}, q[4];
  qd_add(a, b, q);
  r[0] = q[0]; r[1] = q[1]; r[2] = fadd(q[2], q[3]);
}

static void td_mul(const double* x, const double* y, double* r) {
  double a[4] = {x[0], x[1], x[2], 0.0}, b[4] = {y[0], y[1], y[2], 0.0}, q[4];
  qd_mul(a, b, q);
  r[0] = q[0]; r[1] = q[1]; r[2] = fadd(q[2], q[3]);
}

/* Algorithm 5 (TDmulD), TD times binary64.  Readings: (s1,s2) is a TwoSum;
 * after ThreeSum the middle output q1 is of the same order as q2 and is kept,
 * s3 = q1 + (q2 + p2); Renorm4 returns three components. */
static void td_mul_d(const double* x, double y, double* r) {
  double p0, p1, p2, q0, q1, q2;
  two_prod(x[0], y, &p0, &q0);
  two_prod(x[1], y, &p1, &q1);
  two_prod(x[2], y, &p2, &q2);
  double s0 = p0, s1, s2;
  two_sum(q0, p1, &s1, &s2);
  three_sum(&s2, &q1, &p2);
  double s3 = fadd(q1, fadd(q2, p2));
  renorm4(s0, s1, s2, s3, r);
}

/* ------------------------------------------------------------------------- */
/* Precision-generic scalar operations.  L = 1 (binary64), 2, 3, 4.           */
/* ------------------------------------------------------------------------- */
static void mp_add(int L, const double* a, const double* b, double* r) {
  switch (L) {
    case 1: r[0] = fadd(a[0], b[0]); break;
    case 2: dd_add(a, b, r); break;
    case 3: td_add(a, b, r); break;
    default: qd_add(a, b, r); break;
  }
}
static void mp_mul(int L, const double* a, const double* b, double* r) {
  switch (L) {
    case 1: r[0] = fmul(a[0], b[0]); break;
    case 2: dd_mul(a, b, r); break;
    case 3: td_mul(a, b, r); break;
    default: qd_mul(a, b, r); break;
  }
}
static void mp_mul_d(int L, const double* a, double b, double* r) {
  switch (L) {
    case 1: r[0] = fmul(a[0], b); break;
    case 2: dd_mul_d(a, b, r); break;
    case 3: td_mul_d(a, b, r); break;
    default: qd_mul_d(a, b, r); break;
  }
}
static void mp_neg(int L, const double* a, double* r) {
  for (int l = 0; l < L; l++) r[l] = -a[l];
}
static void mp_sub(int L, const double* a, const double* b, double* r) {
  double nb[4];
  mp_neg(L, b, nb);
  mp_add(L, a, nb, r);
}
static void mp_zero(int L, double* r) {
  for (int l = 0; l < L; l++) r[l] = 0.0;
}
static void mp_copy(int L, const double* a, double* r) {
  for (int l = 0; l < L; l++) r[l] = a[l];
}

/* Division a/b by long division: L+1 binary64 quotient digits, each followed
 * by the exact-order update r := r - q_k*b in the working precision, then a
 * renormalisation (Hida, Li and Bailey 2001).  The paper needs division only
 * for the Krylov scalars and does not print an algorithm. */
static void mp_div(int L, const double* a, const double* b, double* r) {
  if (L == 1) { r[0] = fdiv(a[0], b[0]); return; }
  double q[5] = {0, 0, 0, 0, 0}, rem[4], t[4];
  mp_copy(L, a, rem);
  for (int k = 0; k <= L; k++) {
    q[k] = fdiv(rem[0], b[0]);
    if (k == L) break;
    mp_mul_d(L, b, q[k], t);
    mp_sub(L, rem, t, rem);
  }
  if (L == 2) {
    double s, e;
    quick_two_sum(q[0], q[1], &s, &e);
    e = fadd(e, q[2]);
    quick_two_sum(s, e, &r[0], &r[1]);
  } else if (L == 3) {
    renorm4(q[0], q[1], q[2], q[3], r);
  } else {
    renorm5(q[0], q[1], q[2], q[3], q[4], r);
  }
}

/* Complex scalar helpers: z = (re[0..L), im[0..L)). */
static void cmp_mul(int L, const double* ar, const double* ai, const double* br, const double* bi,
                    double* rr, double* ri) {
  double t1[4], t2[4], t3[4], t4[4];
  mp_mul(L, ar, br, t1);
  mp_mul(L, ai, bi, t2);
  mp_mul(L, ar, bi, t3);
  mp_mul(L, ai, br, t4);
  mp_sub(L, t1, t2, rr);
  mp_add(L, t3, t4, ri);
}
/* (a/b) = a*conj(b)/|b|^2, with a and b first scaled by the same power of
 * two (exact, component by component) so that the larger part of b is near
 * 1: |b|^2 then stays in range when b is tiny or huge (scalars of a
 * converged Krylov iteration reach 1e-200 and below). */
static void cmp_div(int L, const double* ar, const double* ai, const double* br, const double* bi,
                    double* rr, double* ri) {
  double nbi[4], nr[4], ni[4], d[4], t1[4], t2[4];
  double as_r[4], as_i[4], bs_r[4], bs_i[4];
  double m = fmax(fabs(br[0]), fabs(bi[0]));
  int e = (m > 0.0 && isfinite(m)) ? ilogb(m) : 0;
  for (int l = 0; l < L; l++) {
    as_r[l] = scalbn(ar[l], -e);
    as_i[l] = scalbn(ai[l], -e);
    bs_r[l] = scalbn(br[l], -e);
    bs_i[l] = scalbn(bi[l], -e);
  }
  mp_neg(L, bs_i, nbi);
  cmp_mul(L, as_r, as_i, bs_r, nbi, nr, ni);
  mp_mul(L, bs_r, bs_r, t1);
  mp_mul(L, bs_i, bs_i, t2);
  mp_add(L, t1, t2, d);
  mp_div(L, nr, d, rr);
  mp_div(L, ni, d, ri);
}

/* ------------------------------------------------------------------------- */
/* Exported scalar entry points (used by the oracle's own tests).            */
/* ------------------------------------------------------------------------- */
void oracle_two_sum(double a, double b, double* s, double* e) { two_sum(a, b, s, e); }
void oracle_quick_two_sum(double a, double b, double* s, double* e) { quick_two_sum(a, b, s, e); }
void oracle_two_prod(double a, double b, double* p, double* e) { two_prod(a, b, p, e); }
void oracle_three_sum(double* a, double* b, double* c) { three_sum(a, b, c); }
void oracle_three_sum2(double* a, double* b, double c) { three_sum2(a, b, c); }
void oracle_renorm5(const double* c, double* r) { renorm5(c[0], c[1], c[2], c[3], c[4], r); }
void oracle_renorm4(const double* c, double* r) { renorm4(c[0], c[1], c[2], c[3], r); }
void oracle_mp_add(int L, const double* a, const double* b, double* r) { mp_add(L, a, b, r); }
void oracle_mp_mul(int L, const double* a, const double* b, double* r) { mp_mul(L, a, b, r); }
void oracle_mp_mul_d(int L, const double* a, double b, double* r) { mp_mul_d(L, a, b, r); }
void oracle_mp_div(int L, const double* a, const double* b, double* r) { mp_div(L, a, b, r); }

/* ------------------------------------------------------------------------- */
/* COO -> CSR (Section 3 worked example: data, indices, indptr).              */
/* Triplets are sorted by (row, col), stable in input order; duplicates are   */
/* summed in the working precision in that order.                             */
/* ------------------------------------------------------------------------- */
typedef struct { int64_t row, col, pos; } trip_t;
static int trip_cmp(const void* pa, const void* pb) {
  const trip_t* a = (const trip_t*)pa;
  const trip_t* b = (const trip_t*)pb;
  if (a->row != b->row) return a->row < b->row ? -1 : 1;
  if (a->col != b->col) return a->col < b->col ? -1 : 1;
  return a->pos < b->pos ? -1 : (a->pos > b->pos ? 1 : 0);
}

/* val: P planes of nnz (P = L, or 2L when complex); out_data: P planes of nnz
 * (capacity nnz); returns the number of stored entries, or -1 on a bad index. */
int64_t oracle_coo_to_csr(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t* row, const int64_t* col,
                          const double* val, int L, int cplx, int64_t* indptr, int32_t* indices,
                          double* out_data) {
  int P = cplx ? 2 * L : L;
  trip_t* t = (trip_t*)malloc(sizeof(trip_t) * (size_t)(nnz > 0 ? nnz : 1));
  for (int64_t k = 0; k < nnz; k++) {
    if (row[k] < 0 || row[k] >= nrows || col[k] < 0 || col[k] >= ncols) { free(t); return -1; }
    t[k].row = row[k]; t[k].col = col[k]; t[k].pos = k;
  }
  qsort(t, (size_t)nnz, sizeof(trip_t), trip_cmp);
  int64_t m = 0;
  for (int64_t i = 0; i <= nrows; i++) indptr[i] = 0;
  for (int64_t k = 0; k < nnz; k++) {
    int64_t src = t[k].pos;
    double vr[4], vi[4];
    for (int l = 0; l < L; l++) vr[l] = val[(int64_t)l * nnz + src];
    if (cplx) for (int l = 0; l < L; l++) vi[l] = val[(int64_t)(L + l) * nnz + src];
    if (m > 0 && k > 0 && t[k].row == t[k - 1].row && t[k].col == t[k - 1].col) {
      double ar[4], ai[4], sr[4], si[4];
      for (int l = 0; l < L; l++) ar[l] = out_data[(int64_t)l * nnz + m - 1];
      mp_add(L, ar, vr, sr);
      for (int l = 0; l < L; l++) out_data[(int64_t)l * nnz + m - 1] = sr[l];
      if (cplx) {
        for (int l = 0; l < L; l++) ai[l] = out_data[(int64_t)(L + l) * nnz + m - 1];
        mp_add(L, ai, vi, si);
        for (int l = 0; l < L; l++) out_data[(int64_t)(L + l) * nnz + m - 1] = si[l];
      }
      continue;
    }
    indices[m] = (int32_t)t[k].col;
    for (int p = 0; p < P; p++) out_data[(int64_t)p * nnz + m] = val[(int64_t)p * nnz + src];
    indptr[t[k].row + 1]++;
    m++;
  }
  for (int64_t i = 0; i < nrows; i++) indptr[i + 1] += indptr[i];
  free(t);
  (void)P;
  return m;
}

/* ------------------------------------------------------------------------- */
/* SpMV (Section 3, Eq. complex_spmv).  data: P planes with plane stride      */
/* dstride; x: P planes with stride xs; y: P planes with stride ys.           */
/* Each row is accumulated left to right: s := s + a_k * x_{col_k}.           */
/* mixed != 0: the matrix has one binary64 plane (two if complex) and the     */
/* products use the MP x binary64 forms (Algorithms 3-5, "M" mode).           */
/* ------------------------------------------------------------------------- */
static void spmv_row(int L, int cplx, int mixed, int64_t i, const int64_t* indptr, const int32_t* indices,
                     const double* data, int64_t dstride, const double* x, int64_t xs, double* sr, double* si) {
  double a[4], ai[4], xr[4], xi[4], t[4];
  mp_zero(L, sr);
  mp_zero(L, si);
  for (int64_t k = indptr[i]; k < indptr[i + 1]; k++) {
    int64_t j = indices[k];
    for (int l = 0; l < L; l++) xr[l] = x[(int64_t)l * xs + j];
    if (cplx) for (int l = 0; l < L; l++) xi[l] = x[(int64_t)(L + l) * xs + j];
    if (mixed) {
      double ad = data[k];
      mp_mul_d(L, xr, ad, t);
      mp_add(L, sr, t, sr);
      if (cplx) {
        double aid = data[dstride + k];
        mp_mul_d(L, xi, aid, t);
        mp_neg(L, t, t);
        mp_add(L, sr, t, sr);
        mp_mul_d(L, xi, ad, t);
        mp_add(L, si, t, si);
        mp_mul_d(L, xr, aid, t);
        mp_add(L, si, t, si);
      }
    } else {
      for (int l = 0; l < L; l++) a[l] = data[(int64_t)l * dstride + k];
      mp_mul(L, a, xr, t);
      mp_add(L, sr, t, sr);
      if (cplx) {
        for (int l = 0; l < L; l++) ai[l] = data[(int64_t)(L + l) * dstride + k];
        mp_mul(L, ai, xi, t);     /* re -= A_im x_im */
        mp_neg(L, t, t);
        mp_add(L, sr, t, sr);
        mp_mul(L, a, xi, t);      /* im += A_re x_im */
        mp_add(L, si, t, si);
        mp_mul(L, ai, xr, t);     /* im += A_im x_re */
        mp_add(L, si, t, si);
      }
    }
  }
}

void oracle_spmv(int L, int cplx, int mixed, int64_t nrows, const int64_t* indptr, const int32_t* indices,
                 const double* data, int64_t dstride, const double* x, int64_t xs, double* y, int64_t ys) {
  double sr[4], si[4];
  for (int64_t i = 0; i < nrows; i++) {
    spmv_row(L, cplx, mixed, i, indptr, indices, data, dstride, x, xs, sr, si);
    for (int l = 0; l < L; l++) y[(int64_t)l * ys + i] = sr[l];
    if (cplx) for (int l = 0; l < L; l++) y[(int64_t)(L + l) * ys + i] = si[l];
  }
}

/* SpTMV y = A^T x (Section 4, "A^T v"; complex: transpose, no conjugation),
 * in the row-oriented scatter form: rows i in increasing order, and each
 * stored entry a_ik of row i adds a_ik x_i into y_k.  Every y_k therefore
 * sums its products in increasing i, starting from zero.  x: P planes of
 * nrows (stride xs); y: P planes of ncols (stride ys), overwritten.  The
 * products and signs of one entry follow spmv_row. */
void oracle_spmtv(int L, int cplx, int mixed, int64_t nrows, int64_t ncols, const int64_t* indptr,
                  const int32_t* indices, const double* data, int64_t dstride, const double* x, int64_t xs,
                  double* y, int64_t ys) {
  int P = cplx ? 2 * L : L;
  for (int p = 0; p < P; p++)
    for (int64_t j = 0; j < ncols; j++) y[(int64_t)p * ys + j] = 0.0;
  for (int64_t i = 0; i < nrows; i++) {
    double xr[4], xi[4], a[4], ai[4], t[4], yr[4], yi[4];
    for (int l = 0; l < L; l++) xr[l] = x[(int64_t)l * xs + i];
    if (cplx) for (int l = 0; l < L; l++) xi[l] = x[(int64_t)(L + l) * xs + i];
    for (int64_t k = indptr[i]; k < indptr[i + 1]; k++) {
      int64_t j = indices[k];
      for (int l = 0; l < L; l++) yr[l] = y[(int64_t)l * ys + j];
      if (cplx) for (int l = 0; l < L; l++) yi[l] = y[(int64_t)(L + l) * ys + j];
      if (mixed) {
        double ad = data[k];
        mp_mul_d(L, xr, ad, t);
        mp_add(L, yr, t, yr);
        if (cplx) {
          double aid = data[dstride + k];
          mp_mul_d(L, xi, aid, t);
          mp_neg(L, t, t);
          mp_add(L, yr, t, yr);
          mp_mul_d(L, xi, ad, t);
          mp_add(L, yi, t, yi);
          mp_mul_d(L, xr, aid, t);
          mp_add(L, yi, t, yi);
        }
      } else {
        for (int l = 0; l < L; l++) a[l] = data[(int64_t)l * dstride + k];
        mp_mul(L, a, xr, t);
        mp_add(L, yr, t, yr);
        if (cplx) {
          for (int l = 0; l < L; l++) ai[l] = data[(int64_t)(L + l) * dstride + k];
          mp_mul(L, ai, xi, t);
          mp_neg(L, t, t);
          mp_add(L, yr, t, yr);
          mp_mul(L, a, xi, t);
          mp_add(L, yi, t, yi);
          mp_mul(L, ai, xr, t);
          mp_add(L, yi, t, yi);
        }
      }
      for (int l = 0; l < L; l++) y[(int64_t)l * ys + j] = yr[l];
      if (cplx) for (int l = 0; l < L; l++) y[(int64_t)(L + l) * ys + j] = yi[l];
    }
  }
}

/* Selected rows only: y is P planes of nsel (row rows[s] goes to column s). */
void oracle_spmv_rows(int L, int cplx, int mixed, int64_t nsel, const int64_t* rows, const int64_t* indptr,
                      const int32_t* indices, const double* data, int64_t dstride, const double* x, int64_t xs,
                      double* y) {
  double sr[4], si[4];
  for (int64_t s = 0; s < nsel; s++) {
    spmv_row(L, cplx, mixed, rows[s], indptr, indices, data, dstride, x, xs, sr, si);
    for (int l = 0; l < L; l++) y[(int64_t)l * nsel + s] = sr[l];
    if (cplx) for (int l = 0; l < L; l++) y[(int64_t)(L + l) * nsel + s] = si[l];
  }
}

/* SpMM: Y(:,c) = A X(:,c) for c < k.  X plane p, row j, column c sits at
 * X[p*xplane + j*ldx + c]; Y likewise with yplane and ldy. */
void oracle_spmm(int L, int cplx, int64_t nrows, int64_t ncols, const int64_t* indptr, const int32_t* indices,
                 const double* data, int64_t dstride, int k, const double* X, int64_t ldx, int64_t xplane,
                 double* Y, int64_t ldy, int64_t yplane) {
  int P = cplx ? 2 * L : L;
  double* xc = (double*)malloc(sizeof(double) * (size_t)(P * (ncols > 0 ? ncols : 1)));
  double* yc = (double*)malloc(sizeof(double) * (size_t)(P * (nrows > 0 ? nrows : 1)));
  for (int c = 0; c < k; c++) {
    for (int p = 0; p < P; p++)
      for (int64_t j = 0; j < ncols; j++) xc[(int64_t)p * ncols + j] = X[(int64_t)p * xplane + j * ldx + c];
    oracle_spmv(L, cplx, 0, nrows, indptr, indices, data, dstride, xc, ncols, yc, nrows);
    for (int p = 0; p < P; p++)
      for (int64_t i = 0; i < nrows; i++) Y[(int64_t)p * yplane + i * ldy + c] = yc[(int64_t)p * nrows + i];
  }
  free(xc);
  free(yc);
}

/* ------------------------------------------------------------------------- */
/* Vector operations for the Krylov methods.  A vector is P planes of n.      */
/* ------------------------------------------------------------------------- */
typedef struct {
  int L, cplx;
  int64_t n;
} vshape_t;

static void vget(const vshape_t* s, const double* v, int64_t i, double* re, double* im) {
  for (int l = 0; l < s->L; l++) re[l] = v[(int64_t)l * s->n + i];
  if (s->cplx) for (int l = 0; l < s->L; l++) im[l] = v[(int64_t)(s->L + l) * s->n + i];
  else mp_zero(s->L, im);
}
static void vset(const vshape_t* s, double* v, int64_t i, const double* re, const double* im) {
  for (int l = 0; l < s->L; l++) v[(int64_t)l * s->n + i] = re[l];
  if (s->cplx) for (int l = 0; l < s->L; l++) v[(int64_t)(s->L + l) * s->n + i] = im[l];
}

/* dot = sum_i conj(u_i) v_i, accumulated in index order. */
static void vdot(const vshape_t* s, const double* u, const double* v, double* dr, double* di) {
  int L = s->L;
  mp_zero(L, dr);
  mp_zero(L, di);
  for (int64_t i = 0; i < s->n; i++) {
    double ur[4], ui[4], vr[4], vi[4], t[4];
    vget(s, u, i, ur, ui);
    vget(s, v, i, vr, vi);
    mp_mul(L, ur, vr, t);
    mp_add(L, dr, t, dr);
    if (s->cplx) {
      mp_mul(L, ui, vi, t);      /* re += u_im v_im */
      mp_add(L, dr, t, dr);
      mp_mul(L, ur, vi, t);      /* im += u_re v_im */
      mp_add(L, di, t, di);
      mp_mul(L, ui, vr, t);      /* im -= u_im v_re */
      mp_neg(L, t, t);
      mp_add(L, di, t, di);
    }
  }
}

/* w := u + alpha * v  (w may alias u or v) */
static void vaxpy(const vshape_t* s, const double* ar, const double* ai, const double* u, const double* v,
                  double* w) {
  int L = s->L;
  for (int64_t i = 0; i < s->n; i++) {
    double ur[4], ui[4], vr[4], vi[4], tr[4], ti[4], rr[4], ri[4];
    vget(s, u, i, ur, ui);
    vget(s, v, i, vr, vi);
    if (s->cplx) {
      cmp_mul(L, ar, ai, vr, vi, tr, ti);
      mp_add(L, ur, tr, rr);
      mp_add(L, ui, ti, ri);
    } else {
      mp_mul(L, ar, vr, tr);
      mp_add(L, ur, tr, rr);
    }
    vset(s, w, i, rr, ri);
  }
}

/* binary64 value of ||v||_2 from the MP sum of squares. */
static double vnorm(const vshape_t* s, const double* v) {
  double dr[4], di[4];
  vdot(s, v, v, dr, di);
  double t = 0.0;
  for (int l = s->L - 1; l >= 0; l--) t += dr[l];
  if (isnan(t)) return t;  /* a NaN must not read as a zero norm */
  return sqrt(t > 0.0 ? t : 0.0);
}

typedef struct {
  int L, cplx, mixed;
  int64_t n;
  const int64_t* indptr;
  const int32_t* indices;
  const double* data;
  int64_t dstride;
} mat_t;

static void matvec(const mat_t* A, const double* x, double* y) {
  oracle_spmv(A->L, A->cplx, A->mixed, A->n, A->indptr, A->indices, A->data, A->dstride, x, A->n, y, A->n);
}

/* r := b - A x */
static void residual(const mat_t* A, const vshape_t* s, const double* b, const double* x, double* r) {
  double one_r[4] = {-1.0, 0, 0, 0}, zero[4] = {0, 0, 0, 0};
  matvec(A, x, r);
  vaxpy(s, one_r, zero, b, r, r);
}

/* Status codes shared in meaning (not in code) with the CUDA library. */
#define OR_OK 0
#define OR_EBREAKDOWN (-5)
#define OR_ENOCONV (-6)

static int mp_is_zero(int L, const double* a) { (void)L; return a[0] == 0.0; }

/* Conjugate gradient (Hestenes-Stiefel), x0 = the given x.  Stops when the
 * recurrence residual satisfies ||r_k|| <= rtol*||b|| + atol (Section 4.2
 * stopping test with its constants as parameters).  Real only.
 * Outputs: iterations taken, and the binary64 norm of the true residual
 * b - A x at exit relative to ||b||. */
int oracle_cg(int L, int64_t n, const int64_t* indptr, const int32_t* indices, const double* data,
              int64_t dstride, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
              double* relres) {
  vshape_t s = {L, 0, n};
  mat_t A = {L, 0, 0, n, indptr, indices, data, dstride};
  size_t bytes = sizeof(double) * (size_t)(L * (n > 0 ? n : 1));
  double *r = malloc(bytes), *p = malloc(bytes), *q = malloc(bytes);
  double zero[4] = {0, 0, 0, 0};
  int status = OR_ENOCONV, k = 0;
  double bnorm = vnorm(&s, b);
  double tol = rtol * bnorm + atol;
  residual(&A, &s, b, x, r);
  memcpy(p, r, bytes);
  double rho[4], di[4];
  vdot(&s, r, r, rho, di);
  if (vnorm(&s, r) <= tol) status = OR_OK;
  while (status != OR_OK && k < maxit) {
    double pq[4], alpha[4], nalpha[4], rho1[4], beta[4];
    matvec(&A, p, q);
    vdot(&s, p, q, pq, di);
    if (mp_is_zero(L, pq) || !isfinite(pq[0])) { status = OR_EBREAKDOWN; break; }
    mp_div(L, rho, pq, alpha);
    vaxpy(&s, alpha, zero, x, p, x);
    mp_neg(L, alpha, nalpha);
    vaxpy(&s, nalpha, zero, r, q, r);
    vdot(&s, r, r, rho1, di);
    k++;
    double t = 0.0;
    for (int l = L - 1; l >= 0; l--) t += rho1[l];
    if (!isfinite(t)) { status = OR_EBREAKDOWN; break; }
    if (sqrt(t > 0 ? t : 0) <= tol) { status = OR_OK; break; }
    if (mp_is_zero(L, rho)) { status = OR_EBREAKDOWN; break; }
    mp_div(L, rho1, rho, beta);
    vaxpy(&s, beta, zero, r, p, p);
    mp_copy(L, rho1, rho);
  }
  residual(&A, &s, b, x, r);
  *iters = k;
  *relres = bnorm > 0 ? vnorm(&s, r) / bnorm : vnorm(&s, r);
  free(r); free(p); free(q);
  return status;
}

/* BiCGSTAB (van der Vorst 1992), real or complex, r_hat = r_0, x0 = the given
 * x; stopping test as in oracle_cg. */
int oracle_bicgstab(int L, int cplx, int64_t n, const int64_t* indptr, const int32_t* indices,
                    const double* data, int64_t dstride, const double* b, double* x, double rtol, double atol,
                    int maxit, int* iters, double* relres) {
  vshape_t s = {L, cplx, n};
  mat_t A = {L, cplx, 0, n, indptr, indices, data, dstride};
  int P = cplx ? 2 * L : L;
  size_t bytes = sizeof(double) * (size_t)(P * (n > 0 ? n : 1));
  double *r = malloc(bytes), *rh = malloc(bytes), *p = calloc(1, bytes), *v = calloc(1, bytes);
  double *sv = malloc(bytes), *t = malloc(bytes);
  int status = OR_ENOCONV, k = 0;
  double bnorm = vnorm(&s, b);
  double tol = rtol * bnorm + atol;
  residual(&A, &s, b, x, r);
  memcpy(rh, r, bytes);
  double rho_r[4] = {1, 0, 0, 0}, rho_i[4] = {0, 0, 0, 0};
  double al_r[4] = {1, 0, 0, 0}, al_i[4] = {0, 0, 0, 0};
  double om_r[4] = {1, 0, 0, 0}, om_i[4] = {0, 0, 0, 0};
  if (vnorm(&s, r) <= tol) status = OR_OK;
  while (status != OR_OK && k < maxit) {
    double r1r[4], r1i[4], tr[4], ti[4], br[4], bi[4], nr[4], ni[4], dr[4], di[4];
    vdot(&s, rh, r, r1r, r1i);
    if (mp_is_zero(L, r1r) && (!cplx || mp_is_zero(L, r1i))) { status = OR_EBREAKDOWN; break; }
    /* beta = (rho1/rho) * (alpha/omega) */
    if (cplx) {
      cmp_div(L, r1r, r1i, rho_r, rho_i, tr, ti);
      cmp_div(L, al_r, al_i, om_r, om_i, nr, ni);
      cmp_mul(L, tr, ti, nr, ni, br, bi);
    } else {
      mp_div(L, r1r, rho_r, tr);
      mp_div(L, al_r, om_r, nr);
      mp_mul(L, tr, nr, br);
      mp_zero(L, bi);
    }
    /* p = r + beta * (p - omega v) */
    mp_neg(L, om_r, nr);
    mp_neg(L, om_i, ni);
    vaxpy(&s, nr, ni, p, v, p);
    vaxpy(&s, br, bi, r, p, p);
    matvec(&A, p, v);
    vdot(&s, rh, v, dr, di);
    if (mp_is_zero(L, dr) && (!cplx || mp_is_zero(L, di))) { status = OR_EBREAKDOWN; break; }
    if (cplx) cmp_div(L, r1r, r1i, dr, di, al_r, al_i);
    else { mp_div(L, r1r, dr, al_r); mp_zero(L, al_i); }
    /* s = r - alpha v */
    mp_neg(L, al_r, nr);
    mp_neg(L, al_i, ni);
    vaxpy(&s, nr, ni, r, v, sv);
    k++;
    double snorm = vnorm(&s, sv);
    if (!isfinite(snorm)) { status = OR_EBREAKDOWN; break; }
    if (snorm <= tol) {
      vaxpy(&s, al_r, al_i, x, p, x);
      status = OR_OK;
      break;
    }
    matvec(&A, sv, t);
    double ttr[4], tti[4];
    vdot(&s, t, sv, nr, ni);
    vdot(&s, t, t, ttr, tti);
    if (mp_is_zero(L, ttr)) { status = OR_EBREAKDOWN; break; }
    if (cplx) cmp_div(L, nr, ni, ttr, tti, om_r, om_i);
    else { mp_div(L, nr, ttr, om_r); mp_zero(L, om_i); }
    /* x = x + alpha p + omega s ; r = s - omega t */
    vaxpy(&s, al_r, al_i, x, p, x);
    vaxpy(&s, om_r, om_i, x, sv, x);
    mp_neg(L, om_r, nr);
    mp_neg(L, om_i, ni);
    vaxpy(&s, nr, ni, sv, t, r);
    double rn = vnorm(&s, r);
    if (!isfinite(rn)) { status = OR_EBREAKDOWN; break; }
    if (rn <= tol) { status = OR_OK; break; }
    if (mp_is_zero(L, om_r) && (!cplx || mp_is_zero(L, om_i))) { status = OR_EBREAKDOWN; break; }
    mp_copy(L, r1r, rho_r);
    mp_copy(L, r1i, rho_i);
  }
  residual(&A, &s, b, x, r);
  *iters = k;
  *relres = bnorm > 0 ? vnorm(&s, r) / bnorm : vnorm(&s, r);
  (void)P;
  free(r); free(rh); free(p); free(v); free(sv); free(t);
  return status;
}

/* ------------------------------------------------------------------------- */
/* BiCG, CGS and GPBiCG: the other product-type Krylov methods of Section     */
/* 4.2, in their textbook forms, every vector and scalar in the working       */
/* precision, inner products (u, v) = sum conj(u_i) v_i, x0 = the given x,    */
/* stopping test as in oracle_cg (recurrence residual).                       */
/* ------------------------------------------------------------------------- */
typedef struct {
  double re[4], im[4];
} cscal_t;

static cscal_t cs_real(int L, double v) {
  cscal_t a;
  mp_zero(L, a.re);
  mp_zero(L, a.im);
  a.re[0] = v;
  return a;
}
static int cs_is_zero(int L, int cplx, const cscal_t* a) {
  return mp_is_zero(L, a->re) && (!cplx || mp_is_zero(L, a->im));
}
static cscal_t cs_mul(int L, int cplx, const cscal_t* a, const cscal_t* b) {
  cscal_t r;
  if (cplx) {
    cmp_mul(L, a->re, a->im, b->re, b->im, r.re, r.im);
  } else {
    mp_mul(L, a->re, b->re, r.re);
    mp_zero(L, r.im);
  }
  return r;
}
static cscal_t cs_div(int L, int cplx, const cscal_t* a, const cscal_t* b) {
  cscal_t r;
  if (cplx) {
    cmp_div(L, a->re, a->im, b->re, b->im, r.re, r.im);
  } else {
    mp_div(L, a->re, b->re, r.re);
    mp_zero(L, r.im);
  }
  return r;
}
static cscal_t cs_sub(int L, const cscal_t* a, const cscal_t* b) {
  cscal_t r;
  mp_sub(L, a->re, b->re, r.re);
  mp_sub(L, a->im, b->im, r.im);
  return r;
}
static cscal_t cs_neg(int L, const cscal_t* a) {
  cscal_t r;
  mp_neg(L, a->re, r.re);
  mp_neg(L, a->im, r.im);
  return r;
}
static cscal_t cs_conj(int L, const cscal_t* a) {
  cscal_t r;
  mp_copy(L, a->re, r.re);
  mp_neg(L, a->im, r.im);
  return r;
}
static cscal_t cs_dot(const vshape_t* s, const double* u, const double* v) {
  cscal_t r;
  vdot(s, u, v, r.re, r.im);
  return r;
}
/* w := u + alpha v */
static void cs_axpy(const vshape_t* s, const cscal_t* alpha, const double* u, const double* v, double* w) {
  vaxpy(s, alpha->re, alpha->im, u, v, w);
}
/* w := a v */
static void vscale(const vshape_t* s, const cscal_t* a, const double* v, double* w) {
  int L = s->L;
  for (int64_t i = 0; i < s->n; i++) {
    double vr[4], vi[4], rr[4], ri[4];
    vget(s, v, i, vr, vi);
    if (s->cplx) {
      cmp_mul(L, a->re, a->im, vr, vi, rr, ri);
    } else {
      mp_mul(L, a->re, vr, rr);
    }
    vset(s, w, i, rr, ri);
  }
}
/* v := conj(v) (negate the imaginary planes) */
static void vconj(const vshape_t* s, double* v) {
  if (!s->cplx) return;
  for (int64_t q = (int64_t)s->L * s->n; q < (int64_t)2 * s->L * s->n; q++) v[q] = -v[q];
}

/* y := A^H x = conj(A^T conj(x)) (the definition, through the transpose
 * product oracle_spmtv); tmp has the size of x. */
static void matvec_adj(const mat_t* A, const vshape_t* s, const double* x, double* y, double* tmp) {
  size_t bytes = sizeof(double) * (size_t)((s->cplx ? 2 : 1) * s->L * s->n);
  memcpy(tmp, x, bytes);
  vconj(s, tmp);
  oracle_spmtv(A->L, A->cplx, A->mixed, A->n, A->n, A->indptr, A->indices, A->data, A->dstride, tmp, A->n, y,
               A->n);
  vconj(s, y);
}

/* BiCG (Fletcher 1976): shadow residual r~_0 = r_0, shadow products with A^H.
 *   q = A p, q~ = A^H p~, alpha = rho / (p~, q),
 *   x += alpha p, r -= alpha q, r~ -= conj(alpha) q~,
 *   rho' = (r~, r), beta = rho' / rho, p = r + beta p, p~ = r~ + conj(beta) p~. */
int oracle_bicg(int L, int cplx, int64_t n, const int64_t* indptr, const int32_t* indices, const double* data,
                int64_t dstride, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
                double* relres) {
  vshape_t s = {L, cplx, n};
  mat_t A = {L, cplx, 0, n, indptr, indices, data, dstride};
  size_t bytes = sizeof(double) * (size_t)((cplx ? 2 : 1) * L * (n > 0 ? n : 1));
  double *r = malloc(bytes), *rt = malloc(bytes), *p = malloc(bytes), *pt = malloc(bytes);
  double *q = malloc(bytes), *qt = malloc(bytes), *tmp = malloc(bytes);
  int status = OR_ENOCONV, k = 0;
  double bnorm = vnorm(&s, b);
  double tol = rtol * bnorm + atol;
  residual(&A, &s, b, x, r);
  memcpy(rt, r, bytes);
  memcpy(p, r, bytes);
  memcpy(pt, rt, bytes);
  cscal_t rho = cs_dot(&s, rt, r);
  if (vnorm(&s, r) <= tol) status = OR_OK;
  while (status != OR_OK && k < maxit) {
    if (cs_is_zero(L, cplx, &rho)) { status = OR_EBREAKDOWN; break; }
    matvec(&A, p, q);
    matvec_adj(&A, &s, pt, qt, tmp);
    cscal_t sigma = cs_dot(&s, pt, q);
    if (cs_is_zero(L, cplx, &sigma) || !isfinite(sigma.re[0])) { status = OR_EBREAKDOWN; break; }
    cscal_t alpha = cs_div(L, cplx, &rho, &sigma);
    cscal_t nalpha = cs_neg(L, &alpha);
    cscal_t nalpha_c = cs_conj(L, &nalpha);
    cs_axpy(&s, &alpha, x, p, x);
    cs_axpy(&s, &nalpha, r, q, r);
    cs_axpy(&s, &nalpha_c, rt, qt, rt);
    k++;
    double rn = vnorm(&s, r);
    if (!isfinite(rn)) { status = OR_EBREAKDOWN; break; }
    if (rn <= tol) { status = OR_OK; break; }
    cscal_t rho1 = cs_dot(&s, rt, r);
    cscal_t beta = cs_div(L, cplx, &rho1, &rho);
    cscal_t beta_c = cs_conj(L, &beta);
    cs_axpy(&s, &beta, r, p, p);
    cs_axpy(&s, &beta_c, rt, pt, pt);
    rho = rho1;
  }
  residual(&A, &s, b, x, r);
  *iters = k;
  *relres = bnorm > 0 ? vnorm(&s, r) / bnorm : vnorm(&s, r);
  free(r); free(rt); free(p); free(pt); free(q); free(qt); free(tmp);
  return status;
}

/* CGS (Sonneveld 1989), r^ = r_0:
 *   v = A p, alpha = rho / (r^, v), q = u - alpha v, w = u + q,
 *   x += alpha w, r -= alpha A w, rho' = (r^, r), beta = rho' / rho,
 *   u = r + beta q, p = u + beta (q + beta p). */
int oracle_cgs(int L, int cplx, int64_t n, const int64_t* indptr, const int32_t* indices, const double* data,
               int64_t dstride, const double* b, double* x, double rtol, double atol, int maxit, int* iters,
               double* relres) {
  vshape_t s = {L, cplx, n};
  mat_t A = {L, cplx, 0, n, indptr, indices, data, dstride};
  size_t bytes = sizeof(double) * (size_t)((cplx ? 2 : 1) * L * (n > 0 ? n : 1));
  double *r = malloc(bytes), *rh = malloc(bytes), *p = malloc(bytes), *u = malloc(bytes);
  double *v = malloc(bytes), *q = malloc(bytes), *w = malloc(bytes), *t = malloc(bytes);
  int status = OR_ENOCONV, k = 0;
  cscal_t one = cs_real(L, 1.0);
  double bnorm = vnorm(&s, b);
  double tol = rtol * bnorm + atol;
  residual(&A, &s, b, x, r);
  memcpy(rh, r, bytes);
  memcpy(u, r, bytes);
  memcpy(p, r, bytes);
  cscal_t rho = cs_dot(&s, rh, r);
  if (vnorm(&s, r) <= tol) status = OR_OK;
  while (status != OR_OK && k < maxit) {
    if (cs_is_zero(L, cplx, &rho)) { status = OR_EBREAKDOWN; break; }
    matvec(&A, p, v);
    cscal_t sigma = cs_dot(&s, rh, v);
    if (cs_is_zero(L, cplx, &sigma) || !isfinite(sigma.re[0])) { status = OR_EBREAKDOWN; break; }
    cscal_t alpha = cs_div(L, cplx, &rho, &sigma);
    cscal_t nalpha = cs_neg(L, &alpha);
    cs_axpy(&s, &nalpha, u, v, q);
    cs_axpy(&s, &one, u, q, w);
    cs_axpy(&s, &alpha, x, w, x);
    matvec(&A, w, t);
    cs_axpy(&s, &nalpha, r, t, r);
    k++;
    double rn = vnorm(&s, r);
    if (!isfinite(rn)) { status = OR_EBREAKDOWN; break; }
    if (rn <= tol) { status = OR_OK; break; }
    cscal_t rho1 = cs_dot(&s, rh, r);
    cscal_t beta = cs_div(L, cplx, &rho1, &rho);
    cs_axpy(&s, &beta, r, q, u);
    cs_axpy(&s, &beta, q, p, p);
    cs_axpy(&s, &beta, u, p, p);
    rho = rho1;
  }
  residual(&A, &s, b, x, r);
  *iters = k;
  *relres = bnorm > 0 ? vnorm(&s, r) / bnorm : vnorm(&s, r);
  free(r); free(rh); free(p); free(u); free(v); free(q); free(w); free(t);
  return status;
}

/* GPBiCG (Zhang 1997), r^ = r_0, t_{-1} = w_{-1} = u_{-1} = z_{-1} = 0,
 * beta_{-1} = 0.  Per iteration k:
 *   p = r + beta (p - u), alpha = rho / (r^, A p),
 *   y = t_prev - r - alpha w + alpha A p, t = r - alpha A p
 *   (if ||t|| meets the test: x += alpha p and stop),
 *   zeta, eta minimise || t - zeta A t - eta y || (eta = 0 when k = 0):
 *     a = (At, At), b = (y, y), c = (At, y), d = (At, t), e = (y, t),
 *     det = a b - c conj(c), zeta = (b d - c e) / det, eta = (a e - conj(c) d) / det,
 *   u = zeta A p + eta (t_prev - r + beta u), z = zeta r + eta z - alpha u,
 *   x += alpha p + z, r = t - eta y - zeta A t,
 *   beta = (alpha / zeta) (r^, r_new) / (r^, r_old), w = A t + beta A p. */
int oracle_gpbicg(int L, int cplx, int64_t n, const int64_t* indptr, const int32_t* indices,
                  const double* data, int64_t dstride, const double* b, double* x, double rtol, double atol,
                  int maxit, int* iters, double* relres) {
  vshape_t s = {L, cplx, n};
  mat_t A = {L, cplx, 0, n, indptr, indices, data, dstride};
  size_t bytes = sizeof(double) * (size_t)((cplx ? 2 : 1) * L * (n > 0 ? n : 1));
  double *r = malloc(bytes), *rh = malloc(bytes), *p = calloc(1, bytes), *u = calloc(1, bytes);
  double *z = calloc(1, bytes), *w = calloc(1, bytes), *tp = calloc(1, bytes), *t = malloc(bytes);
  double *ap = malloc(bytes), *at = malloc(bytes), *y = malloc(bytes), *tmp = malloc(bytes);
  int status = OR_ENOCONV, k = 0;
  const cscal_t one = cs_real(L, 1.0), mone = cs_real(L, -1.0);
  cscal_t beta = cs_real(L, 0.0);
  double bnorm = vnorm(&s, b);
  double tol = rtol * bnorm + atol;
  residual(&A, &s, b, x, r);
  memcpy(rh, r, bytes);
  cscal_t rho = cs_dot(&s, rh, r);
  if (vnorm(&s, r) <= tol) status = OR_OK;
  while (status != OR_OK && k < maxit) {
    if (cs_is_zero(L, cplx, &rho)) { status = OR_EBREAKDOWN; break; }
    cs_axpy(&s, &mone, p, u, tmp);            /* p = r + beta (p - u) */
    cs_axpy(&s, &beta, r, tmp, p);
    matvec(&A, p, ap);
    cscal_t sigma = cs_dot(&s, rh, ap);
    if (cs_is_zero(L, cplx, &sigma) || !isfinite(sigma.re[0])) { status = OR_EBREAKDOWN; break; }
    cscal_t alpha = cs_div(L, cplx, &rho, &sigma);
    cscal_t nalpha = cs_neg(L, &alpha);
    cs_axpy(&s, &mone, tp, r, y);             /* y = t_prev - r - alpha w + alpha A p */
    cs_axpy(&s, &nalpha, y, w, y);
    cs_axpy(&s, &alpha, y, ap, y);
    cs_axpy(&s, &nalpha, r, ap, t);           /* t = r - alpha A p */
    /* t is the residual of x + alpha p: stop there when it already meets
       the test (as BiCGSTAB stops on s); the minimisation below would
       otherwise work on rounding-level vectors */
    double tn = vnorm(&s, t);
    if (!isfinite(tn)) { status = OR_EBREAKDOWN; break; }
    if (tn <= tol) {
      cs_axpy(&s, &alpha, x, p, x);
      k++;
      status = OR_OK;
      break;
    }
    matvec(&A, t, at);
    cscal_t zeta, eta;
    if (k == 0) {
      cscal_t d = cs_dot(&s, at, t), a = cs_dot(&s, at, at);
      if (cs_is_zero(L, cplx, &a)) { status = OR_EBREAKDOWN; break; }
      zeta = cs_div(L, cplx, &d, &a);
      eta = cs_real(L, 0.0);
    } else {
      cscal_t a = cs_dot(&s, at, at), bb = cs_dot(&s, y, y), c = cs_dot(&s, at, y);
      cscal_t d = cs_dot(&s, at, t), e = cs_dot(&s, y, t);
      cscal_t cc = cs_conj(L, &c);
      cscal_t ab = cs_mul(L, cplx, &a, &bb), c2 = cs_mul(L, cplx, &c, &cc);
      cscal_t det = cs_sub(L, &ab, &c2);
      if (cs_is_zero(L, cplx, &det)) { status = OR_EBREAKDOWN; break; }
      cscal_t bd = cs_mul(L, cplx, &bb, &d), ce = cs_mul(L, cplx, &c, &e);
      cscal_t ae = cs_mul(L, cplx, &a, &e), cd = cs_mul(L, cplx, &cc, &d);
      cscal_t zn = cs_sub(L, &bd, &ce), en = cs_sub(L, &ae, &cd);
      zeta = cs_div(L, cplx, &zn, &det);
      eta = cs_div(L, cplx, &en, &det);
    }
    if (cs_is_zero(L, cplx, &zeta)) { status = OR_EBREAKDOWN; break; }
    cscal_t neta = cs_neg(L, &eta), nzeta = cs_neg(L, &zeta);
    cs_axpy(&s, &mone, tp, r, tmp);           /* u = zeta A p + eta (t_prev - r + beta u) */
    cs_axpy(&s, &beta, tmp, u, tmp);
    vscale(&s, &eta, tmp, tmp);
    cs_axpy(&s, &zeta, tmp, ap, u);
    vscale(&s, &eta, z, z);                   /* z = zeta r + eta z - alpha u */
    cs_axpy(&s, &zeta, z, r, z);
    cs_axpy(&s, &nalpha, z, u, z);
    cs_axpy(&s, &alpha, x, p, x);             /* x += alpha p + z */
    cs_axpy(&s, &one, x, z, x);
    cs_axpy(&s, &neta, t, y, r);              /* r = t - eta y - zeta A t */
    cs_axpy(&s, &nzeta, r, at, r);
    k++;
    double rn = vnorm(&s, r);
    if (!isfinite(rn)) { status = OR_EBREAKDOWN; break; }
    if (rn <= tol) { status = OR_OK; break; }
    cscal_t rho1 = cs_dot(&s, rh, r);
    cscal_t az = cs_div(L, cplx, &alpha, &zeta), rr = cs_div(L, cplx, &rho1, &rho);
    beta = cs_mul(L, cplx, &az, &rr);
    cs_axpy(&s, &beta, at, ap, w);            /* w = A t + beta A p */
    memcpy(tp, t, bytes);
    rho = rho1;
  }
  residual(&A, &s, b, x, r);
  *iters = k;
  *relres = bnorm > 0 ? vnorm(&s, r) / bnorm : vnorm(&s, r);
  free(r); free(rh); free(p); free(u); free(z); free(w); free(tp); free(t);
  free(ap); free(at); free(y); free(tmp);
  return status;
}

/* Exported vector helpers for tests. */
void oracle_dot(int L, int cplx, int64_t n, const double* u, const double* v, double* dr, double* di) {
  vshape_t s = {L, cplx, n};
  vdot(&s, u, v, dr, di);
}
void oracle_axpy(int L, int cplx, int64_t n, const double* ar, const double* ai, const double* u,
                 const double* v, double* w) {
  vshape_t s = {L, cplx, n};
  vaxpy(&s, ar, ai, u, v, w);
}
