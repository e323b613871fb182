"""Exact dyadic reference for multiple-precision SpMV (test infrastructure).

Every component of a DD/TD/QD number is a binary64, i.e. an integer times
2**-1074, so a row sum  y_i = sum_k a_k * x_{col_k}  of such numbers is an exact
integer multiple of 2**-2148.  This module evaluates it with Python integers,
rounds an exact value greedily to L binary64 components (hi = RN(y),
next = RN(y - hi), ...), and checks the componentwise acceptance bound

    |y_i - y_exact,i| <= c * m * u * (|A| |x|)_i ,

with m the maximum number of stored entries in a row and u = 2**-104,
2**-155, 2**-207 for DD, TD, QD (2**-53 for binary64).  For complex data the
bound for each component uses the sum of the moduli of the real products that
enter it (Eq. complex_spmv): |A_re||x_re| + |A_im||x_im| for the real part and
|A_re||x_im| + |A_im||x_re| for the imaginary part, with 2m terms.

Also builds the paper's sample vector v = sqrt(2)[1..n] (real) and
v = sqrt(2+3i)[1..n] (complex), Eq. sample_vector, from integer square roots
at 1200 bits.
"""
import math
from fractions import Fraction

import numpy as np

SCALE = 1074  # every binary64 is an integer multiple of 2**-1074
U = {1: 2.0 ** -53, 2: 2.0 ** -104, 3: 2.0 ** -155, 4: 2.0 ** -207}


def f2i(v):
    """Exact integer N with v = N * 2**-1074."""
    v = float(v)
    if v == 0.0 or not math.isfinite(v):
        if not math.isfinite(v):
            raise ValueError("non-finite value")
        return 0
    m, e = math.frexp(v)            # v = m * 2**e, 0.5 <= |m| < 1
    mi = int(m * (1 << 53))         # exact: 53-bit integer mantissa
    sh = e - 53 + SCALE
    return mi << sh if sh >= 0 else mi >> (-sh)  # sh < 0 never drops bits for binary64


def limbs_to_int(limbs):
    """Exact value of sum(limbs) as an integer multiple of 2**-1074."""
    return sum(f2i(v) for v in limbs)


def int_to_frac(N, scale):
    return Fraction(N, 1 << scale)


def round_greedy(value, L):
    """Greedy round-to-nearest of an exact Fraction to L binary64 components."""
    out = []
    rem = Fraction(value)
    for _ in range(L):
        h = float(rem) if rem != 0 else 0.0   # Fraction -> float is correctly rounded
        out.append(h)
        rem -= Fraction(h)
    return np.array(out)


def exact_rows(A, x, rows=None):
    """Exact row values of A x.  Returns (num_re, num_im, abs_re, abs_im) as
    lists of integers in units of 2**-2148; abs_* are (|A||x|)-style sums of
    the moduli of the products entering each component.  ``A`` is an
    ``oracle.CSR``; ``x`` has shape (P, ncols)."""
    L, cplx = A.L, A.cplx
    if rows is None:
        rows = range(A.nrows)
    xi = {}

    def xval(j):
        if j not in xi:
            re = limbs_to_int(x[:L, j])
            im = limbs_to_int(x[L:2 * L, j]) if cplx else 0
            xi[j] = (re, im)
        return xi[j]

    out_re, out_im, abs_re, abs_im = [], [], [], []
    for i in rows:
        sr = si = ar_ = ai_ = 0
        for k in range(A.indptr[i], A.indptr[i + 1]):
            j = int(A.indices[k])
            a_re = limbs_to_int(A.data[:L, k])
            a_im = limbs_to_int(A.data[L:2 * L, k]) if cplx else 0
            x_re, x_im = xval(j)
            p1 = a_re * x_re
            sr += p1
            ar_ += abs(p1)
            if cplx:
                p2, p3, p4 = a_im * x_im, a_re * x_im, a_im * x_re
                sr -= p2
                ar_ += abs(p2)
                si += p3 + p4
                ai_ += abs(p3) + abs(p4)
        out_re.append(sr)
        out_im.append(si)
        abs_re.append(ar_)
        abs_im.append(ai_)
    return out_re, out_im, abs_re, abs_im


def bound_ratio(y, A, x, rows=None, factor=8.0):
    """Max over the given rows and components of
    |y - y_exact| / (factor * m * u * (|A||x|)), computed exactly.  ``y`` has
    shape (P, len(rows)) (or (P, nrows) when rows is None).  A ratio <= 1
    means the bound holds.  Rows whose |A||x| is zero must have y == 0
    exactly (ratio 0 if so, inf otherwise)."""
    L, cplx = A.L, A.cplx
    rows = list(range(A.nrows)) if rows is None else list(rows)
    ex_re, ex_im, ab_re, ab_im = exact_rows(A, x, rows)
    rl = np.diff(A.indptr)
    m = int(rl.max()) if len(rl) else 0
    mm = 2 * m if cplx else m
    u = Fraction(U[L])
    worst = 0.0
    comps = [(ex_re, ab_re, 0)] + ([(ex_im, ab_im, L)] if cplx else [])
    for ex, ab, off in comps:
        for s in range(len(rows)):
            got = limbs_to_int(y[off:off + L, s]) << SCALE   # units of 2**-2148
            err = abs(got - ex[s])
            if ab[s] == 0:
                if err != 0:
                    return math.inf
                continue
            r = Fraction(err) / (Fraction(ab[s]) * u * Fraction(factor) * max(mm, 1))
            worst = max(worst, float(r))
    return worst


def exact_round_rows(A, x, rows=None):
    """Greedy L-component rounding of the exact row values, shape (P, nsel)."""
    L, cplx = A.L, A.cplx
    rows = list(range(A.nrows)) if rows is None else list(rows)
    ex_re, ex_im, _, _ = exact_rows(A, x, rows)
    P = 2 * L if cplx else L
    out = np.zeros((P, len(rows)))
    den = 2 * SCALE
    for s in range(len(rows)):
        out[:L, s] = round_greedy(Fraction(ex_re[s], 1 << den), L)
        if cplx:
            out[L:, s] = round_greedy(Fraction(ex_im[s], 1 << den), L)
    return out


# --------------------------------------------------------------------------
# The paper's sample vector (Eq. sample_vector)
# --------------------------------------------------------------------------
_BITS = 1200


def _isqrt_fixed(num, den, bits=_BITS):
    """floor(sqrt(num/den) * 2**bits) for non-negative integers."""
    return math.isqrt((num << (2 * bits)) // den)


def sqrt2_fixed(bits=_BITS):
    return _isqrt_fixed(2, 1, bits)


def sqrt_2p3i_fixed(bits=_BITS):
    """Principal square root of 2+3i, each part as floor(part * 2**bits).
    sqrt(a+bi) = sqrt((|z|+a)/2) + i sqrt((|z|-a)/2) for b > 0, |z| = sqrt(13)."""
    mod = math.isqrt(13 << (2 * (bits + 8)))          # |z| * 2**(bits+8)
    two = 2 << (bits + 8)
    re2 = (mod + two) // 2                            # (|z|+2)/2 * 2**(bits+8)
    im2 = (mod - two) // 2
    re = math.isqrt(re2 << (bits - 8))                # sqrt(v * 2**(bits+8) * 2**(bits-8))
    im = math.isqrt(im2 << (bits - 8))
    return re, im


def sample_vector(n, L, cplx=False):
    """v_j = c * j (j = 1..n) with c = sqrt(2) or sqrt(2+3i), rounded
    greedily to L components; shape (P, n).  The truncation of c at 1200
    bits is far below every format's unit roundoff."""
    P = 2 * L if cplx else L
    v = np.zeros((P, n))
    if cplx:
        cr, ci = sqrt_2p3i_fixed()
        parts = [(cr, 0), (ci, L)]
    else:
        parts = [(sqrt2_fixed(), 0)]
    for c, off in parts:
        for j in range(1, n + 1):
            v[off:off + L, j - 1] = round_greedy(Fraction(c * j, 1 << _BITS), L)
    return v


def to_fraction(limbs):
    return sum((Fraction(float(v)) for v in limbs), Fraction(0))
