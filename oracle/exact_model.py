"""Exact model of the exact-accumulation arithmetic (MPSPMV_EXACT_ACC), for
the parity checks of that path (test infrastructure, like the rest of this
package: only tests/, smoke() and bench.py's oracle leg use it).

The variant is defined by its terms, not by the paper's operation sequence:
every term is an integer times 2^-2148 (binary64 values are integers times
2^-1074); a stored entry a . x contributes the exact products a_i x_j below
the format's unit roundoff plus one FMA chain over the next order (for a
binary64 value a: the exact a x_j for j < L - 1 plus the rounded a x_{L-1});
a row (or a vector update u + alpha v) is the exact sum of its terms, cut to
L binary64 components by truncation of its magnitude.  The accumulator that
computes it keeps D digits of 32 bits and is exact while the terms span at
most 32 (D - 2) + 1 bits; comparisons use rows and elements within that
span.  Written with Python integers, independently of the CUDA sources.
"""
import math
from fractions import Fraction

import numpy as np

from . import exact
from . import two_prod as _two_prod

SC = 2 * exact.SCALE  # terms and products are integers times 2^-2148
DIGITS = {1: 4, 2: 6, 3: 8, 4: 10}  # accumulator digits per L (binary64, DD, TD, QD)


def window_bits(L):
    return 32 * (DIGITS[L] - 2) + 1


def rn_fma(a, b, c):
    """fl(a b + c) with one rounding (Fraction -> float rounds correctly)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def term(kind, a, b, neg):
    """kind 0: the binary64 a; kind 1: the exact product a b."""
    v = exact.f2i(a) << exact.SCALE if kind == 0 else exact.f2i(a) * exact.f2i(b)
    return -v if neg else v


def entry_terms(L, mode, a, x):
    """The terms one stored entry adds (mode 0: MP value a, mode 1: binary64
    value a[0]): exact products a_i x_j for i + j < L - 1 (a x_j for j < L - 1)
    and the FMA chain over i + j = L - 1 (the rounded a x_{L-1}); L = 1 with
    an MP value: the TwoProd pair."""
    if mode == 1:
        if L == 1:
            return [exact.f2i(a[0] * x[0]) << exact.SCALE]
        return [exact.f2i(a[0]) * exact.f2i(x[j]) for j in range(L - 1)] + [exact.f2i(a[0] * x[L - 1]) << exact.SCALE]
    if L == 1:
        p, e = _two_prod(a[0], x[0])
        return [exact.f2i(p) << exact.SCALE, exact.f2i(e) << exact.SCALE]
    terms = [exact.f2i(a[i]) * exact.f2i(x[j]) for i in range(L) for j in range(L) if i + j < L - 1]
    c = a[L - 1] * x[0]
    for i in range(L - 2, -1, -1):
        c = rn_fma(a[i], x[L - 1 - i], c)
    return terms + [exact.f2i(c) << exact.SCALE]


def cut(V, L):
    """V * 2^-2148 cut to L components by truncation of its magnitude."""
    out = np.zeros(L)
    if V == 0:
        return out
    s = -1.0 if V < 0 else 1.0
    m = abs(V)
    top = m.bit_length() - 1
    for l in range(L):
        lsb = top - 52 - 53 * l
        chunk = (m >> lsb) & ((1 << 53) - 1) if lsb >= 0 else (m << -lsb) & ((1 << 53) - 1)
        out[l] = s * math.ldexp(chunk, lsb - SC)
    return out


def span(terms):
    """Bits from the lowest set bit of any term to the top bit of the largest."""
    nz = [abs(t) for t in terms if t]
    if not nz:
        return 0
    lo = min((t & -t).bit_length() - 1 for t in nz)
    hi = max(t.bit_length() - 1 for t in nz)
    return hi - lo + 1


def row_model(L, mode, A, x, r):
    """(cut value, fits) of row r of the oracle CSR A against x (P x ncols):
    the exact model of the row (real: L components; complex: the real part's
    L components, then the imaginary part's) and whether the terms of every
    part fit the window.  Complex entries follow the kernels' pattern:
    re += a_re x_re - a_im x_im, im += a_re x_im + a_im x_re."""
    def part(k, p):  # components of plane group p (0 real, 1 imaginary) of entry k
        return A.data[p * L:p * L + L, k] if mode == 0 else A.data[p * L:p * L + 1, k]
    if not A.cplx:
        terms = []
        for k in range(A.indptr[r], A.indptr[r + 1]):
            terms += entry_terms(L, mode, part(k, 0), x[:L, int(A.indices[k])])
        return cut(sum(terms), L), span(terms) <= window_bits(L)
    re, im = [], []
    for k in range(A.indptr[r], A.indptr[r + 1]):
        c = int(A.indices[k])
        xr, xi = x[:L, c], x[L:2 * L, c]
        re += entry_terms(L, mode, part(k, 0), xr)
        re += [-t for t in entry_terms(L, mode, part(k, 1), xi)]
        im += entry_terms(L, mode, part(k, 0), xi)
        im += entry_terms(L, mode, part(k, 1), xr)
    fits = span(re) <= window_bits(L) and span(im) <= window_bits(L)
    return np.concatenate([cut(sum(re), L), cut(sum(im), L)]), fits


def axpy_model(L, alpha_re, alpha_im, u, v, cplx):
    """(cut value, fits) of one element of w = u + alpha v on an exact
    handle (the vector kernels' form): u's components added exactly, the
    products alpha v in the decomposed form (complex: re takes
    a_re v_re - a_im v_im, im takes a_re v_im + a_im v_re), each part cut once.
    u and v hold P components of the element."""
    def limbs(w):
        return [exact.f2i(c) << exact.SCALE for c in w]
    re = limbs(u[:L]) + entry_terms(L, 0, alpha_re, v[:L])
    if not cplx:
        return cut(sum(re), L), span(re) <= window_bits(L)
    re += [-t for t in entry_terms(L, 0, alpha_im, v[L:2 * L])]
    im = limbs(u[L:2 * L]) + entry_terms(L, 0, alpha_re, v[L:2 * L]) + entry_terms(L, 0, alpha_im, v[:L])
    fits = span(re) <= window_bits(L) and span(im) <= window_bits(L)
    return np.concatenate([cut(sum(re), L), cut(sum(im), L)]), fits


# ---------------------------------------------------------------------------
# The wide-x form of the exact arithmetic (single-vector products of exact
# handles whose values are binary64: one stored value plane).  Each column's
# x (and each of its real and imaginary parts) is first turned into one
# fixed-point number X = s M 2^E with a W-word mantissa (W = 4 / 5 / 7 words
# of 32 bits for DD / TD / QD); an entry then adds the one product a X,
# without the product's lowest 32-bit word, to the row's exact sum, which is
# cut to L components as before.  X is x truncated toward zero to 32 W bits
# below its top bit, so |a X - a x| < 2^(1-32W) |a x|: below the unit
# roundoff of every format (2^-127, 2^-159, 2^-223 against u = 2^-104,
# 2^-155, 2^-207).
# ---------------------------------------------------------------------------
WIDE_WORDS = {2: 4, 3: 5, 4: 7}
WIDE_DIGITS = {2: 8, 3: 9, 4: 11}  # row accumulator digits of the wide form
WIDE_MARGIN = 32  # bits the window keeps above a product when it is placed or moved
WSC = 4400  # wide-form terms are integers times 2^-4400


def _top_exp(c):
    """Bit the accumulator assumes for the top of a non-zero binary64's
    mantissa: e0 + 52 with c = m 2^e0 (subnormals: e0 = -1074)."""
    m, e = math.frexp(abs(c))
    return max(e - 1, -1022)


def wide_record(comps, L):
    """(s, M, E) of one part of one column: comps are its L binary64
    components.  The components are added into D = W + 2 digits of 32 bits
    whose base puts the largest component's top bit (e0 + 52) in the last
    bit of digit D - 2; each component's magnitude is truncated below the
    base (exact when the components span at most 32 (D - 1) bits).  The sum
    V (an integer times 2^base) is then cut to the 32 W bits below its top
    bit: M = floor(|V| / 2^(t - 32W + 1)), t the top bit of |V|, E = base +
    t - 32W + 1, s the sign of V.  Returns None for a non-finite component
    (the products then give NaN) and (0, 0, 0) for a zero sum."""
    W = WIDE_WORDS[L]
    D = W + 2
    if any(not math.isfinite(float(c)) for c in comps):
        return None
    nz = [float(c) for c in comps if float(c) != 0.0]
    if not nz:
        return 0, 0, 0
    t0 = max(_top_exp(c) for c in nz)
    base = t0 - (32 * (D - 1) - 1)
    V = 0
    for c in nz:
        N = abs(exact.f2i(c))          # |c| = N 2^-1074
        sh = -exact.SCALE - base       # |c| / 2^base = N 2^sh
        mag = N << sh if sh >= 0 else N >> (-sh)
        V += -mag if c < 0 else mag
    if V == 0:
        return 0, 0, 0
    m = abs(V)
    t = m.bit_length() - 1
    lsb = t - 32 * W + 1
    M = m >> lsb if lsb >= 0 else m << (-lsb)
    return (-1 if V < 0 else 1), M, base + lsb


def wide_product(a, rec):
    """(sign, P, e0) of one entry a . X: P = floor(m_a M / 2^32) (the
    product of the mantissas without its lowest 32-bit word), its last bit
    weighing 2^e0 with e0 = e_a + E + 32, a = s_a m_a 2^e_a (binary64); None
    for a zero product."""
    if a == 0.0 or rec[1] == 0:
        return None
    s, M, E = rec
    N = exact.f2i(a)                   # a = N 2^-1074 = s_a m_a 2^e_a with m_a < 2^53
    ma, ea = abs(N), -exact.SCALE
    while ma >= (1 << 53):             # normal values: 53-bit mantissa, e_a >= -1074
        ma >>= 1                       # (exact: N carries trailing zeros there)
        ea += 1
    return (1 if a > 0 else -1) * s, (ma * M) >> 32, ea + E + 32


def wide_term(a, rec, neg=False):
    """The term of one entry a . X in units of 2^-WSC."""
    pr = wide_product(a, rec)
    if pr is None:
        return 0
    sg, P, e0 = pr
    sh = e0 + WSC
    v = P << sh if sh >= 0 else P >> (-sh)
    return sg * (-1 if neg else 1) * v


def wide_sum(L, prods):
    """The row accumulator of the wide form, step by step: prods are the
    (sign, P, e0) of a row's products in the kernels' order.  Two
    non-negative digit arrays (positive and negative terms) of D digits with
    a common base: the first product's top bit (e0 + 20 + 32 W, the bound on
    P), raised by the margin, anchors the window in the last bit of digit
    D - 2; a product whose top would reach digit D - 1 moves the window up
    by whole digits so that its top, raised by the margin, fits below digit
    D - 1, each array's value then floor-divided by 2^32 per digit (all
    digits cleared for a move of D or more); a product's bits below the base
    are truncated.  Returns the sum, cut to L components."""
    W, D = WIDE_WORDS[L], WIDE_DIGITS[L]
    base = None
    vp = vn = 0
    for sg, P, e0 in prods:
        top = e0 + 20 + 32 * W
        if base is None:
            base = top + WIDE_MARGIN - (32 * (D - 1) - 1)
        elif e0 - base > 32 * (D - 1) - 21 - 32 * W:
            sd = (top + WIDE_MARGIN - base - (32 * (D - 1) - 1) + 31) >> 5
            if sd >= D:
                vp = vn = 0
            else:
                vp >>= 32 * sd
                vn >>= 32 * sd
            base += 32 * sd
        pos = e0 - base
        c = P << pos if pos >= 0 else P >> (-pos)
        if sg > 0:
            vp += c
        else:
            vn += c
    if base is None:
        return np.zeros(L)
    return cut_scaled(vp - vn, L, -base)


def wide_window_bits(L):
    return 32 * (WIDE_DIGITS[L] - 2) + 1


def cut_scaled(V, L, scale):
    """V * 2^-scale cut to L components by truncation of its magnitude."""
    out = np.zeros(L)
    if V == 0:
        return out
    s = -1.0 if V < 0 else 1.0
    m = abs(V)
    top = m.bit_length() - 1
    for l in range(L):
        lsb = top - 52 - 53 * l
        chunk = (m >> lsb) & ((1 << 53) - 1) if lsb >= 0 else (m << -lsb) & ((1 << 53) - 1)
        try:
            out[l] = s * math.ldexp(chunk, lsb - scale)
        except OverflowError:          # beyond the binary64 range: infinity, like scalbn
            out[l] = s * math.inf
    return out


def row_model_wide(L, A, x, r):
    """(value, exact) of row r of the oracle CSR A (binary64 values in
    component 0 of each part) against x, in the wide-x form: the row
    accumulator of wide_sum over the entries' products (complex, the kernels'
    order per entry: re += a_re X_re, im += a_im X_re, re -= a_im X_im,
    im += a_re X_im).  exact: whether the accumulator kept every bit (the
    terms span at most 32 (D - 2) + 1 bits), i.e. the value is the exact sum
    cut to L components.  A non-finite x component in the row gives NaN in
    the first component of each part."""
    def rec(c, p):
        return wide_record(x[p * L:p * L + L, c], L)

    def flip(pr):
        return None if pr is None else (-pr[0], pr[1], pr[2])

    def terms_of(prods):
        return [pr[0] * (pr[1] << (pr[2] + WSC)) for pr in prods]

    if not A.cplx:
        prods = []
        for k in range(A.indptr[r], A.indptr[r + 1]):
            R = rec(int(A.indices[k]), 0)
            if R is None:
                out = np.zeros(L)
                out[0] = np.nan
                return out, True
            pr = wide_product(float(A.data[0, k]), R)
            if pr is not None:
                prods.append(pr)
        return wide_sum(L, prods), span(terms_of(prods)) <= wide_window_bits(L)
    re, im = [], []
    for k in range(A.indptr[r], A.indptr[r + 1]):
        c = int(A.indices[k])
        Rr, Ri = rec(c, 0), rec(c, 1)
        if Rr is None or Ri is None:
            out = np.zeros(2 * L)
            out[0] = out[L] = np.nan
            return out, True
        ar, ai = float(A.data[0, k]), float(A.data[L, k])
        for acc, pr in ((re, wide_product(ar, Rr)), (im, wide_product(ai, Rr)),
                        (re, flip(wide_product(ai, Ri))), (im, wide_product(ar, Ri))):
            if pr is not None:
                acc.append(pr)
    ex = span(terms_of(re)) <= wide_window_bits(L) and span(terms_of(im)) <= wide_window_bits(L)
    return np.concatenate([wide_sum(L, re), wide_sum(L, im)]), ex
