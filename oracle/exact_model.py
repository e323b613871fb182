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
