"""Pins of oracle/exact_model.py (the exact model of the exact-accumulation
arithmetic) against what mathematics fixes, independently of the CUDA code:

* cut(): the components are 53-bit chunks of the magnitude, non-overlapping
  and consecutive, their sum is the value truncated to 53 L bits below its
  top bit (so the remainder is below one unit of the last place), and the
  sign is the value's;
* entry_terms(): integer operands give the exact product; the terms of an
  MP product differ from the full product by the dropped products and one
  rounding of the FMA chain, within a few unit roundoffs; for a binary64
  value only the last product is rounded, within one unit roundoff;
* span(): the bit span of single powers of two and of a pair;
* row_model() and axpy_model(): a one-entry row is that entry; a sum that
  cancels exactly gives zeros; complex parts follow (a + bi)(c + di).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads
from oracle import exact
from oracle import exact_model as em

SC = em.SC


def as_int(v):
    """v (binary64) as an integer in units of 2^-2148."""
    return exact.f2i(v) << exact.SCALE


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_cut_is_truncation_to_53L_bits(L):
    rng = np.random.default_rng(L)
    for _ in range(500):
        # values between 2^-1000 and 2^900 (units of 2^-2148), with low bits set
        V = int(rng.integers(1, 1 << 62)) << int(rng.integers(1148, 2950))
        V = V * int(rng.integers(1, 1 << 60)) + int(rng.integers(0, 1 << 62))
        V = -V if rng.random() < 0.5 else V
        out = em.cut(V, L)
        m = abs(V)
        top = m.bit_length() - 1
        s = sum(as_int(abs(c)) for c in out)
        # the magnitude cut below bit top - 53 L + 1, in one piece
        lsb = top - 53 * L + 1
        want = (m >> lsb) << lsb if lsb > 0 else m
        assert s == want
        assert all((c < 0) == (V < 0) or c == 0 for c in out)
        # consecutive 53-bit chunks: each component's top bit sits 53 bits
        # below the previous one's (or the component is zero)
        for l in range(L):
            if out[l] != 0:
                assert abs(as_int(out[l])) < 1 << (top - 53 * l + 1)
    assert not em.cut(0, L).any()


@pytest.mark.parametrize("L", [2, 3, 4])
def test_entry_terms_of_integers_are_the_exact_product(L):
    rng = np.random.default_rng(10 + L)
    for _ in range(300):
        a = np.zeros(L)
        x = np.zeros(L)
        a[0] = float(rng.integers(-1 << 20, 1 << 20))
        x[0] = float(rng.integers(-1 << 20, 1 << 20))
        for mode in (0, 1):
            assert sum(em.entry_terms(L, mode, a, x)) == exact.f2i(a[0]) * exact.f2i(x[0])


@pytest.mark.parametrize("L", [2, 3, 4])
def test_entry_terms_stay_within_a_few_unit_roundoffs(L):
    rng = np.random.default_rng(20 + L)
    u = Fraction(exact.U[L])
    for _ in range(300):
        a = workloads.full_limb_vector(1, L, seed=int(rng.integers(1 << 30)))[:, 0] * 2.0 ** int(rng.integers(-50, 50))
        x = workloads.full_limb_vector(1, L, seed=int(rng.integers(1 << 30)))[:, 0] * 2.0 ** int(rng.integers(-50, 50))
        full = exact.limbs_to_int(a) * exact.limbs_to_int(x)
        got = sum(em.entry_terms(L, 0, a, x))
        scale = abs(exact.limbs_to_int(a)) * abs(exact.limbs_to_int(x))
        assert Fraction(abs(got - full), scale) <= 3 * u
        # binary64 value: exact up to the one rounded product of the last component
        got = sum(em.entry_terms(L, 1, a[:1], x))
        full = exact.f2i(a[0]) * exact.limbs_to_int(x)
        assert Fraction(abs(got - full), abs(exact.f2i(a[0])) * abs(exact.limbs_to_int(x))) <= u


def test_span():
    assert em.span([1 << 10]) == 1
    assert em.span([(1 << 10) + 1]) == 11
    assert em.span([1 << 10, -(1 << 3)]) == 8
    assert em.span([0, 0]) == 0


@pytest.mark.parametrize("L", [2, 4])
def test_row_and_axpy_models_special_cases(L):
    x = workloads.full_limb_vector(3, L, seed=5)
    a = workloads.full_limb_vector(3, L, seed=6)
    # a one-entry row is that entry's terms, cut
    A = oracle.CSR(1, 3, np.array([0, 1]), np.array([2]), a[:, :1], L, False)
    want = em.cut(sum(em.entry_terms(L, 0, a[:, 0], x[:, 2])), L)
    got, fits = em.row_model(L, 0, A, x, 0)
    assert fits and np.array_equal(got, want)
    # a row a x - a x cancels exactly
    A = oracle.CSR(1, 3, np.array([0, 2]), np.array([1, 1]), np.stack([a[:, 0], -a[:, 0]], axis=1), L, False)
    got, _ = em.row_model(L, 0, A, x, 0)
    assert not got.any()
    # u + alpha v with alpha = 0 returns u cut (u's components sum exactly)
    got, fits = em.axpy_model(L, np.zeros(L), np.zeros(L), x[:, 0], x[:, 1], False)
    assert fits and np.array_equal(got, em.cut(exact.limbs_to_int(x[:, 0]) << exact.SCALE, L))
    # complex: (a + bi) with integer parts times (c + di), no rounding anywhere
    ar, ai = np.zeros(L), np.zeros(L)
    ar[0], ai[0] = 3.0, -2.0
    v = np.zeros(2 * L)
    v[0], v[L] = 5.0, 7.0
    u = np.zeros(2 * L)
    got, fits = em.axpy_model(L, ar, ai, u, v, True)
    assert fits and got[0] == 3 * 5 - (-2) * 7 and got[L] == 3 * 7 + (-2) * 5
    assert not got[1:L].any() and not got[L + 1:].any()
    assert math.isclose(got[0], 29.0)


# ---------------------------------------------------------------------------
# The wide-x form (single-vector products of binary64-valued exact handles)
# ---------------------------------------------------------------------------
def _rec_value(rec):
    """X = s M 2^E of a record as a Fraction."""
    s, M, E = rec
    return Fraction(s * M) * (Fraction(2) ** E)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_wide_record_is_x_truncated_to_32W_bits(L):
    """X has a mantissa of exactly 32 W bits (top bit set), the sign of x,
    |X| <= |x| < |X| + 2^E (truncation toward zero below the last kept bit),
    and X = x whenever x needs no more than 32 W bits; zero and non-finite
    components give the zero record and None."""
    W = em.WIDE_WORDS[L]
    rng = np.random.default_rng(100 + L)
    for i in range(300):
        x = workloads.full_limb_vector(1, L, rng=rng)[:, 0] * 2.0 ** int(rng.integers(-900, 900))
        if i % 7 == 0:
            x[1:] = -x[1:]                    # lower components of the other sign
        ex = sum((Fraction(float(c)) for c in x), Fraction(0))
        rec = em.wide_record(x, L)
        s, M, E = rec
        assert M.bit_length() == 32 * W and s == (1 if ex > 0 else -1)
        X = _rec_value(rec)
        assert abs(X) <= abs(ex) < abs(X) + Fraction(2) ** E
    for v in (3.0, -1.5, 2.0 ** -1060, 12345678901.0):
        comps = np.zeros(L)
        comps[0] = v
        assert _rec_value(em.wide_record(comps, L)) == Fraction(v)
    # an integer spread over components that fits 32 W bits is exact
    comps = np.zeros(L)
    comps[0], comps[1] = 2.0 ** 60, 7.0
    assert _rec_value(em.wide_record(comps, L)) == Fraction(2 ** 60 + 7)
    assert em.wide_record(np.zeros(L), L) == (0, 0, 0)
    comps = np.zeros(L)
    comps[0], comps[1] = 1.0, -1.0
    assert em.wide_record(comps, L) == (0, 0, 0)
    comps[1] = float("inf")
    assert em.wide_record(comps, L) is None


@pytest.mark.parametrize("L", [2, 3, 4])
def test_wide_term_error_and_integer_exactness(L):
    """A term a X differs from a x by less than 2^(2-32W) |a x| (X's
    truncation plus the dropped lowest product word), and equals a x exactly
    for integer a and x of a few bits; the sign follows a x."""
    W = em.WIDE_WORDS[L]
    rng = np.random.default_rng(200 + L)
    unit = Fraction(1, 2 ** em.WSC)
    for _ in range(300):
        a = float(rng.standard_normal()) * 2.0 ** int(rng.integers(-400, 400))
        x = workloads.full_limb_vector(1, L, rng=rng)[:, 0] * 2.0 ** int(rng.integers(-400, 400))
        ax = Fraction(a) * sum((Fraction(float(c)) for c in x), Fraction(0))
        t = em.wide_term(a, em.wide_record(x, L)) * unit
        assert abs(t - ax) < Fraction(2) ** (2 - 32 * W) * abs(ax)
        assert (t > 0) == (ax > 0)
    for a, xv in ((3.0, 5.0), (-7.0, 11.0), (2.0 ** 40, -3.0), (1.0, 2.0 ** 52 + 1.0)):
        comps = np.zeros(L)
        comps[0] = xv
        assert em.wide_term(a, em.wide_record(comps, L)) * unit == Fraction(a) * Fraction(xv)
    assert em.wide_term(0.0, em.wide_record(np.array([1.0] + [0.0] * (L - 1)), L)) == 0


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_wide_rows_within_bound_and_integer_rows_exact(L, cplx):
    """Rows of the wide form meet the componentwise bound 8 m u (|A||x|)_i
    against the exact row value (m the longest row, 2m terms for complex);
    integer-valued rows are exact (the cut of an exact integer sum that fits
    L components is that sum)."""
    coo = workloads.random_sparse(60, 50, 12, seed=7 + L, cplx=cplx, empty_frac=0.1)
    A = oracle.coo_to_csr(60, 50, coo.row, coo.col, coo.promoted(L), L, cplx)
    x = workloads.full_limb_vector(50, L, seed=8 + L, cplx=cplx)
    P = 2 * L if cplx else L
    y = np.zeros((P, 60))
    for r in range(60):
        y[:, r], _ = em.row_model_wide(L, A, x, r)
    assert exact.bound_ratio(y, A, x) <= 1.0
    icoo = workloads.integer_matrix(40, 40, 0.2, seed=3 + L, cplx=cplx)
    Ai = oracle.coo_to_csr(40, 40, icoo.row, icoo.col, icoo.promoted(L), L, cplx)
    xi = workloads.integer_vector(40, L, seed=4 + L, cplx=cplx)
    want = oracle.spmv(Ai, xi)                # integer data: the oracle's rows are exact
    for r in range(40):
        got, fits = em.row_model_wide(L, Ai, xi, r)
        assert fits and np.array_equal(got, want[:, r])


def test_wide_nan_rows():
    """A non-finite x component referenced by a row gives NaN in the first
    component of each part of that row."""
    L = 2
    coo = workloads.COO(2, 3, np.array([0, 0, 1]), np.array([0, 2, 1]), np.array([[1.0, 0.0, 2.0]]))
    A = oracle.coo_to_csr(2, 3, coo.row, coo.col, coo.promoted(L), L)
    x = np.zeros((L, 3))
    x[0] = 1.0
    x[1, 2] = float("nan")
    y0, fits = em.row_model_wide(L, A, x, 0)
    assert fits and np.isnan(y0[0]) and y0[1] == 0.0
    y1, _ = em.row_model_wide(L, A, x, 1)
    assert y1[0] == 2.0
