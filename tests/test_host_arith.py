"""The device arithmetic, compiled for the host (tests/host_build): the same
csrc/mp_arith.cuh and csrc/fixacc.cuh the kernels compile, run on the CPU
with IEEE 754 binary64 and no FMA contraction.  This checks, without a GPU,
millions of operations that the GPU tests sample:

* the paper-order MP add, mul, mul_d and div (Algorithms 1-5, QD sloppy
  forms, long division) are bit-identical to the oracle's;
* the exact accumulators (shared-memory digits with their window, and the
  register digits at a common base) return the exact sum of their terms cut
  to L components by truncation, whenever the terms fit the window: signs,
  cancellation to zero, carries into the head-room digit, window moves,
  106-bit integer products, subnormal terms, non-finite terms;
* the terms of one stored entry (exact_prod.cuh: the exact products a_i x_j
  below the format's unit roundoff plus one FMA chain, for MP and binary64
  matrix values) add up to exactly that decomposition, and stay within a
  few units of the unit roundoff of the full product;
* the integer assembly of a component from its 53-bit chunk
  (chunk_to_double) equals chunk * 2^e, including the subnormal and
  overflow ends.
"""
import ctypes
import math
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads
from oracle import exact
from oracle import exact_model as model
from oracle.exact_model import SC
from oracle.exact_model import cut as _cut
from oracle.exact_model import entry_terms as _entry_term_list
from oracle.exact_model import rn_fma as _rn_fma  # noqa: F401
from oracle.exact_model import span as _span
from oracle.exact_model import term as _term


def _entry_terms(L, mode, a, x):
    return sum(_entry_term_list(L, mode, a, x))

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2412_17510_gb300", "csrc")

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("host_build") / "libhostarith.so")
    cmd = [cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-Wno-unknown-pragmas", "-shared",
           "-fPIC", "-I", os.path.join(HERE, "host_build"), "-I", CSRC, os.path.join(HERE, "host_build", "harness.cpp"),
           "-o", out]
    subprocess.run(cmd, check=True, capture_output=True)
    h = ctypes.CDLL(out)
    h.host_mp_ops.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _dp, _dp, _dp]
    h.host_fas_sum.argtypes = [ctypes.c_int, ctypes.c_int, _ip, _dp, _dp, _ip, _dp]
    h.host_fa_sum.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp]
    h.host_chunk_to_double.argtypes = [ctypes.c_ulonglong, ctypes.c_int, ctypes.c_int]
    h.host_chunk_to_double.restype = ctypes.c_double
    h.host_entry_sum.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
    _up = ctypes.POINTER(ctypes.c_ulonglong)
    h.host_flush.argtypes = [ctypes.c_int, _up, _up, ctypes.c_int, _dp]
    h.host_flush_wide.argtypes = [ctypes.c_int, _up, _up, ctypes.c_int, _dp]
    h.host_row_sum.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
    h.host_row_sum_c.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    h.host_axpy_elem.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
    DIGITS.update({L: h.host_acc_digits(L) for L in (1, 2, 3, 4)})
    assert DIGITS == model.DIGITS  # the model's table is the kernels' one
    return h


DIGITS = {}  # accumulator digits per L, read from the kernels' table


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


# --------------------------------------------------------------------------
# paper-order MP operations against the oracle
# --------------------------------------------------------------------------
OPS = {0: lambda L, a, b: oracle.mp_add(L, a, b), 1: lambda L, a, b: oracle.mp_mul(L, a, b),
       2: lambda L, a, b: oracle.mp_mul_d(L, a, b[0]), 3: lambda L, a, b: oracle.mp_div(L, a, b)}


def _operands(n, L, seed):
    rng = np.random.default_rng(seed)
    a = workloads.full_limb_vector(n, L, seed=seed).T.copy()
    b = workloads.full_limb_vector(n, L, seed=seed + 1).T.copy()
    a *= (2.0 ** rng.integers(-60, 61, n))[:, None]
    b *= (2.0 ** rng.integers(-60, 61, n))[:, None]
    # near-cancellation for the additions: b = -a with its last component moved
    k = n // 4
    b[:k] = -a[:k]
    b[:k, L - 1] *= 1.0 + 2.0 ** -20
    # integers (exact products and sums) and a binary64 first operand
    a[k:2 * k] = np.floor(a[k:2 * k] * 1e6)
    a[k:2 * k, 1:] = 0.0
    return a, b


@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_mp_ops_bit_identical_to_oracle(lib, L, op):
    n = 2000
    a, b = _operands(n, L, seed=10 * L + op)
    r = np.zeros((n, L))
    assert lib.host_mp_ops(L, op, n, _d(a), _d(b), _d(r)) == 0
    for i in range(n):
        ref = OPS[op](L, a[i], b[i])
        assert np.array_equal(r[i], ref), (L, op, i, a[i], b[i], r[i], ref)


# --------------------------------------------------------------------------
# exact accumulators against exact integer sums
# --------------------------------------------------------------------------
def _fas(lib, L, kind, a, b, neg):
    n = len(kind)
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    neg = np.ascontiguousarray(neg, dtype=np.int32)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros(L)
    assert lib.host_fas_sum(L, n, _i(kind), _d(a), _d(b), _i(neg), _d(out)) == 0
    return out


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_shared_digit_accumulator_is_exact_within_its_window(lib, L):
    """Random mixtures of binary64 terms and exact products, both signs,
    exponent ranges chosen so that every term fits the window the
    accumulator guarantees after any move (32 (D - 2) + 1 bits below the
    largest term); the first term is often a small one, so the window moves
    up."""
    rng = np.random.default_rng(100 + L)
    D = DIGITS[L]
    guaranteed = 32 * (D - 2) + 1
    checked = 0
    for case in range(400):
        n = int(rng.integers(1, 120))
        prods = L >= 2 and case % 2 == 1
        kind = (rng.random(n) < 0.6).astype(np.int32) if prods else np.zeros(n, dtype=np.int32)
        spread = max(1, (guaranteed - (106 if prods else 53) - 8) // 2)
        a = rng.standard_normal(n) * 2.0 ** rng.integers(-spread, spread + 1, n)
        b = np.where(kind == 1, rng.standard_normal(n) * 2.0 ** rng.integers(-spread // 2, spread // 2 + 1, n), 0.0)
        if prods:  # the product's exponent range is a's plus b's: narrow a for products
            a = np.where(kind == 1, rng.standard_normal(n) * 2.0 ** rng.integers(-spread // 2, spread // 2 + 1, n), a)
        neg = (rng.random(n) < 0.5).astype(np.int32)
        terms = [_term(k, x, y, g) for k, x, y, g in zip(kind, a, b, neg)]
        if _span(terms) > guaranteed:
            continue
        got = _fas(lib, L, kind, a, b, neg)
        assert np.array_equal(got, _cut(sum(terms), L)), (L, case)
        checked += 1
    assert checked >= 300


@pytest.mark.parametrize("L", [2, 3, 4])
def test_shared_digit_accumulator_special_cases(lib, L):
    x = workloads.full_limb_vector(1, L, seed=4)[:, 0]
    # exact cancellation: x - x, its components in another order
    kind = np.zeros(2 * L, dtype=np.int32)
    a = np.concatenate([x, x[::-1]])
    neg = np.array([0] * L + [1] * L, dtype=np.int32)
    assert not _fas(lib, L, kind, a, np.zeros(2 * L), neg).any()
    # a product that cancels a TwoProd pair: a b - fl(a b) - err(a b) = 0
    p, e = oracle.two_prod(x[0], 3.0 + 2.0 ** -40)
    got = _fas(lib, L, [1, 0, 0], [x[0], p, e], [3.0 + 2.0 ** -40, 0, 0], [0, 1, 1])
    assert not got.any()
    # carries into the head-room digit: 1000 copies of a value with all bits set
    v = 2.0 ** 53 - 1.0
    got = _fas(lib, L, np.zeros(1000, dtype=np.int32), np.full(1000, v), np.zeros(1000), np.zeros(1000, dtype=np.int32))
    assert np.array_equal(got, _cut(1000 * (exact.f2i(v) << exact.SCALE), L))
    # a negative sum whose magnitude has a long run of ones below its second
    # component: the magnitude is cut, the sign kept (the smallest term sits
    # inside the window: 32 (D - 2) + 1 - 58 bits below the largest)
    g = 32 * (DIGITS[L] - 2) + 1
    terms = [1.0, -3.0 * 2.0 ** -60, 2.0 ** -(g - 60), -2.0 ** -(g - 59)]
    kind = np.zeros(4, dtype=np.int32)
    neg = np.array([1, 0, 0, 0], dtype=np.int32)
    got = _fas(lib, L, kind, terms, np.zeros(4), neg)
    V = sum(_term(0, t, 0.0, g) for t, g in zip(terms, neg))
    assert V < 0 and np.array_equal(got, _cut(V, L))
    # the same sum with the two smallest terms below the window: they are
    # dropped (the sum is exact up to the window), so the result differs from
    # the cut exact sum, by less than 2^(2 - 53 L) times the largest term
    if L == 2:
        terms = [1.0, -3.0 * 2.0 ** -60, 2.0 ** -200, -2.0 ** -201]
        got = _fas(lib, L, kind, terms, np.zeros(4), neg)
        V = sum(_term(0, t, 0.0, g) for t, g in zip(terms, neg))
        assert not np.array_equal(got, _cut(V, L))
        err = abs(sum(exact.f2i(c) << exact.SCALE for c in got) - V)
        assert err <= (exact.f2i(1.0) << exact.SCALE) >> (53 * L - 2)
    # subnormal terms only (the out-of-line general path)
    sub = np.array([5e-324, 3 * 5e-324, -7 * 5e-324, 2.0 ** -1030, -(2.0 ** -1060)])
    got = _fas(lib, L, np.zeros(5, dtype=np.int32), sub, np.zeros(5), np.zeros(5, dtype=np.int32))
    assert np.array_equal(got, _cut(sum(exact.f2i(s) << exact.SCALE for s in sub), L))
    # non-finite terms give NaN in the first component
    for bad in (math.inf, -math.inf, math.nan):
        got = _fas(lib, L, [0, 0], [1.0, bad], [0.0, 0.0], [0, 0])
        assert math.isnan(got[0]) and not got[1:].any()
    # zero terms only
    assert not _fas(lib, L, [0, 1], [0.0, 0.0], [0.0, 5.0], [0, 1]).any()


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_register_digit_sum_is_exact_within_its_window(lib, L):
    """The combine kernels' and block sums' form: every term at the base of
    the largest one (32 (D - 1) bits of window below its top)."""
    rng = np.random.default_rng(200 + L)
    D = DIGITS[L]
    window = 32 * (D - 1)
    checked = 0
    for case in range(300):
        n = int(rng.integers(1, 200))
        spread = max(1, (window - 53 - 8) // 2)
        a = rng.standard_normal(n) * 2.0 ** rng.integers(-spread, spread + 1, n)
        terms = [_term(0, x, 0.0, False) for x in a]
        if _span(terms) > window:
            continue
        a = np.ascontiguousarray(a)
        out = np.zeros(L)
        assert lib.host_fa_sum(L, n, _d(a), _d(out)) == 0
        assert np.array_equal(out, _cut(sum(terms), L)), (L, case)
        checked += 1
    assert checked >= 250


def test_chunk_to_double(lib):
    rng = np.random.default_rng(7)
    for _ in range(20000):
        chunk = int(rng.integers(0, 1 << 53, dtype=np.int64))
        e = int(rng.integers(-1180, 1000))
        neg = int(rng.integers(0, 2))
        got = lib.host_chunk_to_double(chunk, e, neg)
        try:
            want = math.ldexp(chunk, e)
        except OverflowError:
            want = math.inf
        want = -want if neg else want
        assert got == want and math.copysign(1.0, got) == math.copysign(1.0, want), (chunk, e, neg)


# --------------------------------------------------------------------------
# the terms of one stored entry (exact_prod.cuh)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("mode", [0, 1])
def test_entry_products_match_their_decomposition(lib, L, mode):
    n = 1500
    rng = np.random.default_rng(300 + 10 * L + mode)
    A = workloads.full_limb_vector(n, L, seed=L + 20).T.copy()
    X = workloads.full_limb_vector(n, L, seed=L + 30).T.copy()
    A *= (2.0 ** rng.integers(-100, 101, n))[:, None]
    X *= (2.0 ** rng.integers(-100, 101, n))[:, None]
    if mode == 1:
        A[:, 1:] = 0.0
    u = exact.U[L]
    worst = 0.0
    for i in range(n):
        out = np.zeros(L)
        assert lib.host_entry_sum(L, mode, _d(np.ascontiguousarray(A[i])), _d(np.ascontiguousarray(X[i])),
                                  _d(out)) == 0
        assert np.array_equal(out, _cut(_entry_terms(L, mode, A[i], X[i]), L)), (L, mode, i)
        full = exact.limbs_to_int(A[i]) * exact.limbs_to_int(X[i])
        got = sum(exact.f2i(c) for c in out) << exact.SCALE
        scale = abs(exact.limbs_to_int(A[i])) * abs(exact.limbs_to_int(X[i]))
        worst = max(worst, float(Fraction(abs(got - full), scale) / Fraction(u)))
    # dropped products, the chain's rounding and the final truncation
    assert worst <= 4.0, worst


@pytest.mark.parametrize("L", [2, 4])
def test_products_at_the_ends_of_the_exponent_range(lib, L):
    """Exact products far below the binary64 range (the digits hold them; the
    cut components round into the subnormal range or to zero, as chunk * 2^e
    does) and far above it (components overflow to infinity)."""
    cases = [
        ([1, 1], [2.0 ** -600, -(2.0 ** -601) * 3], [2.0 ** -500, 2.0 ** -499]),  # sum 2^-1100 (1 - 3)
        ([1, 0], [2.0 ** -540 * 1.5, 2.0 ** -1074], [2.0 ** -530, 0.0]),          # 1.5 2^-1070 + 2^-1074
        ([1, 1], [2.0 ** 600 * 1.25, 2.0 ** 600], [2.0 ** 500, -(2.0 ** 500)]),    # 0.25 2^1100 -> inf
    ]
    for kind, a, b in cases:
        kind = np.array(kind, dtype=np.int32)
        neg = np.zeros(len(kind), dtype=np.int32)
        got = _fas(lib, L, kind, a, b, neg)
        V = sum(_term(k, x, y, 0) for k, x, y in zip(kind, a, b))
        m = abs(V)
        if V and m.bit_length() - 1 - SC > 1023:
            assert math.isinf(got[0]) and (got[0] > 0) == (V > 0)
        else:
            assert np.array_equal(got, _cut(V, L)), (a, b, got)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_mp_ops_non_finite_operands_like_the_oracle(lib, L):
    """Infinite and NaN leading components: the kernels' operations give the
    oracle's result (NaN where it has NaN, the same infinity otherwise)."""
    x = workloads.full_limb_vector(1, L, seed=9)[:, 0]
    specials = []
    for s in (math.inf, -math.inf, math.nan):
        v = np.zeros(L)
        v[0] = s
        specials.append(v)
    pairs = [(p, x) for p in specials] + [(x, p) for p in specials] + [(p, q) for p in specials for q in specials]
    for op in (0, 1, 2, 3):
        for a, b in pairs:
            a = np.ascontiguousarray(a)
            b = np.ascontiguousarray(b)
            r = np.zeros(L)
            lib.host_mp_ops(L, op, 1, _d(a), _d(b), _d(r))
            ref = OPS[op](L, a, b)
            same = [(math.isnan(g) and math.isnan(w)) or g == w for g, w in zip(r, ref)]
            assert all(same), (L, op, a, b, r, ref)


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_flush_of_random_digit_arrays(lib, L):
    """The end-of-row flush on arbitrary digit contents (each digit below
    2^63, as the accumulator keeps them; the head-room digit small enough that
    the value stays below 2^(32 D)): one signed carry pass, negation of a
    negative sum, the components cut by truncation.  Against the exact value
    sum_j (dp_j - dn_j) 2^(32 j + base)."""
    D = DIGITS[L]
    rng = np.random.default_rng(400 + L)
    up = ctypes.POINTER(ctypes.c_ulonglong)
    for case in range(3000):
        dp = rng.integers(0, 2 ** 62, D, dtype=np.uint64) >> rng.integers(0, 62, D).astype(np.uint64)
        dn = rng.integers(0, 2 ** 62, D, dtype=np.uint64) >> rng.integers(0, 62, D).astype(np.uint64)
        zero = rng.random(D) < 0.3
        dp[zero & (rng.random(D) < 0.5)] = 0
        dn[zero] = 0
        dp[D - 1] >>= np.uint64(34)  # keep |value| below 2^(32 D - 2): the head-room digit holds carries only
        dn[D - 1] >>= np.uint64(34)
        base = int(rng.integers(-1300, 700))
        out = np.zeros(L)
        dpc, dnc = np.ascontiguousarray(dp), np.ascontiguousarray(dn)
        lib.host_flush(L, dpc.ctypes.data_as(up), dnc.ctypes.data_as(up), base, _d(out))
        V = sum((int(a) - int(b)) << (32 * j) for j, (a, b) in enumerate(zip(dp, dn)))
        # V * 2^base in units of 2^-2148
        shift = base + SC
        assert shift >= 0
        want = _cut(V << shift, L)
        assert np.array_equal(out, want), (L, case)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_staged_digit_differences_flush_like_the_accumulator(lib, L):
    """The finishing pass of staged rows flushes the digit differences
    dp_j - dn_j, stored as 64-bit two's complement words, with the negative
    digits zero, where the run kernel flushed the pair (dp, dn) itself
    (wide-x row accumulator, D digits).  Both give the same components, and
    both are the exact value sum_j (dp_j - dn_j) 2^(32 j + base) cut to L
    components: random digit contents of either sign, and rows whose digits
    cancel to zero."""
    D = lib.host_wide_digits(L)
    rng = np.random.default_rng(900 + L)
    up = ctypes.POINTER(ctypes.c_ulonglong)
    zeros = np.zeros(D, dtype=np.uint64)
    for case in range(3000):
        dp = rng.integers(0, 2 ** 62, D, dtype=np.uint64) >> rng.integers(0, 62, D).astype(np.uint64)
        dn = rng.integers(0, 2 ** 62, D, dtype=np.uint64) >> rng.integers(0, 62, D).astype(np.uint64)
        dp[rng.random(D) < 0.2] = 0
        dn[rng.random(D) < 0.2] = 0
        if case % 10 == 0:
            dn = dp.copy()  # a row that cancels exactly
        dp[D - 1] >>= np.uint64(34)  # keep |value| below 2^(32 D - 2)
        dn[D - 1] >>= np.uint64(34)
        base = int(rng.integers(-1300, 1020 - 32 * D))  # the value stays inside the binary64 range
        pair, staged = np.zeros(L), np.zeros(L)
        dpc, dnc = np.ascontiguousarray(dp), np.ascontiguousarray(dn)
        lib.host_flush_wide(L, dpc.ctypes.data_as(up), dnc.ctypes.data_as(up), base, _d(pair))
        diff = np.ascontiguousarray(np.subtract(dp, dn))  # wraps modulo 2^64: the two's complement word
        lib.host_flush_wide(L, diff.ctypes.data_as(up), zeros.ctypes.data_as(up), base, _d(staged))
        assert np.array_equal(pair, staged), (L, case)
        V = sum((int(a) - int(b)) << (32 * j) for j, (a, b) in enumerate(zip(dp, dn)))
        shift = base + SC
        assert shift >= 0
        assert np.array_equal(pair, _cut(V << shift, L)), (L, case)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_shared_digit_accumulator_bound_over_the_whole_exponent_range(lib, L):
    """Terms and products anywhere in the binary64 range (subnormal operands
    included), so the window moves often and small terms fall below it.  The
    dropped parts are below the window, whose lower end stays within
    32 (D - 2) bits of the largest term's top bit, so the result is within
    n 2^(T - 32 (D - 2) + 1) of the exact sum (T: the largest term's top bit)
    plus one unit of its last component."""
    rng = np.random.default_rng(500 + L)
    D = DIGITS[L]
    for case in range(400):
        n = int(rng.integers(1, 60))
        kind = (rng.random(n) < 0.5).astype(np.int32)
        a = rng.standard_normal(n) * 2.0 ** rng.integers(-1070, 1000, n).astype(np.float64)
        b = np.where(kind == 1, rng.standard_normal(n) * 2.0 ** rng.integers(-1070, 20, n).astype(np.float64), 0.0)
        sub = rng.random(n) < 0.1
        a[sub] = rng.integers(1, 1 << 40, int(sub.sum())) * 5e-324
        neg = (rng.random(n) < 0.5).astype(np.int32)
        terms = [_term(k, x, y, g) for k, x, y, g in zip(kind, a, b, neg)]
        if any(not math.isfinite(x * y) for k, x, y in zip(kind, a, b) if k == 1):
            continue
        got = _fas(lib, L, kind, a, b, neg)
        V = sum(terms)
        T = max((abs(t).bit_length() - 1 for t in terms if t), default=0)
        if V and abs(V).bit_length() - 1 - SC > 1023:
            continue  # beyond the binary64 range: components overflow
        top_v = abs(V).bit_length() - 1 if V else 0
        bound = n * (1 << max(T - 32 * (D - 2) + 1, 0)) + (1 << max(top_v - 53 * L + 2, 0))
        err = abs(sum(exact.f2i(c) for c in got) * (1 << exact.SCALE) - V)
        # components below 2^-1074 are rounded by the conversion, not truncated
        tiny = 1 << (SC - 1074 + 1)
        assert err <= bound + L * tiny, (L, case, err, bound)



@pytest.mark.parametrize("L,mode", [(2, 0), (3, 0), (4, 0), (1, 1), (2, 1), (3, 1), (4, 1)])
def test_row_sums_equal_the_exact_model(lib, L, mode):
    """Whole rows as one thread sums them (stencil-like lengths, N(0,1)
    matrix values, full-limb x): the device code returns exactly the cut sum
    of the entries' decomposed terms whenever all of them fit the window.
    This is the model a row of the exact kernels follows.  (Binary64 sums of
    binary64 products, L = 1 with an MP value, add TwoProd pairs whose 106
    bits exceed the 4-digit window: their tails are cut, within the bound.)"""
    rng = np.random.default_rng(600 + 10 * L + mode)
    D = DIGITS[L]
    g = 32 * (D - 2) + 1
    checked = 0
    for case in range(150):
        n = int(rng.integers(1, 40))
        if mode == 1:
            A = np.zeros((n, L))
            A[:, 0] = rng.standard_normal(n)
        else:
            A = workloads.full_limb_vector(n, L, seed=int(rng.integers(1 << 30))).T.copy()
            A *= rng.standard_normal(n)[:, None]
        X = workloads.full_limb_vector(n, L, seed=int(rng.integers(1 << 30))).T.copy()
        terms = [t for k in range(n) for t in _entry_term_list(L, mode, A[k], X[k])]
        if _span(terms) > g:
            continue
        out = np.zeros(L)
        assert lib.host_row_sum(L, mode, n, _d(np.ascontiguousarray(A)), _d(np.ascontiguousarray(X)), _d(out)) == 0
        want = _cut(sum(_entry_terms(L, mode, A[k], X[k]) for k in range(n)), L)
        assert np.array_equal(out, want), (L, mode, case)
        checked += 1
    assert checked >= 100



@pytest.mark.parametrize("L,mode", [(2, 0), (3, 0), (4, 0), (2, 1), (3, 1), (4, 1)])
def test_complex_row_sums_equal_the_exact_model(lib, L, mode):
    """Complex rows in the kernels' per-entry pattern (re += a_re x_re -
    a_im x_im, im += a_re x_im + a_im x_re) against the model's complex row
    (oracle/exact_model.py), for rows whose terms fit the window."""
    rng = np.random.default_rng(700 + 10 * L + mode)
    checked = 0
    for case in range(80):
        n = int(rng.integers(1, 30))
        if mode == 1:
            data = np.zeros((2 * L, n))
            data[0] = rng.standard_normal(n)
            data[L] = rng.standard_normal(n)
        else:
            data = workloads.full_limb_vector(n, L, seed=int(rng.integers(1 << 30)), cplx=True)
        x = workloads.full_limb_vector(n, L, seed=int(rng.integers(1 << 30)), cplx=True)
        A = oracle.CSR(1, n, np.array([0, n]), np.arange(n), data, L, True)
        want, fits = model.row_model(L, mode, A, x, 0)
        if not fits:
            continue
        ore, oim = np.zeros(L), np.zeros(L)
        c = np.ascontiguousarray
        assert lib.host_row_sum_c(L, mode, n, _d(c(data[:L].T)), _d(c(data[L:].T)), _d(c(x[:L].T)),
                                  _d(c(x[L:].T)), _d(ore), _d(oim)) == 0
        assert np.array_equal(np.concatenate([ore, oim]), want), (L, mode, case)
        checked += 1
    assert checked >= 60



@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_axpy_elements_equal_the_exact_model(lib, L, cplx):
    """Elements of w = u + alpha v in the vector kernels' form against the
    model's axpy element (oracle/exact_model.py), whenever they fit the
    window."""
    n = 400
    P = 2 * L if cplx else L
    u = workloads.full_limb_vector(n, L, seed=80 + L, cplx=cplx)
    v = workloads.full_limb_vector(n, L, seed=90 + L, cplx=cplx)
    a = workloads.full_limb_vector(1, L, seed=99, cplx=cplx)[:, 0]
    ar, ai = a[:L], (a[L:] if cplx else np.zeros(L))
    checked = 0
    for i in range(n):
        want, fits = model.axpy_model(L, ar, ai, u[:, i], v[:, i], cplx)
        if not fits:
            continue
        out = np.zeros(P)
        c = np.ascontiguousarray
        assert lib.host_axpy_elem(L, int(cplx), _d(c(a)), _d(c(u[:, i])), _d(c(v[:, i])), _d(out)) == 0
        assert np.array_equal(out, want), (L, cplx, i)
        checked += 1
    assert checked >= n // 2


# ---------------------------------------------------------------------------
# wide-x form (csrc/wide.cuh) against the model's wide_record / row_model_wide
# ---------------------------------------------------------------------------
def _wide_lib(lib):
    _u32 = ctypes.POINTER(ctypes.c_uint32)
    lib.host_wide_rec.argtypes = [ctypes.c_int, _dp, _u32]
    lib.host_wide_row.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
    lib.host_wide_row_c.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
    for L in (2, 3, 4):
        assert lib.host_wide_words(L) == model.WIDE_WORDS[L]
        assert lib.host_wide_digits(L) == model.WIDE_DIGITS[L]
    return lib


def _dptr(a):
    return a.ctypes.data_as(_dp)


def _host_record(lib, c, L):
    w = np.zeros(8, dtype=np.uint32)
    c = np.ascontiguousarray(c, dtype=np.float64)
    lib.host_wide_rec(L, _dptr(c), w.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    meta = int(w[7])
    if meta & 1:
        return None
    W = model.WIDE_WORDS[L]
    M = sum(int(w[i]) << (32 * i) for i in range(W))
    if M == 0:
        return 0, 0, 0
    E = ctypes.c_int32(meta).value >> 2
    return (-1 if meta & 2 else 1), M, E


def _wide_x_cases(L, rng, n):
    """Column components of many kinds: full-limb values over the exponent
    range, lower components of either sign, overlapping (non-canonical)
    components, exact cancellation, zeros, subnormals, gaps wider than the
    record's window."""
    out = []
    for i in range(n):
        x = workloads.full_limb_vector(1, L, rng=rng)[:, 0] * 2.0 ** int(rng.integers(-1000, 1000))
        k = i % 8
        if k == 1:
            x[1:] = -x[1:]
        elif k == 2:
            x[1] = x[0] * float(rng.uniform(-0.9, 0.9))                 # overlapping
        elif k == 3:
            x[1] = -x[0]                                                # cancellation
        elif k == 4:
            x[:] = 0.0
            x[L - 1] = float(rng.uniform(-1, 1)) * 2.0 ** -1070         # subnormal only
        elif k == 5:
            x[L - 1] = x[0] * 2.0 ** -400                               # beyond the window
        elif k == 6:
            x[0] = 0.0
        out.append(x)
    return out


@pytest.mark.parametrize("L", [2, 3, 4])
def test_wide_records_equal_the_model(lib, L):
    """The record the kernels build for a column equals the model's
    (s, M, E) for 2,400 columns of every kind, and non-finite components give
    the NaN record."""
    h = _wide_lib(lib)
    rng = np.random.default_rng(300 + L)
    for x in _wide_x_cases(L, rng, 2400):
        assert _host_record(h, x, L) == model.wide_record(x, L), x
    x = np.zeros(L)
    x[0] = float("inf")
    assert _host_record(h, x, L) is None


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_wide_rows_equal_the_model(lib, L, cplx):
    """Rows of the wide form (records built per entry, products added in the
    row accumulator, cut to L components) equal the model bit for bit --
    the model follows the accumulator's window moves and truncations step by
    step -- and meet the bound 8 m u (|A||x|): rows of 1-40 entries with
    binary64 values over narrow and wide spreads of exponents."""
    h = _wide_lib(lib)
    rng = np.random.default_rng(400 + L + (10 if cplx else 0))
    compared = 0
    for i in range(400):
        n = int(rng.integers(1, 41))
        spread = 10 if i % 2 else 200
        ar = rng.standard_normal(n) * 2.0 ** rng.integers(-spread, spread + 1, n)
        ai = rng.standard_normal(n) * 2.0 ** rng.integers(-spread, spread + 1, n)
        xr = np.stack([workloads.full_limb_vector(1, L, rng=rng)[:, 0] * 2.0 ** int(rng.integers(-spread, spread + 1))
                       for _ in range(n)])
        xi = np.stack([workloads.full_limb_vector(1, L, rng=rng)[:, 0] * 2.0 ** int(rng.integers(-spread, spread + 1))
                       for _ in range(n)])
        V = 2 if cplx else 1
        vals = np.zeros((V * L, n))
        vals[0] = ar
        if cplx:
            vals[L] = ai
        A = oracle.CSR(1, n, np.array([0, n]), np.arange(n, dtype=np.int32), vals, L, cplx)
        x = np.concatenate([xr.T, xi.T]) if cplx else xr.T
        want, fits = model.row_model_wide(L, A, x, 0)
        if cplx:
            ore, oim = np.zeros(L), np.zeros(L)
            h.host_wide_row_c(L, n, _dptr(ar), _dptr(ai), _dptr(np.ascontiguousarray(xr)),
                              _dptr(np.ascontiguousarray(xi)), _dptr(ore), _dptr(oim))
            got = np.concatenate([ore, oim])
        else:
            got = np.zeros(L)
            h.host_wide_row(L, n, _dptr(ar), _dptr(np.ascontiguousarray(xr)), _dptr(got))
        assert np.array_equal(got, want), (i, got, want)
        compared += 1
        assert exact.bound_ratio(got[:, None], A, x) <= 1.0
    assert compared == 400


@pytest.mark.parametrize("L", [2, 3, 4])
def test_self_products_doubled_equal_the_plain_products(lib, L):
    """Self inner products (u, u) take each symmetric pair u_i u_j + u_j u_i
    once at twice the weight (add_prod_self): the same exact sum as
    add_prod(u, u), the same FMA chain, so the same bits -- on single
    elements over the exponent range (subnormal, zero and huge components
    included) and on sums of elements of similar magnitude."""
    lib.host_self_sum.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp]
    rng = np.random.default_rng(500 + L)
    cases = []
    for i in range(3000):
        u = workloads.full_limb_vector(1, L, rng=rng)[:, 0] * 2.0 ** int(rng.integers(-500, 500))
        if i % 9 == 1:
            u[1:] = -u[1:]
        elif i % 9 == 2:
            u[L - 1] = 0.0
        elif i % 9 == 3:
            u = workloads.full_limb_vector(1, L, rng=rng)[:, 0] * 2.0 ** -1040   # lower parts subnormal
        elif i % 9 == 4:
            u = workloads.full_limb_vector(1, L, rng=rng)[:, 0] * 2.0 ** 500
        cases.append((1, u))
    for i in range(300):
        n = int(rng.integers(2, 20))
        U = workloads.full_limb_vector(n, L, rng=rng).T * 2.0 ** int(rng.integers(-200, 200))
        cases.append((n, U.reshape(-1)))
    for n, U in cases:
        U = np.ascontiguousarray(U, dtype=np.float64)
        a, b = np.zeros(L), np.zeros(L)
        lib.host_self_sum(L, 1, n, U.ctypes.data_as(_dp), a.ctypes.data_as(_dp))
        lib.host_self_sum(L, 0, n, U.ctypes.data_as(_dp), b.ctypes.data_as(_dp))
        assert np.array_equal(a, b), (n, U, a, b)
