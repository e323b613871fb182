"""Pins for the oracle's scalar arithmetic (Section 2: EFTs, Algorithms 1-5,
QD sloppy add/mul, TD as QD with a zero fourth component).

Every check compares against exact rational arithmetic (fractions) or, where
noted, an independent 600-bit mpmath evaluation -- never against the oracle
itself.
"""
import math
import random
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from oracle import exact

U = {2: F(1, 2 ** 104), 3: F(1, 2 ** 155), 4: F(1, 2 ** 207)}


def fr(limbs):
    return sum((F(float(v)) for v in limbs), F(0))


def rand_mp(rng, L, scale_exp=0):
    """Random L-component number with every component random (c14 recipe)."""
    out = [rng.uniform(-1, 1) * 2.0 ** scale_exp]
    for _ in range(1, L):
        out.append(rng.uniform(-1, 1) * 2.0 ** -53 * abs(out[-1]))
    return np.array(out)


ADVERSARIAL = [
    (1.0, 2.0 ** -53), (1.0, -2.0 ** -54), (2.0 ** 60, 1.0), (1e300, 1e-300), (-0.0, 0.0),
    (5e-324, 5e-324), (1.0, -1.0), (3.0, 2.0 ** -52 + 2.0 ** -104), (2.0 ** -1022, -2.0 ** -1060),
    (1.0 + 2.0 ** -52, -(1.0 + 2.0 ** -51)), (float.fromhex("0x1.fffffffffffffp+1023"), -1e308),
]


def _pairs(n=400, seed=1):
    rng = random.Random(seed)
    out = list(ADVERSARIAL)
    for _ in range(n):
        a = rng.uniform(-1, 1) * 2.0 ** rng.randint(-60, 60)
        b = rng.uniform(-1, 1) * 2.0 ** rng.randint(-60, 60)
        out.append((a, b))
    return out


def test_two_sum_is_error_free():
    for a, b in _pairs():
        s, e = oracle.two_sum(a, b)
        assert s == a + b
        assert F(s) + F(e) == F(a) + F(b)


def test_quick_two_sum_is_error_free_when_ordered():
    for a, b in _pairs(seed=2):
        if abs(a) < abs(b):
            a, b = b, a
        if not math.isfinite(a + b):
            continue
        s, e = oracle.quick_two_sum(a, b)
        assert s == a + b
        assert F(s) + F(e) == F(a) + F(b)


def test_two_prod_is_error_free():
    rng = random.Random(3)
    for _ in range(500):
        a = rng.uniform(-1, 1) * 2.0 ** rng.randint(-200, 200)
        b = rng.uniform(-1, 1) * 2.0 ** rng.randint(-200, 200)
        p, e = oracle.two_prod(a, b)
        assert p == a * b
        assert F(p) + F(e) == F(a) * F(b)


def test_three_sum_preserves_sum_and_three_sum2_rounds_tail_only():
    rng = random.Random(4)
    for _ in range(300):
        a, b, c = (rng.uniform(-1, 1) * 2.0 ** rng.randint(-80, 0) for _ in range(3))
        x, y, z = oracle.three_sum(a, b, c)
        assert F(x) + F(y) + F(z) == F(a) + F(b) + F(c)
        assert x == (a + b) + c or x == c + (a + b)  # leading term is the rounded sum
        p, q = oracle.three_sum2(a, b, c)
        exact_sum = F(a) + F(b) + F(c)
        # only the final addition of the two error terms is rounded
        assert abs(F(p) + F(q) - exact_sum) <= abs(F(q)) * F(1, 2 ** 52) + F(0)


@pytest.mark.parametrize("n_in,fn", [(5, oracle.renorm5), (4, oracle.renorm4)])
def test_renorm_preserves_value_and_separates_components(n_in, fn):
    rng = random.Random(5)
    for _ in range(300):
        c = [rng.uniform(-1, 1)]
        for k in range(1, n_in):
            c.append(rng.uniform(-1, 1) * 2.0 ** (-50 * k) * rng.choice([1, 4, 0.25]))
        r = fn(np.array(c))
        total = sum(F(v) for v in c)
        # value kept to the weight of the last output component
        err = abs(fr(r) - total)
        assert err <= abs(F(float(r[-1]))) * F(1, 2 ** 50) + abs(total) * F(1, 2 ** (53 * (n_in - 1) + 2))
        # non-overlapping: each component is at most half an ulp of the previous
        for k in range(1, len(r)):
            if r[k - 1] != 0:
                assert abs(r[k]) <= math.ulp(r[k - 1]) / 2 * (1 + 2 ** -52)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_add_within_sloppy_bound(L):
    rng = np.random.default_rng(10 + L)
    worst = 0
    for t in range(400):
        a = rand_mp(rng, L, int(rng.integers(-3, 3)))
        b = rand_mp(rng, L, int(rng.integers(-3, 3)))
        if t % 4 == 0:            # heavy cancellation
            b = -a.copy()
            b[-1] *= 0.5
        r = oracle.mp_add(L, a, b)
        err = abs(fr(r) - (fr(a) + fr(b)))
        scale = abs(fr(a)) + abs(fr(b))
        if scale:
            worst = max(worst, err / (U[L] * scale))
    assert worst <= 4, float(worst)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_mul_within_bound(L):
    rng = np.random.default_rng(20 + L)
    worst = 0
    for _ in range(400):
        a = rand_mp(rng, L, int(rng.integers(-20, 20)))
        b = rand_mp(rng, L, int(rng.integers(-20, 20)))
        r = oracle.mp_mul(L, a, b)
        err = abs(fr(r) - fr(a) * fr(b))
        worst = max(worst, err / (U[L] * abs(fr(a) * fr(b))))
    assert worst <= 8, float(worst)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_mul_d_exact_for_power_of_two_and_bounded_otherwise(L):
    """Algorithms 3-5.  With y = 2^k the product x*y is representable, so a
    correct MP x binary64 product returns it exactly; the printed DDmulD step
    'p2 := x[1] + p2' (no multiply) would fail this immediately."""
    rng = np.random.default_rng(30 + L)
    for k in (-3, 0, 1, 7):
        x = rand_mp(rng, L)
        r = oracle.mp_mul_d(L, x, 2.0 ** k)
        assert fr(r) == fr(x) * F(2) ** k
    worst = 0
    for _ in range(400):
        x = rand_mp(rng, L, int(rng.integers(-10, 10)))
        y = float(rng.uniform(-4, 4))
        r = oracle.mp_mul_d(L, x, y)
        err = abs(fr(r) - fr(x) * F(y))
        worst = max(worst, err / (U[L] * abs(fr(x) * F(y))))
    assert worst <= 8, float(worst)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_div_within_bound(L):
    rng = np.random.default_rng(40 + L)
    worst = 0
    for _ in range(200):
        a = rand_mp(rng, L, int(rng.integers(-10, 10)))
        b = rand_mp(rng, L, int(rng.integers(-10, 10)))
        q = oracle.mp_div(L, a, b)
        err = abs(fr(q) - fr(a) / fr(b))
        worst = max(worst, err / (U[L] * abs(fr(a) / fr(b))))
    assert worst <= 16, float(worst)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_integer_arithmetic_is_exact(L):
    """Integer operands with results below 2^53: every operation is exact and
    the lower components come out zero."""
    rng = np.random.default_rng(50 + L)
    for _ in range(200):
        a, b = (float(v) for v in rng.integers(-2 ** 20, 2 ** 20, 2))
        A = np.zeros(L); A[0] = a
        B = np.zeros(L); B[0] = b
        s = oracle.mp_add(L, A, B)
        p = oracle.mp_mul(L, A, B)
        assert s[0] == a + b and not s[1:].any()
        assert p[0] == a * b and not p[1:].any()


def test_sqrt2_squared_matches_two():
    """sqrt(2) rounded to L components, squared in the working precision, is
    2 within the format's unit roundoff (closed form)."""
    for L in (2, 3, 4):
        v = exact.sample_vector(1, L)[:, 0]
        r = oracle.mp_mul(L, v, v)
        assert abs(fr(r) - 2) <= 8 * U[L] * 2


# Operation counts of the algorithms as implemented (binary64 add, sub, mul,
# fma, div each count one).  They fix the algorithmic work per nonzero used by
# the roofline: one MP multiply and one MP add per stored entry (P mode).
OPS = {
    ("add", 2): 11, ("mul", 2): 9, ("mul_d", 2): 6,    # Algorithms 1, 2, 3
    ("add", 3): 88, ("mul", 3): 124, ("mul_d", 3): 50,  # TDaddq, TDmulq, Algorithm 5
    ("add", 4): 87, ("mul", 4): 123, ("mul_d", 4): 69,  # QD sloppy add, mul, Algorithm 4
}


@pytest.mark.parametrize("L", [2, 3, 4])
def test_operation_counts(L):
    rng = np.random.default_rng(60)
    a, b = rand_mp(rng, L), rand_mp(rng, L)
    oracle.ops_reset(); oracle.mp_add(L, a, b, counting=True)
    assert oracle.ops_get() == OPS[("add", L)]
    oracle.ops_reset(); oracle.mp_mul(L, a, b, counting=True)
    assert oracle.ops_get() == OPS[("mul", L)]
    oracle.ops_reset(); oracle.mp_mul_d(L, a, 1.7, counting=True)
    assert oracle.ops_get() == OPS[("mul_d", L)]


def test_qd_and_td_against_mpmath_600():
    mpmath = pytest.importorskip("mpmath")
    from oracle import mpref
    rng = np.random.default_rng(70)
    for L in (3, 4):
        for _ in range(50):
            a, b = rand_mp(rng, L), rand_mp(rng, L)
            with mpmath.workprec(600):
                ref_p = mpref.mpf_of(a) * mpref.mpf_of(b)
                ref_s = mpref.mpf_of(a) + mpref.mpf_of(b)
            assert mpref.rel_err(oracle.mp_mul(L, a, b), ref_p) <= 8 * float(U[L])
            e = mpref.rel_err(oracle.mp_add(L, a, b), ref_s)
            assert e * abs(float(ref_s)) <= 4 * float(U[L]) * (abs(a[0]) + abs(b[0])) * 1.01
