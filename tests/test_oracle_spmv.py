"""Pins for the oracle's COO->CSR build and SpMV/SpMM (Section 3, Eq.
complex_spmv, Eq. sample_vector).  References: the paper's worked 5x5 example,
closed forms, exact big-integer evaluation, and mpmath at 600 bits."""
import json
import os
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
import workloads
from oracle import exact

GOLD = os.path.join(os.path.dirname(__file__), "golden", "worked_example_5x5.json")


def worked():
    with open(GOLD) as f:
        return json.load(f)


def _csr_from(coo, L):
    """Binary64 triplets promoted to L components (P mode)."""
    return oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.promoted(L), L, coo.cplx)


def test_coo_to_csr_matches_paper_worked_example():
    g = worked()
    A = oracle.coo_to_csr(5, 5, g["coo"]["row"], g["coo"]["col"], np.array([g["coo"]["data"]], float), 1)
    assert A.indptr.tolist() == g["csr"]["indptr"]
    assert A.indices.tolist() == g["csr"]["indices"]
    assert A.data[0].tolist() == g["csr"]["data"]


def test_coo_to_csr_any_order_and_duplicates():
    g = worked()
    rng = np.random.default_rng(0)
    perm = rng.permutation(8)
    row = np.array(g["coo"]["row"])[perm]
    col = np.array(g["coo"]["col"])[perm]
    dat = np.array(g["coo"]["data"], float)[perm]
    # split every value into two duplicate triplets that sum to it
    row2 = np.concatenate([row, row])
    col2 = np.concatenate([col, col])
    dat2 = np.concatenate([dat - 1.0, np.ones(8)])
    for L in (1, 2, 4):
        v = np.zeros((L, 16)); v[0] = dat2
        A = oracle.coo_to_csr(5, 5, row2, col2, v, L)
        assert A.indptr.tolist() == g["csr"]["indptr"]
        assert A.indices.tolist() == g["csr"]["indices"]
        assert A.data[0].tolist() == g["csr"]["data"]
    with pytest.raises(ValueError):
        oracle.coo_to_csr(5, 5, [0, 5], [0, 0], np.ones((1, 2)), 1)


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_worked_example_integer_vector_exact(L):
    g = worked()
    v = np.zeros((L, 8)); v[0] = g["coo"]["data"]
    A = oracle.coo_to_csr(5, 5, g["coo"]["row"], g["coo"]["col"], v, L)
    x = np.zeros((L, 5)); x[0] = [1, 2, 3, 4, 5]
    y = oracle.spmv(A, x)
    assert y[0].tolist() == g["A_times_1_to_5"]["value"]
    assert not y[1:].any()


@pytest.mark.parametrize("L", [2, 3, 4])
def test_worked_example_sample_vector_closed_form(L):
    """A (sqrt2 [1..5]) = sqrt2 [7,-14,15,-22,40] (Eq. sample_vector): the
    result equals the closed form within the componentwise bound."""
    g = worked()
    v = np.zeros((L, 8)); v[0] = g["coo"]["data"]
    A = oracle.coo_to_csr(5, 5, g["coo"]["row"], g["coo"]["col"], v, L)
    x = exact.sample_vector(5, L)
    y = oracle.spmv(A, x)
    s2 = F(exact.sqrt2_fixed(), 1 << 1200)
    for i, c in enumerate(g["A_times_1_to_5"]["value"]):
        absax = sum(abs(F(a)) * exact.to_fraction(x[:, j]) for a, j in
                    zip(A.data[0][A.indptr[i]:A.indptr[i + 1]], A.indices[A.indptr[i]:A.indptr[i + 1]]))
        err = abs(exact.to_fraction(y[:, i]) - s2 * c)
        assert err <= 8 * 2 * F(exact.U[L]) * absax + abs(s2 * c) * F(1, 2 ** 1100)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_worked_example_complex_closed_form(L):
    """Complex sample vector sqrt(2+3i)[1..5] with A real (A_im = 0), and with
    A purely imaginary (A_re = 0): results are sqrt(2+3i) * [7,...] and
    i * sqrt(2+3i) * [7,...].  A sign error in Eq. complex_spmv breaks one."""
    g = worked()
    cr, ci = exact.sqrt_2p3i_fixed()
    zr, zi = F(cr, 1 << 1200), F(ci, 1 << 1200)
    x = exact.sample_vector(5, L, cplx=True)
    for imag in (False, True):
        v = np.zeros((2 * L, 8)); v[L if imag else 0] = g["coo"]["data"]
        A = oracle.coo_to_csr(5, 5, g["coo"]["row"], g["coo"]["col"], v, L, cplx=True)
        y = oracle.spmv(A, x)
        for i, c in enumerate(g["A_times_1_to_5"]["value"]):
            er, ei = zr * c, zi * c
            if imag:
                er, ei = -ei, er
            tol = 64 * F(exact.U[L]) * (abs(er) + abs(ei)) * 8
            assert abs(exact.to_fraction(y[:L, i]) - er) <= tol
            assert abs(exact.to_fraction(y[L:, i]) - ei) <= tol


@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_integer_matrices_bit_exact(L, cplx):
    """Integer-valued A and x with all partial sums far below 2^53: the MP
    result is the exact integer in component 0 and zero below."""
    coo = workloads.integer_matrix(60, 50, 0.2, seed=L, cplx=cplx)
    A = _csr_from(coo, L)
    x = workloads.integer_vector(50, L, seed=7, cplx=cplx)
    y = oracle.spmv(A, x)
    Ad = np.zeros((60, 50), dtype=np.int64 if not cplx else np.complex128)
    for i in range(60):
        for k in range(A.indptr[i], A.indptr[i + 1]):
            Ad[i, A.indices[k]] = A.data[0, k] + (1j * A.data[L, k] if cplx else 0)
    xv = x[0] + (1j * x[L] if cplx else 0)
    ref = Ad @ xv
    assert np.array_equal(y[0], np.real(ref))
    if cplx:
        assert np.array_equal(y[L], np.imag(ref))
        assert not y[1:L].any() and not y[L + 1:].any()
    else:
        assert not y[1:].any()


@pytest.mark.parametrize("L", [2, 3, 4])
def test_diagonal_matrix_reduces_to_scalar_mul(L):
    rng = np.random.default_rng(L)
    n = 40
    d = workloads.full_limb_vector(n, L, seed=11)
    d[0, :5] = [2.0, -4.0, 0.5, 1.0, -1.0]
    d[1:, :5] = 0.0
    A = oracle.coo_to_csr(n, n, np.arange(n), np.arange(n), d, L)
    x = workloads.full_limb_vector(n, L, seed=12)
    y = oracle.spmv(A, x)
    for i in range(n):
        # adding a product to zero only renormalises it: value is the product
        p = oracle.mp_mul(L, d[:, i], x[:, i])
        assert exact.to_fraction(y[:, i]) == exact.to_fraction(p)
    for i in range(5):   # powers of two: exact
        assert exact.to_fraction(y[:, i]) == exact.to_fraction(d[:, i]) * exact.to_fraction(x[:, i])
    del rng


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_random_full_limb_within_bound(L, cplx):
    """Brute force with exact integers on a small matrix whose every
    component is random, with empty rows."""
    coo = workloads.random_sparse(48, 40, 12, seed=3 + L, cplx=cplx, L=L, full_limb=True, empty_frac=0.1)
    A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, L, cplx)
    x = workloads.full_limb_vector(40, L, seed=5, cplx=cplx)
    y = oracle.spmv(A, x)
    assert exact.bound_ratio(y, A, x) <= 1.0
    empty = np.nonzero(np.diff(A.indptr) == 0)[0]
    assert len(empty) > 0 and not y[:, empty].any()


@pytest.mark.parametrize("L", [2, 3, 4])
def test_laplacian_64x64_against_exact_and_mpmath(L):
    """Config: 2D 5-point Laplacian 64x64 (n = 4096, nnz = 20,224), binary64
    values promoted, x with every component random."""
    coo = workloads.laplacian_2d(64)
    assert coo.nnz == 20224
    A = _csr_from(coo, L)
    x = workloads.full_limb_vector(4096, L, seed=0)
    y = oracle.spmv(A, x)
    assert exact.bound_ratio(y, A, x) <= 1.0
    mpmath = pytest.importorskip("mpmath")
    from oracle import mpref
    rows = list(range(0, 4096, 97))
    re, _ = mpref.rows(A, x, rows)
    rnd = exact.exact_round_rows(A, x, rows)
    for s, i in enumerate(rows):
        # exact module and mpmath agree to 600 bits on the reference value
        assert mpref.rel_err(rnd[:, s], re[s]) <= 2.0 ** (-53 * L + 1)
        ab = sum(abs(mpref.mpf_of(A.data[:, k]) * mpref.mpf_of(x[:, A.indices[k]]))
                 for k in range(A.indptr[i], A.indptr[i + 1]))
        with mpmath.workprec(600):
            err = abs(mpref.mpf_of(y[:, i]) - re[s])
        assert err <= 8 * 5 * exact.U[L] * ab


def test_spmm_equals_columnwise_spmv():
    for L, cplx in ((2, False), (4, True)):
        coo = workloads.random_sparse(30, 25, 6, seed=1, cplx=cplx, L=L, full_limb=True)
        A = oracle.coo_to_csr(30, 25, coo.row, coo.col, coo.val, L, cplx)
        P = A.P
        X = np.stack([workloads.full_limb_vector(25, L, seed=c, cplx=cplx) for c in range(5)], axis=-1)
        Y = oracle.spmm(A, X)
        for c in range(5):
            assert np.array_equal(Y[:, :, c], oracle.spmv(A, X[:, :, c]))
        assert Y.shape == (P, 30, 5)


def test_spmv_rows_equals_full():
    coo = workloads.random_sparse(50, 50, 9, seed=2, L=3, full_limb=True)
    A = oracle.coo_to_csr(50, 50, coo.row, coo.col, coo.val, 3)
    x = workloads.full_limb_vector(50, 3, seed=9)
    y = oracle.spmv(A, x)
    rows = [0, 7, 49, 3]
    assert np.array_equal(oracle.spmv_rows(A, x, rows), y[:, rows])


@pytest.mark.parametrize("L", [2, 4])
def test_mixed_mode_within_bound(L):
    """M mode (binary64 A with Algorithms 3-5) agrees with the exact product
    within the same bound."""
    coo = workloads.random_sparse(40, 40, 10, seed=8)
    A1 = oracle.coo_to_csr(40, 40, coo.row, coo.col, coo.val, 1)
    x = workloads.full_limb_vector(40, L, seed=4)
    Am = oracle.CSR(40, 40, A1.indptr, A1.indices, A1.data, L, False)
    y = oracle.spmv(Am, x, mixed=True)
    Ap = oracle.coo_to_csr(40, 40, coo.row, coo.col, coo.promoted(L), L)
    assert exact.bound_ratio(y, Ap, x) <= 1.0


def test_exact_module_pins():
    """The exact module itself: f2i on edge values and greedy rounding."""
    assert exact.f2i(5e-324) == 1
    assert exact.f2i(1.0) == 1 << 1074
    assert exact.f2i(-0.75) == -(3 << 1072)
    r = exact.round_greedy(F(1, 3), 3)
    assert r[0] == 1 / 3 and abs(exact.to_fraction(r) - F(1, 3)) < F(1, 2 ** 160)
    s = F(exact.sqrt2_fixed(), 1 << 1200)
    assert abs(s * s - 2) < F(1, 2 ** 1190)
    cr, ci = exact.sqrt_2p3i_fixed()
    zr, zi = F(cr, 1 << 1200), F(ci, 1 << 1200)
    assert abs(zr * zr - zi * zi - 2) < F(1, 2 ** 1180) and abs(2 * zr * zi - 3) < F(1, 2 ** 1180)


# ---------------------------------------------------------------------------
# SpTMV y = A^T x (Section 4, "A^T v"): the oracle's row-oriented scatter
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_spmtv_worked_example_brute_force(L):
    g = worked()
    v = np.zeros((L, 8)); v[0] = g["coo"]["data"]
    A = oracle.coo_to_csr(5, 5, g["coo"]["row"], g["coo"]["col"], v, L)
    x = np.zeros((L, 5)); x[0] = [1, 2, 3, 4, 5]
    y = oracle.spmtv(A, x)
    ref = [sum(d * (r + 1) for d, r, c in zip(g["coo"]["data"], g["coo"]["row"], g["coo"]["col"]) if c == j)
           for j in range(5)]
    assert y[0].tolist() == ref
    assert not y[1:].any()


@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_spmtv_equals_spmv_of_the_transpose(L, cplx):
    """The scatter sums each y_j in increasing row order, the order of row j
    of the transposed CSR: bit-identical to the row sum of A^T built from the
    swapped triplets, and within the exact bound."""
    coo = workloads.random_sparse(70, 50, 8, seed=20 + L, cplx=cplx, L=L, full_limb=True, empty_frac=0.1)
    A = oracle.coo_to_csr(70, 50, coo.row, coo.col, coo.val, L, cplx)
    AT = oracle.coo_to_csr(50, 70, coo.col, coo.row, coo.val, L, cplx)
    x = workloads.full_limb_vector(70, L, seed=5, cplx=cplx)
    y = oracle.spmtv(A, x)
    assert y.shape == (A.P, 50)
    assert np.array_equal(y, oracle.spmv(AT, x))
    assert exact.bound_ratio(y, AT, x) <= 1.0


@pytest.mark.parametrize("L", [2, 4])
def test_spmtv_mixed_mode_and_duplicates(L):
    coo = workloads.random_sparse(40, 30, 10, seed=9)
    A1 = oracle.coo_to_csr(40, 30, coo.row, coo.col, coo.val, 1)
    AT1 = oracle.coo_to_csr(30, 40, coo.col, coo.row, coo.val, 1)
    Am = oracle.CSR(40, 30, A1.indptr, A1.indices, A1.data, L, False)
    ATm = oracle.CSR(30, 40, AT1.indptr, AT1.indices, AT1.data, L, False)
    x = workloads.full_limb_vector(40, L, seed=6)
    assert np.array_equal(oracle.spmtv(Am, x, mixed=True), oracle.spmv(ATm, x, mixed=True))
    # integer data with duplicated triplets: exact
    ic = workloads.integer_matrix(30, 25, 0.2, seed=3, dup_frac=0.3)
    Ai = oracle.coo_to_csr(30, 25, ic.row, ic.col, ic.promoted(L), L)
    xi = workloads.integer_vector(30, L, seed=2)
    dense = np.zeros((30, 25))
    np.add.at(dense, (ic.row, ic.col), ic.val[0])
    ref = dense.T @ xi[0]
    yi = oracle.spmtv(Ai, xi)
    assert np.array_equal(yi[0], ref) and not yi[1:].any()
