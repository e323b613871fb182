"""Pins for the oracle's Krylov solvers (Section 4.2: CG on an SPD matrix,
BiCGSTAB on a nonsymmetric one; x0 = 0; stopping test on the residual norm)
and its vector kernels.  References: exact rational solves, exact residuals
computed with big integers, closed forms."""
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
import workloads
from oracle import exact


def dense_exact(A):
    n = A.nrows
    M = [[F(0)] * n for _ in range(n)]
    for i in range(n):
        for k in range(A.indptr[i], A.indptr[i + 1]):
            M[i][A.indices[k]] = exact.to_fraction(A.data[:A.L, k])
    return M


def solve_exact(M, b):
    """Gaussian elimination in rationals (small n)."""
    n = len(M)
    Aug = [row[:] + [b[i]] for i, row in enumerate(M)]
    for c in range(n):
        p = next(r for r in range(c, n) if Aug[r][c] != 0)
        Aug[c], Aug[p] = Aug[p], Aug[c]
        for r in range(n):
            if r != c and Aug[r][c] != 0:
                f = Aug[r][c] / Aug[c][c]
                Aug[r] = [a - f * b_ for a, b_ in zip(Aug[r], Aug[c])]
    return [Aug[i][n] / Aug[i][i] for i in range(n)]


def exact_residual_norm2(A, x, b):
    """||b - A x||^2 exactly (real or complex), as a Fraction."""
    L = A.L
    ex_re, ex_im, _, _ = exact.exact_rows(A, x)
    den = 1 << (2 * exact.SCALE)
    tot = F(0)
    for i in range(A.nrows):
        br = exact.to_fraction(b[:L, i])
        tot += (br - F(ex_re[i], den)) ** 2
        if A.cplx:
            bi = exact.to_fraction(b[L:, i])
            tot += (bi - F(ex_im[i], den)) ** 2
    return tot


def norm2(v, L, cplx):
    t = sum(exact.to_fraction(v[:L, i]) ** 2 for i in range(v.shape[1]))
    if cplx:
        t += sum(exact.to_fraction(v[L:, i]) ** 2 for i in range(v.shape[1]))
    return t


@pytest.mark.parametrize("L", [2, 3, 4])
def test_cg_solves_spd_system_exactly_checked(L):
    coo = workloads.laplacian_2d(5)      # n = 25, SPD
    A = oracle.coo_to_csr(25, 25, coo.row, coo.col, coo.promoted(L), L)
    xt = np.arange(1, 26, dtype=float)
    b = np.zeros((L, 25)); b[0] = oracle.spmv(oracle.coo_to_csr(25, 25, coo.row, coo.col, coo.val, 1),
                                               xt[None, :])[0]
    st, x, it, rr = oracle.cg(A, b, rtol=1e-28 if L > 2 else 1e-28, maxit=200)
    assert st == 0 and it <= 26
    xs = solve_exact(dense_exact(A), [exact.to_fraction(b[:, i]) for i in range(25)])
    assert xs == [F(int(v)) for v in xt]
    err = max(abs(exact.to_fraction(x[:, i]) - xs[i]) for i in range(25))
    assert err <= F(1, 10 ** 24) * 25
    assert exact_residual_norm2(A, x, b) <= (F(1, 10 ** 28) ** 2) * norm2(b, L, False) * 4
    assert rr <= 2e-28


def test_cg_diagonal_converges_in_one_iteration():
    n = 10
    d = np.zeros((2, n)); d[0] = np.arange(1, n + 1)
    A = oracle.coo_to_csr(n, n, np.arange(n), np.arange(n), d, 2)
    b = np.zeros((2, n)); b[0, 3] = 5.0
    st, x, it, rr = oracle.cg(A, b, rtol=1e-30, maxit=10)
    assert st == 0 and it == 1
    assert x[0, 3] == 5.0 / 4.0 and rr == 0.0


def test_cg_iteration_counts_do_not_grow_with_precision():
    """Section 4.2: as the precision rises the CG iteration count settles; on
    an ill-conditioned SPD system the higher formats never need more steps."""
    rng = np.random.default_rng(1)
    n = 60
    coo = workloads.laplacian_2d(6, 10)
    scale = 10.0 ** rng.uniform(-3, 3, n)
    its = []
    for L in (2, 3, 4):
        # D A D with a graded diagonal scaling: SPD, condition ~1e9
        v = coo.val[0] * (scale[coo.row] * scale[coo.col])   # exactly symmetric
        vv = np.zeros((L, coo.nnz)); vv[0] = v
        A = oracle.coo_to_csr(n, n, coo.row, coo.col, vv, L)
        b = np.zeros((L, n)); b[0] = 1.0
        st, x, it, rr = oracle.cg(A, b, rtol=1e-25, maxit=2000)
        assert st == 0 and rr <= 1e-24
        its.append(it)
    assert its[0] >= its[1] >= its[2]


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_bicgstab_nonsymmetric_exact_residual(L, cplx):
    n = 30
    coo = workloads.random_sparse(n, n, 5, seed=20 + L, cplx=cplx, L=1)
    # make it diagonally dominant-ish with a shift
    rows = np.concatenate([coo.row, np.arange(n)])
    cols = np.concatenate([coo.col, np.arange(n)])
    shift = np.zeros((coo.val.shape[0], n)); shift[0] = 8.0
    if cplx:
        shift[1] = 2.0
    vals = np.concatenate([coo.val, shift], axis=1)
    V = vals.shape[0]
    vv = np.zeros((V * L, vals.shape[1]))
    for c in range(V):
        vv[c * L] = vals[c]
    A = oracle.coo_to_csr(n, n, rows, cols, vv, L, cplx)
    b = workloads.full_limb_vector(n, L, seed=3, cplx=cplx)
    st, x, it, rr = oracle.bicgstab(A, b, rtol=1e-25, maxit=300)
    assert st == 0 and it < 100
    assert exact_residual_norm2(A, x, b) <= (F(10) ** -50) * norm2(b, L, cplx) * 4
    assert rr <= 2e-25
    if not cplx:
        xs = solve_exact(dense_exact(A), [exact.to_fraction(b[:, i]) for i in range(n)])
        err = max(abs(exact.to_fraction(x[:, i]) - xs[i]) for i in range(n))
        assert err <= F(1, 10 ** 20)


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_dot_and_axpy_against_exact(L, cplx):
    n = 50
    u = workloads.full_limb_vector(n, L, seed=1, cplx=cplx)
    v = workloads.full_limb_vector(n, L, seed=2, cplx=cplx)
    dr, di = oracle.dot(L, u, v, cplx)
    er = sum(exact.to_fraction(u[:L, i]) * exact.to_fraction(v[:L, i]) for i in range(n))
    ab = sum(abs(exact.to_fraction(u[:L, i]) * exact.to_fraction(v[:L, i])) for i in range(n))
    if cplx:   # conj(u) v
        er += sum(exact.to_fraction(u[L:, i]) * exact.to_fraction(v[L:, i]) for i in range(n))
        ei = sum(exact.to_fraction(u[:L, i]) * exact.to_fraction(v[L:, i])
                 - exact.to_fraction(u[L:, i]) * exact.to_fraction(v[:L, i]) for i in range(n))
        ab *= 4
        assert abs(exact.to_fraction(di) - ei) <= 8 * 2 * n * F(exact.U[L]) * ab
    assert abs(exact.to_fraction(dr) - er) <= 8 * 2 * n * F(exact.U[L]) * ab
    a = workloads.full_limb_vector(1, L, seed=3)[:, 0]
    w = oracle.axpy(L, a, u, v, alpha_im=(a * 0.5 if cplx else None), cplx=cplx)
    for i in range(0, n, 7):
        ur, vr = exact.to_fraction(u[:L, i]), exact.to_fraction(v[:L, i])
        A_ = exact.to_fraction(a)
        if cplx:
            ui, vi = exact.to_fraction(u[L:, i]), exact.to_fraction(v[L:, i])
            Ai = A_ / 2
            wr, wi = ur + A_ * vr - Ai * vi, ui + A_ * vi + Ai * vr
            sc = abs(ur) + abs(ui) + 2 * (abs(A_) + abs(Ai)) * (abs(vr) + abs(vi))
            assert abs(exact.to_fraction(w[L:, i]) - wi) <= 32 * F(exact.U[L]) * sc
        else:
            wr = ur + A_ * vr
            sc = abs(ur) + abs(A_ * vr)
        assert abs(exact.to_fraction(w[:L, i]) - wr) <= 32 * F(exact.U[L]) * sc


# ---------------------------------------------------------------------------
# BiCG, CGS, GPBiCG (the other product-type methods of Section 4.2)
# ---------------------------------------------------------------------------
def shifted_nonsym(n, L, cplx, seed):
    coo = workloads.random_sparse(n, n, 5, seed=seed, cplx=cplx, L=1)
    rows = np.concatenate([coo.row, np.arange(n)])
    cols = np.concatenate([coo.col, np.arange(n)])
    shift = np.zeros((coo.val.shape[0], n)); shift[0] = 8.0
    if cplx:
        shift[1] = 2.0
    vals = np.concatenate([coo.val, shift], axis=1)
    vv = np.zeros((vals.shape[0] * L, vals.shape[1]))
    for c in range(vals.shape[0]):
        vv[c * L] = vals[c]
    return oracle.coo_to_csr(n, n, rows, cols, vv, L, cplx)


SOLVERS = {"bicg": oracle.bicg, "cgs": oracle.cgs, "gpbicg": oracle.gpbicg}


@pytest.mark.parametrize("method", sorted(SOLVERS))
@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_product_type_methods_exact_residual_and_solution(method, L, cplx):
    n = 30
    A = shifted_nonsym(n, L, cplx, seed=40 + L)
    b = workloads.full_limb_vector(n, L, seed=4, cplx=cplx)
    st, x, it, rr = SOLVERS[method](A, b, rtol=1e-25, maxit=300)
    assert st == 0 and 0 < it < 100
    assert exact_residual_norm2(A, x, b) <= (F(10) ** -50) * norm2(b, L, cplx) * 4
    assert rr <= 2e-25
    if not cplx:
        xs = solve_exact(dense_exact(A), [exact.to_fraction(b[:, i]) for i in range(n)])
        err = max(abs(exact.to_fraction(x[:, i]) - xs[i]) for i in range(n))
        assert err <= F(1, 10 ** 20)


@pytest.mark.parametrize("L", [2, 4])
def test_bicg_reduces_to_cg_on_symmetric_matrices(L):
    """For real symmetric A and r~_0 = r_0 the shadow recurrences repeat the
    primal ones (A^T p is the same row sum as A p), so BiCG is CG step for
    step: same iterations, bit-identical iterates."""
    coo = workloads.laplacian_2d(9, 7)
    A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.promoted(L), L)
    b = workloads.full_limb_vector(coo.nrows, L, seed=2)
    st1, x1, it1, rr1 = oracle.cg(A, b, rtol=1e-20, maxit=500)
    st2, x2, it2, rr2 = oracle.bicg(A, b, rtol=1e-20, maxit=500)
    assert st1 == st2 == 0 and it1 == it2 and rr1 == rr2
    assert np.array_equal(x1, x2)


@pytest.mark.parametrize("method", sorted(SOLVERS) + ["bicgstab"])
@pytest.mark.parametrize("cplx", [False, True])
def test_finite_termination_with_few_distinct_eigenvalues(method, cplx):
    """A diagonal matrix with m = 3 distinct eigenvalues: the Krylov space of
    any b has dimension 3, so every method reaches the QD-level residual in at
    most 3 iterations (the polynomial methods' termination property)."""
    L, n = 4, 24
    ev = [(2.0, 0.5), (3.0, -1.0), (7.0, 0.25)]
    V = 2 if cplx else 1
    vals = np.zeros((V * L, n))
    for i in range(n):
        vals[0, i] = ev[i % 3][0]
        if cplx:
            vals[L, i] = ev[i % 3][1]
    A = oracle.coo_to_csr(n, n, np.arange(n), np.arange(n), vals, L, cplx)
    b = workloads.full_limb_vector(n, L, seed=9, cplx=cplx)
    solver = oracle.bicgstab if method == "bicgstab" else SOLVERS[method]
    st, x, it, rr = solver(A, b, rtol=1e-50, maxit=10)
    assert st == 0 and it <= 3
    assert exact_residual_norm2(A, x, b) <= (F(10) ** -98) * norm2(b, L, cplx)
