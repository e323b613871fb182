"""Pins of the selector's feature oracle (oracle/features.py) against values
derived by hand from the feature definitions, on matrices whose statistics
have closed forms.  A slip in any single feature (a sign in the Gershgorin
bounds, population against sample deviation, the bandwidth normalisation,
row against column sums, the dominance caps) changes one of the numbers
below.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import workloads
from oracle import features as fo


def _csr(coo):
    return oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.promoted(1), 1)


def _lg(v):
    return math.log10(v)


@pytest.mark.parametrize("N", [4, 7, 64])
def test_laplacian_closed_forms(N):
    """2D 5-point Laplacian on an N x N grid (diagonal 4, neighbours -1):
    rows of 3 (4 corners), 4 (4(N-2) edge cells) and 5 ((N-2)^2 interior
    cells) entries; every off-diagonal sum is 2, 3 or 4 against a diagonal
    of 4, so ||A||_1 = ||A||_inf = 8 and the Gershgorin interval is [0, 8]."""
    n = N * N
    coo = workloads.laplacian_2d(N)
    A = _csr(coo)
    b = np.ones(n)
    f = fo.features(A, b)
    counts = {3: 4, 4: 4 * (N - 2), 5: (N - 2) ** 2}
    nnz = 5 * n - 4 * N
    assert A.nnz == nnz
    mean = nnz / n
    var = sum(c * (k - mean) ** 2 for k, c in counts.items()) / n        # population variance
    m3 = sum(c * (k - mean) ** 3 for k, c in counts.items()) / n
    sd = math.sqrt(var)
    edges = 2 * N * (N - 1)                                               # neighbour pairs
    dom_mean = (4 * 2.0 + 4 * (N - 2) * (4.0 / 3.0) + (N - 2) ** 2 * 1.0) / n
    want = {
        0: _lg(n), 1: _lg(nnz), 2: mean, 3: sd, 4: 3.0, 5: 5.0, 6: sd / mean, 7: m3 / sd ** 3, 8: 0.0,
        9: N / n,                                  # the vertical neighbour is N columns away
        10: _lg(1.0),                              # interior: 4 / 4
        11: _lg(dom_mean),
        12: _lg(2.0),                              # corners: 4 / 2
        13: 1.0,                                   # every row weakly dominant
        14: _lg(8.0), 15: _lg(8.0),
        16: _lg(math.sqrt(16 * n + 2 * edges)),
        17: _lg(4.0), 18: _lg(4.0), 19: 0.0,
        20: 0.0,                                   # min(4 - R_i) = 4 - 4
        21: 1.0,                                   # max(4 + R_i) / ||A||_inf = 8 / 8
        31: _lg(math.sqrt(16 * n + 2 * edges)) - _lg(4.0),
    }
    for i, v in want.items():
        assert f[i] == pytest.approx(v, rel=1e-12, abs=1e-12), i


def test_nonsymmetric_small_closed_forms():
    """A = [[2, -7, 0], [0, 3, 1], [0, 0, -5]]: row sums 9, 4, 5 and column
    sums 2, 10, 6 separate ||A||_inf from ||A||_1; the row lengths 2, 2, 1
    separate the population from the sample deviation; a negative diagonal
    and a zero off-diagonal sum exercise the dominance caps."""
    row = np.array([0, 0, 1, 1, 2])
    col = np.array([0, 1, 1, 2, 2])
    val = np.array([[2.0, -7.0, 3.0, 1.0, -5.0]])
    A = _csr(workloads.COO(3, 3, row, col, val))
    f = fo.features(A, np.array([1.0, -1.0, 0.5]))
    mean = 5.0 / 3.0
    sd = math.sqrt(2.0 / 9.0)                       # population: ((1/3)^2 * 2 + (2/3)^2) / 3
    m3 = ((1.0 / 3.0) ** 3 * 2 + (-2.0 / 3.0) ** 3) / 3.0
    want = {
        0: _lg(3), 1: _lg(5), 2: mean, 3: sd, 4: 1.0, 5: 2.0, 6: sd / mean, 7: m3 / sd ** 3, 8: 0.0,
        9: 1.0 / 3.0,
        10: _lg(2.0 / 7.0),
        11: _lg((2.0 / 7.0 + 3.0 + 1e6) / 3.0),     # the empty off-diagonal row counts as 1e6 in the mean
        12: 30.0,                                   # ... and as 1e30 in the maximum
        13: 2.0 / 3.0,
        14: _lg(10.0), 15: _lg(9.0),
        16: _lg(math.sqrt(4 + 49 + 9 + 1 + 25)),
        17: _lg(5.0), 18: _lg(2.0), 19: _lg(5.0) - _lg(2.0),
        20: -5.0 / 9.0,                             # min(a_ii - R_i) = min(2 - 7, 3 - 1, -5 - 0)
        21: 1.0,                                    # max(a_ii + R_i) = 2 + 7 over ||A||_inf = 9
        31: _lg(math.sqrt(88.0)) - _lg(5.0),
    }
    for i, v in want.items():
        assert f[i] == pytest.approx(v, rel=1e-12, abs=1e-12), i


def test_diagonal_matrix_and_exact_cg_step():
    """A = diag(-7, 1, 2, 5, 1): no off-diagonal entries (dominance 1e30,
    bandwidth 0, row lengths constant); the largest |a_ii| is negative, so
    the upper Gershgorin bound (5) differs from max |a_ii| (7).  And binary64
    CG on diag(1, 3) with b = (1, 1): alpha = 2 / 4, r_1 = (1/2, -1/2),
    ||r_1|| / ||b|| = 1/2, all exact in binary64; on 2^k I it stops after
    one step with r_1 = 0 exactly (every later entry is the -300 of a zero
    norm)."""
    d = np.array([-7.0, 1.0, 2.0, 5.0, 1.0])
    n = d.size
    A = _csr(workloads.COO(n, n, np.arange(n), np.arange(n), d[None, :]))
    f = fo.features(A, np.ones(n))
    want = {2: 1.0, 3: 0.0, 4: 1.0, 5: 1.0, 6: 0.0, 7: 0.0, 8: 0.0, 9: 0.0, 10: 30.0, 11: 6.0, 12: 30.0, 13: 1.0,
            14: _lg(7.0), 15: _lg(7.0), 16: _lg(math.sqrt(80.0)), 17: _lg(7.0), 18: 0.0, 19: _lg(7.0),
            20: -1.0, 21: 5.0 / 7.0}
    for i, v in want.items():
        assert f[i] == pytest.approx(v, rel=1e-12, abs=1e-12), i

    h = fo.cg_history(np.array([0, 1, 2]), np.array([0, 1]), np.array([1.0, 3.0]), np.array([1.0, 1.0]), 1)
    assert h[0] == 0.5

    with np.errstate(all="ignore"):
        A8 = _csr(workloads.COO(4, 4, np.arange(4), np.arange(4), np.full((1, 4), 8.0)))
        f8 = fo.features(A8, np.array([0.3, -1.7, 2.2, 0.9]))
    assert np.all(f8[22:30] == -300.0)
    assert f8[30] == pytest.approx(0.0, abs=1e-12)


def _krylov_residuals(M, b, k):
    """||b - A x_j|| / ||b|| for x_j the A-norm minimiser over the Krylov
    space K_j(A, b) (the characterisation of CG iterates), from an
    orthonormal basis of [b, Ab, ..., A^(j-1) b] and a j x j solve."""
    out = []
    for j in range(1, k + 1):
        K = np.empty((len(b), j))
        v = b.copy()
        for t in range(j):
            K[:, t] = v
            v = M @ v
        Q, _ = np.linalg.qr(K)
        y = np.linalg.solve(Q.T @ M @ Q, Q.T @ b)
        out.append(np.linalg.norm(b - M @ (Q @ y)) / np.linalg.norm(b))
    return np.array(out)


def test_cg_history_is_the_krylov_minimiser():
    """Features 22-29: the residual norms of the first 8 CG steps equal those
    of the A-norm minimisers over the Krylov spaces, computed by dense
    projection (a different definition of the same iterates); feature 30 is
    their least-squares slope against the step number."""
    rng = np.random.default_rng(5)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(1.0, 30.0, n)
    M = (Q * lam) @ Q.T
    M = 0.5 * (M + M.T)
    r, c = np.nonzero(np.ones((n, n)))
    A = _csr(workloads.COO(n, n, r, c, M[r, c][None, :]))
    b = rng.uniform(-1, 1, n)
    f = fo.features(A, b)
    want = _krylov_residuals(M, b, 8)
    np.testing.assert_allclose(10.0 ** f[22:30], want, rtol=1e-7)
    slope = np.linalg.lstsq(np.stack([np.arange(1, 9), np.ones(8)], axis=1), f[22:30], rcond=None)[0][0]
    assert f[30] == pytest.approx(slope, rel=1e-10)
