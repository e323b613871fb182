"""GPU parity of the multiple-precision SpMV / SpMM (C ABI) against the oracle.

Two levels (arXiv 2412.17510, Section 3):
  * rows whose entries one thread sums end to end are computed with the same
    operation sequence as the oracle's row sweep: they must agree limb for
    limb (values compared as binary64, so +0 == -0);
  * every row must meet the componentwise bound 8 m u (|A||x|)_i against the
    exact value (big-integer evaluation).
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle import exact
from tests._util import csr_pair, gpu_spmv, to_dev, unsplit_rows

pytestmark = pytest.mark.gpu

mps = pytest.importorskip("paper_2412_17510_gb300")
torch = pytest.importorskip("torch")

FLAG = {False: 0, True: 1}


def _check(A, h, x, y):
    K = mps.mpspmv_get_info(h)["chunk"]
    ref = oracle.spmv(A, x)
    rows = unsplit_rows(A, K)
    assert np.array_equal(y[:, rows], ref[:, rows]), "run-internal rows differ from the oracle"
    assert exact.bound_ratio(y, A, x) <= 1.0
    return ref


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_random_full_limb_matrix(L, cplx):
    """Every component random, several tiles of runs plus a ragged tail, empty
    rows, and a few long rows that span many runs."""
    coo = workloads.random_sparse(700, 650, 24, seed=L, cplx=cplx, L=L, full_limb=True, empty_frac=0.1)
    # add three long rows (200-400 entries)
    rng = np.random.default_rng(1)
    extra_r, extra_c = [], []
    for r, ln in ((5, 400), (300, 200), (699, 333)):
        extra_r.append(np.full(ln, r))
        extra_c.append(np.sort(rng.choice(650, ln, replace=False)))
    er, ec = np.concatenate(extra_r), np.concatenate(extra_c)
    keep = ~np.isin(coo.row, [5, 300, 699])
    row = np.concatenate([coo.row[keep], er])
    col = np.concatenate([coo.col[keep], ec])
    P = coo.val.shape[0]
    ev = workloads.full_limb_vector(er.shape[0], L, seed=9, cplx=cplx)
    val = np.concatenate([coo.val[:, keep], ev], axis=1)
    big = workloads.COO(700, 650, row, col, val)
    A, h = csr_pair(big, L, vals=val, flags=FLAG[cplx])
    try:
        info = mps.mpspmv_get_info(h)
        assert info["nsplit_rows"] > 3 and info["nchunks"] > 64
        x = workloads.full_limb_vector(650, L, seed=2, cplx=cplx)
        y = gpu_spmv(h, x, P, 700)
        _check(A, h, x, y)
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_laplacian_64x64(L):
    """2D 5-point Laplacian 64x64 (n = 4096, nnz = 20,224), binary64 values
    promoted, x with every component random."""
    coo = workloads.laplacian_2d(64)
    A, h = csr_pair(coo, L)
    try:
        x = workloads.full_limb_vector(4096, L, seed=0)
        y = gpu_spmv(h, x, L, 4096)
        _check(A, h, x, y)
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_integer_matrices_bit_exact(L, cplx):
    coo = workloads.integer_matrix(300, 280, 0.05, seed=L, cplx=cplx)
    A, h = csr_pair(coo, L, flags=FLAG[cplx])
    try:
        x = workloads.integer_vector(280, L, seed=7, cplx=cplx)
        y = gpu_spmv(h, x, A.P, 300)
        ref = oracle.spmv(A, x)
        assert np.array_equal(y, ref)
        lo = [p for p in range(A.P) if p % L != 0]
        assert not y[lo].any()
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_worked_example_5x5(L, cplx):
    """Section 3 example: A [1..5] = [7,-14,15,-22,40] exactly, and the sample
    vector of Eq. sample_vector against the oracle."""
    data = np.array([1, 2, 3, -4, 5, 6, -7, 8], float)
    row = np.array([0, 0, 1, 1, 2, 3, 3, 4])
    col = np.array([0, 2, 1, 4, 2, 0, 3, 4])
    V = 2 if cplx else 1
    val = np.zeros((V, 8)); val[0] = data
    coo = workloads.COO(5, 5, row, col, val)
    A, h = csr_pair(coo, L, flags=FLAG[cplx])
    try:
        x = np.zeros((A.P, 5)); x[0] = [1, 2, 3, 4, 5]
        y = gpu_spmv(h, x, A.P, 5)
        assert y[0].tolist() == [7, -14, 15, -22, 40] and not y[1:].any()
        v = exact.sample_vector(5, L, cplx=cplx)
        y = gpu_spmv(h, v, A.P, 5)
        assert np.array_equal(y, oracle.spmv(A, v))
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_mixed_mode(L, cplx):
    coo = workloads.random_sparse(400, 400, 30, seed=4, cplx=cplx)
    A1 = oracle.coo_to_csr(400, 400, coo.row, coo.col, coo.val, 1, cplx)
    Am = oracle.CSR(400, 400, A1.indptr, A1.indices, A1.data, L, cplx)
    Ap = oracle.coo_to_csr(400, 400, coo.row, coo.col, coo.promoted(L), L, cplx)
    h = mps.mpspmv_create_csr(400, 400, coo.row, coo.col, coo.val, L, FLAG[cplx] | mps.MPSPMV_MIXED, val_limbs=1)
    try:
        x = workloads.full_limb_vector(400, L, seed=3, cplx=cplx)
        y = gpu_spmv(h, x, Ap.P, 400)
        K = mps.mpspmv_get_info(h)["chunk"]
        ref = oracle.spmv(Am, x, mixed=True)
        rows = unsplit_rows(Ap, K)
        assert np.array_equal(y[:, rows], ref[:, rows])
        assert exact.bound_ratio(y, Ap, x) <= 1.0
    finally:
        mps.mpspmv_destroy(h)


def test_edge_shapes():
    L = 2
    # no stored entry at all
    h = mps.mpspmv_create_csr(7, 5, np.zeros(0), np.zeros(0), np.zeros((1, 0)), L)
    try:
        y = gpu_spmv(h, np.ones((L, 5)), L, 7)
        assert not y.any()
    finally:
        mps.mpspmv_destroy(h)
    # leading / trailing empty rows, one stored entry
    h = mps.mpspmv_create_csr(9, 3, [4], [2], np.array([[3.0]]), L)
    try:
        x = np.zeros((L, 3)); x[0] = [1, 2, 5]
        y = gpu_spmv(h, x, L, 9)
        assert y[0].tolist() == [0, 0, 0, 0, 15, 0, 0, 0, 0] and not y[1].any()
    finally:
        mps.mpspmv_destroy(h)
    # single long row and many empty rows, rectangular
    n = 3000
    coo = workloads.COO(50, n, np.full(n, 17), np.arange(n), np.random.default_rng(0).standard_normal((1, n)))
    A, h = csr_pair(coo, 3)
    try:
        x = workloads.full_limb_vector(n, 3, seed=5)
        y = gpu_spmv(h, x, 3, 50)
        assert exact.bound_ratio(y, A, x) <= 1.0
        assert not np.delete(y, 17, axis=1).any()
    finally:
        mps.mpspmv_destroy(h)


def test_unsorted_duplicates_symmetric_one_based():
    rng = np.random.default_rng(3)
    coo = workloads.integer_matrix(80, 80, 0.08, seed=2, dup_frac=0.3)
    L = 2
    A, h = csr_pair(coo, L)
    try:
        x = workloads.full_limb_vector(80, L, seed=1)
        y = gpu_spmv(h, x, L, 80)
        ref = oracle.spmv(A, x)
        K = mps.mpspmv_get_info(h)["chunk"]
        rows = unsplit_rows(A, K)
        assert np.array_equal(y[:, rows], ref[:, rows])
        assert exact.bound_ratio(y, A, x) <= 1.0
    finally:
        mps.mpspmv_destroy(h)
    # symmetric lower triangle, 1-based indices == the full matrix, 0-based
    n = 40
    full = workloads.laplacian_2d(8, 5)
    low = full.row >= full.col
    h1 = mps.mpspmv_create_csr(n, n, full.row[low] + 1, full.col[low] + 1, full.val[:, low], L,
                               mps.MPSPMV_SYMMETRIC | mps.MPSPMV_ONE_BASED)
    A2, h2 = csr_pair(full, L)
    try:
        x = workloads.full_limb_vector(n, L, seed=4)
        assert np.array_equal(gpu_spmv(h1, x, L, n), gpu_spmv(h2, x, L, n))
        assert mps.mpspmv_get_info(h1)["nnz"] == full.nnz
    finally:
        mps.mpspmv_destroy(h1)
        mps.mpspmv_destroy(h2)
    del rng


@pytest.mark.parametrize("L,cplx", [(2, False), (3, False), (4, True)])
def test_spmm_columns_equal_spmv(L, cplx):
    coo = workloads.random_sparse(500, 450, 40, seed=6, cplx=cplx, L=L, full_limb=True, empty_frac=0.05)
    A, h = csr_pair(coo, L, vals=coo.val, flags=FLAG[cplx])
    try:
        for k, ld in ((1, 1), (5, 7), (32, 32)):
            X = np.stack([workloads.full_limb_vector(450, L, seed=10 + c, cplx=cplx) for c in range(k)], axis=-1)
            Xp = np.zeros((A.P, 450, ld)); Xp[:, :, :k] = X
            Xd = to_dev(Xp)
            Yd = torch.full((A.P, 500, ld + 1), float("nan"), dtype=torch.float64, device="cuda")
            mps.mpspmv_spmm(h, k, Xd, ld, Yd, ld + 1)
            torch.cuda.synchronize()
            Y = Yd.cpu().numpy()
            for c in range(k):
                assert np.array_equal(Y[:, :, c], gpu_spmv(h, X[:, :, c], A.P, 500))
            assert np.isnan(Y[:, :, k:]).all()
    finally:
        mps.mpspmv_destroy(h)


def test_host_buffer_entry_point():
    coo = workloads.laplacian_2d(32)
    A, h = csr_pair(coo, 4)
    try:
        x = workloads.full_limb_vector(1024, 4, seed=8)
        y = np.zeros((4, 1024))
        mps.mpspmv_spmv_host(h, np.ascontiguousarray(x), y)
        assert np.array_equal(y, gpu_spmv(h, x, 4, 1024))
    finally:
        mps.mpspmv_destroy(h)


def test_async_host_buffer_entry_point_on_two_streams():
    """mpspmv_spmv_host_async: products of three handles (paper order, exact
    on binary64 values, complex) enqueued on two streams with pinned host
    buffers, twice in a row; after the streams complete, every y equals the
    device-buffer product of the same handle."""
    cases = []
    coo = workloads.laplacian_2d(40)
    cases.append((coo, 3, 0, coo.val))
    coo2 = workloads.power_law(2000, seed=4)
    cases.append((coo2, 4, mps.MPSPMV_EXACT_ACC, coo2.val))
    coo3 = workloads.complex_sym_banded(900, 5, 0.5, seed=2)
    cases.append((coo3, 2, mps.MPSPMV_COMPLEX, coo3.val))
    hs, xs, ys = [], [], []
    try:
        for c, L, fl, v in cases:
            h = mps.mpspmv_create_csr(c.nrows, c.ncols, c.row, c.col, v, L, fl, val_limbs=1)
            P = mps.mpspmv_get_info(h)["planes"]
            hs.append((h, P, c))
            xs.append(torch.from_numpy(workloads.full_limb_vector(c.ncols, L, seed=12, cplx=c.cplx)).pin_memory())
            ys.append(torch.full((P, c.nrows), float("nan"), dtype=torch.float64).pin_memory())
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        for _ in range(2):
            for i, ((h, P, c), xh, yh) in enumerate(zip(hs, xs, ys)):
                mps.mpspmv_spmv_host_async(h, xh, yh, streams[i % 2])
        for s in streams:
            s.synchronize()
        for (h, P, c), xh, yh in zip(hs, xs, ys):
            assert np.array_equal(yh.numpy(), gpu_spmv(h, xh.numpy(), P, c.nrows))
    finally:
        for h, _, _ in hs:
            mps.mpspmv_destroy(h)


def test_invalid_arguments():
    with pytest.raises(mps.MpspmvError) as e:
        mps.mpspmv_create_csr(5, 5, [0, 5], [0, 0], np.ones((1, 2)), 2)
    assert e.value.status == mps.MPSPMV_EINVAL
    with pytest.raises(mps.MpspmvError):
        mps.mpspmv_create_csr(5, 5, [0], [0], np.array([[np.inf]]), 2)
    with pytest.raises(mps.MpspmvError):
        mps.mpspmv_create_csr(5, 5, [0], [0], np.ones((3, 1)), 2)   # 3 limbs for DD
    h = mps.mpspmv_create_csr(5, 5, [0], [0], np.ones((1, 1)), 2)
    try:
        x = to_dev(np.ones((2, 5)))
        with pytest.raises(mps.MpspmvError):
            mps.mpspmv_spmm(h, 33, x, 33, x, 33)
        with pytest.raises(mps.MpspmvError):
            mps.mpspmv_spmv(h, 0, x)
    finally:
        mps.mpspmv_destroy(h)
