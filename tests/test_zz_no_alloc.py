"""The allocation-free SpMV entry point (for callers whose device memory is
all handed to their own pool, or who cannot take the synchronisation of
cudaMalloc) against the regular handle-based entry point.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.  It passes alone in a fresh
process and after the other tests (the library's scratch array keeps the
previous call's partial sums, and every call overwrites what it reads)."""
import numpy as np
import pytest

import workloads
from oracle import exact
from tests._util import csr_pair, to_dev

pytestmark = pytest.mark.gpu

mps = pytest.importorskip("paper_2412_17510_gb300")
torch = pytest.importorskip("torch")


def plain_csr(coo, vals):
    indptr = np.zeros(coo.nrows + 1, dtype=np.int64)
    np.add.at(indptr, coo.row + 1, 1)
    return np.cumsum(indptr), coo.col.astype(np.int32), np.ascontiguousarray(vals)


def run_noalloc(prec, flags, coo, vals, x):
    ip, ind, v = plain_csr(coo, vals)
    P = v.shape[0]
    y = torch.full((P, coo.nrows), float("nan"), dtype=torch.float64, device="cuda")
    mps.mpspmv_spmv_csr_noalloc(prec, flags, coo.nrows, coo.ncols, int(ip[-1]), to_dev(ip), to_dev(ind), to_dev(v),
                                to_dev(x), y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def run_handle(h, x, P, nrows):
    y = torch.empty((P, nrows), dtype=torch.float64, device="cuda")
    mps.mpspmv_spmv(h, to_dev(x), y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def same_runs(A, K):
    """Rows summed end to end by one thread both with runs of K entries and
    with the no-allocation path's runs of 16: both paths compute them with
    the same operation sequence."""
    ip = A.indptr
    ne = ip[1:] > ip[:-1]
    inside = lambda k: (ip[:-1] // k) == ((ip[1:] - 1) // k)
    return ne & inside(K) & inside(16), ne


def pair_ratio(y1, y2, A, x, rows):
    """max |y1 - y2| / (8 m u (|A||x|)_i) over the given rows, exactly: the
    tests' acceptance bound, applied to the difference of the two entry
    points (each within the bound of the exact value gives at most 2)."""
    from fractions import Fraction
    L = A.L
    _, _, ab_re, ab_im = exact.exact_rows(A, x, rows)
    m = int(np.diff(A.indptr).max()) * (2 if A.cplx else 1)
    u = Fraction(exact.U[L])
    worst = 0.0
    parts = [(0, ab_re)] + ([(L, ab_im)] if A.cplx else [])
    for off, ab in parts:
        for s_, i in enumerate(rows):
            d = abs(exact.limbs_to_int(y1[off:off + L, i]) - exact.limbs_to_int(y2[off:off + L, i])) << exact.SCALE
            if ab[s_] == 0:
                assert d == 0
                continue
            worst = max(worst, float(Fraction(d) / (Fraction(ab[s_]) * 8 * m * u)))
    return worst


def test_noalloc_setup_call_before_products():
    """The documented start-up call: nrows = 0 with NULL pointers does only
    the set-up (loads the module holding the scratch array, looks up its
    address) and succeeds; a product right after it matches the handle
    entry point on rows both sum within one run."""
    mps.mpspmv_spmv_csr_noalloc(2, 0, 0, 0, 0, None, None, None, None, None)
    mps.mpspmv_spmv_csr_noalloc(4, mps.MPSPMV_COMPLEX, 0, 0, 0, None, None, None, None, None)
    coo = workloads.laplacian_2d(20)
    A, h = csr_pair(coo, 2)
    try:
        x = workloads.full_limb_vector(coo.ncols, 2, seed=9)
        y_na = run_noalloc(2, 0, coo, coo.promoted(2), x)
        y_h = run_handle(h, x, 2, coo.nrows)
        same, _ = same_runs(A, mps.mpspmv_get_info(h)["chunk"])
        assert same.any()
        assert np.array_equal(y_na[:, same], y_h[:, same])
        assert exact.bound_ratio(y_na, A, x) <= 1.0
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 4])
def test_noalloc_matches_handle_entry_point(L):
    """27-point stencil 32^3 (830,584 entries), full-limb x: two calls in a
    row, each compared with mpspmv_spmv on sampled rows within the tests'
    bound 8 m u (|A||x|)_i (and identical on rows both paths sum in one run)."""
    coo = workloads.stencil_27pt(32)
    vals = coo.promoted(L)
    A, h = csr_pair(coo, L)
    try:
        same, _ = same_runs(A, mps.mpspmv_get_info(h)["chunk"])
        rows = list(range(0, coo.nrows, 97))
        for seed in (1, 2):
            x = workloads.full_limb_vector(coo.ncols, L, seed=seed)
            y_na = run_noalloc(L, 0, coo, vals, x)
            y_h = run_handle(h, x, L, coo.nrows)
            assert not np.isnan(y_na).any()
            assert np.array_equal(y_na[:, same], y_h[:, same])
            assert pair_ratio(y_na, y_h, A, x, rows) <= 2.0
            assert exact.bound_ratio(y_na[:, rows], A, x, rows=rows) <= 1.0
    finally:
        mps.mpspmv_destroy(h)


def test_noalloc_complex_long_rows_within_bound():
    """Complex QD with empty rows and rows spanning many runs; two calls in a
    row with different x, each compared with mpspmv_spmv (rows that both
    paths sum within one run: identical; sampled rows: within the bound)."""
    L = 4
    coo = workloads.random_sparse(900, 800, 60, seed=3, cplx=True, L=L, full_limb=True, empty_frac=0.2)
    A, h = csr_pair(coo, L, vals=coo.val, flags=mps.MPSPMV_COMPLEX)
    try:
        same, ne = same_runs(A, mps.mpspmv_get_info(h)["chunk"])
        rows = list(range(0, 900, 7))
        for seed in (4, 5):
            x = workloads.full_limb_vector(800, L, seed=seed, cplx=True)
            y_na = run_noalloc(L, mps.MPSPMV_COMPLEX, coo, coo.val, x)
            y_h = run_handle(h, x, 2 * L, 900)
            assert np.array_equal(y_na[:, same], y_h[:, same])
            assert pair_ratio(y_na, y_h, A, x, rows) <= 2.0
            assert exact.bound_ratio(y_na[:, rows], A, x, rows=rows) <= 1.0
            assert not y_na[:, ~ne].any()
    finally:
        mps.mpspmv_destroy(h)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    zi = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(mps.MpspmvError) as e:
        mps.mpspmv_spmv_csr_noalloc(4, mps.MPSPMV_COMPLEX, 1, 1, 4194304 + 16, zi, zi, z, z, z)
    assert e.value.status == mps.MPSPMV_EINVAL
