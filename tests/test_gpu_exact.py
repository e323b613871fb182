"""The exact-accumulation arithmetic (MPSPMV_EXACT_ACC): error-free products
on the binary64 pipe, exact fixed-point row sums on the integer pipe.  It
must meet the same componentwise bound 8 m u (|A||x|)_i as the paper-order
arithmetic against the exact value (it is not bit-identical to it)."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import exact
from oracle import exact_model as model
from tests._util import csr_pair, gpu_spmv, to_dev, unsplit_rows

pytestmark = pytest.mark.gpu

mps = pytest.importorskip("paper_2412_17510_gb300")
torch = pytest.importorskip("torch")

EX = 16  # MPSPMV_EXACT_ACC


@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_full_limb_random_within_bound(L, cplx):
    coo = workloads.random_sparse(600, 500, 40, seed=10 + L, cplx=cplx, L=L, full_limb=True, empty_frac=0.1)
    A, h = csr_pair(coo, L, vals=coo.val, flags=EX | (1 if cplx else 0))
    try:
        x = workloads.full_limb_vector(500, L, seed=3, cplx=cplx)
        y = gpu_spmv(h, x, A.P, 600)
        assert exact.bound_ratio(y, A, x) <= 1.0
        empty = np.diff(A.indptr) == 0
        assert not y[:, empty].any()
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_mixed_mode_within_bound(L, cplx):
    coo = workloads.random_sparse(400, 400, 30, seed=4, cplx=cplx)
    Ap = oracle.coo_to_csr(400, 400, coo.row, coo.col, coo.promoted(L), L, cplx)
    h = mps.mpspmv_create_csr(400, 400, coo.row, coo.col, coo.val, L, EX | mps.MPSPMV_MIXED | (1 if cplx else 0),
                              val_limbs=1)
    try:
        x = workloads.full_limb_vector(400, L, seed=3, cplx=cplx)
        y = gpu_spmv(h, x, Ap.P, 400)
        assert exact.bound_ratio(y, Ap, x) <= 1.0
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_integer_matrices_bit_exact(L, cplx):
    coo = workloads.integer_matrix(300, 280, 0.05, seed=L, cplx=cplx)
    A, h = csr_pair(coo, L, flags=EX | (1 if cplx else 0))
    try:
        x = workloads.integer_vector(280, L, seed=7, cplx=cplx)
        y = gpu_spmv(h, x, A.P, 300)
        assert np.array_equal(y, oracle.spmv(A, x))
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_wide_exponent_range_and_long_rows(L):
    """Rows whose products span 2^-900 .. 2^900 (the accumulation window has
    to move up several times) and rows spanning many runs."""
    rng = np.random.default_rng(5)
    n, m = 64, 300
    ncol = 512
    rows, cols, vals = [], [], []
    for i in range(n):
        k = m if i % 8 == 0 else 20
        c = np.sort(rng.choice(ncol, k, replace=False))
        v = rng.standard_normal(k) * 2.0 ** rng.integers(-450, 450, k)
        rows.append(np.full(k, i)); cols.append(c); vals.append(v)
    coo = workloads.COO(n, ncol, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals)[None, :])
    A, h = csr_pair(coo, L, flags=EX)
    try:
        x = workloads.full_limb_vector(ncol, L, seed=9)
        x[:, ::3] *= 2.0 ** 400
        y = gpu_spmv(h, x, L, n)
        assert exact.bound_ratio(y, A, x) <= 1.0
    finally:
        mps.mpspmv_destroy(h)


def test_non_finite_x_gives_nan_rows():
    coo = workloads.laplacian_2d(8)
    A, h = csr_pair(coo, 2, flags=EX)
    try:
        x = workloads.full_limb_vector(64, 2, seed=1)
        x[0, 10] = np.inf
        y = gpu_spmv(h, x, 2, 64)
        bad_rows = [i for i in range(64) if 10 in A.indices[A.indptr[i]:A.indptr[i + 1]]]
        assert all(np.isnan(y[0, i]) for i in bad_rows)
        good = [i for i in range(64) if i not in bad_rows]
        assert np.isfinite(y[:, good]).all()
    finally:
        mps.mpspmv_destroy(h)


def test_spmm_and_batch_equal_spmv():
    L = 4
    coo = workloads.random_sparse(500, 500, 30, seed=6, L=L, full_limb=True)
    A, h = csr_pair(coo, L, vals=coo.val, flags=EX)
    try:
        k = 5
        X = np.stack([workloads.full_limb_vector(500, L, seed=20 + c) for c in range(k)], axis=-1)
        Xd = to_dev(X)
        Yd = torch.empty((L, 500, k), dtype=torch.float64, device="cuda")
        mps.mpspmv_spmm(h, k, Xd, k, Yd, k)
        torch.cuda.synchronize()
        Y = Yd.cpu().numpy()
        for c in range(k):
            assert np.array_equal(Y[:, :, c], gpu_spmv(h, X[:, :, c], L, 500))
        b = mps.mpspmv_batch_create([h], [k], 0)
        try:
            Yb = torch.empty_like(Yd)
            mps.mpspmv_batch_spmm(b, [Xd], [Yb])
            torch.cuda.synchronize()
            assert np.array_equal(Yb.cpu().numpy(), Y)
        finally:
            mps.mpspmv_batch_destroy(b)
    finally:
        mps.mpspmv_destroy(h)


def test_stencil_full_size_sampled_rows():
    """27-point stencil 64^3 (n = 262,144), DD and QD, exact accumulation vs
    the paper-order arithmetic: both within the bound on sampled rows."""
    coo = workloads.stencil_27pt(64)
    rows = list(range(0, coo.nrows, 4099))
    for L in (2, 4):
        A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.promoted(L), L)
        x = workloads.full_limb_vector(coo.ncols, L, seed=0)
        for flags in (0, EX):
            h = mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, L, flags, val_limbs=1)
            try:
                y = gpu_spmv(h, x, L, coo.nrows)
                assert exact.bound_ratio(y[:, rows], A, x, rows=rows) <= 1.0
            finally:
                mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_binary64_storage_forms(L, cplx):
    """Exact accumulation on binary64 data stores the leading components
    only.  Its multi-right-hand-side products use the MP x binary64 forms,
    whose left-out products are exactly zero, so they equal those of the
    full P-mode storage (the same values passed with explicit zero lower
    components) bit for bit; its single-vector products take the wide-x
    form, which meets the same bound."""
    coo = workloads.random_sparse(700, 650, 40, seed=30 + L, cplx=cplx, empty_frac=0.1)
    fl = EX | (1 if cplx else 0)
    h1 = mps.mpspmv_create_csr(700, 650, coo.row, coo.col, coo.val, L, fl, val_limbs=1)
    h2 = mps.mpspmv_create_csr(700, 650, coo.row, coo.col, coo.promoted(L), L, fl, val_limbs=L)
    try:
        assert mps.mpspmv_get_info(h1)["value_planes"] == (2 if cplx else 1)
        assert mps.mpspmv_get_info(h2)["value_planes"] == (2 * L if cplx else L)
        P = 2 * L if cplx else L
        x = workloads.full_limb_vector(650, L, seed=8, cplx=cplx)
        X = np.ascontiguousarray(np.stack([x, x], axis=-1))
        Ys = []
        for h in (h1, h2):
            Yd = torch.empty((P, 700, 2), dtype=torch.float64, device="cuda")
            mps.mpspmv_spmm(h, 2, to_dev(X), 2, Yd, 2)
            torch.cuda.synchronize()
            Ys.append(Yd.cpu().numpy())
        assert np.array_equal(Ys[0], Ys[1])
        A = oracle.coo_to_csr(700, 650, coo.row, coo.col, coo.promoted(L), L, cplx)
        y1 = gpu_spmv(h1, x, P, 700)
        assert exact.bound_ratio(y1, A, x) <= 1.0
        assert exact.bound_ratio(Ys[0][:, :, 0], A, x) <= 1.0
    finally:
        mps.mpspmv_destroy(h1)
        mps.mpspmv_destroy(h2)


def _near_uniform(n, ncols, lo, hi, empty_frac, seed, cplx, L):
    """Rows of lo..hi entries (a few empty): short, evenly sized rows, the
    kind that gets the one-row-per-thread copy."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(lo, hi + 1, n)
    lens[rng.random(n) < empty_frac] = 0
    rows = np.repeat(np.arange(n), lens)
    cols = np.concatenate([np.sort(rng.choice(ncols, k, replace=False)) for k in lens])
    P = 2 * L if cplx else L
    vals = workloads.full_limb_vector(rows.shape[0], L, seed=seed + 1, cplx=cplx)
    return workloads.COO(n, ncols, rows, cols, vals), P


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_row_per_thread_copy_within_bound(L, cplx):
    """Exact handles with short, evenly sized rows multiply one vector from a
    sliced-ELL copy (whole rows per thread): every row meets the bound and
    empty rows give zeros."""
    n, ncols = 2000 + 13, 1500
    coo, P = _near_uniform(n, ncols, 7, 8, 0.03, seed=40 + L, cplx=cplx, L=L)
    A, h = csr_pair(coo, L, vals=coo.val, flags=EX | (1 if cplx else 0))
    try:
        assert mps.mpspmv_get_info(h)["sell_slots"] > 0
        x = workloads.full_limb_vector(ncols, L, seed=5, cplx=cplx)
        y = gpu_spmv(h, x, P, n)
        assert exact.bound_ratio(y, A, x) <= 1.0
        empty = np.diff(A.indptr) == 0
        assert empty.any() and not y[:, empty].any()
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_row_per_thread_copy_matches_runs(L, cplx):
    """Rows that the run layout sums inside one run (the layout SpMM uses)
    agree bit for bit with the one-row-per-thread product: the same exact sum
    of the same terms, cut once.  8M entries, so that runs hold 16 entries
    and about half of the 7..8-entry rows lie inside one run."""
    rng = np.random.default_rng(60 + L)
    n, ncols = 1_100_000, 900_000
    lens = rng.integers(7, 9, n)
    rows = np.repeat(np.arange(n), lens)
    j = np.arange(rows.shape[0]) - np.repeat(np.cumsum(lens) - lens, lens)
    cols = (rows * 7 + 37 * j) % ncols
    P = 2 * L if cplx else L
    vals = workloads.full_limb_vector(rows.shape[0], L, seed=61, cplx=cplx)
    h = mps.mpspmv_create_csr(n, ncols, rows, cols, vals, L, EX | (1 if cplx else 0))
    try:
        info = mps.mpspmv_get_info(h)
        assert info["chunk"] == 16 and info["sell_slots"] > 0
        x = workloads.full_limb_vector(ncols, L, seed=6, cplx=cplx)
        y = gpu_spmv(h, x, P, n)
        X = np.ascontiguousarray(np.stack([x, x], axis=-1))
        Yd = torch.empty((P, n, 2), dtype=torch.float64, device="cuda")
        mps.mpspmv_spmm(h, 2, to_dev(X), 2, Yd, 2)
        torch.cuda.synchronize()
        Y = Yd.cpu().numpy()[:, :, 0]
        indptr = np.concatenate([[0], np.cumsum(lens)])
        same = (indptr[:-1] // 16) == ((indptr[1:] - 1) // 16)
        assert same.sum() > n // 4
        assert np.array_equal(y[:, same], Y[:, same])
        # split rows: the run partials are cut before the exact combine, so
        # they may differ in the last component only
        d = np.abs(y[0] - Y[0])
        assert (d <= 1e-12 * np.abs(Y[0]) + 1e-300).all()
    finally:
        mps.mpspmv_destroy(h)


def _model_case(L, layout, mode, cplx):
    """Matrix, its oracle CSR and the values passed to the handle for one
    case of the exact-model test."""
    if layout == "rows":
        coo = workloads.stencil_27pt(12)
        if cplx:
            im = np.random.default_rng(70 + L).standard_normal(coo.nnz)
            coo = workloads.COO(coo.nrows, coo.ncols, coo.row, coo.col, np.stack([coo.val[0], im]))
    else:
        coo = workloads.random_sparse(3000, 3000, 6, seed=40 + L, cplx=cplx)
    if mode == 0:
        vals, limbs = workloads.full_limb_vector(coo.nnz, L, seed=50 + L, cplx=cplx), L
        A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, vals, L, cplx)
    else:
        vals, limbs = coo.val, 1
        A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.promoted(L), L, cplx)
    return coo, A, vals, limbs


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("layout", ["rows", "runs"])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("cplx", [False, True])
def test_rows_bit_identical_to_the_exact_model(L, layout, mode, cplx):
    """Rows that one thread sums end to end equal the exact model bit for bit
    (oracle/exact_model.py).  MP values (every component random, mode 0):
    the exact sum of the entries' decomposed terms (exact products below the
    unit roundoff plus one FMA chain), cut to L components by truncation,
    for every row whose terms fit the window.  Binary64 values (leading
    component stored, mode 1): the wide-x form (x turned into one W-word
    fixed-point number per column, one product a X per entry), the model
    following the row accumulator step by step, for every row.  Complex data
    in the pattern re += a_re x_re - a_im x_im, im += a_re x_im + a_im x_re.
    Layouts: the row-per-thread copy of a 27-point stencil (every row) and
    the run layout of short random rows (the rows inside one run)."""
    coo, A, vals, limbs = _model_case(L, layout, mode, cplx)
    P = 2 * L if cplx else L
    h = mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, vals, L,
                              EX | (mps.MPSPMV_COMPLEX if cplx else 0), val_limbs=limbs)
    try:
        info = mps.mpspmv_get_info(h)
        x = workloads.full_limb_vector(coo.ncols, L, seed=60 + L, cplx=cplx)
        y = gpu_spmv(h, x, P, coo.nrows)
    finally:
        mps.mpspmv_destroy(h)
    if layout == "rows":
        assert info["sell_slots"] > 0
        rows = np.arange(coo.nrows)
    else:
        assert info["sell_slots"] == 0
        rows = unsplit_rows(A, info["chunk"])
    compared = 0
    for r in rows:
        if mode == 1:
            want, fits = model.row_model_wide(L, A, x, int(r))
            fits = True
        else:
            want, fits = model.row_model(L, mode, A, x, int(r))
        if fits:
            assert np.array_equal(y[:, r], want), (L, layout, mode, cplx, int(r), y[:, r], want)
            compared += 1
    assert compared >= max(100, len(rows) // 2)
    if mode == 1:
        assert compared == len(rows)


@pytest.mark.parametrize("L", [2, 3, 4])
def test_wide_form_edge_cases(L):
    """Wide-x form on binary64 data: x with zero, subnormal, cancelling,
    overflowing and non-finite columns; entries far below a row's largest
    (the truncating path below the window) and window moves; empty rows.
    Rows that one run holds equal the model bit for bit (rows cut by runs are
    combined from their runs' L-component partials); every row that
    references a non-finite x is NaN; the rest meet the bound."""
    rng = np.random.default_rng(90 + L)
    n, ncols = 600, 64
    near, _ = _near_uniform(n, ncols, 7, 8, 0.03, seed=91 + L, cplx=False, L=1)
    coo = workloads.COO(n, ncols, near.row, near.col, rng.standard_normal((1, near.nnz)))
    vals = coo.val.copy()
    vals[0, ::5] *= 2.0 ** rng.integers(-300, 300, vals[0, ::5].shape[0])
    coo = workloads.COO(n, ncols, coo.row, coo.col, vals)
    x = workloads.full_limb_vector(ncols, L, seed=92 + L)
    x[:, 3] = 0.0
    x[:, 5] = 0.0
    x[L - 1, 5] = 2.0 ** -1070
    x[1, 7] = -x[0, 7]
    x[0, 9] = float("inf")
    x[:, 11] *= 2.0 ** 900
    A = oracle.coo_to_csr(n, ncols, coo.row, coo.col, coo.promoted(L), L)
    h = mps.mpspmv_create_csr(n, ncols, coo.row, coo.col, coo.val, L, EX, val_limbs=1)
    try:
        info = mps.mpspmv_get_info(h)
        y = gpu_spmv(h, x, L, n)
    finally:
        mps.mpspmv_destroy(h)
    assert info["sell_slots"] > 0  # short, even rows: one row per thread, every row compared
    one = set(range(n))
    compared = 0
    finite = []
    for r in range(n):
        want, _ = model.row_model_wide(L, A, x, r)
        if np.isnan(want[0]):
            assert np.isnan(y[0, r])
        elif r in one:
            assert np.array_equal(y[:, r], want), (L, r, y[:, r], want)
            compared += 1
        # the bound needs results whose L components lie in the normal range
        # (a subnormal result cannot carry them)
        if np.isfinite(want).all() and (want[0] == 0.0 or abs(want[0]) > 2.0 ** -800):
            finite.append(r)
    assert compared >= n // 2
    assert not y[:, np.diff(A.indptr) == 0].any()
    xb = x.copy()
    xb[:, 9] = 0.0  # the rows checked do not reference the non-finite column
    assert exact.bound_ratio(y[:, finite], A, xb, rows=finite) <= 1.0
