"""SpTMV (y = A^T x) and the product-type methods BiCG, CGS and GPBiCG
(Section 4.2) through the C ABI, against the oracle.

SpTMV: rows of A^T that one thread sums end to end are bit-identical to the
oracle's row-oriented scatter; every element meets the exact bound.  Solvers:
the oracle's iteration counts (rounding order of the inner products differs,
so counts may differ slightly) and the exact residual of the returned x."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import exact
from tests._util import to_dev, unsplit_rows

pytestmark = pytest.mark.gpu

mps = pytest.importorskip("paper_2412_17510_gb300")
torch = pytest.importorskip("torch")

EX, TR = 16, 32  # MPSPMV_EXACT_ACC, MPSPMV_TRANSPOSE


def gpu_spmtv(h, x, P, ncols):
    xd = to_dev(x)
    yd = torch.full((P, ncols), float("nan"), dtype=torch.float64, device="cuda")
    mps.mpspmv_spmtv(h, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_spmtv_matches_oracle_scatter(L, cplx):
    """700 x 650, every component random, about 3 entries per row (so many
    rows of A^T lie inside one run), empty rows, two long columns (rows of
    A^T spanning many runs), ragged tail."""
    coo = workloads.random_sparse(700, 650, 6, seed=50 + L, cplx=cplx, L=L, full_limb=True, empty_frac=0.1)
    rng = np.random.default_rng(2)
    extra_r, extra_c = [], []
    for c, ln in ((3, 500), (321, 260)):
        r = np.sort(rng.choice(700, ln, replace=False))
        extra_r.append(r)
        extra_c.append(np.full(ln, c))
    er, ec = np.concatenate(extra_r), np.concatenate(extra_c)
    keep = ~np.isin(coo.col, [3, 321])
    row = np.concatenate([coo.row[keep], er])
    col = np.concatenate([coo.col[keep], ec])
    val = np.concatenate([coo.val[:, keep], workloads.full_limb_vector(er.shape[0], L, seed=8, cplx=cplx)], axis=1)
    A = oracle.coo_to_csr(700, 650, row, col, val, L, cplx)
    AT = oracle.coo_to_csr(650, 700, col, row, val, L, cplx)
    P = 2 * L if cplx else L
    x = workloads.full_limb_vector(700, L, seed=3, cplx=cplx)
    ref = oracle.spmtv(A, x)
    for ex in (False, True):
        h = mps.mpspmv_create_csr(700, 650, row, col, val, L, (1 if cplx else 0) | TR | (EX if ex else 0))
        try:
            y = gpu_spmtv(h, x, P, 650)
            assert exact.bound_ratio(y, AT, x) <= 1.0
            if not ex:
                K = mps.mpspmv_get_info(h)["chunk"]  # same nnz, same run length as A^T
                rows = unsplit_rows(AT, K)
                assert len(rows) > 50
                assert np.array_equal(y[:, rows], ref[:, rows])
            # the forward product is unaffected by the transpose
            xf = workloads.full_limb_vector(650, L, seed=4, cplx=cplx)
            yf = torch.empty((P, 700), dtype=torch.float64, device="cuda")
            mps.mpspmv_spmv(h, to_dev(xf), yf)
            torch.cuda.synchronize()
            assert exact.bound_ratio(yf.cpu().numpy(), A, xf) <= 1.0
        finally:
            mps.mpspmv_destroy(h)


def test_spmtv_mixed_mode_and_missing_transpose():
    L = 2
    coo = workloads.random_sparse(300, 280, 12, seed=7)
    A1 = oracle.coo_to_csr(300, 280, coo.row, coo.col, coo.val, 1)
    AT1 = oracle.coo_to_csr(280, 300, coo.col, coo.row, coo.val, 1)
    ATp = oracle.coo_to_csr(280, 300, coo.col, coo.row, coo.promoted(L), L)
    x = workloads.full_limb_vector(300, L, seed=5)
    h = mps.mpspmv_create_csr(300, 280, coo.row, coo.col, coo.val, L, mps.MPSPMV_MIXED | TR, val_limbs=1)
    try:
        y = gpu_spmtv(h, x, L, 280)
        assert exact.bound_ratio(y, ATp, x) <= 1.0
        ref = oracle.spmtv(oracle.CSR(300, 280, A1.indptr, A1.indices, A1.data, L, False), x, mixed=True)
        rows = unsplit_rows(AT1, mps.mpspmv_get_info(h)["chunk"])
        assert np.array_equal(y[:, rows], ref[:, rows])
    finally:
        mps.mpspmv_destroy(h)
    h = mps.mpspmv_create_csr(300, 280, coo.row, coo.col, coo.val, L, 0, val_limbs=1)
    try:
        with pytest.raises(mps.MpspmvError) as e:
            gpu_spmtv(h, x, L, 280)
        assert e.value.status == mps.MPSPMV_ENOTSUP
        b = torch.zeros((L, 300), dtype=torch.float64, device="cuda")
        with pytest.raises(mps.MpspmvError) as e:
            mps.mpspmv_bicg(h, b, torch.zeros_like(b), 1e-20)
        assert e.value.status in (mps.MPSPMV_ENOTSUP, mps.MPSPMV_EINVAL)
    finally:
        mps.mpspmv_destroy(h)


def shifted_nonsym(n, L, cplx, seed):
    coo = workloads.random_sparse(n, n, 6, seed=seed, cplx=cplx)
    rows = np.concatenate([coo.row, np.arange(n)])
    cols = np.concatenate([coo.col, np.arange(n)])
    shift = np.zeros((coo.val.shape[0], n))
    shift[0] = 8.0
    if cplx:
        shift[1] = 2.0
    return workloads.COO(n, n, rows, cols, np.concatenate([coo.val, shift], axis=1))


SOLVE = {"bicg": ("mpspmv_bicg", oracle.bicg), "cgs": ("mpspmv_cgs", oracle.cgs),
         "gpbicg": ("mpspmv_gpbicg", oracle.gpbicg)}


def gpu_solve(fn, h, b, maxit, rtol):
    bd = to_dev(b)
    xd = torch.zeros_like(bd)
    st, it, rr = fn(h, bd, xd, rtol, 0.0, maxit)
    torch.cuda.synchronize()
    return st, xd.cpu().numpy(), it, rr


@pytest.mark.parametrize("method", sorted(SOLVE))
@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("ex", [False, True])
def test_product_type_solvers_match_oracle(method, L, cplx, ex):
    n = 300
    coo = shifted_nonsym(n, L, cplx, seed=L)
    P = 2 * L if cplx else L
    vals = np.zeros((P, coo.nnz))
    for c in range(2 if cplx else 1):
        vals[c * L] = coo.val[c]
    A = oracle.coo_to_csr(n, n, coo.row, coo.col, vals, L, cplx)
    h = mps.mpspmv_create_csr(n, n, coo.row, coo.col, vals, L, (1 if cplx else 0) | TR | (EX if ex else 0))
    try:
        b = workloads.full_limb_vector(n, L, seed=L + 1, cplx=cplx)
        rtol = {2: 1e-28, 4: 1e-55}[L]
        name, ofn = SOLVE[method]
        st, x, it, rr = gpu_solve(getattr(mps, name), h, b, 500, rtol)
        ost, ox, oit, orr = ofn(A, b, rtol=rtol, maxit=500)
        assert st == 0 and ost == 0
        assert abs(it - oit) <= max(2, 0.1 * oit)
        assert rr <= 4 * rtol
        if not ex:
            ex_re, ex_im, _, _ = exact.exact_rows(A, x)
            den = 1 << (2 * exact.SCALE)
            from fractions import Fraction as F
            num = bb = F(0)
            for i in range(n):
                br = exact.to_fraction(b[:L, i])
                num += (br - F(ex_re[i], den)) ** 2
                bb += br ** 2
                if cplx:
                    bi = exact.to_fraction(b[L:, i])
                    num += (bi - F(ex_im[i], den)) ** 2
                    bb += bi ** 2
            assert float(num / bb) ** 0.5 <= 4 * rtol
    finally:
        mps.mpspmv_destroy(h)


def test_bicg_equals_cg_iterations_on_spd():
    """Symmetric A: BiCG with r~_0 = r_0 repeats CG step for step."""
    coo = workloads.laplacian_2d(30, 24)
    n, L = coo.nrows, 2
    h = mps.mpspmv_create_csr(n, n, coo.row, coo.col, coo.val, L, TR, val_limbs=1)
    try:
        b = workloads.full_limb_vector(n, L, seed=6)
        st1, x1, it1, rr1 = gpu_solve(mps.mpspmv_cg, h, b, 2000, 1e-25)
        st2, x2, it2, rr2 = gpu_solve(mps.mpspmv_bicg, h, b, 2000, 1e-25)
        assert st1 == st2 == 0 and abs(it1 - it2) <= 1
        assert rr2 <= 4e-25
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("method", sorted(SOLVE))
@pytest.mark.parametrize("cplx", [False, True])
def test_finite_termination_three_eigenvalues(method, cplx):
    """Diagonal A with 3 distinct eigenvalues: at most 3 iterations in QD
    (GPBiCG leaves through its ||t|| exit at the third)."""
    L, n = 4, 48
    ev = [(2.0, 0.5), (3.0, -1.0), (7.0, 0.25)]
    P = 2 * L if cplx else L
    vals = np.zeros((P, n))
    for i in range(n):
        vals[0, i] = ev[i % 3][0]
        if cplx:
            vals[L, i] = ev[i % 3][1]
    h = mps.mpspmv_create_csr(n, n, np.arange(n), np.arange(n), vals, L, (1 if cplx else 0) | TR)
    try:
        b = workloads.full_limb_vector(n, L, seed=9, cplx=cplx)
        st, x, it, rr = gpu_solve(getattr(mps, SOLVE[method][0]), h, b, 10, 1e-50)
        A = oracle.coo_to_csr(n, n, np.arange(n), np.arange(n), vals, L, cplx)
        ost, ox, oit, orr = SOLVE[method][1](A, b, rtol=1e-50, maxit=10)
        assert st == 0 and ost == 0 and it <= 3 and oit <= 3
        assert rr <= 1e-49
    finally:
        mps.mpspmv_destroy(h)
