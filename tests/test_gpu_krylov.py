"""GPU CG / BiCGSTAB (C ABI) against the oracle's solvers and exact residuals
(Section 4.2: x0 = 0, stopping test ||r|| <= rtol ||b|| + atol)."""
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
import workloads
from oracle import exact
from tests._util import csr_pair, to_dev

pytestmark = pytest.mark.gpu

mps = pytest.importorskip("paper_2412_17510_gb300")
torch = pytest.importorskip("torch")


def exact_relres(A, x, b):
    ex_re, ex_im, _, _ = exact.exact_rows(A, x)
    L = A.L
    den = 1 << (2 * exact.SCALE)
    num = F(0)
    bb = F(0)
    for i in range(A.nrows):
        br = exact.to_fraction(b[:L, i])
        num += (br - F(ex_re[i], den)) ** 2
        bb += br ** 2
        if A.cplx:
            bi = exact.to_fraction(b[L:, i])
            num += (bi - F(ex_im[i], den)) ** 2
            bb += bi ** 2
    return float(num / bb) ** 0.5


def gpu_solve(fn, h, b, maxit, rtol, atol=0.0):
    bd = to_dev(b)
    xd = torch.zeros_like(bd)
    st, it, rr = fn(h, bd, xd, rtol, atol, maxit)
    torch.cuda.synchronize()
    return st, xd.cpu().numpy(), it, rr


def spd_system(L, nx=12, ny=10, grade=0.0, seed=0):
    coo = workloads.laplacian_2d(nx, ny)
    n = nx * ny
    rng = np.random.default_rng(seed)
    if grade:
        d = 10.0 ** rng.uniform(-grade, grade, n)
        coo = workloads.COO(n, n, coo.row, coo.col, (coo.val[0] * (d[coo.row] * d[coo.col]))[None, :])
    b = np.zeros((L, n))
    b[0] = rng.uniform(-1, 1, n)
    return coo, b


@pytest.mark.parametrize("L", [2, 3, 4])
def test_cg_matches_oracle(L):
    coo, b = spd_system(L, grade=1.5)
    A, h = csr_pair(coo, L)
    try:
        # targets well above the attainable accuracy u * cond(A) (cond ~ 1e8)
        rtol = {2: 1e-20, 3: 1e-35, 4: 1e-48}[L]
        st, x, it, rr = gpu_solve(mps.mpspmv_cg, h, b, 2000, rtol)
        ost, ox, oit, orr = oracle.cg(A, b, rtol=rtol, maxit=2000)
        assert st == mps.MPSPMV_OK and ost == 0
        # cond(A) ~ 1e8: in finite precision the CG iteration count depends on
        # the rounding of the inner products (their summation order differs);
        # it settles as the precision rises (Section 4.2)
        assert abs(it - oit) <= max(2, 0.05 * oit)
        assert rr <= 4 * rtol and orr <= 4 * rtol
        assert exact_relres(A, x, b) <= 4 * rtol
        # the two solutions agree to cond(A) * rtol (cond ~ 1e8 here)
        scale = np.abs(ox[0]).max()
        assert np.abs((x[0] - ox[0]) + (x[1] - ox[1])).max() <= 1e10 * rtol * scale
    finally:
        mps.mpspmv_destroy(h)


def test_cg_large_poisson_1e30():
    """64x64 Laplacian (n = 4096, cond ~ 1.7e3) to a recurrence residual of
    1e-30: DD reaches it with a true residual near u_DD * cond (~1e-29), TD
    with a true residual below 2e-30."""
    coo, b = spd_system(3, 64, 64)
    for L, true_tol in ((2, 1e-28), (3, 2e-30)):
        A, h = csr_pair(coo, L)
        try:
            st, x, it, rr = gpu_solve(mps.mpspmv_cg, h, b[:L], 5000, 1e-30)
            ost, ox, oit, orr = oracle.cg(A, b[:L], rtol=1e-30, maxit=5000)
            assert st == 0 and ost == 0 and abs(it - oit) <= max(2, 0.05 * oit)
            assert rr <= true_tol and orr <= true_tol
        finally:
            mps.mpspmv_destroy(h)


def test_cg_diagonal_one_iteration_and_limits():
    n = 10
    d = np.zeros((2, n)); d[0] = np.arange(1, n + 1)
    h = mps.mpspmv_create_csr(n, n, np.arange(n), np.arange(n), d, 2)
    try:
        b = np.zeros((2, n)); b[0, 3] = 5.0
        st, x, it, rr = gpu_solve(mps.mpspmv_cg, h, b, 10, 1e-30)
        assert st == 0 and it == 1 and x[0, 3] == 1.25 and rr == 0.0
        # zero right-hand side: converged before the first iteration
        st, x, it, rr = gpu_solve(mps.mpspmv_cg, h, np.zeros((2, n)), 10, 1e-30)
        assert st == 0 and it == 0 and not x.any()
    finally:
        mps.mpspmv_destroy(h)
    coo, b = spd_system(2, 20, 20)
    A, h = csr_pair(coo, 2)
    try:
        for maxit in (1, 3, 8, 9):
            st, x, it, rr = gpu_solve(mps.mpspmv_cg, h, b, maxit, 1e-30)
            assert st == mps.MPSPMV_ENOCONV and it == maxit
            ost, ox, oit, _ = oracle.cg(A, b, rtol=1e-30, maxit=maxit)
            assert ost == -6 and oit == maxit
    finally:
        mps.mpspmv_destroy(h)


def test_cg_breakdown_and_unsupported():
    n = 6
    # a matrix of explicit zeros: p'Ap = 0 in the first iteration
    h = mps.mpspmv_create_csr(n, n, np.arange(n), np.arange(n), np.zeros((1, n)), 2)
    try:
        b = np.ones((2, n)); b[1] = 0
        with pytest.raises(mps.MpspmvError) as e:
            gpu_solve(mps.mpspmv_cg, h, b, 10, 1e-20)
        assert e.value.status == mps.MPSPMV_EBREAKDOWN
    finally:
        mps.mpspmv_destroy(h)
    h = mps.mpspmv_create_csr(n, n, np.arange(n), np.arange(n), np.ones((2, n)), 2, mps.MPSPMV_COMPLEX)
    try:
        with pytest.raises(mps.MpspmvError) as e:
            gpu_solve(mps.mpspmv_cg, h, np.ones((4, n)), 10, 1e-20)
        assert e.value.status == mps.MPSPMV_ENOTSUP
    finally:
        mps.mpspmv_destroy(h)


def nonsym_system(L, n, cplx, seed):
    coo = workloads.random_sparse(n, n, 6, seed=seed, cplx=cplx)
    rows = np.concatenate([coo.row, np.arange(n)])
    cols = np.concatenate([coo.col, np.arange(n)])
    shift = np.zeros((coo.val.shape[0], n)); shift[0] = 8.0
    if cplx:
        shift[1] = 2.0
    vals = np.concatenate([coo.val, shift], axis=1)
    full = workloads.COO(n, n, rows, cols, vals)
    b = workloads.full_limb_vector(n, L, seed=seed + 1, cplx=cplx)
    return full, b


@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_bicgstab_matches_oracle(L, cplx):
    coo, b = nonsym_system(L, 300, cplx, seed=L)
    A, h = csr_pair(coo, L, flags=mps.MPSPMV_COMPLEX if cplx else 0)
    try:
        rtol = {2: 1e-28, 3: 1e-40, 4: 1e-55}[L]
        st, x, it, rr = gpu_solve(mps.mpspmv_bicgstab, h, b, 500, rtol)
        ost, ox, oit, orr = oracle.bicgstab(A, b, rtol=rtol, maxit=500)
        assert st == 0 and ost == 0
        assert abs(it - oit) <= 1
        assert rr <= 4 * rtol
        assert exact_relres(A, x, b) <= 4 * rtol
    finally:
        mps.mpspmv_destroy(h)


def test_bicgstab_complex_shifted_band_1e28():
    """Complex-symmetric band, half-bandwidth 48, 30% fill, shift 50+10i (a
    small instance of the complex workload), DD and QD to 1e-28."""
    coo = workloads.complex_sym_banded(3000, 48, 0.3, seed=0, shift=50 + 10j)
    for L in (2, 4):
        A, h = csr_pair(coo, L, flags=mps.MPSPMV_COMPLEX)
        try:
            rng = np.random.default_rng(5)
            xt = workloads.full_limb_vector(3000, L, seed=6, cplx=True)
            b = oracle.spmv(A, xt)
            st, x, it, rr = gpu_solve(mps.mpspmv_bicgstab, h, b, 1000, 1e-28)
            ost, ox, oit, orr = oracle.bicgstab(A, b, rtol=1e-28, maxit=1000)
            assert st == 0 and ost == 0 and abs(it - oit) <= 2
            assert rr <= 1e-28 * 2
            del rng
        finally:
            mps.mpspmv_destroy(h)
