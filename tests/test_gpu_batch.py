"""Batched persistent SpMM and batched CG (C ABI) against the single-matrix
entry points and the oracle: 7-point finite-volume diffusion matrices with
log-uniform coefficients (the batched workload's kind), uneven sizes and
1..32 right-hand sides."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import exact
from tests._util import to_dev

pytestmark = pytest.mark.gpu

mps = pytest.importorskip("paper_2412_17510_gb300")
torch = pytest.importorskip("torch")


def make_batch(L, count=10, seed=0, nmax=3000, ks=None, kappa=(1e-3, 1e3), flags=0):
    specs = workloads.batch_specs(count, n_range=(150, nmax), k_range=(1, 9), seed=seed)
    mats, coos, kk = [], [], []
    for i, (nx, ny, nz, k, sd) in enumerate(specs):
        coo = workloads.diffusion_7pt(nx, ny, nz, kappa_range=kappa, seed=sd)
        h = mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, L, flags, val_limbs=1)
        mats.append(h)
        coos.append(coo)
        kk.append(ks[i] if ks else k)
    return mats, coos, kk


def rhs_block(n, k, L, seed):
    X = np.stack([workloads.full_limb_vector(n, L, seed=seed + c) for c in range(k)], axis=-1)  # (L, n, k)
    return np.ascontiguousarray(X)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("tune", [False, True])
def test_batch_spmm_equals_single_matrix(L, tune):
    mats, coos, ks = make_batch(L, count=10, seed=L, ks=[1, 3, 32, 5, 8, 2, 17, 4, 1, 9])
    try:
        b = mps.mpspmv_batch_create(mats, ks, mps.MPSPMV_BATCH_AUTOTUNE if tune else 0)
        try:
            K, w = mps.mpspmv_batch_get_plan(b, len(mats))
            assert all(k in (4, 8, 16, 32, 64) for k in K) and all(v in (1, 2, 4, 8) for v in w)
            Xs = [to_dev(rhs_block(c.ncols, k, L, 10 * i)) for i, (c, k) in enumerate(zip(coos, ks))]
            Ys = [torch.full((L, c.nrows, k), float("nan"), dtype=torch.float64, device="cuda")
                  for c, k in zip(coos, ks)]
            for _ in range(2):  # second call replays the cached graph
                mps.mpspmv_batch_spmm(b, Xs, Ys)
            torch.cuda.synchronize()
            for i, (h, c, k) in enumerate(zip(mats, coos, ks)):
                Yr = torch.empty_like(Ys[i])
                mps.mpspmv_spmm(h, k, Xs[i], k, Yr, k)
                torch.cuda.synchronize()
                Yb = Ys[i].cpu().numpy()
                assert np.array_equal(Yb, Yr.cpu().numpy()), i
                A = oracle.coo_to_csr(c.nrows, c.ncols, c.row, c.col, c.promoted(L), L)
                X = Xs[i].cpu().numpy()
                rows = list(range(0, c.nrows, 13))
                for col in sorted({0, k - 1}):
                    assert exact.bound_ratio(Yb[:, rows, col], A, X[:, :, col], rows=rows) <= 1.0
        finally:
            mps.mpspmv_batch_destroy(b)
    finally:
        for h in mats:
            mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 3])
def test_batch_cg_matches_single_cg(L):
    # milder coefficient contrast keeps the CPU oracle's solves short
    mats, coos, ks = make_batch(L, count=6, seed=7, nmax=600, kappa=(0.1, 10.0))
    rtol = {2: 1e-25, 3: 1e-35}[L]
    try:
        b = mps.mpspmv_batch_create(mats, ks, 0)
        try:
            Bs = [to_dev(rhs_block(c.ncols, k, L, 100 + 10 * i)) for i, (c, k) in enumerate(zip(coos, ks))]
            Xs = [torch.zeros_like(B) for B in Bs]
            nsys = sum(ks)
            st, it, rr, ss = mps.mpspmv_batch_cg(b, Bs, Xs, nsys, rtol, 0.0, 20000)
            assert st == mps.MPSPMV_OK and (ss == 0).all()
            q = 0
            for i, (h, c, k) in enumerate(zip(mats, coos, ks)):
                X = Xs[i].cpu().numpy()
                Bh = Bs[i].cpu().numpy()
                for col in range(k):
                    bcol = to_dev(Bh[:, :, col])
                    xcol = torch.zeros_like(bcol)
                    st1, it1, rr1 = mps.mpspmv_cg(h, bcol, xcol, rtol, 0.0, 20000)
                    assert st1 == 0
                    assert abs(it[q] - it1) <= max(3, 0.05 * it1), (i, col, it[q], it1)
                    assert rr[q] <= 50 * rtol and rr1 <= 50 * rtol
                    q += 1
                # one system per matrix against the oracle's CG
                A = oracle.coo_to_csr(c.nrows, c.ncols, c.row, c.col, c.promoted(L), L)
                ost, ox, oit, orr = oracle.cg(A, Bh[:, :, 0], rtol=rtol, maxit=20000)
                assert ost == 0 and abs(it[q - k] - oit) <= max(3, 0.05 * oit)
                assert np.isfinite(X).all()
        finally:
            mps.mpspmv_batch_destroy(b)
    finally:
        for h in mats:
            mps.mpspmv_destroy(h)


def test_batch_cg_maxit_and_invalid():
    mats, coos, ks = make_batch(2, count=3, seed=11, nmax=400, kappa=(0.1, 10.0))
    try:
        b = mps.mpspmv_batch_create(mats, ks, 0)
        try:
            Bs = [to_dev(rhs_block(c.ncols, k, 2, 7)) for c, k in zip(coos, ks)]
            Xs = [torch.zeros_like(B) for B in Bs]
            st, it, rr, ss = mps.mpspmv_batch_cg(b, Bs, Xs, sum(ks), 1e-30, 0.0, 5)
            assert st == mps.MPSPMV_ENOCONV and (it == 5).all() and (ss == mps.MPSPMV_ENOCONV).all()
        finally:
            mps.mpspmv_batch_destroy(b)
        with pytest.raises(mps.MpspmvError):
            mps.mpspmv_batch_create(mats, [1, 33, 2], 0)
        h4 = mps.mpspmv_create_csr(5, 5, np.arange(5), np.arange(5), np.ones((1, 5)), 4)
        try:
            with pytest.raises(mps.MpspmvError):
                mps.mpspmv_batch_create([mats[0], h4], [1, 1], 0)   # mixed precisions
        finally:
            mps.mpspmv_destroy(h4)
    finally:
        for h in mats:
            mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 4])
def test_batch_cg_exact_accumulation(L):
    """Batches of MPSPMV_EXACT_ACC handles: exact products and exact vector
    kernels.  Every system converges with about the iteration count of the
    single-handle exact CG and of the oracle's CG, to the target."""
    mats, coos, ks = make_batch(L, count=5, seed=13, nmax=2500, kappa=(0.1, 10.0), flags=16)
    rtol = {2: 1e-25, 4: 1e-50}[L]
    try:
        b = mps.mpspmv_batch_create(mats, ks, 0)
        try:
            Bs = [to_dev(rhs_block(c.ncols, k, L, 300 + 10 * i)) for i, (c, k) in enumerate(zip(coos, ks))]
            Xs = [torch.zeros_like(B) for B in Bs]
            st, it, rr, ss = mps.mpspmv_batch_cg(b, Bs, Xs, sum(ks), rtol, 0.0, 20000)
            assert st == mps.MPSPMV_OK and (ss == 0).all()
            assert (rr <= 50 * rtol).all()
            q = 0
            for i, (h, c, k) in enumerate(zip(mats, coos, ks)):
                Bh = Bs[i].cpu().numpy()
                bcol = to_dev(Bh[:, :, 0])
                xcol = torch.zeros_like(bcol)
                st1, it1, rr1 = mps.mpspmv_cg(h, bcol, xcol, rtol, 0.0, 20000)
                assert st1 == 0 and abs(it[q] - it1) <= max(3, 0.05 * it1), (i, it[q], it1)
                A = oracle.coo_to_csr(c.nrows, c.ncols, c.row, c.col, c.promoted(L), L)
                ost, ox, oit, orr = oracle.cg(A, Bh[:, :, 0], rtol=rtol, maxit=20000)
                assert ost == 0 and abs(it[q] - oit) <= max(3, 0.05 * oit)
                # the batched solution of this system solves it to the target (exact residual)
                x = Xs[i].cpu().numpy()[:, :, 0]
                ex_re, _, _, _ = exact.exact_rows(A, x)
                from fractions import Fraction as F
                den = 1 << (2 * exact.SCALE)
                num = sum((exact.to_fraction(Bh[:, j, 0]) - F(ex_re[j], den)) ** 2 for j in range(c.nrows))
                bb = sum(exact.to_fraction(Bh[:, j, 0]) ** 2 for j in range(c.nrows))
                assert float(num / bb) ** 0.5 <= 50 * rtol
                q += k
        finally:
            mps.mpspmv_batch_destroy(b)
    finally:
        for h in mats:
            mps.mpspmv_destroy(h)
