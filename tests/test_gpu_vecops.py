"""Krylov vector operations through the C ABI (mpspmv_dot, mpspmv_axpy) and
the solvers of MPSPMV_EXACT_ACC handles.

The inner products and updates of Section 4.2's CG and BiCGSTAB, in DD / TD /
QD: paper order against the oracle's vector routines (axpy element by element,
bit for bit), both arithmetics against exact rational values of
sum conj(u_i) v_i and u + alpha v."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads
from oracle import exact
from oracle import exact_model as model
from tests._util import csr_pair, to_dev

pytestmark = pytest.mark.gpu

mps = pytest.importorskip("paper_2412_17510_gb300")
torch = pytest.importorskip("torch")

EX = 16  # MPSPMV_EXACT_ACC


def vec_handle(L, cplx, ex):
    """A 1 x 1 matrix: the handle only fixes precision and arithmetic."""
    vals = np.zeros((2 if cplx else 1, 1))
    vals[0, 0] = 1.0
    return mps.mpspmv_create_csr(1, 1, [0], [0], vals, L, (EX if ex else 0) | (1 if cplx else 0))


def ints(x, L, cplx):
    """Exact values of the elements (units of 2**-1074): (re list, im list)."""
    n = x.shape[1]
    re = [exact.limbs_to_int(x[:L, i]) for i in range(n)]
    im = [exact.limbs_to_int(x[L:2 * L, i]) for i in range(n)] if cplx else [0] * n
    return re, im


def dot_ratio(got_re, got_im, u, v, L, cplx, factor):
    """max over parts of |got - exact| / (factor u_L sum |products|)."""
    ur, ui = ints(u, L, cplx)
    vr, vi = ints(v, L, cplx)
    sr = si = ar = ai = 0
    for a, b, c, d in zip(ur, ui, vr, vi):  # conj(a + bi) (c + di)
        sr += a * c + b * d
        si += a * d - b * c
        ar += abs(a * c) + abs(b * d)
        ai += abs(a * d) + abs(b * c)
    worst = 0.0
    for got, ex, ab in ((got_re, sr, ar), (got_im, si, ai)):
        err = abs((exact.limbs_to_int(got) << exact.SCALE) - ex)
        if ab == 0:
            if err:
                return math.inf
            continue
        worst = max(worst, float(Fraction(err, ab)) / (exact.U[L] * factor))
    return worst


def axpy_ratio(w, alpha_re, alpha_im, u, v, L, cplx, factor):
    """max over elements and parts of |w - (u + alpha v)| / (factor u_L
    (|u| + |alpha||v|)), the moduli taken per real product."""
    a = exact.limbs_to_int(alpha_re)
    b = exact.limbs_to_int(alpha_im) if cplx else 0
    ur, ui = ints(u, L, cplx)
    vr, vi = ints(v, L, cplx)
    wr, wi = ints(w, L, cplx)
    S = 1 << exact.SCALE
    worst = 0.0
    for i in range(u.shape[1]):
        parts = [(wr[i], ur[i] * S + a * vr[i] - b * vi[i], abs(ur[i]) * S + abs(a * vr[i]) + abs(b * vi[i]))]
        if cplx:
            parts.append((wi[i], ui[i] * S + a * vi[i] + b * vr[i], abs(ui[i]) * S + abs(a * vi[i]) + abs(b * vr[i])))
        for got, ex, ab in parts:
            err = abs(got * S - ex)
            if ab == 0:
                if err:
                    return math.inf
                continue
            worst = max(worst, float(Fraction(err, ab)) / (exact.U[L] * factor))
    return worst


def alpha_of(L, cplx, seed):
    a = workloads.full_limb_vector(1, L, seed=seed, cplx=cplx)[:, 0]
    return a[:L], (a[L:] if cplx else np.zeros(L))


@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_axpy_paper_order_bit_identical_to_oracle(L, cplx):
    n = 5000 + 17
    u = workloads.full_limb_vector(n, L, seed=1, cplx=cplx)
    v = workloads.full_limb_vector(n, L, seed=2, cplx=cplx)
    ar, ai = alpha_of(L, cplx, 3)
    h = vec_handle(L, cplx, False)
    try:
        ud, vd = to_dev(u), to_dev(v)
        wd = torch.full_like(ud, float("nan"))
        mps.mpspmv_axpy(h, n, ar, ud, vd, wd, alpha_im=ai if cplx else None)
        torch.cuda.synchronize()
        ref = oracle.axpy(L, ar, u, v, alpha_im=ai, cplx=cplx)
        assert np.array_equal(wd.cpu().numpy(), ref)
        # in place (w = u)
        mps.mpspmv_axpy(h, n, ar, ud, vd, ud, alpha_im=ai if cplx else None)
        torch.cuda.synchronize()
        assert np.array_equal(ud.cpu().numpy(), ref)
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_axpy_exact_within_bound(L, cplx):
    n = 3000 + 5
    u = workloads.full_limb_vector(n, L, seed=4, cplx=cplx)
    v = workloads.full_limb_vector(n, L, seed=5, cplx=cplx)
    ar, ai = alpha_of(L, cplx, 6)
    h = vec_handle(L, cplx, True)
    try:
        ud, vd = to_dev(u), to_dev(v)
        wd = torch.full_like(ud, float("nan"))
        mps.mpspmv_axpy(h, n, ar, ud, vd, wd, alpha_im=ai if cplx else None)
        torch.cuda.synchronize()
        w = wd.cpu().numpy()
        assert axpy_ratio(w, ar, ai, u, v, L, cplx, 4.0) <= 1.0
        # v in place (w = v)
        mps.mpspmv_axpy(h, n, ar, ud, vd, vd, alpha_im=ai if cplx else None)
        torch.cuda.synchronize()
        assert np.array_equal(vd.cpu().numpy(), w)
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 4])
def test_axpy_exact_cancellation(L):
    """u = -alpha v up to the last components: the exact form keeps the
    small difference to the format's precision; the bound is relative to
    |u| + |alpha v| and holds for both arithmetics."""
    n = 2000
    v = workloads.full_limb_vector(n, L, seed=7)
    ar, _ = alpha_of(L, False, 8)
    u = -oracle.axpy(L, ar, np.zeros_like(v), v)
    u[L - 1] *= 1.0 + 2.0 ** -30  # a perturbation of the last component
    for ex in (False, True):
        h = vec_handle(L, False, ex)
        try:
            ud, vd = to_dev(u), to_dev(v)
            wd = torch.empty_like(ud)
            mps.mpspmv_axpy(h, n, ar, ud, vd, wd)
            torch.cuda.synchronize()
            assert axpy_ratio(wd.cpu().numpy(), ar, np.zeros(L), u, v, L, False, 4.0) <= 1.0
        finally:
            mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [1, 2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("ex", [False, True])
def test_dot_within_bound(L, cplx, ex):
    n = 4096 + 33
    u = workloads.full_limb_vector(n, L, seed=10, cplx=cplx)
    v = workloads.full_limb_vector(n, L, seed=11, cplx=cplx)
    h = vec_handle(L, cplx, ex)
    try:
        re, im = mps.mpspmv_dot(h, n, to_dev(u), to_dev(v))
        factor = 8.0 * (math.ceil(math.log2(n)) + 2)
        assert dot_ratio(re, im, u, v, L, cplx, factor) <= 1.0
        if not cplx:
            assert not im.any()
        # the self product of a complex vector has an exactly zero imaginary
        # part in the exact arithmetic
        if cplx and ex:
            ud = to_dev(u)
            re2, im2 = mps.mpspmv_dot(h, n, ud, ud)
            assert not im2.any() and re2[0] > 0
        # n = 0: zero
        z_re, z_im = mps.mpspmv_dot(h, 0, to_dev(u), to_dev(v))
        assert not z_re.any() and not z_im.any()
    finally:
        mps.mpspmv_destroy(h)


def test_dot_exact_many_elements_per_thread():
    """n well above the exact kernels' thread count (each thread sums several
    elements exactly before the block tree): QD, within the bound."""
    L, n = 4, 400_000 + 3
    u = workloads.full_limb_vector(n, L, seed=12)
    v = workloads.full_limb_vector(n, L, seed=13)
    h = vec_handle(L, False, True)
    try:
        re, im = mps.mpspmv_dot(h, n, to_dev(u), to_dev(v))
        assert dot_ratio(re, im, u, v, L, False, 8.0 * (math.ceil(math.log2(n)) + 2)) <= 1.0
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("ex", [False, True])
def test_dot_non_finite_gives_non_finite(ex):
    L, n = 2, 1000
    u = workloads.full_limb_vector(n, L, seed=14)
    v = workloads.full_limb_vector(n, L, seed=15)
    u[0, 123] = np.inf
    h = vec_handle(L, False, ex)
    try:
        re, _ = mps.mpspmv_dot(h, n, to_dev(u), to_dev(v))
        assert not np.isfinite(re[0])
    finally:
        mps.mpspmv_destroy(h)


def test_vector_ops_argument_errors():
    h = vec_handle(2, False, True)
    try:
        u = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
        with pytest.raises(mps.MpspmvError) as e:
            mps.mpspmv_dot(h, -1, u, u)
        assert e.value.status == mps.MPSPMV_EINVAL
        with pytest.raises(mps.MpspmvError) as e:
            mps.mpspmv_axpy(h, 4, 1.0, u, None, u)
        assert e.value.status == mps.MPSPMV_EINVAL
        mps.mpspmv_axpy(h, 0, 1.0, None, None, None)  # nothing to do
    finally:
        mps.mpspmv_destroy(h)


# ---------------------------------------------------------------------------
# Solvers of exact-accumulation handles (exact SpMV and vector kernels)
# ---------------------------------------------------------------------------
def gpu_solve(fn, h, b, maxit, rtol):
    bd = to_dev(b)
    xd = torch.zeros_like(bd)
    st, it, rr = fn(h, bd, xd, rtol, 0.0, maxit)
    torch.cuda.synchronize()
    return st, xd.cpu().numpy(), it, rr


@pytest.mark.parametrize("L", [2, 3, 4])
def test_cg_exact_handle(L):
    coo = workloads.laplacian_2d(24, 20)
    n = coo.nrows
    b = np.zeros((L, n))
    b[0] = np.random.default_rng(0).uniform(-1, 1, n)
    rtol = {2: 1e-25, 3: 1e-40, 4: 1e-55}[L]
    A, h = csr_pair(coo, L, flags=EX)
    try:
        st, x, it, rr = gpu_solve(mps.mpspmv_cg, h, b, 3000, rtol)
        ost, ox, oit, orr = oracle.cg(A, b, rtol=rtol, maxit=3000)
        assert st == mps.MPSPMV_OK and ost == 0
        assert abs(it - oit) <= max(2, 0.05 * oit)
        assert rr <= 4 * rtol
        # the solutions agree to about cond(A) rtol (cond ~ 250 here), compared
        # exactly component sum against component sum
        scale = np.abs(ox[0]).max()
        d = max(abs(exact.limbs_to_int(x[:, i]) - exact.limbs_to_int(ox[:, i])) for i in range(n))
        assert float(Fraction(d, 1 << exact.SCALE)) <= 1e4 * rtol * scale
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_bicgstab_exact_handle(L, cplx):
    n = 300
    coo = workloads.random_sparse(n, n, 6, seed=L, cplx=cplx)
    rows = np.concatenate([coo.row, np.arange(n)])
    cols = np.concatenate([coo.col, np.arange(n)])
    shift = np.zeros((coo.val.shape[0], n))
    shift[0] = 8.0
    if cplx:
        shift[1] = 2.0
    full = workloads.COO(n, n, rows, cols, np.concatenate([coo.val, shift], axis=1))
    b = workloads.full_limb_vector(n, L, seed=L + 1, cplx=cplx)
    rtol = {2: 1e-28, 4: 1e-55}[L]
    A, h = csr_pair(full, L, flags=EX | (1 if cplx else 0))
    try:
        st, x, it, rr = gpu_solve(mps.mpspmv_bicgstab, h, b, 500, rtol)
        ost, ox, oit, orr = oracle.bicgstab(A, b, rtol=rtol, maxit=500)
        assert st == 0 and ost == 0
        assert abs(it - oit) <= 2
        assert rr <= 4 * rtol
    finally:
        mps.mpspmv_destroy(h)



@pytest.mark.parametrize("L", [2, 3, 4])
@pytest.mark.parametrize("cplx", [False, True])
def test_axpy_exact_bit_identical_to_the_exact_model(L, cplx):
    """w = u + alpha v on an exact handle equals the exact model element by
    element (oracle/exact_model.py: u's components plus the decomposed
    products alpha v, each part cut once by truncation), for every element
    whose terms fit the accumulator's window."""
    n = 3000 + 5
    u = workloads.full_limb_vector(n, L, seed=80 + L, cplx=cplx)
    v = workloads.full_limb_vector(n, L, seed=90 + L, cplx=cplx)
    ar, ai = alpha_of(L, cplx, 99)
    h = vec_handle(L, cplx, True)
    try:
        ud, vd = to_dev(u), to_dev(v)
        wd = torch.full_like(ud, float("nan"))
        mps.mpspmv_axpy(h, n, ar, ud, vd, wd, alpha_im=ai if cplx else None)
        torch.cuda.synchronize()
        w = wd.cpu().numpy()
    finally:
        mps.mpspmv_destroy(h)
    compared = 0
    for i in range(n):
        want, fits = model.axpy_model(L, ar, ai, u[:, i], v[:, i], cplx)
        if fits:
            assert np.array_equal(w[:, i], want), (L, cplx, i, w[:, i], want)
            compared += 1
    assert compared >= n // 2
