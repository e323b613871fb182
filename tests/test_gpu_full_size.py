"""Parity at the benchmark's full sizes, in the launch configuration that
bench.py times: the 27-point stencil on a 128^3 grid, the power-law matrix
with n = 1e6 (Zipf 1.5 row lengths, clipped to 20,000) and the complex-
symmetric band with n = 500,000; binary64 triplet values, DD / TD / QD,
paper-order and exact-accumulation handles, one mpspmv_spmv on device
buffers.  The oracle cannot multiply these matrices whole in a test's time,
so the check runs on sampled rows: about 120 random rows plus the first, the
last and the longest one (so the bound's m is the whole matrix's maximum row
length).  Every sampled component meets |y - y_exact| <= 8 m u (|A||x|)
against the exact rational value; in paper order, the sampled rows that one
run holds are bit-identical to the oracle's row sums (most band rows span two
runs, so there the bitwise part covers few rows).  The measured ratio to the
bound is printed for every case."""
import numpy as np
import pytest

import oracle
import workloads
from oracle import exact
from tests._util import gpu_spmv

pytestmark = pytest.mark.gpu

mps = pytest.importorskip("paper_2412_17510_gb300")
torch = pytest.importorskip("torch")

EX = 16  # MPSPMV_EXACT_ACC

MATRICES = {
    "stencil27_128^3": lambda: workloads.stencil_27pt(128),
    "powerlaw_1e6_zipf1.5": lambda: workloads.power_law(1000000),
    "complex_band_5e5": lambda: workloads.complex_sym_banded(500000, 48, 0.3, seed=0),
}

_cache = {}


def matrix(name):
    """The triplets, their row starts and the sampled rows (built once per
    module run; the power-law matrix alone holds 2.2e8 entries)."""
    if name not in _cache:
        _cache.clear()
        coo = MATRICES[name]()
        n = coo.nrows
        counts = np.bincount(coo.row, minlength=n)
        ip = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(counts, out=ip[1:])
        rng = np.random.default_rng(17)
        rows = np.unique(np.concatenate([rng.choice(n, 120, replace=False), [0, n - 1, int(np.argmax(counts))]]))
        mask = np.isin(coo.row, rows, kind="table")
        sub = workloads.COO(len(rows), coo.ncols, np.searchsorted(rows, coo.row[mask]), coo.col[mask],
                            coo.val[:, mask])
        _cache[name] = (coo, ip, rows, sub)
    return _cache[name]


@pytest.mark.parametrize("name,L", [(m, L) for m in MATRICES for L in ((2, 4) if m.startswith("complex") else (2, 3, 4))])
def test_full_size_sampled_rows(name, L):
    coo, ip, rows, sub = matrix(name)
    cplx = name.startswith("complex")
    P = 2 * L if cplx else L
    A_rows = oracle.coo_to_csr(sub.nrows, sub.ncols, sub.row, sub.col, sub.promoted(L), L, cplx)
    assert A_rows.nrows == len(rows)
    assert int(A_rows.row_lengths().max()) == int(np.diff(ip).max())
    x = workloads.full_limb_vector(coo.ncols, L, seed=0, cplx=cplx)
    ref = oracle.spmv(A_rows, x)
    worst = {}
    for arith, fl in (("paper", 0), ("exact", EX)):
        h = mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, L,
                                  fl | (mps.MPSPMV_COMPLEX if cplx else 0), val_limbs=1)
        try:
            y = gpu_spmv(h, x, P, coo.nrows)[:, rows]
            K = mps.mpspmv_get_info(h)["chunk"]
        finally:
            mps.mpspmv_destroy(h)
        worst[arith] = exact.bound_ratio(y, A_rows, x)
        assert worst[arith] <= 1.0, (arith, worst[arith])
        if arith == "paper":
            one_run = (ip[rows] // K == (ip[rows + 1] - 1) // K) & (ip[rows + 1] > ip[rows])
            # the band's 15M entries give runs of 16, shorter than most of its rows
            assert one_run.sum() >= (1 if cplx else 50)
            assert np.array_equal(y[:, one_run], ref[:, one_run])
    print("%s L=%d max |y - y_exact| / (8 m u |A||x|): paper %.3g, exact %.3g" % (name, L, worst["paper"],
                                                                               worst["exact"]))
