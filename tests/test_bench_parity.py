"""The parity report of bench.py's oracle leg (host logic, no GPU): the
sampled rows include the longest one, results that equal the oracle's give
bit identity and ratios within the bound, and a perturbed result is caught."""
import importlib.util
import os

import numpy as np

import oracle
import workloads
from oracle import exact
from oracle import exact_model as em

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _setup(bench):
    mats = {"stencil": workloads.stencil_27pt(6), "powerlaw": workloads.power_law(400, seed=3)}
    xs = {m: {L: workloads.full_limb_vector(c.ncols, L, seed=0) for L in bench.PRECS} for m, c in mats.items()}
    rows_of = {m: bench.sample_rows(c, n=40) for m, c in mats.items()}
    ysamp, chunk_of = {}, {}
    for m, c in mats.items():
        rows = rows_of[m]
        counts = np.bincount(c.row, minlength=c.nrows)
        assert int(np.argmax(counts)) in rows and 0 in rows and c.nrows - 1 in rows
        for L in bench.PRECS:
            A = oracle.coo_to_csr(c.nrows, c.ncols, c.row, c.col, c.promoted(L), L)
            ysamp[("paper", m, L)] = oracle.spmv(A, xs[m][L])[:, rows]
            sub = oracle.CSR(len(rows), c.ncols, np.concatenate([[0], np.cumsum(np.diff(A.indptr)[rows])]),
                             np.concatenate([A.indices[A.indptr[r]:A.indptr[r + 1]] for r in rows]),
                             np.concatenate([A.data[:, A.indptr[r]:A.indptr[r + 1]] for r in rows], axis=1), L,
                             False)
            ysamp[("exact", m, L)] = np.stack([em.row_model_wide(L, sub, xs[m][L], i)[0] for i in range(len(rows))],
                                              axis=1)
            chunk_of[("paper", m, L)] = chunk_of[("exact", m, L)] = 64
    return mats, xs, rows_of, ysamp, chunk_of


def test_parity_report_accepts_oracle_results():
    bench = _bench()
    mats, xs, rows_of, ysamp, chunk_of = _setup(bench)
    sell_of = {k: k[1] == "stencil" for k in ysamp}
    rep = bench.parity_report(mats, xs, rows_of, ysamp, chunk_of, sell_of)
    assert rep["paper_one_run_rows_bit_identical"] is True and rep["paper_one_run_rows"] > 0
    assert rep["exact_model_rows_bit_identical"] is True and rep["exact_model_rows"] > 100
    for ar in ("paper", "exact"):
        assert len(rep["max_bound_ratio"][ar]) == 6
        assert all(0.0 <= r <= 1.0 for r in rep["max_bound_ratio"][ar].values())


def test_parity_report_catches_a_wrong_result():
    bench = _bench()
    mats, xs, rows_of, ysamp, chunk_of = _setup(bench)
    rep0 = bench.parity_report(mats, xs, rows_of, ysamp, chunk_of)
    # one ulp in the second component of every sampled stencil row (most of
    # them lie inside one run of 64 entries), a relative 2^-30 in a QD result
    y = ysamp[("paper", "stencil", 2)].copy()
    y[1] = np.nextafter(y[1], np.inf)
    ysamp[("paper", "stencil", 2)] = y
    y = ysamp[("exact", "powerlaw", 4)].copy()
    y[0] *= 1.0 + 2.0 ** -30
    ysamp[("exact", "powerlaw", 4)] = y
    sell_of = {k: k[1] == "stencil" for k in ysamp}
    rep = bench.parity_report(mats, xs, rows_of, ysamp, chunk_of, sell_of)
    assert rep["paper_one_run_rows_bit_identical"] is False
    assert rep["exact_model_rows_bit_identical"] is False
    assert rep["max_bound_ratio"]["exact"]["powerlaw/QD"] > 1.0
    assert rep["max_bound_ratio"]["exact"]["stencil/DD"] == rep0["max_bound_ratio"]["exact"]["stencil/DD"]


def test_oracle_sampler_slices_and_rates():
    """The CPU baseline's sampler (one method for both bench arms): slices
    start at evenly spaced rows, do not overlap, hold the requested entries
    where the matrix allows, and the measured rates are the oracle's own
    (a slice's product equals the oracle on the same rows)."""
    import multiprocessing as mp
    import bench  # by its own name: the spawned workers import the sampler's function from it
    mats = {"powerlaw": workloads.power_law(3000, seed=3), "stencil": workloads.stencil_27pt(10)}
    xs = {m: {L: workloads.full_limb_vector(c.ncols, L, seed=0) for L in bench.PRECS} for m, c in mats.items()}
    want = {2: 5000, 3: 800, 4: 800}
    sampler = bench.OracleSampler(mats, xs, 4, slice_entries=want)
    try:
        for (m, L), tl in sampler.tasks.items():
            coo = mats[m]
            ip = np.concatenate([[0], np.cumsum(np.bincount(coo.row, minlength=coo.nrows))])
            assert len(tl) == 4
            for i, (_, _, L2, a, b) in enumerate(tl):
                assert L2 == L and a == int(i * coo.nrows / 4) and b > a
                assert i == 3 or b <= tl[i + 1][3]
                assert ip[b] - ip[a] >= min(want[L], ip[tl[i + 1][3] if i < 3 else coo.nrows] - ip[a]) or b == a + 1
            e, t = bench._oracle_slice(tl[1])
            assert e == ip[tl[1][4]] - ip[tl[1][3]] and t > 0
        with mp.get_context("spawn").Pool(2) as pool:
            rates = sampler.rates(pool)
            single = sampler.single_rates(pool)
        assert set(rates) == set(sampler.tasks) and all(r > 0 for r in rates.values())
        assert all(r > 0 for r in single.values())
    finally:
        sampler.close()
    assert not os.path.exists(sampler.dir)
