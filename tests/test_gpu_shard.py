"""Sharded SpMV and CG on the GPU (two gloo ranks as processes that share
cuda:0; no kernel waits on another, every exchange is a host collective),
and the scalar entry points they use, through the C ABI against the oracle."""
import os
import socket
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads
from oracle import exact

pytestmark = pytest.mark.gpu

mps = pytest.importorskip("paper_2412_17510_gb300")
torch = pytest.importorskip("torch")


def _frac(limbs):
    return sum((Fraction(float(v)) for v in limbs), Fraction(0))


def _mp_scalars(count, L, seed):
    rng = np.random.default_rng(seed)
    out = np.zeros((count, 2 * L))
    for i in range(count):
        for c in range(2):
            v = workloads.full_limb_vector(1, L, rng=rng)[:, 0] * 2.0 ** int(rng.integers(-40, 40))
            out[i, c * L:(c + 1) * L] = v
    return out


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_scalar_sum_and_div_paper_order_match_oracle(L):
    """Paper order: the rank-ordered sum is the oracle's MP additions from
    left to right and the quotient the oracle's MP division, bit for bit."""
    coo = workloads.laplacian_2d(4)
    h = mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, L, 0, val_limbs=1)
    try:
        parts = _mp_scalars(7, L, seed=L)
        parts[:, L:] = 0.0
        re, im = mps.mpspmv_scalar_sum(h, parts)
        want = parts[0, :L]
        for p in parts[1:]:
            want = oracle.mp_add(L, want, p[:L])
        assert np.array_equal(re, want) and not im.any()
        re1, _ = mps.mpspmv_scalar_sum(h, parts[:1])
        assert np.array_equal(re1, parts[0, :L])
        q, _ = mps.mpspmv_scalar_div(h, parts[2], parts[5])
        assert np.array_equal(q, oracle.mp_div(L, parts[2, :L], parts[5, :L]))
        with pytest.raises(mps.MpspmvError) as e:
            mps.mpspmv_scalar_div(h, parts[2], np.zeros(2 * L))
        assert e.value.status == mps.MPSPMV_EBREAKDOWN
    finally:
        mps.mpspmv_destroy(h)


@pytest.mark.parametrize("L", [2, 4])
def test_scalar_sum_exact_and_complex_div(L):
    """MPSPMV_EXACT_ACC: the sum of all components exactly, cut to L
    components (truncation: below the exact value in magnitude, within
    2^(1-53L) of it).  Complex division: within 16 u of a conj(b) / |b|^2."""
    coo = workloads.complex_sym_banded(20, 2, 0.5, seed=0)
    h = mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, L,
                              mps.MPSPMV_COMPLEX | mps.MPSPMV_EXACT_ACC, val_limbs=1)
    try:
        parts = _mp_scalars(9, L, seed=10 + L)
        re, im = mps.mpspmv_scalar_sum(h, parts)
        for got, off in ((re, 0), (im, L)):
            ex = sum((_frac(p[off:off + L]) for p in parts), Fraction(0))
            g = _frac(got)
            assert abs(g) <= abs(ex) and abs(ex - g) <= abs(ex) * Fraction(2) ** (1 - 53 * L)
        a, b = parts[1], parts[4]
        qr, qi = mps.mpspmv_scalar_div(h, a, b)
        ar, ai, br, bi = _frac(a[:L]), _frac(a[L:]), _frac(b[:L]), _frac(b[L:])
        den = br * br + bi * bi
        wr, wi = (ar * br + ai * bi) / den, (ai * br - ar * bi) / den
        tol = 16 * Fraction(exact.U[L]) * max(abs(wr), abs(wi))
        assert abs(_frac(qr) - wr) <= tol and abs(_frac(qi) - wi) <= tol
    finally:
        mps.mpspmv_destroy(h)


# ---------------------------------------------------------------------------
# two gloo ranks on cuda:0
# ---------------------------------------------------------------------------
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(fn, rank, world, port, out, *args):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = fn(dist, rank, world, *args)
    finally:
        dist.destroy_process_group()


def _spawn(fn, world, *args):
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(fn, r, world, port, out) + args) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
        assert p.exitcode == 0
    return dict(out)


def _matrix(name):
    return {"powerlaw": lambda: workloads.power_law(3000, seed=1),
            "laplace": lambda: workloads.laplacian_2d(40),
            "cband": lambda: workloads.complex_sym_banded(2000, 9, 0.4, seed=1)}[name]()


def _gpu_spmv_rank(dist, rank, world, name, L, flags):
    import torch as th
    import paper_2412_17510_gb300 as m
    from paper_2412_17510_gb300 import shard
    th.cuda.set_device(0)
    coo = _matrix(name)
    fl = flags | (m.MPSPMV_COMPLEX if coo.cplx else 0)
    plan = shard.ShardPlan.build(coo.nrows, coo.ncols, coo.row, coo.col, world, rank)
    be = shard.GpuBackend(L, fl)
    A = shard.ShardedMatrix(plan, shard.TorchComm(dist), be, coo.row, coo.col, coo.val, val_limbs=1)
    try:
        x = workloads.full_limb_vector(coo.ncols, L, seed=3, cplx=coo.cplx)
        y = be.zeros(plan.nlocal)
        A.spmv(be.asvec(x[:, plan.r0:plan.r1]), y)
        th.cuda.synchronize()
        K = m.mpspmv_get_info(A.h)["chunk"]
        return plan.r0, plan.r1, y.cpu().numpy(), K
    finally:
        A.free()


@pytest.mark.parametrize("name,L,flags", [("powerlaw", 2, 0), ("powerlaw", 4, 16), ("laplace", 3, 0),
                                          ("laplace", 4, 16), ("cband", 2, 0), ("cband", 4, 16)])
def test_sharded_spmv_two_ranks(name, L, flags):
    """Rows are split over two ranks; paper order: rows that one run of the
    rank's handle holds equal the oracle's rows bit for bit; every row (both
    arithmetics) meets the bound 8 m u (|A||x|)_i."""
    coo = _matrix(name)
    res = _spawn(_gpu_spmv_rank, 2, name, L, flags)
    A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.promoted(L), L, coo.cplx)
    x = workloads.full_limb_vector(coo.ncols, L, seed=3, cplx=coo.cplx)
    y = np.concatenate([res[r][2] for r in range(2)], axis=1)
    assert exact.bound_ratio(y, A, x) <= 1.0
    if not flags:
        ref = oracle.spmv(A, x)
        ip = A.indptr
        for r in range(2):
            r0, r1, _, K = res[r]
            loc = ip[r0:r1 + 1] - ip[r0]
            one = (loc[1:] > loc[:-1]) & ((loc[:-1] // K) == ((loc[1:] - 1) // K))
            rows = np.arange(r0, r1)[one]
            assert rows.size > 0
            assert np.array_equal(y[:, rows], ref[:, rows])


def _gpu_cg_rank(dist, rank, world, L, flags, rtol):
    import torch as th
    from paper_2412_17510_gb300 import shard
    th.cuda.set_device(0)
    coo = workloads.diffusion_7pt(12, 11, 10, kappa_range=(0.1, 10.0), seed=2)
    plan = shard.ShardPlan.build(coo.nrows, coo.ncols, coo.row, coo.col, world, rank)
    be = shard.GpuBackend(L, flags)
    A = shard.ShardedMatrix(plan, shard.TorchComm(dist), be, coo.row, coo.col, coo.val, val_limbs=1)
    try:
        b = workloads.full_limb_vector(coo.ncols, L, seed=4)
        x = be.zeros(plan.nlocal)
        st, it, rr = shard.sharded_cg(A, be.asvec(b[:, plan.r0:plan.r1]), x, rtol, 0.0, 3000)
        return st, it, rr
    finally:
        A.free()


@pytest.mark.parametrize("L,flags,rtol", [(2, 0, 1e-25), (2, 16, 1e-25), (4, 16, 1e-50)])
def test_sharded_cg_two_ranks_matches_single_handle(L, flags, rtol):
    """CG over two ranks (x exchanged per product, inner products summed in
    rank order) against mpspmv_cg on one handle of the whole matrix: the
    same iteration count within one, both converged, and the recomputed
    residual of the sharded solve within 10 rtol."""
    coo = workloads.diffusion_7pt(12, 11, 10, kappa_range=(0.1, 10.0), seed=2)
    h = mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.val, L, flags, val_limbs=1)
    try:
        b = torch.from_numpy(workloads.full_limb_vector(coo.ncols, L, seed=4)).cuda()
        x = torch.zeros_like(b)
        st0, it0, rr0 = mps.mpspmv_cg(h, b, x, rtol, 0.0, 3000)
        assert st0 == mps.MPSPMV_OK
    finally:
        mps.mpspmv_destroy(h)
    res = _spawn(_gpu_cg_rank, 2, L, flags, rtol)
    assert res[0][1] == res[1][1]
    assert abs(res[0][1] - it0) <= 1
    for r in range(2):
        assert res[r][0] == 0 and res[r][2] <= 10 * rtol
