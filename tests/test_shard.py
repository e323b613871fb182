"""Row-block sharding of the SpMV and CG (paper_2412_17510_gb300/shard.py):
the partition, the exchange plan, and the sharded product and solve run as
gloo ranks on the CPU with the oracle as each rank's local arithmetic.

Every row belongs to one block and keeps its entries' order, so the sharded
product equals the single-process oracle product bit for bit on every row;
the rank-ordered sums of the inner products change only the rounding of the
scalars, so CG takes the same iterations within one and meets its target."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads

shard = pytest.importorskip("paper_2412_17510_gb300.shard")


class OracleBackend:
    """One rank's local operations on the CPU through the oracle (test
    infrastructure): the same interface as shard.GpuBackend."""

    def __init__(self, L, cplx=False):
        self.L, self.cplx = L, cplx
        self.P = 2 * L if cplx else L

    def create(self, nrows, ncols, row, col, val, val_limbs):
        V = 2 if self.cplx else 1
        vals = np.zeros((self.P, len(row)))
        for c in range(V):
            vals[c * self.L:c * self.L + val_limbs] = val[c * val_limbs:(c + 1) * val_limbs]
        return oracle.coo_to_csr(nrows, ncols, row, col, vals, self.L, self.cplx)

    def destroy(self, h):
        pass

    def zeros(self, n):
        return np.zeros((self.P, n))

    def asvec(self, a):
        return np.array(a, dtype=np.float64)

    def host(self, v):
        return v

    def copy_cols(self, dst, doff, src, soff, count):
        dst[:, doff:doff + count] = src[:, soff:soff + count]

    def to_comm(self, v, on_device):
        import torch
        return torch.from_numpy(np.ascontiguousarray(v))

    def from_comm(self, t):
        return t.numpy()

    def comm_scalar(self, parts, on_device):
        import torch
        return torch.from_numpy(np.array(parts, dtype=np.float64))

    def spmv(self, h, x, y):
        y[:, :h.nrows] = oracle.spmv(h, x)

    def dot(self, h, n, u, v):
        re, im = oracle.dot(self.L, u[:, :n], v[:, :n], self.cplx)
        return np.concatenate([re, im])

    def axpy(self, h, n, alpha, u, v, w):
        L = self.L
        w[:, :n] = oracle.axpy(L, alpha[:L], u[:, :n], v[:, :n], alpha[L:] if self.cplx else None, self.cplx)

    def scalar_sum(self, h, parts):
        L = self.L
        re, im = parts[0][:L].copy(), parts[0][L:].copy()
        for p in parts[1:]:
            re = oracle.mp_add(L, re, p[:L])
            im = oracle.mp_add(L, im, p[L:]) if self.cplx else im
        return np.concatenate([re, im])

    def scalar_div(self, h, a, b):
        L = self.L
        return np.concatenate([oracle.mp_div(L, a[:L], b[:L]), np.zeros(L)])


# ---------------------------------------------------------------------------
# host logic
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("world", [1, 2, 3, 4, 7])
def test_partition_balances_entries(world):
    coo = workloads.power_law(5000, seed=2)
    counts = np.bincount(coo.row, minlength=coo.nrows)
    b = shard.partition_rows(counts, world)
    assert b[0] == 0 and b[-1] == coo.nrows and np.all(np.diff(b) >= 0)
    w = np.concatenate([[0], np.cumsum(counts + 1)])
    ideal = w[-1] / world
    for k in range(world):
        # a block misses its share by at most one row's weight at each end
        assert abs((w[b[k + 1]] - w[b[k]]) - ideal) <= 2 * (counts.max() + 1)


def _plans(coo, world):
    return [shard.ShardPlan.build(coo.nrows, coo.ncols, coo.row, coo.col, world, r) for r in range(world)]


@pytest.mark.parametrize("world", [2, 3, 5])
def test_plan_covers_each_window_once(world):
    """Every window is covered exactly once by the process's own block and
    the ranges it receives; what a process receives from a peer is what that
    peer sends it; local column indices lie inside the window."""
    coo = workloads.random_sparse(300, 300, 30, seed=4, empty_frac=0.2)
    plans = _plans(coo, world)
    for p in plans:
        cover = np.zeros(p.wlen, dtype=int)
        woff, boff, cnt = p.own_in_window()
        cover[woff:woff + cnt] += 1
        for peer, a, b in p.recv:
            cover[a - p.c0:b - p.c0] += 1
            assert (p.rank, a, b) in plans[peer].send
        assert np.all(cover == 1)
        lr, lc, _ = p.local_triplets(coo.row, coo.col, coo.val)
        assert lr.min(initial=0) >= 0 and lr.max(initial=-1) < p.nlocal
        assert lc.min(initial=0) >= 0 and lc.max(initial=-1) < max(p.wlen, 1)
    assert sum(p.nlocal for p in plans) == coo.nrows


def test_stencil_window_is_a_halo():
    """For the 2D 5-point Laplacian on an N x N grid the window of a block
    reaches one grid line into each neighbouring block and no further."""
    N, world = 24, 4
    coo = workloads.laplacian_2d(N)
    for p in _plans(coo, world):
        peers = {peer: b - a for peer, a, b in p.recv}
        assert set(peers) <= {p.rank - 1, p.rank + 1}
        assert all(v == N for v in peers.values())


def test_square_only():
    with pytest.raises(ValueError):
        shard.ShardPlan.build(4, 5, np.array([0]), np.array([4]), 2, 0)


# ---------------------------------------------------------------------------
# gloo ranks on the CPU
# ---------------------------------------------------------------------------
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


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
        p.join(300)
        assert p.exitcode == 0
    assert sorted(out.keys()) == list(range(world))
    return dict(out)


def _rank_main(fn, rank, world, port, out, *args):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = fn(dist, rank, world, *args)
    finally:
        dist.destroy_process_group()


def _cases():
    return {
        "random_empty_rows": workloads.random_sparse(257, 257, 40, seed=6, empty_frac=0.3),
        "powerlaw": workloads.power_law(600, seed=3),
        "laplace": workloads.laplacian_2d(18),
        "cband": workloads.complex_sym_banded(300, 7, 0.5, seed=2),
    }


def _spmv_rank(dist, rank, world, name, L):
    coo = _cases()[name]
    cplx = coo.cplx
    comm = shard.TorchComm(dist)
    plan = shard.ShardPlan.build(coo.nrows, coo.ncols, coo.row, coo.col, world, rank)
    be = OracleBackend(L, cplx)
    A = shard.ShardedMatrix(plan, comm, be, coo.row, coo.col, coo.val, val_limbs=1)
    x = workloads.full_limb_vector(coo.ncols, L, seed=5, cplx=cplx)
    y = be.zeros(plan.nlocal)
    A.spmv(x[:, plan.r0:plan.r1].copy(), y)
    d = A.dot(x[:, plan.r0:plan.r1].copy(), x[:, plan.r0:plan.r1].copy())
    part = be.dot(A.h, plan.nlocal, x[:, plan.r0:plan.r1], x[:, plan.r0:plan.r1])
    return plan.r0, plan.r1, y, d, part


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("name,L", [("random_empty_rows", 2), ("powerlaw", 4), ("laplace", 3), ("cband", 4)])
def test_sharded_spmv_equals_single_process(world, name, L):
    """Every row of the sharded product equals the oracle's single-process
    row bit for bit; the sharded inner product is the rank-ordered MP sum of
    the blocks' partials and identical on every rank."""
    coo = _cases()[name]
    res = _spawn(_spmv_rank, world, name, L)
    A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.promoted(L), L, coo.cplx)
    x = workloads.full_limb_vector(coo.ncols, L, seed=5, cplx=coo.cplx)
    ref = oracle.spmv(A, x)
    y = np.concatenate([res[r][2] for r in range(world)], axis=1)
    assert np.array_equal(y, ref)
    parts = [res[r][4] for r in range(world)]
    re, im = parts[0][:L], parts[0][L:]
    for p in parts[1:]:
        re = oracle.mp_add(L, re, p[:L])
        im = oracle.mp_add(L, im, p[L:])
    want = np.concatenate([re, im]) if coo.cplx else np.concatenate([re, np.zeros(L)])
    for r in range(world):
        assert np.array_equal(res[r][3], want)
    # the ordered sum differs from the one-pass dot only in rounding
    full_re, _ = oracle.dot(L, x, x, coo.cplx)
    assert abs(float(re[0]) - float(full_re[0])) <= 1e-25 * abs(float(full_re[0]))


def _cg_rank(dist, rank, world, L, rtol):
    coo = workloads.diffusion_7pt(7, 6, 5, kappa_range=(0.1, 10.0), seed=3)
    comm = shard.TorchComm(dist) if world > 1 else None
    plan = shard.ShardPlan.build(coo.nrows, coo.ncols, coo.row, coo.col, world, rank)
    be = OracleBackend(L)
    A = shard.ShardedMatrix(plan, comm, be, coo.row, coo.col, coo.val, val_limbs=1)
    b = workloads.full_limb_vector(coo.ncols, L, seed=8)
    x = np.zeros((L, plan.nlocal))
    st, it, rr = shard.sharded_cg(A, b[:, plan.r0:plan.r1].copy(), x, rtol, 0.0, 2000)
    return st, it, rr, x


@pytest.mark.parametrize("L,rtol", [(2, 1e-25), (4, 1e-50)])
def test_sharded_cg_matches_single_process(L, rtol):
    """One rank: the sharded CG is the oracle's CG step for step (same
    iterate bits).  Two and three gloo ranks: the same iteration count within
    one, converged, and the recomputed residual meets the target."""
    coo = workloads.diffusion_7pt(7, 6, 5, kappa_range=(0.1, 10.0), seed=3)
    A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, coo.promoted(L), L)
    b = workloads.full_limb_vector(coo.ncols, L, seed=8)
    st0, x0, it0, rr0 = oracle.cg(A, b, rtol, 0.0, 2000)
    assert st0 == 0
    # one rank, no communicator: the same operation sequence as the oracle
    st, it, rr, x = _cg_rank(None, 0, 1, L, rtol)
    assert (st, it) == (0, it0) and np.array_equal(x, x0) and rr == rr0
    for world in (2, 3):
        res = _spawn(_cg_rank, world, L, rtol)
        its = {res[r][1] for r in range(world)}
        assert len(its) == 1                     # every rank stops at the same step
        it = its.pop()
        assert abs(it - it0) <= 1
        for r in range(world):
            assert res[r][0] == 0 and res[r][2] <= 10 * rtol
        x = np.concatenate([res[r][3] for r in range(world)], axis=1)
        assert np.max(np.abs(x[0] - x0[0])) <= 1e-12 * np.max(np.abs(x0[0]))
