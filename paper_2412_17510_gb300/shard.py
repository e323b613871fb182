"""Row-block sharding of the multiple-precision SpMV and CG over processes.

The paper parallelises CSR SpMV over rows (Section 3: OpenMP threads over
row blocks) and uses inner products inside its Krylov solvers (Section 4.2).
Across GPUs this becomes:

* a partition of the rows into contiguous blocks balanced by stored entries
  (``partition_rows``); x and y are split by the same blocks;
* per process a handle holding its block of rows, with the columns renumbered
  into the block's column window [c0, c1) (the span of the columns its rows
  reference);
* before every product, an exchange of x: each process receives, from every
  other process, the part of that process's block that falls inside its
  window.  For a stencil or band matrix the window reaches only the
  neighbouring blocks (a halo exchange); for a general matrix it covers most
  of x (an allgather).  One plan (``ShardPlan``) describes both;
* inner products: every process computes the MP partial of its block, the
  partials are all-gathered and summed in rank order with the library's
  ``mpspmv_scalar_sum`` (MP additions left to right, or one exact sum for
  MPSPMV_EXACT_ACC handles), so every process holds the same bits whatever
  order a collective would have summed in.  No binary64 sum of MP limbs is
  ever formed by a collective.

This module is host-side orchestration only: partitioning, plans, the
exchange through ``torch.distributed`` (NCCL for CUDA tensors, gloo for host
tensors) and the CG loop's control flow.  Every arithmetic step runs in the
backend's kernels; the default backend (``GpuBackend``) is the CUDA library.
"""
import numpy as np


def partition_rows(row_counts, world):
    """Contiguous row blocks balanced by work: bounds[0] = 0 <= bounds[1] <=
    ... <= bounds[world] = nrows, each block holding about 1/world of the
    total weight (stored entries plus one per row, so long runs of empty
    rows are shared out too)."""
    counts = np.asarray(row_counts, dtype=np.int64)
    n = counts.shape[0]
    w = np.cumsum(counts + 1)
    total = int(w[-1]) if n else 0
    bounds = np.zeros(world + 1, dtype=np.int64)
    for k in range(1, world):
        bounds[k] = int(np.searchsorted(w, total * k / world, side="left")) + 1 if total else 0
        bounds[k] = min(max(bounds[k], bounds[k - 1]), n)
    bounds[world] = n
    return bounds


class ShardPlan:
    """The layout of one process's share of y = A x.

    rows        [r0, r1): this process's rows (and its block of x and y)
    window      [c0, c1): the columns its rows reference; the local handle's
                columns are renumbered to 0 .. c1 - c0 - 1
    recv        list of (peer, a, b): global columns [a, b) of peer's block
                that this process receives into its window
    send        list of (peer, a, b): global columns [a, b) of this
                process's block that peer needs
    """

    def __init__(self, nrows, ncols, bounds, windows, rank):
        self.nrows, self.ncols = int(nrows), int(ncols)
        self.world = len(bounds) - 1
        self.rank = int(rank)
        self.bounds = np.asarray(bounds, dtype=np.int64)
        self.windows = [(int(a), int(b)) for a, b in windows]
        self.r0, self.r1 = int(self.bounds[rank]), int(self.bounds[rank + 1])
        self.c0, self.c1 = self.windows[rank]
        self.recv, self.send = [], []
        for s in range(self.world):
            if s == rank:
                continue
            a, b = max(self.c0, int(self.bounds[s])), min(self.c1, int(self.bounds[s + 1]))
            if a < b:
                self.recv.append((s, a, b))
            wa, wb = self.windows[s]
            a, b = max(wa, self.r0), min(wb, self.r1)
            if a < b:
                self.send.append((s, a, b))

    @property
    def nlocal(self):
        return self.r1 - self.r0

    @property
    def wlen(self):
        return self.c1 - self.c0

    def own_in_window(self):
        """(offset in the window, offset in the block, count) of the part of
        this process's own block that lies inside its window."""
        a, b = max(self.c0, self.r0), min(self.c1, self.r1)
        if a >= b:
            return 0, 0, 0
        return a - self.c0, a - self.r0, b - a

    @staticmethod
    def build(nrows, ncols, row, col, world, rank, bounds=None):
        """Plan from the global triplets (every process can form the same
        bounds and windows without communication).  Square matrices only:
        x and y share the row blocks."""
        if nrows != ncols:
            raise ValueError("row-block sharding splits x like y: the matrix must be square")
        row = np.asarray(row, dtype=np.int64)
        col = np.asarray(col, dtype=np.int64)
        if bounds is None:
            bounds = partition_rows(np.bincount(row, minlength=nrows), world)
        owner = np.searchsorted(bounds, row, side="right") - 1
        windows = []
        for s in range(world):
            c = col[owner == s]
            windows.append((int(c.min()), int(c.max()) + 1) if c.size else (0, 0))
        return ShardPlan(nrows, ncols, bounds, windows, rank)

    def local_triplets(self, row, col, val):
        """This process's triplets: rows shifted to start at 0, columns
        renumbered into the window (the order of the entries is kept, so each
        row's entries keep their order and their sums the same sequence)."""
        row = np.asarray(row, dtype=np.int64)
        keep = (row >= self.r0) & (row < self.r1)
        val = np.atleast_2d(val)
        return row[keep] - self.r0, np.asarray(col, dtype=np.int64)[keep] - self.c0, val[:, keep]


class TorchComm:
    """Point-to-point exchange and all-gather through torch.distributed.
    Buffers travel as CUDA tensors under NCCL and as host tensors under
    gloo; the backend converts its vectors to and from them."""

    def __init__(self, dist, group=None):
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.on_device = dist.get_backend(group) == "nccl"

    def exchange(self, sends, recvs):
        """sends: {peer: tensor}; recvs: {peer: tensor to fill}.  Posts every
        receive and send, then waits for all."""
        d = self.dist
        ops = [d.P2POp(d.irecv, t, peer, self.group) for peer, t in sorted(recvs.items())]
        ops += [d.P2POp(d.isend, t, peer, self.group) for peer, t in sorted(sends.items())]
        if ops:
            for r in d.batch_isend_irecv(ops):
                r.wait()

    def allgather(self, t):
        """List of world tensors (rank order) of t's shape."""
        import torch
        out = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t, group=self.group)
        return out


class GpuBackend:
    """Local operations of one process on its GPU, through the C ABI:
    vectors are torch CUDA tensors of P planes."""

    def __init__(self, L, flags=0, stream=None):
        import torch
        from . import MPSPMV_COMPLEX
        self.torch = torch
        self.L, self.flags = int(L), int(flags)
        self.P = 2 * self.L if flags & MPSPMV_COMPLEX else self.L
        self.stream = stream

    def create(self, nrows, ncols, row, col, val, val_limbs):
        from . import mpspmv_create_csr
        return mpspmv_create_csr(nrows, ncols, row, col, val, self.L, self.flags, val_limbs=val_limbs,
                                 stream=self.stream)

    def destroy(self, h):
        from . import mpspmv_destroy
        mpspmv_destroy(h)

    def zeros(self, n):
        return self.torch.zeros((self.P, n), dtype=self.torch.float64, device="cuda")

    def asvec(self, a):
        return self.torch.as_tensor(np.ascontiguousarray(a), dtype=self.torch.float64).cuda()

    def host(self, v):
        return v.cpu().numpy()

    def copy_cols(self, dst, doff, src, soff, count):
        if count > 0:
            dst[:, doff:doff + count].copy_(src[:, soff:soff + count])

    def to_comm(self, v, on_device):
        t = v.contiguous()
        return t if on_device else t.cpu()

    def from_comm(self, t):
        return t.cuda()

    def comm_scalar(self, parts, on_device):
        t = self.torch.as_tensor(np.asarray(parts, dtype=np.float64))
        return t.cuda() if on_device else t

    def spmv(self, h, x, y):
        from . import mpspmv_spmv
        mpspmv_spmv(h, x, y, self.stream)

    def dot(self, h, n, u, v):
        from . import mpspmv_dot
        re, im = mpspmv_dot(h, n, u, v, self.stream)
        return np.concatenate([re, im])

    def axpy(self, h, n, alpha, u, v, w):
        from . import mpspmv_axpy
        a = np.asarray(alpha, dtype=np.float64)
        mpspmv_axpy(h, n, a[:self.L], u, v, w, alpha_im=a[self.L:], stream=self.stream)

    def scalar_sum(self, h, parts):
        from . import mpspmv_scalar_sum
        re, im = mpspmv_scalar_sum(h, np.asarray(parts, dtype=np.float64), self.stream)
        return np.concatenate([re, im])

    def scalar_div(self, h, a, b):
        from . import mpspmv_scalar_div
        re, im = mpspmv_scalar_div(h, a, b, self.stream)
        return np.concatenate([re, im])


class ShardedMatrix:
    """One process's block of rows of A, with the x exchange of its plan."""

    def __init__(self, plan, comm, backend, row, col, val, val_limbs=1):
        self.plan, self.comm, self.be = plan, comm, backend
        lr, lc, lv = plan.local_triplets(row, col, val)
        # a process whose rows reference no column still gets a 1-column window
        self.h = backend.create(plan.nlocal, max(plan.wlen, 1), lr, lc, lv, val_limbs)
        self.xwin = backend.zeros(max(plan.wlen, 1))

    def free(self):
        if self.h is not None:
            self.be.destroy(self.h)
            self.h = None

    def gather_window(self, x_local):
        """Fill the column window from this process's block of x and the
        parts of the other blocks it references."""
        p, be, dev = self.plan, self.be, self.comm.on_device if self.comm else True
        woff, boff, cnt = p.own_in_window()
        be.copy_cols(self.xwin, woff, x_local, boff, cnt)
        if self.comm is None or (not p.send and not p.recv):
            return self.xwin
        sends = {}
        for peer, a, b in p.send:
            sl = be.zeros(b - a)
            be.copy_cols(sl, 0, x_local, a - p.r0, b - a)
            sends[peer] = be.to_comm(sl, dev)
        recvs = {peer: be.to_comm(be.zeros(b - a), dev) for peer, a, b in p.recv}
        self.comm.exchange(sends, recvs)
        for peer, a, b in p.recv:
            be.copy_cols(self.xwin, a - p.c0, be.from_comm(recvs[peer]), 0, b - a)
        return self.xwin

    def spmv(self, x_local, y_local):
        """y_local = (A x)[r0:r1]; every process calls it together."""
        self.be.spmv(self.h, self.gather_window(x_local), y_local)

    def dot(self, u, v):
        """Global sum_i conj(u_i) v_i: the blocks' MP partials summed in rank
        order (identical bits on every process)."""
        part = self.be.dot(self.h, self.plan.nlocal, u, v)
        if self.comm is None or self.comm.world == 1:
            return self.be.scalar_sum(self.h, part[None, :])
        dev = self.comm.on_device
        allp = self.comm.allgather(self.be.comm_scalar(part, dev))
        parts = np.stack([t.cpu().numpy() for t in allp])
        return self.be.scalar_sum(self.h, parts)


def _norm(s, L):
    """sqrt of an MP inner product (v, v), components added from the
    smallest as in binary64."""
    t = 0.0
    for l in range(L - 1, -1, -1):
        t += float(s[l])
    if np.isnan(t):
        return t
    return float(np.sqrt(t)) if t > 0 else 0.0


def sharded_cg(A, b, x, rtol, atol=0.0, maxit=1000):
    """Unpreconditioned CG (Hestenes-Stiefel, every vector and scalar in the
    backend's precision, as mpspmv_cg) on the row blocks of every process:
    b, x are this process's blocks (x: initial guess in, last iterate out).
    Stops when ||r_k|| <= rtol ||b|| + atol on the recurrence residual;
    returns (status, iterations, ||b - A x|| / ||b|| recomputed), status 0
    converged, -6 at maxit, -5 on breakdown, the same on every process."""
    be, p = A.be, A.plan
    L, n, h = be.L, p.nlocal, A.h
    zero = np.zeros(2 * L)
    one_neg = zero.copy()
    one_neg[0] = -1.0
    r = be.zeros(max(n, 1))
    q = be.zeros(max(n, 1))
    A.spmv(x, q)
    be.axpy(h, n, one_neg, b, q, r)                # r = b - A x
    pv = be.zeros(max(n, 1))
    be.copy_cols(pv, 0, r, 0, n)
    bnorm = _norm(A.dot(b, b), L)
    tol = rtol * bnorm + atol
    rho = A.dot(r, r)
    status, k = -6, 0
    if _norm(rho, L) <= tol:
        status = 0
    while status != 0 and k < maxit:
        A.spmv(pv, q)
        pq = A.dot(pv, q)
        if pq[0] == 0.0 or not np.isfinite(pq[0]):
            status = -5
            break
        alpha = be.scalar_div(h, rho, pq)
        be.axpy(h, n, alpha, x, pv, x)             # x = x + alpha p
        nalpha = -alpha
        be.axpy(h, n, nalpha, r, q, r)             # r = r - alpha q
        rho1 = A.dot(r, r)
        k += 1
        t = _norm(rho1, L)
        if not np.isfinite(t):
            status = -5
            break
        if t <= tol:
            status = 0
            break
        if rho[0] == 0.0:
            status = -5
            break
        beta = be.scalar_div(h, rho1, rho)
        be.axpy(h, n, beta, r, pv, pv)             # p = r + beta p
        rho = rho1
    A.spmv(x, q)
    be.axpy(h, n, one_neg, b, q, r)
    rn = _norm(A.dot(r, r), L)
    return status, k, (rn / bnorm if bnorm > 0 else rn)
