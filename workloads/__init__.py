"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and lays out sparsity structure; it
holds none of the multiple-precision arithmetic.  Both the CUDA path (tests,
benchmark) and the CPU oracle take their inputs from here.

The paper measures on SuiteSparse matrices (Section 4, 631 real and 16
complex square matrices; tub1000 and nd3k for the Krylov runs).  Those files
are not available here, so the generators below stand in for them with
matrices of the same kinds: stencil (banded, uniform rows), power-law rows,
complex-symmetric banded, and SPD diffusion systems.

Every generator returns COO triplets sorted by (row, col) with int64 indices
and the values as binary64 planes ``val`` of shape (V, nnz): V = 1 for a real
binary64 matrix (the P mode promotes it to L components with zero lower
components), V = 2 for a complex binary64 matrix (real plane, imaginary
plane).
"""
import math

import numpy as np


class COO:
    def __init__(self, nrows, ncols, row, col, val, name=""):
        self.nrows, self.ncols = int(nrows), int(ncols)
        self.row = np.ascontiguousarray(row, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int64)
        self.val = np.ascontiguousarray(np.atleast_2d(val), dtype=np.float64)
        self.name = name

    @property
    def nnz(self):
        return int(self.row.shape[0])

    @property
    def cplx(self):
        return self.val.shape[0] == 2

    def promoted(self, L):
        """Value planes for the P mode at L components: (P, nnz) with the
        binary64 value in component 0 and zeros below (real: P = L; complex:
        P = 2L, real components then imaginary components)."""
        V = self.val.shape[0]
        out = np.zeros((V * L, self.nnz))
        for c in range(V):
            out[c * L] = self.val[c]
        return out


# --------------------------------------------------------------------------
# Vectors
# --------------------------------------------------------------------------
def full_limb_vector(n, L, seed=0, cplx=False, rng=None):
    """x_0 ~ U[-1,1]; x_k = U[-1,1] * 2**-53 * |x_{k-1}| for k >= 1 (every
    component random).  Shape (P, n), P = L or 2L."""
    rng = np.random.default_rng(seed) if rng is None else rng
    P = 2 * L if cplx else L
    out = np.empty((P, n))
    for c in range(2 if cplx else 1):
        prev = rng.uniform(-1.0, 1.0, n)
        out[c * L] = prev
        for k in range(1, L):
            prev = rng.uniform(-1.0, 1.0, n) * 2.0 ** -53 * np.abs(prev)
            out[c * L + k] = prev
    return out


def full_limb_values(coo, L, seed=0):
    """Matrix values with every component random: component 0 is the
    matrix's own binary64 value, component k = U[-1,1] * 2**-53 * |component
    k-1| (the rule of full_limb_vector).  Real matrices only; shape (L, nnz),
    drawn in blocks to bound the temporaries."""
    rng = np.random.default_rng(seed)
    out = np.empty((L, coo.nnz))
    out[0] = coo.val[0]
    step = 1 << 24
    for a in range(0, coo.nnz, step):
        b = min(a + step, coo.nnz)
        for k in range(1, L):
            out[k, a:b] = rng.uniform(-1.0, 1.0, b - a) * 2.0 ** -53 * np.abs(out[k - 1, a:b])
    return out


def integer_vector(n, L, lo=-8, hi=8, seed=0, cplx=False):
    """Integer-valued vector in component 0, zeros below."""
    rng = np.random.default_rng(seed)
    P = 2 * L if cplx else L
    out = np.zeros((P, n))
    for c in range(2 if cplx else 1):
        out[c * L] = rng.integers(lo, hi + 1, n).astype(np.float64)
    return out


# --------------------------------------------------------------------------
# Matrices
# --------------------------------------------------------------------------
def laplacian_2d(nx, ny=None):
    """2D 5-point Laplacian, non-periodic, diagonal 4 and off-diagonals -1
    (n = nx*ny; nnz = 5n - 2nx - 2ny)."""
    ny = nx if ny is None else ny
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    rows, cols, vals = [], [], []
    # offsets in increasing column order: -nx, -1, 0, +1, +nx
    for dy, dx, v in ((-1, 0, -1.0), (0, -1, -1.0), (0, 0, 4.0), (0, 1, -1.0), (1, 0, -1.0)):
        ys, xs = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        ok = (ys + dy >= 0) & (ys + dy < ny) & (xs + dx >= 0) & (xs + dx < nx)
        r = idx[ok]
        c = idx[(ys + dy)[ok], (xs + dx)[ok]]
        rows.append(r)
        cols.append(c)
        vals.append(np.full(r.shape, v))
    return _sorted_coo(n, n, rows, cols, vals, "laplace2d_%dx%d" % (nx, ny))


def convection_diffusion_2d(nx, ny=None, c=0.5):
    """2D 5-point convection-diffusion, -Laplace(u) + b . grad(u) with
    centred convection on a unit-spaced grid: diagonal 4, west/south -1 - c,
    east/north -1 + c (|c| < 1 keeps it an M-matrix).  Nonsymmetric band
    matrix (half-bandwidth nx), a stand-in for the nonsymmetric band
    matrices of the product-type Krylov comparison."""
    ny = nx if ny is None else ny
    n = nx * ny
    idx = np.arange(n).reshape(ny, nx)
    rows, cols, vals = [], [], []
    for dy, dx, v in ((-1, 0, -1.0 - c), (0, -1, -1.0 - c), (0, 0, 4.0), (0, 1, -1.0 + c), (1, 0, -1.0 + c)):
        ys, xs = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        ok = (ys + dy >= 0) & (ys + dy < ny) & (xs + dx >= 0) & (xs + dx < nx)
        r = idx[ok]
        cc = idx[(ys + dy)[ok], (xs + dx)[ok]]
        rows.append(r)
        cols.append(cc)
        vals.append(np.full(r.shape, v))
    return _sorted_coo(n, n, rows, cols, vals, "convdiff2d_%dx%d_c%g" % (nx, ny, c))


def _sorted_coo(nr, nc, rows, cols, vals, name):
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    v = np.concatenate(vals, axis=-1)
    order = np.lexsort((c, r))
    return COO(nr, nc, r[order], c[order], np.atleast_2d(v)[:, order], name)


def stencil_27pt(N, seed=0):
    """3D 27-point stencil on an N^3 grid, non-periodic; off-diagonals N(0,1);
    diagonal = (sum of |off-diagonals| in the row) + 1.  Rows come out in
    increasing column order without a sort (offsets enumerated dz, dy, dx)."""
    rng = np.random.default_rng(seed)
    n = N ** 3
    offs = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    z, y, x = z.ravel(), y.ravel(), x.ravel()
    mask = np.empty((n, 27), dtype=bool)
    colm = np.empty((n, 27), dtype=np.int64)
    base = np.arange(n, dtype=np.int64)
    for t, (dz, dy, dx) in enumerate(offs):
        mask[:, t] = ((z + dz >= 0) & (z + dz < N) & (y + dy >= 0) & (y + dy < N) & (x + dx >= 0) & (x + dx < N))
        colm[:, t] = base + dz * N * N + dy * N + dx
    del z, y, x
    vals = rng.standard_normal((n, 27))
    vals[~mask] = 0.0
    vals[:, 13] = np.abs(vals).sum(axis=1) - np.abs(vals[:, 13]) + 1.0
    row = np.broadcast_to(base[:, None], (n, 27))[mask]
    col = colm[mask]
    val = vals[mask]
    return COO(n, n, row, col, val[None, :], "stencil27_%d^3" % N)


def power_law(n, s=1.5, max_len=20000, seed=0):
    """Rows of Zipf(s) length clipped to [1, max_len], uniform random distinct
    columns (duplicates of a draw are removed, so a row can come out slightly
    shorter), values N(0,1)."""
    rng = np.random.default_rng(seed)
    lens = np.minimum(rng.zipf(s, n), max_len).astype(np.int64)
    total = int(lens.sum())
    row = np.repeat(np.arange(n, dtype=np.int64), lens)
    col = rng.integers(0, n, total, dtype=np.int64)
    key = row * n + col
    key.sort()
    keep = np.ones(total, dtype=bool)
    keep[1:] = key[1:] != key[:-1]
    key = key[keep]
    row = key // n
    col = key - row * n
    val = rng.standard_normal(key.shape[0])
    return COO(n, n, row, col, val[None, :], "powerlaw_n%d_s%g" % (n, s))


def complex_sym_banded(n, half_bw=48, fill=0.3, seed=0, shift=None):
    """Complex-symmetric (A = A^T, not Hermitian) banded matrix: each entry of
    the strict upper band is present with probability ``fill`` and mirrored;
    the diagonal is always present; real and imaginary parts N(0,1).  An
    optional complex ``shift`` is added to the diagonal."""
    rng = np.random.default_rng(seed)
    ur, uc = [], []
    for d in range(1, half_bw + 1):
        m = n - d
        keep = rng.random(m) < fill
        i = np.nonzero(keep)[0].astype(np.int64)
        ur.append(i)
        uc.append(i + d)
    ur = np.concatenate(ur)
    uc = np.concatenate(uc)
    nu = ur.shape[0]
    vre = rng.standard_normal(nu)
    vim = rng.standard_normal(nu)
    dre = rng.standard_normal(n)
    dim = rng.standard_normal(n)
    if shift is not None:
        dre = dre + shift.real
        dim = dim + shift.imag
    diag = np.arange(n, dtype=np.int64)
    rows = [ur, uc, diag]
    cols = [uc, ur, diag]
    vals = [np.stack([vre, vim]), np.stack([vre, vim]), np.stack([dre, dim])]
    return _sorted_coo(n, n, rows, cols, vals, "csymband_n%d_bw%d" % (n, half_bw))


def grid_dims(n):
    """Near-cubic nx*ny*nz whose product is closest to n."""
    best = None
    c = round(n ** (1.0 / 3.0))
    for nz in range(max(1, c - 3), c + 4):
        for ny in range(max(1, c - 3), c + 4):
            nx = max(1, round(n / (ny * nz)))
            p = nx * ny * nz
            key = (abs(p - n), max(nx, ny, nz) - min(nx, ny, nz))
            if best is None or key < best[0]:
                best = (key, (nx, ny, nz))
    return best[1]


def diffusion_7pt(nx, ny, nz, kappa_range=(1e-3, 1e3), seed=0):
    """3D 7-point finite-volume diffusion with per-cell coefficient kappa
    log-uniform in ``kappa_range``; face coefficient = harmonic mean of the two
    cells; Dirichlet boundary (boundary faces use the cell's own kappa).  The
    result is symmetric positive definite."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    lk = rng.uniform(math.log(kappa_range[0]), math.log(kappa_range[1]), n)
    kap = np.exp(lk).reshape(nz, ny, nx)
    idx = np.arange(n, dtype=np.int64).reshape(nz, ny, nx)
    diag = np.zeros((nz, ny, nx))
    rows, cols, vals = [], [], []
    for axis, size in ((0, nz), (1, ny), (2, nx)):
        # interior faces between cell i and i+1 along axis
        sl_a = [slice(None)] * 3
        sl_b = [slice(None)] * 3
        sl_a[axis] = slice(0, size - 1)
        sl_b[axis] = slice(1, size)
        ka, kb = kap[tuple(sl_a)], kap[tuple(sl_b)]
        t = 2.0 * ka * kb / (ka + kb)
        ia, ib = idx[tuple(sl_a)].ravel(), idx[tuple(sl_b)].ravel()
        tv = t.ravel()
        rows += [ia, ib]
        cols += [ib, ia]
        vals += [-tv, -tv]
        np.add.at(diag, tuple(sl_a), t)
        np.add.at(diag, tuple(sl_b), t)
        # Dirichlet boundary faces
        for end in (0, size - 1):
            sl = [slice(None)] * 3
            sl[axis] = slice(end, end + 1)
            diag[tuple(sl)] += 2.0 * kap[tuple(sl)]
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    vals = [v[None, :] for v in vals]
    return _sorted_coo(n, n, rows, cols, vals, "diff7_%dx%dx%d" % (nx, ny, nz))


def batch_specs(count=512, n_range=(1000, 200000), k_range=(1, 32), seed=0):
    """Per-matrix (nx, ny, nz, k, seed) for the batched workload: n
    log-uniform in n_range on a near-cubic grid, k uniform in k_range."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]), count))
    ks = rng.integers(k_range[0], k_range[1] + 1, count)
    out = []
    for i in range(count):
        out.append(grid_dims(int(round(ns[i]))) + (int(ks[i]), seed * 100003 + i + 1))
    return out


def integer_matrix(nrows, ncols, density, lo=-8, hi=8, seed=0, cplx=False, dup_frac=0.0):
    """Random integer-valued sparse matrix (values in [lo, hi], never zero),
    optionally with duplicated triplets in random order (for COO tests)."""
    rng = np.random.default_rng(seed)
    m = max(1, int(nrows * ncols * density))
    r = rng.integers(0, nrows, m)
    c = rng.integers(0, ncols, m)
    key = np.unique(r * ncols + c)
    r, c = key // ncols, key % ncols
    V = 2 if cplx else 1
    v = rng.integers(lo, hi, (V, key.shape[0])).astype(np.float64)
    v[v >= 0] += 1.0
    coo = COO(nrows, ncols, r, c, v, "int_%dx%d" % (nrows, ncols))
    if dup_frac > 0:
        nd = int(coo.nnz * dup_frac)
        pick = rng.integers(0, coo.nnz, nd)
        extra = rng.integers(lo, hi, (V, nd)).astype(np.float64)
        r = np.concatenate([coo.row, coo.row[pick]])
        c = np.concatenate([coo.col, coo.col[pick]])
        v = np.concatenate([coo.val, extra], axis=1)
        perm = rng.permutation(r.shape[0])
        coo = COO(nrows, ncols, r[perm], c[perm], v[:, perm], coo.name + "_dup")
    return coo


def random_sparse(nrows, ncols, row_len_max, seed=0, cplx=False, L=1, full_limb=False, empty_frac=0.0):
    """Random sparse matrix with row lengths uniform in [0, row_len_max]
    (some rows empty), N(0,1) values; with ``full_limb`` every component of
    the L-component values is random (returned as (P, nnz) planes)."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, row_len_max + 1, nrows)
    if empty_frac > 0:
        lens[rng.random(nrows) < empty_frac] = 0
    lens = np.minimum(lens, ncols)
    rows, cols = [], []
    for i in range(nrows):
        if lens[i]:
            c = np.sort(rng.choice(ncols, lens[i], replace=False))
            rows.append(np.full(lens[i], i))
            cols.append(c)
    r = np.concatenate(rows) if rows else np.zeros(0, dtype=np.int64)
    c = np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)
    nnz = r.shape[0]
    if full_limb:
        v = full_limb_vector(nnz, L, rng=rng, cplx=cplx)
    else:
        V = 2 if cplx else 1
        v = rng.standard_normal((V, nnz))
    return COO(nrows, ncols, r, c, v, "rand_%dx%d" % (nrows, ncols))


def selector_system(n, log10_cond, seed=0, nnz_range=(8, 24)):
    """SPD system A = D (L L^T + I) D for the precision selector (stored
    exactly symmetric): L unit lower
    triangular with U{nnz_range} off-diagonal entries per row (positions
    uniform in [0, i), values N(0,1)); D = diag(10^t_i) with t_i graded
    linearly over the rows so that cond(A) is about 10^log10_cond (cond(L L^T
    + I) is of order 1e2 for these sizes, cond(D)^2 supplies the rest).
    Returns (COO, b) with b ~ U[-1, 1] in binary64."""
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    lo, hi = nnz_range
    for i in range(1, n):
        m = min(i, int(rng.integers(lo, hi + 1)))
        c = rng.choice(i, m, replace=False)
        rows.append(np.full(m, i))
        cols.append(c)
        vals.append(rng.standard_normal(m))
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(np.ones(n))
    Lm = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    M = (Lm @ Lm.T + sp.identity(n)).tocsr()
    tau = max(0.0, (log10_cond - 2.0) / 2.0)
    d = 10.0 ** (tau * np.arange(n) / max(n - 1, 1))
    A = (sp.diags(d) @ M @ sp.diags(d)).tocsr()
    # the products round a_ij and a_ji differently; averaging the two makes the
    # stored binary64 matrix exactly symmetric (fl(u + v) = fl(v + u))
    A = ((A + A.T) * 0.5).tocoo()
    order = np.lexsort((A.col, A.row))
    coo = COO(n, n, A.row[order], A.col[order], A.data[order][None, :], "selector_n%d_c%g" % (n, log10_cond))
    b = rng.uniform(-1.0, 1.0, n)
    return coo, b
