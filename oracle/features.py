"""Oracle for the selector's 32 matrix features (test infrastructure).

Written from the feature definitions (row statistics, diagonal dominance,
norms, Gershgorin bounds, and the residual history of a few binary64 CG
steps on the system); numpy float64, independent of the CUDA library.
Feature i:
  0 log10 n; 1 log10 nnz; 2..5 row length mean, std (population), min, max;
  6 coefficient of variation; 7 skewness; 8 fraction of empty rows;
  9 bandwidth max|i-j| / n; 10..12 log10 of the min / mean (each ratio capped
  at 1e6) / max (capped at 1e30) of |a_ii| / sum_{j!=i} |a_ij| (1e30 when the
  off-diagonal sum is 0); 13 fraction of rows with |a_ii| >= sum_{j!=i} |a_ij|;
  14..16 log10 of ||A||_1, ||A||_inf, ||A||_F; 17, 18 log10 max / min |a_ii|;
  19 = 17 - 18; 20, 21 Gershgorin min(a_ii - R_i), max(a_ii + R_i) divided by
  ||A||_inf; 22..29 log10 ||r_k|| / ||b|| of binary64 CG with x0 = 0,
  k = 1..8; 30 least-squares slope of 22..29 against k; 31 log10(||A||_F /
  max|a_ii|).  log10 of a non-positive number is -300.
"""
import numpy as np


def _lg(v):
    return np.log10(v) if v > 0 else -300.0


def cg_history(indptr, indices, data, b, k=8):
    """Plain binary64 CG (x0 = 0) residual norms ||r_j|| / ||b||, j = 1..k."""
    n = len(indptr) - 1
    rows = np.repeat(np.arange(n), np.diff(indptr))

    def matvec(v):
        return np.bincount(rows, weights=data * v[indices], minlength=n)

    x = np.zeros(n)
    r = b.copy()
    p = r.copy()
    rho = r @ r
    bn = np.sqrt(b @ b)
    out = []
    for _ in range(k):
        q = matvec(p)
        alpha = rho / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rho1 = r @ r
        out.append(np.sqrt(rho1) / bn)
        p = r + (rho1 / rho) * p
        rho = rho1
    return np.array(out)


def features(A, b):
    """A: oracle.CSR (leading components used), b: binary64 right-hand side."""
    n = A.nrows
    ip, ind = A.indptr, A.indices.astype(np.int64)
    v = A.data[0]
    lens = np.diff(ip).astype(np.float64)
    rows = np.repeat(np.arange(n), np.diff(ip))
    isdiag = ind == rows
    diag = np.bincount(rows[isdiag], weights=v[isdiag], minlength=n)
    off = np.bincount(rows[~isdiag], weights=np.abs(v[~isdiag]), minlength=n)
    rowabs = off + np.abs(diag)
    fro2 = float(np.sum(v * v))
    colsum = np.bincount(ind, weights=np.abs(v), minlength=A.ncols)
    bw = float(np.max(np.abs(ind - rows))) if len(ind) else 0.0
    ad = np.abs(diag)
    dom = np.where(off > 0, ad / np.where(off > 0, off, 1.0), 1e30)
    mean = lens.mean()
    sd = lens.std()
    m3 = np.mean((lens - mean) ** 3)
    f = np.zeros(32)
    f[0] = _lg(n)
    f[1] = _lg(A.nnz)
    f[2], f[3], f[4], f[5] = mean, sd, lens.min(), lens.max()
    f[6] = sd / mean if mean > 0 else 0
    f[7] = m3 / sd ** 3 if sd > 0 else 0
    f[8] = np.mean(lens == 0)
    f[9] = bw / n
    f[10] = _lg(dom.min())
    f[11] = _lg(np.mean(np.minimum(dom, 1e6)))
    f[12] = _lg(np.max(np.minimum(dom, 1e30)))
    f[13] = np.mean(ad >= off)
    ninf = rowabs.max()
    f[14] = _lg(colsum.max())
    f[15] = _lg(ninf)
    f[16] = _lg(np.sqrt(fro2))
    f[17] = _lg(ad.max())
    f[18] = _lg(ad.min())
    f[19] = f[17] - f[18]
    f[20] = np.min(diag - off) / ninf if ninf > 0 else 0
    f[21] = np.max(diag + off) / ninf if ninf > 0 else 0
    h = cg_history(ip, ind, v, np.asarray(b, dtype=np.float64), 8)
    f[22:30] = [_lg(t) for t in h]
    ks = np.arange(1, 9)
    f[30] = np.polyfit(ks, f[22:30], 1)[0]
    f[31] = _lg(np.sqrt(fro2)) - _lg(ad.max())
    return f
