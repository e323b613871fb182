"""CPU oracle for multiple-precision CSR SpMV / SpMM / CG / BiCGSTAB.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2412_17510_gb300``) and imports nothing from it.

Layers:
  * ``mporacle.c`` (loaded here through ctypes): the paper's algorithms step by
    step in plain binary64 C -- Algorithms 1-5 of Section 2, the QD sloppy add
    and multiply with ThreeSum/ThreeSum2/Renorm, CSR SpMV of Section 3 with the
    complex form of Eq. complex_spmv, and textbook CG / BiCGSTAB (Section 4.2).
  * ``exact``: the exact dyadic value of every SpMV row (big integers), the
    greedy rounding of an exact value to L components, and the componentwise
    error bound used as the acceptance test.
  * ``exact_model``: the exact model of the exact-accumulation arithmetic
    (MPSPMV_EXACT_ACC): the terms an entry contributes and their exact sum cut
    to L components by truncation, for the bit-exact checks of that path.
  * ``mpref``: an independent 600-bit cross-check through mpmath (optional).

Vectors and matrix values are structure-of-limbs float64 arrays of shape
``(P, n)`` with ``P = L`` (real) or ``P = 2L`` (complex: real limbs, then
imaginary limbs).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None
_libc = None

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def _load(counting=False):
    global _lib, _libc
    if counting and _libc is not None:
        return _libc
    if not counting and _lib is not None:
        return _lib
    outs = _build.build()
    lib = ctypes.CDLL(outs[1] if counting else outs[0])
    c_int, c_i64, c_dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sigs = {
        "oracle_two_sum": (None, [c_dbl, c_dbl, _dp, _dp]),
        "oracle_quick_two_sum": (None, [c_dbl, c_dbl, _dp, _dp]),
        "oracle_two_prod": (None, [c_dbl, c_dbl, _dp, _dp]),
        "oracle_three_sum": (None, [_dp, _dp, _dp]),
        "oracle_three_sum2": (None, [_dp, _dp, c_dbl]),
        "oracle_renorm5": (None, [_dp, _dp]),
        "oracle_renorm4": (None, [_dp, _dp]),
        "oracle_mp_add": (None, [c_int, _dp, _dp, _dp]),
        "oracle_mp_mul": (None, [c_int, _dp, _dp, _dp]),
        "oracle_mp_mul_d": (None, [c_int, _dp, c_dbl, _dp]),
        "oracle_mp_div": (None, [c_int, _dp, _dp, _dp]),
        "oracle_coo_to_csr": (c_i64, [c_i64, c_i64, c_i64, _i64p, _i64p, _dp, c_int, c_int, _i64p, _i32p, _dp]),
        "oracle_spmv": (None, [c_int, c_int, c_int, c_i64, _i64p, _i32p, _dp, c_i64, _dp, c_i64, _dp, c_i64]),
        "oracle_spmtv": (None, [c_int, c_int, c_int, c_i64, c_i64, _i64p, _i32p, _dp, c_i64, _dp, c_i64, _dp,
                                c_i64]),
        "oracle_spmv_rows": (None, [c_int, c_int, c_int, c_i64, _i64p, _i64p, _i32p, _dp, c_i64, _dp, c_i64, _dp]),
        "oracle_spmm": (None, [c_int, c_int, c_i64, c_i64, _i64p, _i32p, _dp, c_i64, c_int, _dp, c_i64, c_i64,
                               _dp, c_i64, c_i64]),
        "oracle_cg": (c_int, [c_int, c_i64, _i64p, _i32p, _dp, c_i64, _dp, _dp, c_dbl, c_dbl, c_int,
                              ctypes.POINTER(c_int), _dp]),
        "oracle_bicgstab": (c_int, [c_int, c_int, c_i64, _i64p, _i32p, _dp, c_i64, _dp, _dp, c_dbl, c_dbl, c_int,
                                ctypes.POINTER(c_int), _dp]),
        "oracle_bicg": (c_int, [c_int, c_int, c_i64, _i64p, _i32p, _dp, c_i64, _dp, _dp, c_dbl, c_dbl, c_int,
                                ctypes.POINTER(c_int), _dp]),
        "oracle_cgs": (c_int, [c_int, c_int, c_i64, _i64p, _i32p, _dp, c_i64, _dp, _dp, c_dbl, c_dbl, c_int,
                                ctypes.POINTER(c_int), _dp]),
        "oracle_gpbicg": (c_int, [c_int, c_int, c_i64, _i64p, _i32p, _dp, c_i64, _dp, _dp, c_dbl, c_dbl, c_int,
                                ctypes.POINTER(c_int), _dp]),
        "oracle_dot": (None, [c_int, c_int, c_i64, _dp, _dp, _dp, _dp]),
        "oracle_axpy": (None, [c_int, c_int, c_i64, _dp, _dp, _dp, _dp, _dp]),
        "oracle_ops_get": (ctypes.c_longlong, []),
        "oracle_ops_reset": (None, []),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if counting:
        _libc = lib
    else:
        _lib = lib
    return lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _mp(v, L):
    a = np.zeros(4, dtype=np.float64)
    v = np.atleast_1d(np.asarray(v, dtype=np.float64))
    a[: len(v)] = v
    return a


# --------------------------------------------------------------------------
# Scalar operations
# --------------------------------------------------------------------------
def two_sum(a, b):
    s, e = ctypes.c_double(), ctypes.c_double()
    _load().oracle_two_sum(a, b, ctypes.byref(s), ctypes.byref(e))
    return s.value, e.value


def quick_two_sum(a, b):
    s, e = ctypes.c_double(), ctypes.c_double()
    _load().oracle_quick_two_sum(a, b, ctypes.byref(s), ctypes.byref(e))
    return s.value, e.value


def two_prod(a, b):
    s, e = ctypes.c_double(), ctypes.c_double()
    _load().oracle_two_prod(a, b, ctypes.byref(s), ctypes.byref(e))
    return s.value, e.value


def three_sum(a, b, c):
    x = [ctypes.c_double(a), ctypes.c_double(b), ctypes.c_double(c)]
    _load().oracle_three_sum(*[ctypes.byref(v) for v in x])
    return tuple(v.value for v in x)


def three_sum2(a, b, c):
    x = [ctypes.c_double(a), ctypes.c_double(b)]
    _load().oracle_three_sum2(ctypes.byref(x[0]), ctypes.byref(x[1]), c)
    return tuple(v.value for v in x)


def renorm5(c):
    c = _mp(c, 5) if len(c) <= 4 else np.asarray(c, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    r = np.zeros(4)
    _load().oracle_renorm5(_d(c), _d(r))
    return r


def renorm4(c):
    c = _f64(c)
    r = np.zeros(3)
    _load().oracle_renorm4(_d(c), _d(r))
    return r


def _binop(name, L, a, b, counting):
    lib = _load(counting)
    aa, bb, r = _mp(a, L), _mp(b, L), np.zeros(4)
    getattr(lib, name)(L, _d(aa), _d(bb), _d(r))
    return r[:L].copy()


def mp_add(L, a, b, counting=False):
    return _binop("oracle_mp_add", L, a, b, counting)


def mp_mul(L, a, b, counting=False):
    return _binop("oracle_mp_mul", L, a, b, counting)


def mp_div(L, a, b, counting=False):
    return _binop("oracle_mp_div", L, a, b, counting)


def mp_mul_d(L, a, d, counting=False):
    lib = _load(counting)
    aa, r = _mp(a, L), np.zeros(4)
    lib.oracle_mp_mul_d(L, _d(aa), float(d), _d(r))
    return r[:L].copy()


def ops_reset():
    _load(True).oracle_ops_reset()


def ops_get():
    return int(_load(True).oracle_ops_get())


# --------------------------------------------------------------------------
# Sparse operations
# --------------------------------------------------------------------------
class CSR:
    """Oracle-side CSR: indptr (int64, n+1), indices (int32), data (P, nnz)."""

    def __init__(self, nrows, ncols, indptr, indices, data, L, cplx):
        self.nrows, self.ncols = int(nrows), int(ncols)
        self.indptr = np.ascontiguousarray(indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(indices, dtype=np.int32)
        self.data = _f64(data)
        self.L, self.cplx = int(L), bool(cplx)

    @property
    def nnz(self):
        return int(self.indptr[-1])

    @property
    def P(self):
        return 2 * self.L if self.cplx else self.L

    def row_lengths(self):
        return np.diff(self.indptr)


def coo_to_csr(nrows, ncols, row, col, val, L, cplx=False):
    """Section 3: COO/MTX triplets -> CSR (sorted by (row, col); duplicates
    summed in the working precision).  ``val`` has shape (P, nnz)."""
    row = np.ascontiguousarray(row, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int64)
    val = _f64(val)
    nnz = row.shape[0]
    P = 2 * L if cplx else L
    assert val.shape == (P, nnz)
    indptr = np.zeros(nrows + 1, dtype=np.int64)
    indices = np.zeros(max(nnz, 1), dtype=np.int32)
    data = np.zeros((P, max(nnz, 1)), dtype=np.float64)
    m = _load().oracle_coo_to_csr(nrows, ncols, nnz, row.ctypes.data_as(_i64p), col.ctypes.data_as(_i64p),
                                  _d(val), L, int(cplx), indptr.ctypes.data_as(_i64p),
                                  indices.ctypes.data_as(_i32p), _d(data))
    if m < 0:
        raise ValueError("index out of range")
    # data planes were written with plane stride nnz; keep the first m entries
    data = data[:, :m] if nnz > 0 else np.zeros((P, 0))
    return CSR(nrows, ncols, indptr, indices[:m], data, L, cplx)


def spmv(A, x, mixed=False, counting=False):
    """y = A x in the working precision; x has shape (P, ncols)."""
    lib = _load(counting)
    x = _f64(x)
    y = np.zeros((A.P, A.nrows))
    lib.oracle_spmv(A.L, int(A.cplx), int(mixed), A.nrows, A.indptr.ctypes.data_as(_i64p),
                    A.indices.ctypes.data_as(_i32p), _d(A.data), A.data.shape[1], _d(x), x.shape[1], _d(y), A.nrows)
    return y


def spmtv(A, x, mixed=False):
    """y = A^T x (transpose, no conjugation) in the working precision, by the
    row-oriented scatter; x has shape (P, nrows), y (P, ncols)."""
    x = _f64(x)
    y = np.zeros((A.P, A.ncols))
    _load().oracle_spmtv(A.L, int(A.cplx), int(mixed), A.nrows, A.ncols, A.indptr.ctypes.data_as(_i64p),
                         A.indices.ctypes.data_as(_i32p), _d(A.data), A.data.shape[1], _d(x), x.shape[1], _d(y),
                         A.ncols)
    return y


def spmv_rows(A, x, rows, mixed=False):
    """Rows ``rows`` of A x only; result shape (P, len(rows))."""
    x = _f64(x)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    y = np.zeros((A.P, len(rows)))
    _load().oracle_spmv_rows(A.L, int(A.cplx), int(mixed), len(rows), rows.ctypes.data_as(_i64p),
                             A.indptr.ctypes.data_as(_i64p), A.indices.ctypes.data_as(_i32p), _d(A.data),
                             A.data.shape[1], _d(x), x.shape[1], _d(y))
    return y


def spmm(A, X):
    """Y = A X for X of shape (P, ncols, k) (row-major, right-hand sides
    contiguous); returns (P, nrows, k)."""
    X = _f64(X)
    P, nc, k = X.shape
    Y = np.zeros((P, A.nrows, k))
    _load().oracle_spmm(A.L, int(A.cplx), A.nrows, A.ncols, A.indptr.ctypes.data_as(_i64p),
                        A.indices.ctypes.data_as(_i32p), _d(A.data), A.data.shape[1], k, _d(X), k, nc * k,
                        _d(Y), k, A.nrows * k)
    return Y


def dot(L, u, v, cplx=False):
    u, v = _f64(u), _f64(v)
    dr, di = np.zeros(4), np.zeros(4)
    _load().oracle_dot(L, int(cplx), u.shape[1], _d(u), _d(v), _d(dr), _d(di))
    return dr[:L].copy(), di[:L].copy()


def axpy(L, alpha_re, u, v, alpha_im=None, cplx=False):
    """w = u + alpha v."""
    u, v = _f64(u), _f64(v)
    w = np.zeros_like(u)
    ar, ai = _mp(alpha_re, L), _mp(alpha_im if alpha_im is not None else 0.0, L)
    _load().oracle_axpy(L, int(cplx), u.shape[1], _d(ar), _d(ai), _d(u), _d(v), _d(w))
    return w


def cg(A, b, rtol, atol=0.0, maxit=1000, x0=None):
    """Returns (status, x, iters, relres); status 0 = converged."""
    assert not A.cplx
    b = _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it, rr = ctypes.c_int(), ctypes.c_double()
    st = _load().oracle_cg(A.L, A.nrows, A.indptr.ctypes.data_as(_i64p), A.indices.ctypes.data_as(_i32p),
                           _d(A.data), A.data.shape[1], _d(b), _d(x), rtol, atol, maxit, ctypes.byref(it),
                           ctypes.byref(rr))
    return st, x, it.value, rr.value


def bicgstab(A, b, rtol, atol=0.0, maxit=1000, x0=None):
    b = _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it, rr = ctypes.c_int(), ctypes.c_double()
    st = _load().oracle_bicgstab(A.L, int(A.cplx), A.nrows, A.indptr.ctypes.data_as(_i64p),
                                 A.indices.ctypes.data_as(_i32p), _d(A.data), A.data.shape[1], _d(b), _d(x), rtol,
                                 atol, maxit, ctypes.byref(it), ctypes.byref(rr))
    return st, x, it.value, rr.value


def _krylov(name, A, b, rtol, atol, maxit, x0):
    b = _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it, rr = ctypes.c_int(), ctypes.c_double()
    st = getattr(_load(), name)(A.L, int(A.cplx), A.nrows, A.indptr.ctypes.data_as(_i64p),
                                A.indices.ctypes.data_as(_i32p), _d(A.data), A.data.shape[1], _d(b), _d(x), rtol,
                                atol, maxit, ctypes.byref(it), ctypes.byref(rr))
    return st, x, it.value, rr.value


def bicg(A, b, rtol, atol=0.0, maxit=1000, x0=None):
    """BiCG (shadow products with A^H); returns (status, x, iters, relres)."""
    return _krylov("oracle_bicg", A, b, rtol, atol, maxit, x0)


def cgs(A, b, rtol, atol=0.0, maxit=1000, x0=None):
    """CGS; returns (status, x, iters, relres)."""
    return _krylov("oracle_cgs", A, b, rtol, atol, maxit, x0)


def gpbicg(A, b, rtol, atol=0.0, maxit=1000, x0=None):
    """GPBiCG; returns (status, x, iters, relres)."""
    return _krylov("oracle_gpbicg", A, b, rtol, atol, maxit, x0)
