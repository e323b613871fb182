"""Python binding of ``libmpspmv.so`` (C ABI in ``include/mpspmv.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names; device arrays are passed as torch CUDA
tensors (or raw integer addresses), host arrays as numpy arrays, streams as
``torch.cuda.Stream`` objects (or raw handles).  A non-zero status raises
``MpspmvError``.  Importing this package fails loudly when the compiled
library is missing: there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmpspmv.so")

MPSPMV_OK = 0
MPSPMV_EINVAL = -1
MPSPMV_ENOMEM = -2
MPSPMV_ECUDA = -3
MPSPMV_ENOTSUP = -4
MPSPMV_EBREAKDOWN = -5
MPSPMV_ENOCONV = -6
MPSPMV_ETIMEOUT = -7

MPSPMV_D, MPSPMV_DD, MPSPMV_TD, MPSPMV_QD = 1, 2, 3, 4
MPSPMV_COMPLEX, MPSPMV_MIXED, MPSPMV_SYMMETRIC, MPSPMV_ONE_BASED = 1, 2, 4, 8
MPSPMV_BATCH_AUTOTUNE = 1
MPSPMV_EXACT_ACC = 16
MPSPMV_TRANSPOSE = 32

PREC = {"d": 1, "dd": 2, "td": 3, "qd": 4}


class MpspmvError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, strerror(status), status))


class mpspmv_info(ctypes.Structure):
    _fields_ = [("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("max_row_nnz", ctypes.c_int64), ("nchunks", ctypes.c_int64), ("nsplit_rows", ctypes.c_int64),
                ("prec", ctypes.c_int32), ("planes", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("device_bytes", ctypes.c_int64), ("nlong_rows", ctypes.c_int64),
                ("value_planes", ctypes.c_int64), ("sell_slots", ctypes.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libmpspmv.so is not built (run __graft_entry__.build() or "
                          "python paper_2412_17510_gb300/build.py)")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    sigs = {
        "mpspmv_create_csr": [ctypes.POINTER(vp), i64, i64, i64, vp, vp, vp, c_int, c_int, ctypes.c_uint, vp],
        "mpspmv_destroy": [vp],
        "mpspmv_get_info": [vp, ctypes.POINTER(mpspmv_info)],
        "mpspmv_spmv": [vp, vp, vp, vp],
        "mpspmv_spmtv": [vp, vp, vp, vp],
        "mpspmv_spmv_host": [vp, vp, vp, vp],
        "mpspmv_spmv_host_async": [vp, vp, vp, vp],
        "mpspmv_spmm": [vp, c_int, vp, i64, vp, i64, vp],
        "mpspmv_probe_fp64": [c_int, c_int, ctypes.POINTER(ctypes.c_double), vp],
        "mpspmv_cg": [vp, vp, vp, ctypes.c_double, ctypes.c_double, c_int, ctypes.POINTER(c_int),
                      ctypes.POINTER(ctypes.c_double), vp],
        "mpspmv_bicgstab": [vp, vp, vp, ctypes.c_double, ctypes.c_double, c_int, ctypes.POINTER(c_int),
                            ctypes.POINTER(ctypes.c_double), vp],
        "mpspmv_dot": [vp, i64, vp, vp, vp, vp],
        "mpspmv_axpy": [vp, i64, vp, vp, vp, vp, vp],
        "mpspmv_scalar_sum": [vp, c_int, vp, vp, vp],
        "mpspmv_scalar_div": [vp, vp, vp, vp, vp],
        "mpspmv_bicg": [vp, vp, vp, ctypes.c_double, ctypes.c_double, c_int, ctypes.POINTER(c_int),
                        ctypes.POINTER(ctypes.c_double), vp],
        "mpspmv_cgs": [vp, vp, vp, ctypes.c_double, ctypes.c_double, c_int, ctypes.POINTER(c_int),
                       ctypes.POINTER(ctypes.c_double), vp],
        "mpspmv_gpbicg": [vp, vp, vp, ctypes.c_double, ctypes.c_double, c_int, ctypes.POINTER(c_int),
                          ctypes.POINTER(ctypes.c_double), vp],
        "mpspmv_spmv_csr_noalloc": [c_int, ctypes.c_uint, i64, i64, i64, vp, vp, vp, vp, vp, vp],
        "mpspmv_batch_create": [vp, vp, c_int, ctypes.c_uint, ctypes.POINTER(vp), vp],
        "mpspmv_batch_destroy": [vp],
        "mpspmv_batch_get_plan": [vp, vp, vp],
        "mpspmv_batch_spmm": [vp, vp, vp, vp, vp, vp],
        "mpspmv_batch_cg": [vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, c_int, vp, vp, vp, vp],
        "mpspmv_ladder_solve": [vp, c_int, vp, vp, ctypes.c_double, ctypes.c_double, c_int, vp, vp, vp, vp],
        "mpspmv_cg_history": [vp, vp, c_int, vp, vp],
        "mpspmv_features": [vp, vp, vp, vp],
        "mpspmv_mlp_forward": [vp, c_int, vp, c_int, vp, vp],
        "mpspmv_mlp_grad": [vp, c_int, vp, vp, c_int, vp, vp, vp],
        "mpspmv_mlp_train": [vp, c_int, vp, vp, c_int, c_int, c_int, ctypes.c_float, vp, vp],
        "mpspmv_mlp_standardize": [vp, c_int, vp, vp, vp, vp],
        "mpspmv_mlp_fold": [vp, c_int, vp, vp, vp],
        "mpspmv_select_precision": [vp, vp, c_int, vp, vp, vp, vp],
        "mpspmv_solve_auto": [vp, vp, c_int, vp, vp, ctypes.c_double, ctypes.c_double, c_int, vp, vp, vp, vp, vp],
    }
    for name, args in sigs.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = c_int
    lib.mpspmv_mlp_param_count.argtypes = [c_int]
    lib.mpspmv_mlp_param_count.restype = i64
    lib.mpspmv_strerror.argtypes = [c_int]
    lib.mpspmv_strerror.restype = ctypes.c_char_p
    return lib


_lib = _load()


def _ptr(a):
    """Address of a torch tensor / numpy array / integer."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    raise TypeError("cannot take the address of %r" % type(a))


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(st, where):
    if st != MPSPMV_OK:
        raise MpspmvError(st, where)


def strerror(status):
    return _lib.mpspmv_strerror(status).decode()


def mpspmv_create_csr(nrows, ncols, row, col, val, prec, flags=0, val_limbs=None, stream=None):
    """Create a handle from host COO triplets.  ``val`` is a float64 array of
    shape (val_limbs * V, nnz), V = 2 for complex.  Returns the handle."""
    row = np.ascontiguousarray(row, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int64)
    val = np.ascontiguousarray(np.atleast_2d(val), dtype=np.float64)
    nnz = row.shape[0]
    V = 2 if flags & MPSPMV_COMPLEX else 1
    if val_limbs is None:
        val_limbs = val.shape[0] // V
    if col.shape[0] != nnz or val.shape != (val_limbs * V, nnz):
        raise ValueError("triplet arrays disagree in length or value planes")
    h = ctypes.c_void_p()
    st = _lib.mpspmv_create_csr(ctypes.byref(h), nrows, ncols, nnz, row.ctypes.data, col.ctypes.data,
                                val.ctypes.data, val_limbs, prec, flags, _stream(stream))
    _check(st, "mpspmv_create_csr")
    return h


def mpspmv_destroy(h):
    _check(_lib.mpspmv_destroy(h), "mpspmv_destroy")


def mpspmv_get_info(h):
    info = mpspmv_info()
    _check(_lib.mpspmv_get_info(h, ctypes.byref(info)), "mpspmv_get_info")
    return {k: getattr(info, k) for k, _ in mpspmv_info._fields_}


def mpspmv_spmv(h, x, y, stream=None):
    _check(_lib.mpspmv_spmv(h, _ptr(x), _ptr(y), _stream(stream)), "mpspmv_spmv")


def mpspmv_spmtv(h, x, y, stream=None):
    """y = A^T x (handle created with MPSPMV_TRANSPOSE)."""
    _check(_lib.mpspmv_spmtv(h, _ptr(x), _ptr(y), _stream(stream)), "mpspmv_spmtv")


def mpspmv_spmv_host(h, x_host, y_host, stream=None):
    _check(_lib.mpspmv_spmv_host(h, _ptr(x_host), _ptr(y_host), _stream(stream)), "mpspmv_spmv_host")


def mpspmv_spmv_host_async(h, x_host, y_host, stream=None):
    """Enqueue x -> device, y = A x, y -> host on ``stream`` (pinned host
    buffers, valid until the stream completes)."""
    _check(_lib.mpspmv_spmv_host_async(h, _ptr(x_host), _ptr(y_host), _stream(stream)), "mpspmv_spmv_host_async")


def mpspmv_spmm(h, k, X, ldx, Y, ldy, stream=None):
    _check(_lib.mpspmv_spmm(h, k, _ptr(X), ldx, _ptr(Y), ldy, _stream(stream)), "mpspmv_spmm")


def _solve(fn, name, h, b, x, rtol, atol, maxit, stream, raise_on_noconv):
    it, rr = ctypes.c_int(), ctypes.c_double()
    st = fn(h, _ptr(b), _ptr(x), rtol, atol, maxit, ctypes.byref(it), ctypes.byref(rr), _stream(stream))
    if st not in (MPSPMV_OK, MPSPMV_ENOCONV) or (st == MPSPMV_ENOCONV and raise_on_noconv):
        raise MpspmvError(st, name)
    return st, it.value, rr.value


def mpspmv_cg(h, b, x, rtol, atol=0.0, maxit=1000, stream=None, raise_on_noconv=False):
    """CG in place on x.  Returns (status, iterations, true relative residual)."""
    return _solve(_lib.mpspmv_cg, "mpspmv_cg", h, b, x, rtol, atol, maxit, stream, raise_on_noconv)


def mpspmv_bicgstab(h, b, x, rtol, atol=0.0, maxit=1000, stream=None, raise_on_noconv=False):
    """BiCGSTAB in place on x.  Returns (status, iterations, true relative residual)."""
    return _solve(_lib.mpspmv_bicgstab, "mpspmv_bicgstab", h, b, x, rtol, atol, maxit, stream, raise_on_noconv)


def mpspmv_bicg(h, b, x, rtol, atol=0.0, maxit=1000, stream=None, raise_on_noconv=False):
    """BiCG in place on x (handle created with MPSPMV_TRANSPOSE).  Returns
    (status, iterations, true relative residual)."""
    return _solve(_lib.mpspmv_bicg, "mpspmv_bicg", h, b, x, rtol, atol, maxit, stream, raise_on_noconv)


def mpspmv_cgs(h, b, x, rtol, atol=0.0, maxit=1000, stream=None, raise_on_noconv=False):
    """CGS in place on x.  Returns (status, iterations, true relative residual)."""
    return _solve(_lib.mpspmv_cgs, "mpspmv_cgs", h, b, x, rtol, atol, maxit, stream, raise_on_noconv)


def mpspmv_gpbicg(h, b, x, rtol, atol=0.0, maxit=1000, stream=None, raise_on_noconv=False):
    """GPBiCG in place on x.  Returns (status, iterations, true relative residual)."""
    return _solve(_lib.mpspmv_gpbicg, "mpspmv_gpbicg", h, b, x, rtol, atol, maxit, stream, raise_on_noconv)


def mpspmv_dot(h, n, u, v, stream=None):
    """sum_i conj(u_i) v_i of device vectors (P planes of n) in the handle's
    precision and arithmetic; returns (re, im) as two arrays of L components."""
    L = mpspmv_get_info(h)["prec"]
    out = np.zeros(2 * L)
    _check(_lib.mpspmv_dot(h, n, _ptr(u), _ptr(v), out.ctypes.data, _stream(stream)), "mpspmv_dot")
    return out[:L].copy(), out[L:].copy()


def mpspmv_axpy(h, n, alpha_re, u, v, w, alpha_im=None, stream=None):
    """w = u + alpha v on device vectors; alpha_re / alpha_im are scalars or
    arrays of up to L components."""
    L = mpspmv_get_info(h)["prec"]
    a = np.zeros(2 * L)
    ar = np.atleast_1d(np.asarray(alpha_re, dtype=np.float64))
    a[:ar.size] = ar
    if alpha_im is not None:
        ai = np.atleast_1d(np.asarray(alpha_im, dtype=np.float64))
        a[L:L + ai.size] = ai
    _check(_lib.mpspmv_axpy(h, n, a.ctypes.data, _ptr(u), _ptr(v), _ptr(w), _stream(stream)), "mpspmv_axpy")


def mpspmv_scalar_sum(h, parts, stream=None):
    """Sum of MP scalars in order; ``parts`` is (count, 2L) (each row a
    scalar in mpspmv_dot's layout).  Returns (re, im) as two arrays of L
    components."""
    L = mpspmv_get_info(h)["prec"]
    p = np.ascontiguousarray(np.atleast_2d(parts), dtype=np.float64)
    if p.shape[1] != 2 * L:
        raise ValueError("parts must have 2L columns")
    out = np.zeros(2 * L)
    _check(_lib.mpspmv_scalar_sum(h, p.shape[0], p.ctypes.data, out.ctypes.data, _stream(stream)),
           "mpspmv_scalar_sum")
    return out[:L].copy(), out[L:].copy()


def mpspmv_scalar_div(h, a, b, stream=None):
    """a / b for MP scalars of 2L components each; returns (re, im)."""
    L = mpspmv_get_info(h)["prec"]
    aa = np.ascontiguousarray(a, dtype=np.float64).reshape(2 * L)
    bb = np.ascontiguousarray(b, dtype=np.float64).reshape(2 * L)
    out = np.zeros(2 * L)
    _check(_lib.mpspmv_scalar_div(h, aa.ctypes.data, bb.ctypes.data, out.ctypes.data, _stream(stream)),
           "mpspmv_scalar_div")
    return out[:L].copy(), out[L:].copy()


def mpspmv_spmv_csr_noalloc(prec, flags, nrows, ncols, nnz, indptr, indices, vals, x, y, stream=None):
    """y = A x from caller-owned device CSR arrays, with no device allocation
    (scratch is a fixed array inside the library)."""
    _check(_lib.mpspmv_spmv_csr_noalloc(prec, flags, nrows, ncols, nnz, _ptr(indptr), _ptr(indices), _ptr(vals),
                                        _ptr(x), _ptr(y), _stream(stream)), "mpspmv_spmv_csr_noalloc")


def _ptr_array(items):
    arr = (ctypes.c_void_p * len(items))(*[_ptr(a) for a in items])
    return arr


def mpspmv_batch_create(mats, ks, flags=0, stream=None):
    """Batch of handles ``mats`` with ``ks[i]`` right-hand sides each."""
    hs = (ctypes.c_void_p * len(mats))(*[m.value if isinstance(m, ctypes.c_void_p) else m for m in mats])
    kk = np.ascontiguousarray(ks, dtype=np.int32)
    b = ctypes.c_void_p()
    _check(_lib.mpspmv_batch_create(hs, kk.ctypes.data, len(mats), flags, ctypes.byref(b), _stream(stream)),
           "mpspmv_batch_create")
    return b


def mpspmv_batch_destroy(b):
    _check(_lib.mpspmv_batch_destroy(b), "mpspmv_batch_destroy")


def mpspmv_batch_get_plan(b, count):
    K = np.zeros(count, dtype=np.int32)
    w = np.zeros(count, dtype=np.int32)
    _check(_lib.mpspmv_batch_get_plan(b, K.ctypes.data, w.ctypes.data), "mpspmv_batch_get_plan")
    return K, w


def mpspmv_batch_spmm(b, X, Y, ldx=None, ldy=None, stream=None):
    """X, Y: lists of device arrays (one per matrix)."""
    lx = None if ldx is None else np.ascontiguousarray(ldx, dtype=np.int64)
    ly = None if ldy is None else np.ascontiguousarray(ldy, dtype=np.int64)
    _check(_lib.mpspmv_batch_spmm(b, _ptr_array(X), None if lx is None else lx.ctypes.data, _ptr_array(Y),
                                  None if ly is None else ly.ctypes.data, _stream(stream)), "mpspmv_batch_spmm")


def mpspmv_batch_cg(b, B, X, nsys, rtol, atol=0.0, maxit=1000, stream=None):
    """Batched CG in place on X.  Returns (status, iters[nsys], relres[nsys],
    per-system status[nsys])."""
    it = np.zeros(nsys, dtype=np.int32)
    rr = np.zeros(nsys)
    ss = np.zeros(nsys, dtype=np.int32)
    st = _lib.mpspmv_batch_cg(b, _ptr_array(B), None, _ptr_array(X), None, rtol, atol, maxit, it.ctypes.data,
                              rr.ctypes.data, ss.ctypes.data, _stream(stream))
    if st not in (MPSPMV_OK, MPSPMV_ENOCONV, MPSPMV_EBREAKDOWN):
        raise MpspmvError(st, "mpspmv_batch_cg")
    return st, it, rr, ss


def _handles4(hs):
    return (ctypes.c_void_p * 4)(*[(h.value if isinstance(h, ctypes.c_void_p) else h) if h is not None else None
                                   for h in hs])


def mpspmv_ladder_solve(hs, start_L, b, x, rtol, atol=0.0, maxit=1000, stream=None):
    """Returns (status, final level, iterations per level, relres)."""
    fl = ctypes.c_int()
    it = (ctypes.c_int * 4)()
    rr = ctypes.c_double()
    st = _lib.mpspmv_ladder_solve(_handles4(hs), start_L, _ptr(b), _ptr(x), rtol, atol, maxit, ctypes.byref(fl),
                                  it, ctypes.byref(rr), _stream(stream))
    if st not in (MPSPMV_OK, MPSPMV_ENOCONV):
        raise MpspmvError(st, "mpspmv_ladder_solve")
    return st, fl.value, list(it), rr.value


def mpspmv_cg_history(h, b, k=8, stream=None):
    out = np.zeros(k)
    _check(_lib.mpspmv_cg_history(h, _ptr(b), k, out.ctypes.data, _stream(stream)), "mpspmv_cg_history")
    return out


def mpspmv_features(h, cg_hist=None, stream=None):
    f = np.zeros(32, dtype=np.float32)
    hh = None if cg_hist is None else np.ascontiguousarray(cg_hist, dtype=np.float64)
    _check(_lib.mpspmv_features(h, None if hh is None else hh.ctypes.data, f.ctypes.data, _stream(stream)),
           "mpspmv_features")
    return f


def mpspmv_mlp_param_count(C):
    return int(_lib.mpspmv_mlp_param_count(C))


def mpspmv_mlp_forward(params, C, X, B, logits, stream=None):
    _check(_lib.mpspmv_mlp_forward(_ptr(params), C, _ptr(X), B, _ptr(logits), _stream(stream)), "mpspmv_mlp_forward")


def mpspmv_mlp_grad(params, C, X, y, B, grads, stream=None):
    loss = ctypes.c_float()
    _check(_lib.mpspmv_mlp_grad(_ptr(params), C, _ptr(X), _ptr(y), B, _ptr(grads), ctypes.byref(loss),
                                _stream(stream)), "mpspmv_mlp_grad")
    return loss.value


def mpspmv_mlp_train(params, C, X, y, n, batch, epochs, lr, stream=None):
    losses = np.zeros(max(epochs, 1), dtype=np.float32)
    _check(_lib.mpspmv_mlp_train(_ptr(params), C, _ptr(X), _ptr(y), n, batch, epochs, ctypes.c_float(lr),
                                 losses.ctypes.data, _stream(stream)), "mpspmv_mlp_train")
    return losses[:epochs]


def mpspmv_mlp_standardize(X, n, mu, sd, Xs, stream=None):
    """Device arrays: mu, sd (32 floats) and Xs = (X - mu) / sd."""
    _check(_lib.mpspmv_mlp_standardize(_ptr(X), n, _ptr(mu), _ptr(sd), _ptr(Xs), _stream(stream)),
           "mpspmv_mlp_standardize")


def mpspmv_mlp_fold(params, C, mu, sd, stream=None):
    """Fold the standardisation (mu, sd: device) into W1, b1 of params in place."""
    _check(_lib.mpspmv_mlp_fold(_ptr(params), C, _ptr(mu), _ptr(sd), _stream(stream)), "mpspmv_mlp_fold")


def mpspmv_select_precision(hs, params, C, b, stream=None):
    p = ctypes.c_int()
    f = np.zeros(32, dtype=np.float32)
    _check(_lib.mpspmv_select_precision(_handles4(hs), _ptr(params), C, _ptr(b), ctypes.byref(p), f.ctypes.data,
                                        _stream(stream)), "mpspmv_select_precision")
    return p.value, f


def mpspmv_solve_auto(hs, params, C, b, x, rtol, atol=0.0, maxit=1000, stream=None):
    """Returns (status, chosen level, final level, iterations per level, relres)."""
    ch, fl = ctypes.c_int(), ctypes.c_int()
    it = (ctypes.c_int * 4)()
    rr = ctypes.c_double()
    st = _lib.mpspmv_solve_auto(_handles4(hs), _ptr(params), C, _ptr(b), _ptr(x), rtol, atol, maxit,
                                ctypes.byref(ch), ctypes.byref(fl), it, ctypes.byref(rr), _stream(stream))
    if st not in (MPSPMV_OK, MPSPMV_ENOCONV):
        raise MpspmvError(st, "mpspmv_solve_auto")
    return st, ch.value, fl.value, list(it), rr.value


def mpspmv_probe_fp64(op, iters=4096, stream=None):
    """Measured binary64 instructions per second (op 0 DFMA, 1 DADD, 2 DMUL)."""
    r = ctypes.c_double()
    _check(_lib.mpspmv_probe_fp64(op, iters, ctypes.byref(r), _stream(stream)), "mpspmv_probe_fp64")
    return r.value


def library():
    """The loaded ctypes library (for symbol checks)."""
    return _lib
