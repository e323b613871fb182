"""600-bit cross-check of SpMV rows and scalar operations through mpmath
(test infrastructure; optional -- callers skip when mpmath is absent).

This is independent of ``exact`` (big-integer arithmetic) and of the binary64
oracle: values are converted to mpmath numbers at 600 bits and the row sums
are evaluated there, so a mistake in the exact module would show up as a
disagreement between the two references.
"""
import mpmath

PREC = 600


def mpf_of(limbs):
    with mpmath.workprec(PREC):
        s = mpmath.mpf(0)
        for v in limbs:
            s += mpmath.mpf(float(v))
        return s


def rows(A, x, rows):
    """Return lists (re, im) of mpmath values of rows of A x at 600 bits."""
    L, cplx = A.L, A.cplx
    out_re, out_im = [], []
    with mpmath.workprec(PREC):
        for i in rows:
            sr = mpmath.mpf(0)
            si = mpmath.mpf(0)
            for k in range(A.indptr[i], A.indptr[i + 1]):
                j = int(A.indices[k])
                ar = mpf_of(A.data[:L, k])
                xr = mpf_of(x[:L, j])
                if cplx:
                    ai = mpf_of(A.data[L:, k])
                    xi = mpf_of(x[L:, j])
                    sr += ar * xr - ai * xi
                    si += ar * xi + ai * xr
                else:
                    sr += ar * xr
            out_re.append(sr)
            out_im.append(si)
    return out_re, out_im


def rel_err(limbs, ref):
    """|sum(limbs) - ref| / |ref| at 600 bits (absolute error if ref == 0)."""
    with mpmath.workprec(PREC):
        d = abs(mpf_of(limbs) - ref)
        return float(d / abs(ref)) if ref != 0 else float(d)
