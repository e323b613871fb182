"""Matrix Market files <-> the triplets ``mpspmv_create_csr`` takes and the
structure-of-limbs vectors the products return.

Host-side input plumbing, no arithmetic of the method.  The paper's test
matrices are Matrix Market files (Section 4.1: SuiteSparse), and
``mpspmv_create_csr`` takes COO triplets (Section 3).  ``read_mtx`` parses the
``matrix coordinate`` format with field ``real``, ``integer``, ``complex`` or
``pattern`` and symmetry ``general``, ``symmetric``, ``skew-symmetric`` or
``hermitian``.  The stored triangle of the last three is expanded into both
triangles (negated for skew-symmetric, conjugated for Hermitian), indices
become 0-based, and the result is ready for
``mpspmv_create_csr(nrows, ncols, row, col, val, L, flags, val_limbs=1)``:
``val`` has one plane for real data and two (real, imaginary) for complex
data, and ``flags`` carries ``MPSPMV_COMPLEX`` for complex data.  Duplicate
entries are kept; the library sums them.

``write_mtx`` writes triplets back as a coordinate file (one triangle for the
symmetric forms), and ``write_vector`` / ``read_vector`` store a DD/TD/QD
vector as an ``array`` file with one column per component; every value is
written with enough digits to read back bit for bit.
"""
import io

import numpy as np

from . import MPSPMV_COMPLEX

_FIELDS = ("real", "integer", "complex", "pattern")
_SYMMETRIES = ("general", "symmetric", "skew-symmetric", "hermitian")


class MtxMatrix:
    """Triplets of one Matrix Market file (0-based, both triangles)."""

    def __init__(self, nrows, ncols, row, col, val, field, symmetry):
        self.nrows, self.ncols = nrows, ncols
        self.row, self.col, self.val = row, col, val
        self.field, self.symmetry = field, symmetry

    @property
    def nnz(self):
        return int(self.row.shape[0])

    @property
    def flags(self):
        return MPSPMV_COMPLEX if self.field == "complex" else 0

    def args(self):
        """(nrows, ncols, row, col, val, flags) for mpspmv_create_csr."""
        return self.nrows, self.ncols, self.row, self.col, self.val, self.flags


def _lines(src):
    if isinstance(src, (str, bytes)) and not (isinstance(src, str) and "\n" in src):
        with open(src, "r") as f:
            return f.read().splitlines()
    if isinstance(src, str):
        return src.splitlines()
    if isinstance(src, io.IOBase) or hasattr(src, "read"):
        return src.read().splitlines()
    raise TypeError("read_mtx takes a path, the file's text or a file object")


def read_mtx(src):
    """Parse a Matrix Market coordinate file (a path, its text, or an open
    text file) into an ``MtxMatrix``.  Raises ValueError on a malformed
    file, an index outside the stated shape, a non-zero diagonal in a
    skew-symmetric matrix, or a non-square symmetric matrix."""
    lines = _lines(src)
    if not lines or not lines[0].lower().startswith("%%matrixmarket"):
        raise ValueError("missing %%MatrixMarket header")
    head = lines[0].split()
    if len(head) != 5 or head[1].lower() != "matrix":
        raise ValueError("header must read: %%MatrixMarket matrix <format> <field> <symmetry>")
    fmt, field, sym = head[2].lower(), head[3].lower(), head[4].lower()
    if fmt != "coordinate":
        raise ValueError("only the coordinate format is read (got %r)" % fmt)
    if field not in _FIELDS:
        raise ValueError("unknown field %r" % field)
    if sym not in _SYMMETRIES:
        raise ValueError("unknown symmetry %r" % sym)
    body = [ln for ln in lines[1:] if ln.strip() and not ln.lstrip().startswith("%")]
    if not body:
        raise ValueError("missing size line")
    size = body[0].split()
    if len(size) != 3:
        raise ValueError("size line must hold nrows ncols nnz")
    nrows, ncols, nnz = (int(t) for t in size)
    if nrows < 0 or ncols < 0 or nnz < 0:
        raise ValueError("negative size")
    if sym != "general" and nrows != ncols:
        raise ValueError("a %s matrix must be square" % sym)
    entries = body[1:]
    if len(entries) != nnz:
        raise ValueError("size line announces %d entries, file holds %d" % (nnz, len(entries)))
    width = {"pattern": 2, "real": 3, "integer": 3, "complex": 4}[field]
    counts = np.fromiter((len(ln.split()) for ln in entries), dtype=np.int64, count=nnz)
    if nnz and (counts != width).any():
        k = int(np.argmax(counts != width))
        raise ValueError("entry %d: expected %d fields, got %d" % (k + 1, width, int(counts[k])))
    tok = " ".join(entries).split()
    ij = np.array(tok[0::width] + tok[1::width], dtype=np.int64).reshape(2, nnz) if nnz else np.zeros((2, 0), np.int64)
    tab = np.array([tok[c::width] for c in range(2, width)], dtype=np.float64).reshape(width - 2, nnz)
    row = ij[0] - 1
    col = ij[1] - 1
    if nnz and (row.min() < 0 or col.min() < 0 or row.max() >= nrows or col.max() >= ncols):
        raise ValueError("index outside the stated shape")
    if field == "pattern":
        re, im = np.ones(nnz), None
    elif field == "complex":
        re, im = tab[0].copy(), tab[1].copy()
    else:
        re, im = tab[0].copy(), None
    if sym != "general":
        off = row != col
        if sym == "skew-symmetric" and (~off).any() and (re[~off] != 0).any():
            raise ValueError("skew-symmetric matrix with a non-zero diagonal entry")
        mr, mc = col[off], row[off]
        mre = -re[off] if sym == "skew-symmetric" else re[off]
        if im is not None:
            mim = -im[off] if sym in ("skew-symmetric", "hermitian") else im[off]
            im = np.concatenate([im, mim])
        row, col, re = np.concatenate([row, mr]), np.concatenate([col, mc]), np.concatenate([re, mre])
    val = re[None, :] if im is None else np.stack([re, im])
    return MtxMatrix(nrows, ncols, row, col, np.ascontiguousarray(val), field, sym)


def _fmt(v):
    """Shortest text that reads back as the same binary64 value."""
    return repr(float(v))


def write_mtx(dst, nrows, ncols, row, col, val, symmetry="general", comment=None):
    """Write triplets as a Matrix Market coordinate file (``dst``: a path or
    an open text file).  ``val`` has one plane (field ``real``) or two (real,
    imaginary: field ``complex``) of binary64 values, written with enough
    digits to read back bit for bit; indices are 0-based here and 1-based in
    the file.  For ``symmetric``, ``skew-symmetric`` or ``hermitian`` only
    the entries on or below the diagonal are written (the reader expands
    them again); the caller passes a matrix that has that symmetry."""
    if symmetry not in _SYMMETRIES:
        raise ValueError("unknown symmetry %r" % symmetry)
    row = np.asarray(row, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    val = np.atleast_2d(np.asarray(val, dtype=np.float64))
    if val.shape[0] not in (1, 2) or val.shape[1] != row.shape[0] or col.shape[0] != row.shape[0]:
        raise ValueError("val must hold one or two planes of nnz values")
    if symmetry != "general":
        if nrows != ncols:
            raise ValueError("a %s matrix must be square" % symmetry)
        keep = row >= col
        row, col, val = row[keep], col[keep], val[:, keep]
    field = "complex" if val.shape[0] == 2 else "real"
    out = ["%%%%MatrixMarket matrix coordinate %s %s" % (field, symmetry)]
    if comment:
        out += ["%" + ln for ln in str(comment).splitlines()]
    out.append("%d %d %d" % (nrows, ncols, row.shape[0]))
    for k in range(row.shape[0]):
        out.append(" ".join([str(int(row[k]) + 1), str(int(col[k]) + 1)] + [_fmt(val[c, k]) for c in range(val.shape[0])]))
    text = "\n".join(out) + "\n"
    if hasattr(dst, "write"):
        dst.write(text)
    else:
        with open(dst, "w") as f:
            f.write(text)


def write_vector(dst, v, comment=None):
    """Write a multiple-precision vector (structure of limbs: P planes of n
    binary64 values) as a Matrix Market ``array`` file of n rows and P
    columns, column p holding plane p, with enough digits to read back bit
    for bit: a DD/TD/QD result (real, or real then imaginary components)
    survives the file unchanged."""
    v = np.atleast_2d(np.asarray(v, dtype=np.float64))
    P, n = v.shape
    out = ["%%MatrixMarket matrix array real general"]
    if comment:
        out += ["%" + ln for ln in str(comment).splitlines()]
    out.append("%d %d" % (n, P))
    for p in range(P):  # column-major, as the array format stores it
        out.extend(_fmt(t) for t in v[p])
    text = "\n".join(out) + "\n"
    if hasattr(dst, "write"):
        dst.write(text)
    else:
        with open(dst, "w") as f:
            f.write(text)


def read_vector(src):
    """Read a Matrix Market ``array real general`` file written by
    ``write_vector`` (n rows, P columns) back into P planes of n values."""
    lines = _lines(src)
    if not lines or not lines[0].lower().startswith("%%matrixmarket"):
        raise ValueError("missing %%MatrixMarket header")
    head = lines[0].lower().split()
    if head[1:] != ["matrix", "array", "real", "general"]:
        raise ValueError("expected: %%MatrixMarket matrix array real general")
    body = [ln for ln in lines[1:] if ln.strip() and not ln.lstrip().startswith("%")]
    n, P = (int(t) for t in body[0].split())
    vals = np.array(" ".join(body[1:]).split(), dtype=np.float64)
    if vals.shape[0] != n * P:
        raise ValueError("size line announces %d values, file holds %d" % (n * P, vals.shape[0]))
    return np.ascontiguousarray(vals.reshape(P, n))
