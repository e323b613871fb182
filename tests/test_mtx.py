"""Matrix Market reader (host input plumbing): the paper's worked 5x5
example (Section 3) written as a Matrix Market file gives the printed COO
arrays, and through the oracle the printed CSR arrays and A [1..5]; the
symmetric, skew-symmetric, Hermitian and pattern forms expand to the dense
matrices they describe; malformed files are rejected."""
import io
import json
import os

import numpy as np
import pytest

import oracle

mtx = pytest.importorskip("paper_2412_17510_gb300.mtx")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "worked_example_5x5.json")


def dense(m):
    """Dense matrix of the returned triplets (duplicates summed)."""
    cplx = m.val.shape[0] == 2
    A = np.zeros((m.nrows, m.ncols), dtype=complex if cplx else float)
    for k in range(m.nnz):
        A[m.row[k], m.col[k]] += m.val[0, k] + (1j * m.val[1, k] if cplx else 0)
    return A


def test_worked_example_as_matrix_market():
    g = json.load(open(GOLDEN))
    coo = g["coo"]
    text = "%%MatrixMarket matrix coordinate integer general\n% the 5x5 example of Section 3\n5 5 8\n"
    text += "".join("%d %d %d\n" % (r + 1, c + 1, v) for r, c, v in zip(coo["row"], coo["col"], coo["data"]))
    m = mtx.read_mtx(text)
    assert (m.nrows, m.ncols, m.nnz, m.flags) == (5, 5, 8, 0)
    assert m.row.tolist() == coo["row"] and m.col.tolist() == coo["col"]
    assert m.val[0].tolist() == coo["data"]
    A = oracle.coo_to_csr(*m.args()[:4], m.val, 1)
    assert A.indptr.tolist() == g["csr"]["indptr"]
    assert A.indices.tolist() == g["csr"]["indices"]
    assert A.data[0].tolist() == g["csr"]["data"]
    y = oracle.spmv(A, np.arange(1.0, 6.0)[None, :])
    assert y[0].tolist() == g["A_times_1_to_5"]["value"]
    # the same file through a file object and through a path
    assert mtx.read_mtx(io.StringIO(text)).nnz == 8


def test_path_input(tmp_path):
    p = tmp_path / "a.mtx"
    p.write_text("%%MatrixMarket matrix coordinate real general\n2 3 2\n1 3 2.5\n2 1 -1e-300\n")
    m = mtx.read_mtx(str(p))
    assert np.array_equal(dense(m), np.array([[0, 0, 2.5], [-1e-300, 0, 0]]))


def test_symmetric_forms_expand_to_both_triangles():
    lower = [(1, 1, 4.0), (2, 1, -1.0), (3, 2, 0.5), (3, 3, 2.0)]
    body = "3 3 %d\n" % len(lower) + "".join("%d %d %r\n" % e for e in lower)
    S = dense(mtx.read_mtx("%%MatrixMarket matrix coordinate real symmetric\n" + body))
    assert np.array_equal(S, S.T) and S[0, 1] == -1.0 and S[1, 2] == 0.5 and S[2, 2] == 2.0
    off = [(2, 1, -1.0), (3, 2, 0.5)]
    K = dense(mtx.read_mtx("%%MatrixMarket matrix coordinate real skew-symmetric\n3 3 2\n"
                           + "".join("%d %d %r\n" % e for e in off)))
    assert np.array_equal(K, -K.T) and K[1, 0] == -1.0 and K[0, 1] == 1.0
    H = dense(mtx.read_mtx("%%MatrixMarket matrix coordinate complex hermitian\n2 2 2\n1 1 3 0\n2 1 1 2\n"))
    assert np.array_equal(H, H.conj().T) and H[1, 0] == 1 + 2j and H[0, 1] == 1 - 2j
    C = mtx.read_mtx("%%MatrixMarket matrix coordinate complex symmetric\n2 2 2\n1 1 3 1\n2 1 1 2\n")
    assert C.flags == 1 and C.val.shape == (2, 3)
    D = dense(C)
    assert np.array_equal(D, D.T) and D[0, 1] == 1 + 2j


def test_pattern_entries_are_ones():
    m = mtx.read_mtx("%%MatrixMarket matrix coordinate pattern symmetric\n3 3 2\n2 1\n3 3\n")
    assert np.array_equal(dense(m), np.array([[0, 1, 0], [1, 0, 0], [0, 0, 1.0]]))


@pytest.mark.parametrize("text", [
    "3 3 1\n1 1 1\n",                                                        # no header
    "%%MatrixMarket matrix array real general\n2 2\n1\n2\n3\n4\n",           # dense format
    "%%MatrixMarket matrix coordinate real general\n2 2 1\n3 1 1\n",         # row out of range
    "%%MatrixMarket matrix coordinate real general\n2 2 2\n1 1 1\n",         # fewer entries than announced
    "%%MatrixMarket matrix coordinate real symmetric\n2 3 1\n1 1 1\n",       # non-square symmetric
    "%%MatrixMarket matrix coordinate real skew-symmetric\n2 2 1\n1 1 1\n",  # skew with a diagonal
    "%%MatrixMarket matrix coordinate complex general\n2 2 1\n1 1 1\n",      # missing imaginary part
])
def test_malformed_files_are_rejected(text):
    with pytest.raises(ValueError):
        mtx.read_mtx(text)


@pytest.mark.parametrize("symmetry", ["general", "symmetric", "hermitian", "skew-symmetric"])
def test_writer_round_trip(symmetry, tmp_path):
    """write_mtx then read_mtx gives back the same matrix bit for bit (the
    symmetric forms store one triangle and expand it again)."""
    rng = np.random.default_rng(4)
    n = 30
    cplx = symmetry == "hermitian"
    A = rng.standard_normal((n, n)) * 2.0 ** rng.integers(-60, 60, (n, n))
    A[rng.random((n, n)) < 0.8] = 0.0
    if cplx:
        A = A + 1j * (rng.standard_normal((n, n)) * (A != 0))
    if symmetry == "symmetric":
        A = np.tril(A) + np.tril(A, -1).T
    elif symmetry == "hermitian":
        A = np.tril(A, -1) + np.tril(A, -1).conj().T + np.diag(np.diag(A).real)
    elif symmetry == "skew-symmetric":
        A = np.tril(A, -1) - np.tril(A, -1).T
    r, c = np.nonzero(A)
    val = np.stack([A[r, c].real, A[r, c].imag]) if cplx else A[r, c].real[None, :]
    path = str(tmp_path / "a.mtx")
    mtx.write_mtx(path, n, n, r, c, val, symmetry=symmetry, comment="round trip\nsecond line")
    m = mtx.read_mtx(path)
    assert m.symmetry == symmetry and m.nrows == n and m.ncols == n
    B = dense(m)
    assert np.array_equal(B, A)


def test_vector_round_trip_is_bit_exact(tmp_path):
    """An MP vector (QD, complex: 8 planes, with subnormal and extreme
    components) survives write_vector / read_vector bit for bit."""
    import workloads
    v = workloads.full_limb_vector(50, 4, seed=1, cplx=True)
    v[3, 0] = 5e-324
    v[0, 1] = -1.7976931348623157e308
    v[1, 2] = -0.0
    path = str(tmp_path / "y.mtx")
    mtx.write_vector(path, v, comment="QD complex result")
    w = mtx.read_vector(path)
    assert w.shape == v.shape
    assert np.array_equal(w.view(np.int64), v.view(np.int64))
