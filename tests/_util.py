"""Shared helpers for the GPU parity tests (host-side marshalling only)."""
import numpy as np

import oracle
import workloads


def csr_pair(coo, L, vals=None, flags=0):
    """(oracle CSR, handle) for the same triplets.  ``vals`` defaults to the
    P-mode promotion of binary64 triplet values."""
    import paper_2412_17510_gb300 as mps
    cplx = bool(flags & mps.MPSPMV_COMPLEX)
    v = coo.promoted(L) if vals is None else vals
    A = oracle.coo_to_csr(coo.nrows, coo.ncols, coo.row, coo.col, v, L, cplx)
    h = mps.mpspmv_create_csr(coo.nrows, coo.ncols, coo.row, coo.col, v, L, flags)
    return A, h


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def unsplit_rows(A, K):
    """Rows whose stored entries lie inside one run of K entries (non-empty)."""
    ip = A.indptr
    r = np.arange(A.nrows)
    ne = ip[1:] > ip[:-1]
    same = (ip[:-1] // K) == ((ip[1:] - 1) // K)
    return r[ne & same]


def gpu_spmv(h, x, P, nrows):
    import torch
    import paper_2412_17510_gb300 as mps
    xd = to_dev(x)
    yd = torch.full((P, nrows), float("nan"), dtype=torch.float64, device="cuda")
    mps.mpspmv_spmv(h, xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()
