"""The C-ABI library loads without a GPU and exports every function that
include/*.h declares; host-side argument checks answer without touching the
device."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(mpspmv_[A-Za-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("mpspmv_create_csr", "mpspmv_spmv", "mpspmv_spmm", "mpspmv_destroy", "mpspmv_strerror"):
        assert need in names


def test_library_exports_every_declared_symbol():
    import paper_2412_17510_gb300 as mps
    lib = mps.library()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_validation_without_device():
    import paper_2412_17510_gb300 as mps
    assert mps.strerror(mps.MPSPMV_EINVAL) == "invalid argument"
    cases = [
        dict(nrows=5, ncols=5, row=[0, 5], col=[0, 0], val=np.ones((1, 2)), prec=2),        # row out of range
        dict(nrows=5, ncols=5, row=[0], col=[-1], val=np.ones((1, 1)), prec=2),            # negative col
        dict(nrows=5, ncols=5, row=[0], col=[0], val=np.array([[np.nan]]), prec=2),        # NaN
        dict(nrows=5, ncols=5, row=[0], col=[0], val=np.ones((1, 1)), prec=5),             # bad precision
        dict(nrows=5, ncols=5, row=[0], col=[0], val=np.ones((3, 1)), prec=2),             # 3 limbs for DD
        dict(nrows=5, ncols=4, row=[0], col=[0], val=np.ones((1, 1)), prec=2, flags=4),    # symmetric, not square
        dict(nrows=5, ncols=5, row=[0], col=[0], val=np.ones((1, 1)), prec=2, flags=64),   # unknown flag
        dict(nrows=5, ncols=5, row=[0], col=[0], val=np.ones((1, 1)), prec=2, flags=8),    # one-based index 0
    ]
    for c in cases:
        with pytest.raises(mps.MpspmvError) as e:
            mps.mpspmv_create_csr(**c)
        assert e.value.status == mps.MPSPMV_EINVAL, c


def test_vector_ops_reject_null_handle_on_host():
    import paper_2412_17510_gb300 as mps
    lib = mps.library()
    out = np.zeros(8)
    assert lib.mpspmv_dot(None, 4, None, None, out.ctypes.data, None) == mps.MPSPMV_EINVAL
    assert lib.mpspmv_axpy(None, 4, out.ctypes.data, None, None, None, None) == mps.MPSPMV_EINVAL
