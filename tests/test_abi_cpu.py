"""Host-side checks of the C ABI library: it builds for sm_103a, loads without a GPU, exports every
symbol the public header declares, and the binding declares the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_symbols():
    hdr = open(os.path.join(ROOT, "include", "risrt.h")).read()
    return set(re.findall(r"\b(risrt_[A-Za-z0-9_]+)\s*\(", hdr))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2402_13034_gb300 import build as B
    return B.build()


def test_library_exports_header_symbols(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = _header_symbols()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(lib_path):
    from paper_2402_13034_gb300 import risrt as R
    assert set(R._SIGS) == _header_symbols()
    R.load()


def test_missing_library_fails_loudly(tmp_path):
    from paper_2402_13034_gb300 import risrt as R
    with pytest.raises(R.RisrtError):
        R.load.__wrapped__(str(tmp_path / "nope.so")) if hasattr(R.load, "__wrapped__") else _load_missing(R, tmp_path)


def _load_missing(R, tmp_path):
    saved = R._lib
    try:
        R._lib = None
        R.load(str(tmp_path / "nope.so"))
    finally:
        R._lib = saved


def test_create_without_gpu_reports_error(lib_path):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2402_13034_gb300 import risrt as R
    with pytest.raises(R.RisrtError):
        R.Context(0)


def test_workspace_size_queries_are_host_arithmetic(lib_path):
    """Workspace sizes are answered on the host (no device needed): they grow with every dimension,
    split BF16 needs more than BF16, the FP32 sweep needs none, and bad arguments are rejected."""
    lib = ctypes.CDLL(lib_path)
    lib.risrt_sweep_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_size_t)]
    lib.risrt_grad_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_size_t)]

    def sweep(n, M, C, prec):
        b = ctypes.c_size_t(0)
        rc = lib.risrt_sweep_workspace_size(n, M, C, prec, ctypes.byref(b))
        return rc, b.value

    def grad(nt, B, M, prec):
        b = ctypes.c_size_t(0)
        rc = lib.risrt_grad_workspace_size(nt, B, M, prec, ctypes.byref(b))
        return rc, b.value

    assert sweep(65536, 1024, 4096, 0) == (0, 0)
    rc1, b1 = sweep(65536, 1024, 4096, 1)
    rc2, b2 = sweep(65536, 1024, 4096, 2)
    assert rc1 == rc2 == 0 and 0 < b1 < b2
    assert sweep(65536, 1024, 64, 1)[1] < b1 < sweep(131072, 1024, 4096, 1)[1]
    assert sweep(65536, 512, 4096, 1)[1] < b1
    # the packed matrix alone (n x 2M BF16) is a lower bound
    assert b1 >= 65536 * 2 * 1024 * 2
    for bad in ((0, 1024, 64, 1), (1024, 0, 64, 1), (1024, 64, 0, 1), (1024, 64, 8, 7)):
        assert sweep(*bad)[0] != 0
    rcf, bf = grad(16384, 64, 4096, 0)
    rcb, bb = grad(16384, 64, 4096, 2)
    assert rcf == rcb == 0 and bf > 0 and bb > bf
    assert grad(16384, 64, 4096, 1)[0] != 0 and grad(0, 64, 4096, 0)[0] != 0
