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
