"""The C-ABI library loads and exports every entry point that include/ebr.h
declares (no CUDA work is done here: this runs without a GPU)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "ebr.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ebr_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_10165_b300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def test_header_declares_the_four_calls():
    names = _declared()
    for n in ("ebr_plan", "ebr_classify", "ebr_build_levels", "ebr_reconstruct", "ebr_boundary_forces",
              "ebr_reconstruct_adjoint"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2609_10165_b300 import _lib
    assert sorted(_lib.EXPORTED) == _declared()


def test_binding_fails_loudly_without_the_library(tmp_path):
    from paper_2609_10165_b300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError):
            _lib.load(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def test_null_context_is_rejected_without_touching_the_gpu(lib):
    lib.ebr_last_error.restype = ctypes.c_char_p
    lib.ebr_last_error.argtypes = [ctypes.c_void_p]
    assert lib.ebr_last_error(None) == b"null context"
    lib.ebr_classify.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.ebr_classify(None, None, None) == -1
