"""The C-ABI library builds, loads without a GPU and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "ba.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ba_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2007_01941_gb300 import _ffi, build
    if not _ffi.LIB_PATH.exists():
        build.build()
    return ctypes.CDLL(str(_ffi.LIB_PATH))


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_2007_01941_gb300 import _ffi
    assert sorted(_ffi.EXPORTED) == _declared()


def test_default_options_are_the_papers_constants(lib):
    from paper_2007_01941_gb300 import _ffi
    _ffi._lib = None
    lib2 = _ffi.load()
    o = _ffi.Options()
    lib2.ba_default_options(ctypes.byref(o))
    assert o.max_agg == 20            # Section 3.2
    assert (o.pre_smooth, o.post_smooth) == (2, 2)   # Section 3.4
    assert o.lanczos_steps == 5
    assert (o.cheb_lo, o.cheb_hi) == (0.3, 1.1)
    assert o.lambda_ == 1e-4          # 1 / initial trust radius 1e4 (Section 5)


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    from paper_2007_01941_gb300 import _ffi
    lib2 = _ffi.load()
    h = ctypes.c_void_p()
    assert lib2.ba_create(0, 0, 0, None, None, None, None, ctypes.byref(h)) == _ffi.BA_ERR_INVALID_ARG
    assert lib2.ba_create(4, 4, 3, None, None, None, None, ctypes.byref(h)) == _ffi.BA_ERR_INVALID_ARG
    assert not h.value
