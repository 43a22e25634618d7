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


def test_struct_layouts_match_the_library(lib):
    from paper_2007_01941_gb300 import _ffi
    lib.ba_struct_size.restype = ctypes.c_size_t
    assert lib.ba_struct_size(0) == ctypes.sizeof(_ffi.Options)
    assert lib.ba_struct_size(1) == ctypes.sizeof(_ffi.Info)
    assert lib.ba_struct_size(2) == 0


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
    assert o.loss == _ffi.BA_LOSS_SQUARED and o.loss_scale == 1.0   # Huber a = 1 (Section 5)


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    from paper_2007_01941_gb300 import _ffi
    lib2 = _ffi.load()
    h = ctypes.c_void_p()
    assert lib2.ba_create(0, 0, 0, None, None, None, None, ctypes.byref(h)) == _ffi.BA_ERR_INVALID_ARG
    assert lib2.ba_create(4, 4, 3, None, None, None, None, ctypes.byref(h)) == _ffi.BA_ERR_INVALID_ARG
    assert not h.value
    # option validation runs before any CUDA call
    for bad in (dict(loss=7), dict(loss=_ffi.BA_LOSS_HUBER, loss_scale=-1.0),
                dict(loss=_ffi.BA_LOSS_HUBER, loss_scale=float("inf")), dict(stop_rule=9)):
        o = _ffi.Options()
        lib2.ba_default_options(ctypes.byref(o))
        for k, v in bad.items():
            setattr(o, k, v)
        assert lib2.ba_create(4, 4, 0, None, None, ctypes.byref(o), None, ctypes.byref(h)) == \
            _ffi.BA_ERR_INVALID_ARG, bad
        assert not h.value
