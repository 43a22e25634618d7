import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


_SCENES = {}


def scene(name, **kw):
    """Cached seeded scene from the shared generator."""
    from paper_2007_01941_gb300 import scenes
    key = (name, tuple(sorted(kw.items())))
    if key not in _SCENES:
        _SCENES[key] = getattr(scenes, name)(**kw)
    return _SCENES[key]


@pytest.fixture(scope="session")
def gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2007_01941_gb300 import _ffi, build
    if not _ffi.LIB_PATH.exists():
        build.build()
    _ffi.load()
    return torch.device("cuda:0")
