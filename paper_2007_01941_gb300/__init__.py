"""GB300 (sm_103a) linear solve of Levenberg-Marquardt bundle adjustment with the
unsmoothed-aggregation multigrid preconditioner of "Multigrid for Bundle
Adjustment" (Konolige & Brown).  The numerical work runs in the CUDA library
built from ``csrc/`` (C ABI in ``include/ba.h``); this package holds the build
script, the ctypes binding, the autograd wrapper and the synthetic scene
generator."""
from . import scenes  # noqa: F401

__all__ = ["scenes", "api", "autograd", "build"]


def __getattr__(name):
    if name in ("api", "autograd", "build", "_ffi"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
