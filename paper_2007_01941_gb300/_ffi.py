"""ctypes declarations of the C ABI in include/ba.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
from ctypes import POINTER, c_double, c_int, c_longlong, c_size_t, c_void_p
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "lib" / "libba_gb300.so"

BA_OK, BA_ERR_INVALID_ARG, BA_ERR_CUDA, BA_ERR_OOM, BA_ERR_NOT_SPD, BA_ERR_BREAKDOWN, \
    BA_ERR_NOT_CONVERGED, BA_ERR_LIMIT, BA_ERR_STATE = range(9)
STATUS_NAMES = {0: "BA_OK", 1: "BA_ERR_INVALID_ARG", 2: "BA_ERR_CUDA", 3: "BA_ERR_OOM",
                4: "BA_ERR_NOT_SPD", 5: "BA_ERR_BREAKDOWN", 6: "BA_ERR_NOT_CONVERGED",
                7: "BA_ERR_LIMIT", 8: "BA_ERR_STATE"}
BA_FP64, BA_MIXED = 0, 1
BA_PRECOND_NONE, BA_PRECOND_JACOBI, BA_PRECOND_MG = 0, 1, 2
BA_OP_IMPLICIT, BA_OP_EXPLICIT, BA_OP_AUTO = 0, 1, 2
BA_DAMP_MARQUARDT, BA_DAMP_IDENTITY = 0, 1
BA_KT_SCHUR_FP64, BA_KT_SCHUR_FP32, BA_KT_LINEARIZE, BA_KT_SCHUR_DF = 0, 1, 2, 3
BA_KT_ASSEMBLY, BA_KT_OUTER_BSR, BA_KT_VCYCLE, BA_KT_SCHUR_RECOMPUTE = 4, 5, 6, 7
BA_OUTER_FP64, BA_OUTER_PAIRED_FP32 = 0, 1
BA_STOP_RELRES, BA_STOP_NASH_SOFER = 0, 1
BA_LOSS_SQUARED, BA_LOSS_HUBER = 0, 1

(BA_ARR_RESIDUAL, BA_ARR_JAC_F, BA_ARR_JAC_E, BA_ARR_DAMP_C, BA_ARR_DAMP_P, BA_ARR_CINV,
 BA_ARR_GRAD_C, BA_ARR_GRAD_P, BA_ARR_RHS, BA_ARR_LEVEL_ROWPTR, BA_ARR_LEVEL_COLS,
 BA_ARR_LEVEL_VALS, BA_ARR_LEVEL_W, BA_ARR_STRENGTH_PTR, BA_ARR_STRENGTH_IDX, BA_ARR_AGG,
 BA_ARR_NULLSPACE, BA_ARR_PROLONG, BA_ARR_KEPT, BA_ARR_JACOBI_INV, BA_ARR_COARSE_INV,
 BA_ARR_SCC_INV) = range(22)


class Options(ctypes.Structure):
    _fields_ = [("lambda_", c_double), ("rtol", c_double), ("max_iters", c_int),
                ("precision", c_int), ("preconditioner", c_int), ("damping", c_int),
                ("recompute_jacobian", c_int), ("max_agg", c_int), ("pre_smooth", c_int),
                ("post_smooth", c_int), ("lanczos_steps", c_int), ("coarse_max_nodes", c_int),
                ("max_levels", c_int), ("cheb_lo", c_double), ("cheb_hi", c_double),
                ("level0_operator", c_int), ("fused_vcycle", c_int), ("outer_product", c_int),
                ("stop_rule", c_int), ("tau", c_double), ("overlap_launches", c_int),
                ("loss", c_int), ("loss_scale", c_double),
                ("precond_lambda_min", c_double), ("schur_staging", c_int)]


class Info(ctypes.Structure):
    _fields_ = [("n_levels", c_int), ("level_nodes", c_int * 16), ("level_block", c_int * 16),
                ("level_nnzb", c_int * 16), ("level_lambda_max", c_double * 16),
                ("pcg_iters", c_int), ("pcg_rel_res", c_double), ("cost", c_double),
                ("lambda_", c_double), ("kernel_launches", c_longlong),
                ("level0_explicit", c_int)]


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "ba_default_options": (None, [POINTER(Options)]),
    "ba_struct_size": (c_size_t, [c_int]),
    "ba_create": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p, POINTER(Options), c_void_p,
                          POINTER(c_void_p)]),
    "ba_destroy": (None, [c_void_p]),
    "ba_last_error": (ctypes.c_char_p, [c_void_p]),
    "ba_linearize": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_double)]),
    "ba_schur_setup": (c_int, [c_void_p, c_double]),
    "ba_mg_setup": (c_int, [c_void_p]),
    "ba_pcg_solve": (c_int, [c_void_p, c_void_p, c_void_p, POINTER(c_int), POINTER(c_double)]),
    "ba_back_substitute": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ba_lm_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_double), POINTER(c_int),
                           POINTER(c_double)]),
    "ba_adjoint": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "ba_schur_matvec": (c_int, [c_void_p, c_void_p, c_void_p, c_int]),
    "ba_precond_apply": (c_int, [c_void_p, c_void_p, c_void_p]),
    "ba_get_info": (c_int, [c_void_p, POINTER(Info)]),
    "ba_set_kernel_timing": (c_int, [c_void_p, c_int]),
    "ba_get_kernel_timing": (c_int, [c_void_p, c_int, POINTER(c_double), POINTER(c_longlong)]),
    "ba_get_array": (c_int, [c_void_p, c_int, c_int, c_void_p, c_size_t, POINTER(c_size_t)]),
    "ba_cost_noalloc": (c_int, [c_int, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_void_p]),
    "ba_set_partition": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
}

EXPORTED = tuple(_SIGS)


def load(path: Path | str | None = None):
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"{p} is missing: build it with `python -m paper_2007_01941_gb300.build`")
    lib = ctypes.CDLL(str(p))
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    for which, st in ((0, Options), (1, Info)):
        if lib.ba_struct_size(which) != ctypes.sizeof(st):
            raise RuntimeError(f"{p}: {st.__name__} layout differs from the library's "
                               f"({ctypes.sizeof(st)} vs {lib.ba_struct_size(which)} bytes); rebuild")
    _lib = lib
    return lib


