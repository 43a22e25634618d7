"""Python front end of the C ABI (include/ba.h): one :class:`Problem` per observation
graph.  Arguments are CUDA tensors; every computation runs in the library's
kernels on the stream that was current when the problem was created.  There is no
CPU path: without the built library or a GPU the calls raise.
"""
from __future__ import annotations

import ctypes
from ctypes import byref, c_double, c_int, c_size_t, c_void_p

import torch

from . import _ffi


class BAError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_ffi.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def default_options(**overrides) -> _ffi.Options:
    lib = _ffi.load()
    o = _ffi.Options()
    lib.ba_default_options(byref(o))
    for k, v in overrides.items():
        name = "lambda_" if k in ("lambda", "lam") else k
        if not hasattr(o, name):
            raise KeyError(f"unknown option {k}")
        setattr(o, name, v)
    return o


def _ptr(t: torch.Tensor | None, dtype=torch.float64) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


class Problem:
    """Reduced-camera-system solver for a fixed set of observations.

    cam_idx, pt_idx: int32 CUDA tensors [n_obs] (camera and point of each
    observation).  Options are those of ``ba_options`` (see :func:`default_options`)."""

    def __init__(self, n_cams: int, n_pts: int, cam_idx: torch.Tensor, pt_idx: torch.Tensor,
                 options: _ffi.Options | None = None, **overrides):
        self._lib = _ffi.load()
        if options is None:
            options = default_options(**overrides)
        self.options = options
        self.n_cams, self.n_pts, self.n_obs = int(n_cams), int(n_pts), int(cam_idx.numel())
        self.device = cam_idx.device
        self.stream = torch.cuda.current_stream(self.device)
        h = c_void_p()
        st = self._lib.ba_create(self.n_cams, self.n_pts, self.n_obs, _ptr(cam_idx, torch.int32),
                                 _ptr(pt_idx, torch.int32), byref(options),
                                 c_void_p(self.stream.cuda_stream), byref(h))
        if st != 0:
            raise BAError(st, "ba_create failed")
        self._h = h

    # -- lifetime -------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self._lib.ba_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st: int, allow=()):
        if st != 0 and st not in allow:
            raise BAError(st, self._lib.ba_last_error(self._h).decode())
        return st

    def _empty(self, *shape, dtype=torch.float64):
        return torch.empty(*shape, dtype=dtype, device=self.device)

    # -- the solve ------------------------------------------------------------
    def linearize(self, cams, pts, obs) -> float:
        cost = c_double()
        self._check(self._lib.ba_linearize(self._h, _ptr(cams), _ptr(pts), _ptr(obs), byref(cost)))
        return cost.value

    def schur_setup(self, lam: float):
        self._check(self._lib.ba_schur_setup(self._h, float(lam)))

    def mg_setup(self):
        self._check(self._lib.ba_mg_setup(self._h))

    def pcg_solve(self, rhs=None, out=None, allow_not_converged=False):
        """Returns (delta_c [n_cams, 9], iterations, relative residual)."""
        if out is None:
            out = self._empty(self.n_cams, 9)
        it, rel = c_int(), c_double()
        allow = (_ffi.BA_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        self._check(self._lib.ba_pcg_solve(self._h, _ptr(rhs), _ptr(out), byref(it), byref(rel)), allow)
        return out, it.value, rel.value

    def back_substitute(self, delta_c, out=None):
        if out is None:
            out = self._empty(self.n_pts, 3)
        self._check(self._lib.ba_back_substitute(self._h, _ptr(delta_c), _ptr(out)))
        return out

    def solve(self, cams, pts, obs, lam: float):
        """linearize + schur_setup + mg_setup + pcg_solve; returns (delta_c, delta_p, iters, rel)."""
        self.linearize(cams, pts, obs)
        self.schur_setup(lam)
        self.mg_setup()
        dc, it, rel = self.pcg_solve()
        return dc, self.back_substitute(dc), it, rel

    def lm_step(self, cams, pts, obs, lam: float):
        """One LM step; cams/pts are updated in place when accepted.
        Returns (new lambda, accepted, cost)."""
        lam_c, acc, cost = c_double(lam), c_int(), c_double()
        self._check(self._lib.ba_lm_step(self._h, _ptr(cams), _ptr(pts), _ptr(obs), byref(lam_c),
                                         byref(acc), byref(cost)))
        return lam_c.value, bool(acc.value), cost.value

    def adjoint(self, dL_ddelta, want_obs=True, want_cams=True, want_pts=True):
        """Gradients (dL/dobs [n_obs,2], dL/dcams [n_cams,9], dL/dpts [n_pts,3]) of the
        last solve's delta for the cotangent dL/ddelta (9 n_cams + 3 n_pts)."""
        go = self._empty(self.n_obs, 2) if want_obs else None
        gc = self._empty(self.n_cams, 9) if want_cams else None
        gp = self._empty(self.n_pts, 3) if want_pts else None
        self._check(self._lib.ba_adjoint(self._h, _ptr(dL_ddelta.contiguous()), _ptr(go), _ptr(gc), _ptr(gp)))
        return go, gc, gp

    def set_partition(self, cam_idx_all, pt_idx_all, hook):
        """Makes this problem one rank's part of a point-partitioned solve (ba_set_partition):
        cam_idx_all, pt_idx_all are the whole problem's observations (global point ids;
        host arrays), hook the all-reduce callback (see partition.gloo_allreduce_hook)."""
        import numpy as np
        ci = np.ascontiguousarray(np.asarray(cam_idx_all, dtype=np.int32))
        pi = np.ascontiguousarray(np.asarray(pt_idx_all, dtype=np.int32))
        if ci.shape != pi.shape or ci.ndim != 1:
            raise ValueError("cam_idx_all and pt_idx_all must be 1-D arrays of equal length")
        self._check(self._lib.ba_set_partition(self._h, int(ci.size), ci.ctypes.data, pi.ctypes.data,
                                               ctypes.cast(hook, c_void_p), None))
        self._part = (ci, pi, hook)   # the hook must outlive the problem

    # -- inspection -----------------------------------------------------------
    def schur_matvec(self, x, precision=_ffi.BA_FP64):
        y = torch.empty_like(x)
        self._check(self._lib.ba_schur_matvec(self._h, _ptr(x), _ptr(y), int(precision)))
        return y

    def precond_apply(self, r):
        z = torch.empty_like(r)
        self._check(self._lib.ba_precond_apply(self._h, _ptr(r), _ptr(z)))
        return z

    def set_kernel_timing(self, enable: bool):
        self._check(self._lib.ba_set_kernel_timing(self._h, int(bool(enable))))

    def kernel_timing(self, kernel_class: int):
        """(total ms, launches) of one kernel class since timing was enabled."""
        ms, n = c_double(), ctypes.c_longlong()
        self._check(self._lib.ba_get_kernel_timing(self._h, int(kernel_class), byref(ms), byref(n)))
        return ms.value, n.value

    def info(self) -> dict:
        inf = _ffi.Info()
        self._check(self._lib.ba_get_info(self._h, byref(inf)))
        n = inf.n_levels
        return dict(n_levels=n, level_nodes=list(inf.level_nodes[:n]), level_block=list(inf.level_block[:n]),
                    level_nnzb=list(inf.level_nnzb[:n]), level_lambda_max=list(inf.level_lambda_max[:n]),
                    pcg_iters=inf.pcg_iters, pcg_rel_res=inf.pcg_rel_res, cost=inf.cost,
                    lam=inf.lambda_, kernel_launches=inf.kernel_launches,
                    level0_explicit=bool(inf.level0_explicit))

    _ARR_DTYPE = {
        _ffi.BA_ARR_LEVEL_ROWPTR: torch.int32, _ffi.BA_ARR_LEVEL_COLS: torch.int32,
        _ffi.BA_ARR_LEVEL_W: torch.int64, _ffi.BA_ARR_STRENGTH_PTR: torch.int32,
        _ffi.BA_ARR_STRENGTH_IDX: torch.int32, _ffi.BA_ARR_AGG: torch.int32,
        _ffi.BA_ARR_KEPT: torch.int32,
    }

    def get_array(self, which: int, level: int = 0) -> torch.Tensor:
        need = c_size_t()
        self._check(self._lib.ba_get_array(self._h, which, level, None, 0, byref(need)))
        dt = self._ARR_DTYPE.get(which, torch.float64)
        esz = torch.tensor([], dtype=dt).element_size()
        out = self._empty(max(need.value // esz, 1), dtype=dt)
        self._check(self._lib.ba_get_array(self._h, which, level, c_void_p(out.data_ptr()), need.value, None))
        return out[: need.value // esz]


def from_scene(scene, device="cuda", **overrides):
    """Problem plus device copies (cams, pts, obs) for a generated Scene."""
    ci = torch.as_tensor(scene.cam_idx, dtype=torch.int32, device=device)
    pi = torch.as_tensor(scene.pt_idx, dtype=torch.int32, device=device)
    prob = Problem(scene.n_cams, scene.n_pts, ci, pi, **overrides)
    cams = torch.as_tensor(scene.cams, dtype=torch.float64, device=device).contiguous()
    pts = torch.as_tensor(scene.pts, dtype=torch.float64, device=device).contiguous()
    obs = torch.as_tensor(scene.obs, dtype=torch.float64, device=device).contiguous()
    return prob, cams, pts, obs


