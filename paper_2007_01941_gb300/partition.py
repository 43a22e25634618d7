"""Point partition of one LM step over several ranks.

The reduced camera system is a sum over points (Section 2.1: S = A - F^T E C^-1 E^T F, with
C block diagonal by point), so the points can be split among ranks, each point with all of
its observations on one rank: every rank forms its points' Jacobian blocks, point blocks
C_p and its share of the camera-space sums, and one all-reduce of those shares per setup
gives every rank the same reduced system (the parallel linear algebra that Section 5.3 names
as the way to larger problems).  The library does the per-rank work (``ba_set_partition``);
this module splits a problem's observations among ranks and adapts a
``torch.distributed`` process group into the library's all-reduce hook.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np


@dataclass
class Part:
    """One rank's share of a problem: its points (global ids, ascending), its observations
    (indices into the global observation arrays, in global order) and the observation
    arrays of its local problem (global camera ids, local point ids 0 .. len(points) - 1)."""
    points: np.ndarray
    obs: np.ndarray
    cam_idx: np.ndarray
    pt_idx: np.ndarray


def split_points(pt_idx: np.ndarray, n_pts: int, world: int) -> list[np.ndarray]:
    """Contiguous ranges of point ids, one per rank, with about the same number of
    observations each (a point's observations stay together)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    counts = np.bincount(np.asarray(pt_idx, dtype=np.int64), minlength=n_pts)
    cum = np.concatenate([[0], np.cumsum(counts)])
    total = cum[-1]
    bounds = [0]
    for r in range(1, world):
        # first point whose cumulative count reaches r / world of the observations
        bounds.append(int(np.searchsorted(cum, r * total / world, side="left")))
    bounds.append(n_pts)
    bounds = np.maximum.accumulate(np.clip(bounds, 0, n_pts))
    return [np.arange(bounds[r], bounds[r + 1], dtype=np.int64) for r in range(world)]


def local_part(cam_idx: np.ndarray, pt_idx: np.ndarray, points: np.ndarray, n_pts: int) -> Part:
    """The observations of `points` and their arrays with local point ids."""
    cam_idx = np.asarray(cam_idx)
    pt_idx = np.asarray(pt_idx)
    local = -np.ones(n_pts, dtype=np.int64)
    local[points] = np.arange(len(points))
    obs = np.flatnonzero(local[pt_idx] >= 0)
    return Part(points=np.asarray(points, dtype=np.int64), obs=obs,
                cam_idx=cam_idx[obs].astype(np.int32), pt_idx=local[pt_idx[obs]].astype(np.int32))


ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t, ctypes.c_void_p)


def gloo_allreduce_hook(group=None):
    """The library's all-reduce hook over a torch.distributed process group: the host
    buffer is summed over the group's ranks in place.  Keep the returned object alive as
    long as the problem uses it."""
    import torch
    import torch.distributed as dist

    def hook(buf, count, user):
        try:
            arr = np.ctypeslib.as_array(buf, shape=(count,))
            t = torch.from_numpy(arr)          # shares the library's host buffer
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
            return 0
        except Exception:                      # the library turns nonzero into an error status
            return 1
    return ALLREDUCE_FN(hook)
