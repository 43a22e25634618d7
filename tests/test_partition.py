"""Host side of the point-partitioned solve: the split of points and observations among
ranks, and the all-reduce hook adapter over a torch.distributed (gloo) group on two CPU
processes."""
import ctypes
import os
import socket
from datetime import timedelta

import numpy as np
import pytest

from conftest import scene


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_split_points_balances_observations_and_covers_every_point():
    from paper_2007_01941_gb300 import partition
    s = scene("street_chain", n_cams=300, n_pts=30000)
    for world in (1, 2, 3, 7):
        parts = partition.split_points(s.pt_idx, s.n_pts, world)
        assert len(parts) == world
        allp = np.concatenate(parts)
        assert np.array_equal(allp, np.arange(s.n_pts))              # contiguous, each once
        counts = np.bincount(s.pt_idx, minlength=s.n_pts)
        loads = np.array([counts[p].sum() for p in parts])
        assert loads.sum() == s.n_obs
        assert loads.max() - loads.min() <= 2 * counts.max()          # balanced to a point or two


def test_local_parts_partition_the_observations():
    from paper_2007_01941_gb300 import partition
    s = scene("street_chain", n_cams=300, n_pts=30000)
    parts = [partition.local_part(s.cam_idx, s.pt_idx, p, s.n_pts)
             for p in partition.split_points(s.pt_idx, s.n_pts, 3)]
    obs = np.concatenate([p.obs for p in parts])
    assert np.array_equal(np.sort(obs), np.arange(s.n_obs))            # every observation once
    for p in parts:
        assert np.array_equal(p.cam_idx, s.cam_idx[p.obs])
        assert np.array_equal(p.points[p.pt_idx], s.pt_idx[p.obs])     # local ids map back
        assert p.pt_idx.min() >= 0 and p.pt_idx.max() < len(p.points)


def _hook_rank(rank, world, port):
    import torch.distributed as dist
    from paper_2007_01941_gb300 import partition
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=60))
    try:
        hook = partition.gloo_allreduce_hook()
        buf = (ctypes.c_double * 5)(*[rank + 1.0 + k for k in range(5)])
        assert hook(buf, 5, None) == 0
        expect = [sum(r + 1.0 + k for r in range(world)) for k in range(5)]
        assert list(buf) == expect, (list(buf), expect)
    finally:
        dist.destroy_process_group()


def test_gloo_hook_sums_host_buffers_over_two_ranks():
    import torch.multiprocessing as mp
    mp.spawn(_hook_rank, args=(2, _free_port()), nprocs=2, join=True)
