"""Point-partitioned solve (ba_set_partition): two ranks, each with half of the points and
their observations, sum their shares of the camera-space quantities through the gloo
all-reduce hook, and must reproduce the unpartitioned solve and LM steps.  Both ranks run on
the one test GPU as separate processes; every exchange goes through the host, so no kernel
of one rank waits on the other's."""
import os
import socket
from datetime import timedelta

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CHAIN = dict(n_cams=300, n_pts=30000)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=120))
    try:
        from paper_2007_01941_gb300 import _ffi, api, partition, scenes
        dev = torch.device("cuda:0")
        _ffi.load()
        s = scenes.street_chain(**CHAIN)
        kw = dict(precision=_ffi.BA_FP64, coarse_max_nodes=16, rtol=1e-12, max_iters=5000)
        part = partition.local_part(s.cam_idx, s.pt_idx, partition.split_points(s.pt_idx, s.n_pts, world)[rank],
                                    s.n_pts)
        assert 0 < len(part.obs) < s.n_obs

        # the whole problem, unpartitioned, on this rank
        ref, rc, rp, ro = api.from_scene(s, device=dev, **kw)
        # this rank's part
        prob = api.Problem(s.n_cams, len(part.points), torch.as_tensor(part.cam_idx, device=dev),
                           torch.as_tensor(part.pt_idx, device=dev), **kw)
        hook = partition.gloo_allreduce_hook()
        prob.set_partition(s.cam_idx, s.pt_idx, hook)
        cams = torch.tensor(s.cams, device=dev)
        pts = torch.tensor(s.pts[part.points], device=dev)
        obs = torch.tensor(s.obs[part.obs], device=dev)

        # one solve: same hierarchy (built from the whole graph), same delta_c on every rank,
        # this rank's delta_p; both solves reach rtol 1e-12 on sums that differ only in their
        # rounding order
        dc_r, dp_r, it_r, _ = ref.solve(rc, rp, ro, s.lam)
        dc, dp, it, rel = prob.solve(cams, pts, obs, s.lam)
        assert rel <= 1e-12 and abs(it - it_r) <= 1, (it, it_r)
        assert prob.info()["level_nodes"] == ref.info()["level_nodes"]
        dcr, dpr = dc_r.cpu().numpy(), dp_r.cpu().numpy()[part.points]
        assert np.linalg.norm(dc.cpu().numpy() - dcr) <= 1e-10 * np.linalg.norm(dcr)
        assert np.linalg.norm(dp.cpu().numpy() - dpr) <= 1e-10 * np.linalg.norm(dpr)
        # the same delta_c on both ranks, bit for bit
        g = torch.tensor(dc.cpu().numpy().ravel())
        g0 = g.clone()
        dist.broadcast(g0, src=0)
        assert torch.equal(g, g0)

        # two LM steps: costs (summed over the ranks), acceptance, lambda, cameras, this
        # rank's points
        lam_r = lam = s.lam
        for k in range(2):
            lam_r, acc_r, cost_r = ref.lm_step(rc, rp, ro, lam_r)
            lam, acc, cost = prob.lm_step(cams, pts, obs, lam)
            assert acc == acc_r, k
            assert abs(cost - cost_r) <= 1e-12 * cost_r, (k, cost, cost_r)
            assert abs(lam - lam_r) <= 1e-9 * lam_r, (k, lam, lam_r)
            cr = rc.cpu().numpy()
            assert np.linalg.norm(cams.cpu().numpy() - cr) <= 1e-10 * np.linalg.norm(cr - s.cams), k
            pr = rp.cpu().numpy()[part.points]
            assert np.linalg.norm(pts.cpu().numpy() - pr) <= 1e-10 * np.linalg.norm(pr - s.pts[part.points]), k
        # not available on a partitioned problem
        with pytest.raises(api.BAError):
            prob.adjoint(torch.zeros(9 * s.n_cams + 3 * len(part.points), dtype=torch.float64, device=dev))
        prob.close()
        ref.close()
    finally:
        dist.destroy_process_group()


def test_partitioned_solve_matches_the_whole_problem(gpu):
    import torch.multiprocessing as mp
    mp.spawn(_rank, args=(2, _free_port()), nprocs=2, join=True)
