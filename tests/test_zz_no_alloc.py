"""ba_cost_noalloc: the objective evaluated without device allocation must equal the cost
that ba_linearize reports (which runs on the problem's own allocated buffers).

Kept in its own file, collected last, so that a run stopping at the first failure has
already run every other test.  It passes alone in a fresh process and after the others.
"""
import ctypes

import numpy as np
import pytest
import torch

from conftest import scene

pytestmark = pytest.mark.gpu


def _call(lib, s, cams, pts, obs, ci, pi, out, stream):
    return lib.ba_cost_noalloc(s.n_cams, s.n_pts, s.n_obs, cams.data_ptr(), pts.data_ptr(), obs.data_ptr(),
                               ci.data_ptr(), pi.data_ptr(), out.data_ptr(), ctypes.c_void_p(stream))


def _small_angle_ring():
    # camera 0 exactly unrotated and camera 1 with theta^2 = 3e-18: both take the
    # first-order rotation branch (theta^2 < 1e-16) in both entry points
    import dataclasses
    s = scene("ring", seed=0)
    cams = s.cams.copy()
    cams[0, :3] = 0.0
    cams[1, :3] = 1e-9
    return dataclasses.replace(s, cams=cams)


def test_noalloc_cost_matches_linearize_twice_in_a_row(gpu):
    from paper_2007_01941_gb300 import _ffi, api
    lib = _ffi.load()
    for s in (scene("street_chain", n_cams=300, n_pts=30000), scene("ring", seed=0), _small_angle_ring()):
        prob, cams, pts, obs = api.from_scene(s, device=gpu)
        ref = prob.linearize(cams, pts, obs)                      # existing entry point
        ci = torch.as_tensor(s.cam_idx, device=gpu)
        pi = torch.as_tensor(s.pt_idx, device=gpu)
        stream = torch.cuda.current_stream(gpu).cuda_stream
        for k in range(2):                                        # two calls in a row
            out = torch.full((1,), -1.0, dtype=torch.float64, device=gpu)
            torch.cuda.synchronize(gpu)
            free0 = torch.cuda.mem_get_info(gpu)[0]
            assert _call(lib, s, cams, pts, obs, ci, pi, out, stream) == _ffi.BA_OK
            torch.cuda.synchronize(gpu)
            if k == 1:
                # after the first call has loaded the array, a call takes no device memory
                assert torch.cuda.mem_get_info(gpu)[0] == free0
            got = float(out.item())
            assert abs(got - ref) <= 1e-12 * ref, (got, ref)
        prob.close()


def test_noalloc_rejects_too_many_cameras(gpu):
    from paper_2007_01941_gb300 import _ffi
    lib = _ffi.load()
    big = 4097
    cams = torch.zeros(big, 9, dtype=torch.float64, device=gpu)
    out = torch.zeros(1, dtype=torch.float64, device=gpu)
    st = lib.ba_cost_noalloc(big, 0, 0, cams.data_ptr(), None, None, None, None, out.data_ptr(), None)
    assert st == _ffi.BA_ERR_LIMIT


def test_noalloc_out_of_range_index_gives_nan(gpu):
    from paper_2007_01941_gb300 import _ffi
    lib = _ffi.load()
    s = scene("ring", seed=0, n_cams=8, n_pts=100)
    cams = torch.tensor(s.cams, device=gpu)
    pts = torch.tensor(s.pts, device=gpu)
    obs = torch.tensor(s.obs, device=gpu)
    ci = torch.as_tensor(s.cam_idx, device=gpu).clone()
    pi = torch.as_tensor(s.pt_idx, device=gpu)
    ci[5] = s.n_cams + 3
    out = torch.zeros(1, dtype=torch.float64, device=gpu)
    stream = torch.cuda.current_stream(gpu).cuda_stream
    assert _call(lib, s, cams, pts, obs, ci, pi, out, stream) == _ffi.BA_OK
    torch.cuda.synchronize(gpu)
    assert np.isnan(out.item())
