"""hgs_bin_sort_static: the binning call for callers that cannot allocate
device memory at render time (its scratch is a fixed array inside the
library).  It must produce exactly the lists of hgs_bin_sort, call after
call, through the C ABI.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

import synthetic as S
from paper_2512_02932_gb300 import Rasterizer, SceneTensors, abi

pytestmark = pytest.mark.gpu

CFG = S.RenderConfig()


def _static_lists(r, capacity):
    """Bin r's projected primitives with hgs_bin_sort_static into fresh,
    caller-owned output buffers."""
    vals = torch.full((capacity,), -1, dtype=torch.int32, device="cuda")
    keys = torch.zeros(capacity, dtype=torch.int64, device="cuda")
    ranges = torch.full_like(r.ranges, -1)
    d_count = torch.zeros(1, dtype=torch.int64, device="cuda")
    dev_err = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = abi.hgs_binning(vals.data_ptr(), keys.data_ptr(), ranges.data_ptr(), d_count.data_ptr())
    proj = r.proj_struct()
    st = abi.hgs_bin_sort_static(r.n, C.byref(proj), C.byref(r._cam_s), C.byref(r._cfg_s), capacity,
                                 C.byref(out), C.c_void_p(dev_err.data_ptr()),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == abi.HGS_OK, abi.hgs_status_string(st)
    torch.cuda.synchronize()
    assert int(dev_err.item()) == 0
    K = int(d_count.item())
    return (keys[:K].cpu().numpy().view(np.uint64), vals[:K].cpu().numpy().view(np.uint32),
            ranges.cpu().numpy().view(np.uint32), K)


def _workspace_lists(r):
    K = int(r.d_count.item())
    return (r.keys[:K].cpu().numpy().view(np.uint64), r.vals[:K].cpu().numpy().view(np.uint32),
            r.ranges.cpu().numpy().view(np.uint32), K)


def test_static_scratch_matches_workspace_binning_twice():
    cases = [S.tiny_scene(0), (S.surface_scene(200_000, seed=21), S.orbit_camera(40.0, 15.0, 3.0, 640, 480))]
    for scene, cam in cases:
        r = Rasterizer("cuda", keep_keys=True)
        r.forward(SceneTensors.from_numpy(scene), cam, CFG)
        torch.cuda.synchronize()
        ref = _workspace_lists(r)
        cap = ref[3] + 4096
        for _ in range(2):  # two calls in a row share (and reuse) the array
            got = _static_lists(r, cap)
            assert got[3] == ref[3] > 0
            np.testing.assert_array_equal(got[0], ref[0])
            np.testing.assert_array_equal(got[1], ref[1])
            np.testing.assert_array_equal(got[2], ref[2])


def test_static_scratch_on_a_heavy_tailed_scene():
    """Needles and ribbons (tile sets with many rows, deferred emits): the
    static call produces the workspace call's lists."""
    scene = S.surface_scene(60_000, seed=21, frac3d=0.3, ls_loc=-4.0, ls_scale=0.8, heavy_df=3)
    cam = S.orbit_camera(15.0, 25.0, 2.6, 1024, 640, 55.0)
    r = Rasterizer("cuda", keep_keys=True)
    r.forward(SceneTensors.from_numpy(scene), cam, CFG)
    torch.cuda.synchronize()
    ref = _workspace_lists(r)
    touched = r.touched[: scene.n].cpu().numpy().astype(np.int64)
    assert (touched > 256).sum() > 50
    got = _static_lists(r, ref[3] + 4096)
    assert got[3] == ref[3]
    for a, b in zip(got[:3], ref[:3]):
        np.testing.assert_array_equal(a, b)


def test_static_scratch_rejects_sizes_beyond_its_limit():
    scene, cam = S.tiny_scene(1)
    r = Rasterizer("cuda")
    r.forward(SceneTensors.from_numpy(scene), cam, CFG)
    out = abi.hgs_binning(r.vals.data_ptr(), None, r.ranges.data_ptr(), r.d_count.data_ptr())
    proj = r.proj_struct()
    too_big = abi.HGS_BIN_SORT_STATIC_BYTES // 4  # instances: 3 x 4 B each alone exceed the array
    st = abi.hgs_bin_sort_static(r.n, C.byref(proj), C.byref(r._cam_s), C.byref(r._cfg_s), too_big,
                                 C.byref(out), None, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == abi.HGS_ERR_INVALID_ARG
