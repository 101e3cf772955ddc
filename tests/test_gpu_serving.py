"""Serving: batched rendering of several resident scenes at several
resolutions in one launch, and the continuous-batching loop.  Each result
must be the same alone and in the mix.  Needs a GB300."""
import numpy as np
import pytest
import torch

import synthetic as S
from gpu_util import CFG, assert_images_match, compare_pixels, gpu_pixels
from oracle import native as O
from paper_2512_02932_gb300 import Rasterizer, SceneTensors
from paper_2512_02932_gb300.serving import Server, ServingConfig, render_batch_once

pytestmark = pytest.mark.gpu

KEYS = ("rgb", "depth", "normal", "alpha", "T_final", "n_last")


def _scenes():
    sizes, mixes = (20_000, 50_000, 80_000, 120_000), (0.5, 0.6, 0.7, 0.8)
    host = [S.surface_scene(n, seed=40 + k, frac3d=f) for k, (n, f) in enumerate(zip(sizes, mixes))]
    return host, [SceneTensors.from_numpy(h) for h in host]


def _alone(scene_t, cam):
    r = Rasterizer("cuda")
    out = r.forward(scene_t, cam, CFG)
    torch.cuda.synchronize()
    return {k: v.detach().cpu().numpy() for k, v in out.items()}


def test_batch_equals_alone_bit_for_bit():
    host, dev = _scenes()
    res = [(512, 512), (800, 600), (1280, 720), (1920, 1080), (97, 33)]
    rng = np.random.default_rng(0)
    picks = [(k % 4, res[k % len(res)]) for k in range(7)]
    cams = [S.orbit_camera(float(rng.uniform(0, 360)), float(rng.uniform(-30, 30)),
                           float(rng.uniform(2.5, 4.0)), w, h) for _, (w, h) in picks]
    scenes = [dev[s] for s, _ in picks]
    outs, K = render_batch_once(scenes, cams, CFG)
    assert K > 0
    for (s, _), cam, o in zip(picks, cams, outs):
        ref = _alone(dev[s], cam)
        for k in KEYS:
            np.testing.assert_array_equal(o[k].cpu().numpy(), ref[k], err_msg=k)
    # and one of them against the oracle
    m = O.Oracle(host[picks[4][0]], cams[4], CFG).render_maps()
    g = {k: outs[4][k].cpu().numpy() for k in KEYS}
    assert_images_match(g, m, max_excluded=0.0, label="batched request")


def test_batch_of_heavy_tailed_scenes_matches_alone():
    """A batch of heavy-tailed scenes (needles and ribbons, many rectangles
    over 256 tiles, so the stacked grid's tile sets and deferred emits are
    exercised): each request's images equal the same request rendered alone,
    bit for bit."""
    host = [S.surface_scene(30_000, seed=50 + k, frac3d=0.3, ls_loc=-4.0, ls_scale=0.8, heavy_df=3)
            for k in range(2)]
    dev = [SceneTensors.from_numpy(h) for h in host]
    cams = [S.orbit_camera(15.0, 25.0, 2.6, 1024, 640, 55.0), S.orbit_camera(200.0, 10.0, 2.8, 800, 600, 50.0)]
    o, K = render_batch_once(dev, cams, CFG)
    assert K > 0
    for k in range(2):
        alone, _ = render_batch_once([dev[k]], [cams[k]], CFG)
        for key in KEYS:
            np.testing.assert_array_equal(o[k][key].cpu().numpy(), alone[0][key].cpu().numpy(), err_msg=key)


def test_server_burst_matches_alone():
    host, dev = _scenes()
    rng = np.random.default_rng(1)
    res = S.SERVING_RES
    reqs = []
    for k in range(24):
        w, h = res[int(rng.integers(len(res)))]
        cam = S.orbit_camera(float(rng.uniform(0, 360)), float(rng.uniform(-30, 30)),
                             float(rng.uniform(2.5, 4.0)), w, h)
        reqs.append((0.0005 * k, int(rng.integers(4)), cam))
    srv = Server(dev, CFG, ServingConfig(max_batch=6, streams=2, prim_budget=1_000_000,
                                         capacity=40_000_000))
    out, st = srv.run(reqs, realtime=False, keep=True)
    assert st["requests"] == 24 and st["failed"] == 0
    assert all(r.t_done >= r.t_launch for r in out)  # realtime=False ignores arrival times
    for r in out[::3]:
        ref = _alone(dev[r.scene_id], r.cam)
        for k in KEYS:
            np.testing.assert_array_equal(r.out[k].cpu().numpy(), ref[k], err_msg=k)


def test_plain_server_and_overflow_retry():
    host, dev = _scenes()
    rng = np.random.default_rng(2)
    reqs = [(0.0, int(rng.integers(4)), S.orbit_camera(float(rng.uniform(0, 360)), 10.0, 3.0, 640, 480))
            for _ in range(8)]
    plain = Server(dev, CFG, plain=True)
    _, st = plain.run(reqs, realtime=False)
    assert st["requests"] == 8
    # a capacity that fits one request but not a batch: batches overflow,
    # their requests are retried alone and still complete correctly
    srv = Server(dev, CFG, ServingConfig(max_batch=8, streams=1, prim_budget=1_000_000,
                                         capacity=2_000_000, safety=0.01))
    out, st = srv.run(reqs, realtime=False, keep=True)
    assert st["failed"] == 0
    for r in out[:3]:
        ref = _alone(dev[r.scene_id], r.cam)
        np.testing.assert_array_equal(r.out["rgb"].cpu().numpy(), ref["rgb"])


def test_serving_workload_scenes_against_the_oracle():
    """The serving workload's resident scenes (200k, 500k, 1M and 3M
    primitives, SH degree 3, 3D shares 50-80%) rendered together in one batch
    at the four serving resolutions: every request against the FP64 oracle
    on sampled pixels."""
    host = S.serving_scenes()
    dev = [SceneTensors.from_numpy(h) for h in host]
    rng = np.random.default_rng(17)
    cams = [S.orbit_camera(float(rng.uniform(0, 360)), float(rng.uniform(-30, 30)), float(rng.uniform(2.5, 4.0)),
                           w, h) for (w, h) in S.SERVING_RES]
    outs, K = render_batch_once(dev, cams, CFG)
    assert K > 0
    for k, (sc, cam) in enumerate(zip(host, cams)):
        pix = np.stack([rng.integers(0, cam.width, 1500), rng.integers(0, cam.height, 1500)], 1).astype(np.int32)
        chk = O.Oracle(sc, cam, CFG).render_checked(pix)
        g = gpu_pixels({key: outs[k][key] for key in KEYS}, pix)
        compare_pixels(g, chk, max_excluded=0.0, label=f"serving scene {sc.n} prims {cam.width}x{cam.height}")
