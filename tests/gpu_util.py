"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare it with the oracle."""
import numpy as np
import torch

import synthetic as S
from oracle import native as O
from paper_2512_02932_gb300 import Rasterizer, SceneTensors

CFG = S.RenderConfig()
IMG_MAX_ABS = 1e-3   # per channel, non-ambiguous pixels
IMG_MEAN_ABS = 1e-5


def gpu_forward(scene, cam, cfg=CFG, keep_keys=True, capacity=0):
    r = Rasterizer("cuda", capacity=capacity, keep_keys=keep_keys)
    st = SceneTensors.from_numpy(scene)
    out = r.forward(st, cam, cfg)
    torch.cuda.synchronize()
    r.check()
    host = {k: v.detach().cpu().numpy() for k, v in out.items()}
    return r, st, host


def gpu_lists(r):
    K = int(r.d_count.item())
    keys = r.keys[:K].cpu().numpy().view(np.uint64)
    vals = r.vals[:K].cpu().numpy().view(np.uint32)
    ranges = r.ranges.cpu().numpy().view(np.uint32)
    return keys, vals, ranges


def assert_lists_bitexact(r, scene, cam, cfg=CFG):
    db, rect, touched = O.contract_bin(scene, cam, cfg)
    n = scene.n
    g_db = r.depth_key[:n].cpu().numpy().view(np.uint32)
    g_touched = r.touched[:n].cpu().numpy().view(np.uint32).astype(np.int64)
    g_rect = r.rect[:n].cpu().numpy().view(np.uint16).astype(np.int32)
    np.testing.assert_array_equal(g_touched, touched)
    binned = touched > 0
    np.testing.assert_array_equal(g_db[binned], db[binned])
    np.testing.assert_array_equal(g_rect[binned], rect[binned])
    keys, vals, ranges, _ = O.tile_lists(scene, cam, cfg)
    gk, gv, gr = gpu_lists(r)
    assert len(gk) == len(keys)
    np.testing.assert_array_equal(gk, keys)
    np.testing.assert_array_equal(gv, vals)
    np.testing.assert_array_equal(gr, ranges)
    return len(keys)


def assert_images_match(gpu, orc, amb, max_abs=IMG_MAX_ABS, mean_abs=IMG_MEAN_ABS, max_amb_frac=1e-3):
    ok = ~amb
    assert amb.mean() <= max_amb_frac, f"ambiguous fraction {amb.mean()}"
    report = {}
    for key in ("rgb", "depth", "normal", "alpha"):
        g = gpu[key]
        o = orc[key]
        if g.ndim == 2:
            g, o = g[None], o[None]
        for c in range(g.shape[0]):
            d = np.abs(g[c].astype(np.float64) - o[c])[ok]
            if key == "depth":  # unnormalised depth: bounds relative to max(1, |depth|)
                d = d / np.maximum(1.0, np.abs(o[c][ok]))
            report[f"{key}{c}"] = (float(d.max()) if d.size else 0.0, float(d.mean()) if d.size else 0.0)
            assert d.size == 0 or d.max() <= max_abs, (key, c, d.max(), np.unravel_index(
                np.argmax(np.where(ok, np.abs(g[c] - o[c]), 0)), ok.shape))
            assert d.size == 0 or d.mean() <= mean_abs, (key, c, d.mean())
    return report


def assert_grads_match(g_gpu, g_ref, rel_norm=1e-3, rel_elem=1e-3):
    """Per tensor ||dg|| <= rel_norm ||g||, per element
    |dg| <= rel_elem |g| + rel_elem rms(g)."""
    out = {}
    for k, ref in g_ref.items():
        g = np.asarray(g_gpu[k], np.float64).reshape(ref.shape)
        diff = g - ref
        nrm = np.linalg.norm(ref)
        rel = np.linalg.norm(diff) / max(nrm, 1e-30)
        rms = np.sqrt(np.mean(ref ** 2))
        bad = np.abs(diff) > rel_elem * np.abs(ref) + rel_elem * rms
        out[k] = (rel, int(bad.sum()))
        assert rel <= rel_norm, (k, rel)
        assert not bad.any(), (k, int(bad.sum()), np.argwhere(bad)[:5])
    return out
