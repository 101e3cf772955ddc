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


CHANNELS = ("r", "g", "b", "depth", "nx", "ny", "nz", "alpha")


def gpu_pixels(maps, pixels):
    """GPU maps at `pixels` ((P, 2) x, y) in the oracle's row layout: r, g,
    b, depth, nx, ny, nz, alpha, T_final, n_contrib (P, 10) float64."""
    g = {k: (v.detach().cpu().numpy() if hasattr(v, "detach") else np.asarray(v)) for k, v in maps.items()}
    x, y = pixels[:, 0], pixels[:, 1]
    cols = [g["rgb"][c][y, x] for c in range(3)] + [g["depth"][y, x]] + [g["normal"][c][y, x] for c in range(3)]
    cols += [g["alpha"][y, x], g["T_final"][y, x] if "T_final" in g else np.zeros(len(x)),
             g["n_contrib"][y, x] if "n_contrib" in g else np.full(len(x), -1)]
    return np.stack([np.asarray(c, np.float64) for c in cols], 1)


def _excess(gv, v, tol):
    """|gpu - oracle| beyond the oracle's conditioning tolerance, per
    channel; depth relative to max(1, |depth|) (the depth map is
    unnormalised, reading 15)."""
    d = np.abs(gv[..., :8] - v[..., :8]) - tol[..., :8]
    d[..., 3] = d[..., 3] / np.maximum(1.0, np.abs(v[..., 3]))
    return d


def compare_pixels(g, chk, max_abs=IMG_MAX_ABS, mean_abs=IMG_MEAN_ABS, check_nc=False, max_excluded=0.0,
                   max_loose=0.0, label=""):
    """Compare GPU pixel values g (P, 10) with the oracle's record chk
    (Oracle.render_checked on the same pixels).

    Every pixel is compared with the oracle's correct results: the one with
    every threshold decision taken the FP64 way and, where decisions were
    ambiguous, each listed variant; the pixel passes if one of them matches
    in every channel within max_abs beyond the oracle's conditioning
    tolerance.  Pixels that met more ambiguous decisions than the oracle
    enumerates are excluded and counted (at most max_excluded of them).
    Pixels whose stop point the oracle cannot place (conditioning errors
    larger than T_min: the stop's effect is in the tolerance and the
    contributor count is not compared) are counted too (at most max_loose).
    mean_abs bounds the per-channel mean of the excess.  check_nc: the
    matching result must also have the GPU's contributor count (up to the
    oracle's faint decisions, tol[:, 9]).  Returns a report with the measured
    fractions (widened: a channel's tolerance above max_abs)."""
    out, tol, flags, var = chk["out"], chk["tol"], chk["flags"], chk["variants"]
    P = len(out)
    e = _excess(g, out, tol)
    nc_ok = np.ones(P, bool)
    if check_nc:
        # the matching result's contributor count, up to its faint decisions
        nc_ok = np.abs(g[:, 9] - out[:, 9]) <= tol[:, 9]
    for r, V in var.items():
        ev = _excess(g[r][None], V[:, :10], V[:, 10:])
        score = ev.max(1)
        if check_nc:
            score = np.where(np.abs(V[:, 9] - g[r, 9]) <= V[:, 19], score, np.inf)
        k = int(np.argmin(score))
        e[r] = ev[k]
        nc_ok[r] = np.isfinite(score[k])
    excluded = (flags & 2) != 0
    comp = ~excluded
    ex = np.maximum(e[comp], 0.0)
    report = {"pixels": P, "excluded_frac": float(excluded.mean()) if P else 0.0,
              "ambiguous_frac": float(((flags & 1) != 0).mean()) if P else 0.0,
              "loose_frac": float(((flags & 4) != 0).mean()) if P else 0.0,
              "widened_frac": float((tol[:, :8].max(1) > max_abs).mean()) if P else 0.0}
    for c, name in enumerate(CHANNELS):
        col = ex[:, c]
        report[name] = (float(col.max()) if col.size else 0.0, float(col.mean()) if col.size else 0.0)
    print(f"[parity {label}] " + " ".join(f"{k}={v}" for k, v in report.items()), flush=True)
    assert report["excluded_frac"] <= max_excluded, ("excluded", report["excluded_frac"], max_excluded)
    assert report["loose_frac"] <= max_loose, ("loose", report["loose_frac"], max_loose)
    for c, name in enumerate(CHANNELS):
        mx, mn = report[name]
        if mx > max_abs:
            bad = np.nonzero(comp)[0][int(np.argmax(ex[:, c]))]
            raise AssertionError((label, name, mx, "pixel", chk["pixels"][bad].tolist(), "gpu", g[bad].tolist(),
                                  "oracle", out[bad].tolist(), "flags", int(flags[bad])))
        assert mn <= mean_abs, (label, name, mn)
    if check_nc:
        bad = comp & ~nc_ok
        assert not bad.any(), (label, "n_contrib", int(bad.sum()), chk["pixels"][np.nonzero(bad)[0][:5]].tolist())
    return report


def assert_images_match(gpu, orc, max_abs=IMG_MAX_ABS, mean_abs=IMG_MEAN_ABS, max_excluded=0.0, check_nc=False,
                        max_loose=0.0, label=""):
    """Full-frame comparison: gpu maps against the oracle's render_maps()."""
    chk = orc["checked"]
    g = gpu_pixels(gpu, chk["pixels"])
    return compare_pixels(g, chk, max_abs, mean_abs, check_nc=check_nc, max_excluded=max_excluded,
                          max_loose=max_loose, label=label)


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
