"""Parity at the full workload sizes, in the launch configuration bench.py
times: the 3M-primitive 1600x1064 scene (forward + backward) and the stress
workload (6M primitives, 90% surfels, heavy-tailed scales, 3840x2160).

The oracle cannot render or sort these in full, so the checks are:
  * contract outputs (depth key, tile rectangle, tiles touched) bit-exact for
    every primitive, and every tile's list length;
  * complete sorted lists, bit-exact, for sampled tiles (the oracle builds a
    tile's list from the rectangles and sorts it by (depth bits, id));
  * images on sampled pixels rendered by the FP64 oracle;
  * gradients against FP64 central finite differences of the oracle for
    sampled primitives (only the pixels of each primitive's tiles change).
"""
import numpy as np
import pytest
import torch

import synthetic as S
from gpu_util import CFG, IMG_MAX_ABS, IMG_MEAN_ABS
from oracle import native as O
from paper_2512_02932_gb300 import Rasterizer, SceneTensors

pytestmark = pytest.mark.gpu


def _tile_counts(rect, touched, TX, TY):
    """Instances per tile from the rectangles (2D difference array)."""
    D = np.zeros((TY + 1, TX + 1), np.int64)
    ok = touched > 0
    r = rect[ok]
    np.add.at(D, (r[:, 2], r[:, 0]), 1)
    np.add.at(D, (r[:, 2], r[:, 1] + 1), -1)
    np.add.at(D, (r[:, 3] + 1, r[:, 0]), -1)
    np.add.at(D, (r[:, 3] + 1, r[:, 1] + 1), 1)
    return D.cumsum(0).cumsum(1)[:TY, :TX].reshape(-1)


def _oracle_tile_list(db, rect, touched, t, TX):
    tx, ty = t % TX, t // TX
    m = (touched > 0) & (rect[:, 0] <= tx) & (tx <= rect[:, 1]) & (rect[:, 2] <= ty) & (ty <= rect[:, 3])
    ids = np.nonzero(m)[0]
    order = np.lexsort((ids, db[ids]))
    return ids[order].astype(np.uint32)


def _check_lists(r, scene, cam, n_tiles_sample, seed):
    db, rect, touched = O.contract_bin(scene, cam, CFG)
    n = scene.n
    g_db = r.depth_key[:n].cpu().numpy().view(np.uint32)
    g_touched = r.touched[:n].cpu().numpy().view(np.uint32).astype(np.int64)
    g_rect = r.rect[:n].cpu().numpy().view(np.uint16).astype(np.int32)
    np.testing.assert_array_equal(g_touched, touched)
    b = touched > 0
    np.testing.assert_array_equal(g_db[b], db[b])
    np.testing.assert_array_equal(g_rect[b], rect[b])
    TX, TY = (cam.width + 15) // 16, (cam.height + 15) // 16
    counts = _tile_counts(rect, touched, TX, TY)
    ranges = r.ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    np.testing.assert_array_equal(ranges[:, 1] - ranges[:, 0], counts)
    K = int(r.d_count.item())
    assert K == int(touched.sum())
    rng = np.random.default_rng(seed)
    nonempty = np.nonzero(counts > 0)[0]
    pick = np.unique(np.concatenate([rng.choice(nonempty, n_tiles_sample, replace=False),
                                     nonempty[[0, -1]], [int(np.argmax(counts))]]))
    for t in pick:
        s, e = ranges[t]
        got = r.vals[s:e].cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(got, _oracle_tile_list(db, rect, touched, t, TX))
    return db, rect, touched, K


def _check_pixels(out, scene, cam, npix, seed, orc=None, max_amb=0.05):
    rng = np.random.default_rng(seed)
    pix = np.stack([rng.integers(0, cam.width, npix), rng.integers(0, cam.height, npix)], 1)
    orc = orc or O.Oracle(scene, cam, CFG)
    o, amb = orc.render(pix)
    ok = ~amb
    # dense scenes: every pixel meets hundreds of pairs before it terminates,
    # so a few percent of pixels hold one inside a band (or, with the stress
    # workload's unclipped scales, an ill-conditioned ribbon)
    assert amb.mean() < max_amb, amb.mean()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    x, y = pix[:, 0], pix[:, 1]
    cols = {"rgb": [g["rgb"][c][y, x] for c in range(3)], "depth": [g["depth"][y, x]],
            "normal": [g["normal"][c][y, x] for c in range(3)], "alpha": [g["alpha"][y, x]]}
    ref = {"rgb": [o[:, c] for c in range(3)], "depth": [o[:, 3]],
           "normal": [o[:, 4 + c] for c in range(3)], "alpha": [o[:, 7]]}
    for k in cols:
        for gc, rc in zip(cols[k], ref[k]):
            d = np.abs(gc.astype(np.float64) - rc)[ok]
            if k == "depth":  # unnormalised depth: bounds relative to max(1, |depth|)
                d = d / np.maximum(1.0, np.abs(rc[ok]))
            print(f"{k}: max {d.max():.2e} mean {d.mean():.2e} (ambiguous {amb.mean():.4f})")
            assert d.max() <= IMG_MAX_ABS, (k, d.max())
            assert d.mean() <= IMG_MEAN_ABS, (k, d.mean())
    return orc


def _fd_check(scene, cam, r, st, orc, rect, touched, n_prims, seed, max_tiles=6, rgb_only=False):
    """GPU gradients of L = sum(cot * outputs) against FP64 central
    differences of the oracle, for sampled primitives and parameters.
    rgb_only: the loss sees the rgb map only (the image-loss backward)."""
    rng = np.random.default_rng(seed)
    TX = (cam.width + 15) // 16
    cand = np.nonzero((touched > 0) & (touched <= max_tiles))[0]
    prims = rng.choice(cand, n_prims, replace=False)
    # pixels of each primitive's tiles; union for the ambiguity scan
    def tile_pixels(i):
        tx0, tx1, ty0, ty1 = rect[i]
        ys, xs = np.mgrid[ty0 * 16:min((ty1 + 1) * 16, cam.height), tx0 * 16:min((tx1 + 1) * 16, cam.width)]
        return np.stack([xs.ravel(), ys.ravel()], 1).astype(np.int32)
    pix_of = {int(i): tile_pixels(i) for i in prims}
    allpix = np.unique(np.concatenate(list(pix_of.values())), axis=0)
    _, amb = orc.render(allpix)
    cot = S.random_cotangents(seed + 1, cam.height, cam.width)
    if rgb_only:
        for k in ("depth", "normal", "alpha"):
            cot[k] = np.zeros_like(cot[k])
    for k in cot:
        m = cot[k] if cot[k].ndim == 2 else cot[k]
        if m.ndim == 2:
            m[allpix[amb, 1], allpix[amb, 0]] = 0.0
        else:
            m[:, allpix[amb, 1], allpix[amb, 0]] = 0.0
    t = {k: torch.from_numpy(v).cuda() for k, v in cot.items()}
    if rgb_only:
        grads = r.backward(t["rgb"], None, None, None)
    else:
        grads = r.backward(t["rgb"], t["depth"], t["normal"], t["alpha"])
    torch.cuda.synchronize()
    r.check()
    G = {k: v.cpu().numpy() for k, v in grads.items()}

    def loss(out, pix):
        x, y = pix[:, 0], pix[:, 1]
        return (sum((out[:, c] * cot["rgb"][c][y, x]).sum() for c in range(3))
                + (out[:, 3] * cot["depth"][y, x]).sum()
                + sum((out[:, 4 + c] * cot["normal"][c][y, x]).sum() for c in range(3))
                + (out[:, 7] * cot["alpha"][y, x]).sum())

    checked = skipped = 0
    errs = []
    for i in prims:
        i = int(i)
        pix = pix_of[i]
        base = {"means": scene.means[i].astype(np.float64), "log_scales": scene.log_scales[i].astype(np.float64),
                "quats": scene.quats[i].astype(np.float64), "sh": scene.sh[i].astype(np.float64),
                "opacity_logits": float(scene.opacity_logits[i])}
        fields = ["means", "log_scales", "quats", "opacity_logits", "sh"]
        for fname in rng.choice(fields, 3, replace=False):
            if fname == "opacity_logits":
                comp = ()
            elif fname == "sh":
                comp = (int(rng.integers(scene.sh.shape[1])), int(rng.integers(3)))
            else:
                hi = 2 if (fname == "log_scales" and scene.types[i] == 0) else base[fname].shape[0]
                comp = (int(rng.integers(hi)),)
            h = 1e-5
            Ls, ncs = [], []
            for sgn in (1.0, -1.0):
                p = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in base.items()}
                if fname == "opacity_logits":
                    p[fname] += sgn * h
                else:
                    p[fname][comp] += sgn * h
                orc.set_prim(i, p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["sh"],
                             scene.types[i])
                out, _ = orc.render(pix)
                Ls.append(loss(out, pix))
                ncs.append(out[:, 9].copy())
            orc.set_prim(i, base["means"], base["log_scales"], base["quats"], base["opacity_logits"],
                         base["sh"], scene.types[i])
            if not np.array_equal(ncs[0], ncs[1]):
                skipped += 1
                continue
            fd = (Ls[0] - Ls[1]) / (2 * h)
            g = float(G[fname][i] if fname == "opacity_logits" else G[fname][i][comp])
            errs.append((fname, fd, g))
            checked += 1
    fd = np.array([e[1] for e in errs])
    g = np.array([e[2] for e in errs])
    scale = np.sqrt(np.mean(fd ** 2))
    bad = np.abs(g - fd) > 1e-3 * np.abs(fd) + 1e-3 * scale
    assert checked >= 0.9 * (checked + skipped) and checked > 0.5 * 3 * n_prims
    assert np.linalg.norm(g - fd) <= 1e-3 * np.linalg.norm(fd), np.linalg.norm(g - fd) / np.linalg.norm(fd)
    assert not bad.any(), [errs[k] for k in np.nonzero(bad)[0][:5]]
    return checked


def test_scene_scale_3m_fwd_bwd():
    scene, cam = S.scene_scale()
    r = Rasterizer("cuda", keep_keys=False)
    st = SceneTensors.from_numpy(scene)
    out = r.forward(st, cam, CFG)
    torch.cuda.synchronize()
    r.check()
    db, rect, touched, K = _check_lists(r, scene, cam, n_tiles_sample=40, seed=0)
    assert K > 20_000_000
    orc = _check_pixels(out, scene, cam, npix=3000, seed=1)
    _fd_check(scene, cam, r, st, orc, rect, touched, n_prims=60, seed=2)
    _fd_check(scene, cam, r, st, orc, rect, touched, n_prims=30, seed=3, rgb_only=True)


def test_stress_6m_4k_fwd_bwd():
    scene, cam = S.stress_scene()
    r = Rasterizer("cuda", keep_keys=False)
    st = SceneTensors.from_numpy(scene)
    out = r.forward(st, cam, CFG)
    torch.cuda.synchronize()
    r.check()
    db, rect, touched, K = _check_lists(r, scene, cam, n_tiles_sample=12, seed=3)
    assert K > 1_000_000_000
    orc = _check_pixels(out, scene, cam, npix=1000, seed=4, max_amb=0.10)
    _fd_check(scene, cam, r, st, orc, rect, touched, n_prims=20, seed=5, max_tiles=4)
