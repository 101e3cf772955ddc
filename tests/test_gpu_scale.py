"""Parity at the full workload sizes, in the launch configuration bench.py
times: the 3M-primitive 1600x1064 scene (forward + backward) and the stress
workload (6M primitives, 90% surfels, heavy-tailed scales, 3840x2160).

The oracle cannot render these frames in full, so the checks are:
  * contract outputs (depth key, tile rectangle, tiles touched) bit-exact for
    every primitive; at 3M the complete sorted list and the tile ranges
    bit-exact (the oracle sorts every instance); at the stress size every
    tile's list length and the complete lists of sampled tiles;
  * images on sampled pixels against every correct result the FP64 oracle
    lists for them (ambiguous threshold decisions enumerated, conditioning
    tolerance carried through Eq. 2);
  * gradients against FP64 central finite differences of the oracle, for
    thousands of primitives at 3M and a stratified sample of small, medium
    and screen-sized splats at the stress size.  Each primitive gets its own
    cotangent: random values on a few pixels where it contributes and zero
    elsewhere, so a central difference re-renders only those pixels however
    large the footprint.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from gpu_util import CFG, compare_pixels, gpu_pixels
from oracle import native as O
from paper_2512_02932_gb300 import Rasterizer, SceneTensors

pytestmark = pytest.mark.gpu

FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")


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


def _check_contract(r, scene, cam):
    db, rect, touched = O.contract_bin(scene, cam, CFG)
    n = scene.n
    g_db = r.depth_key[:n].cpu().numpy().view(np.uint32)
    g_touched = r.touched[:n].cpu().numpy().view(np.uint32).astype(np.int64)
    g_rect = r.rect[:n].cpu().numpy().view(np.uint16).astype(np.int32)
    np.testing.assert_array_equal(g_touched, touched)
    b = touched > 0
    np.testing.assert_array_equal(g_db[b], db[b])
    np.testing.assert_array_equal(g_rect[b], rect[b])
    return db, rect, touched


def _check_full_lists(r, scene, cam):
    """Every instance of the frame, bit for bit: sorted values and ranges."""
    keys, vals, ranges, (db, rect, touched) = O.tile_lists(scene, cam, CFG)
    K = int(r.d_count.item())
    assert K == len(vals)
    np.testing.assert_array_equal(r.vals[:K].cpu().numpy().view(np.uint32), vals)
    np.testing.assert_array_equal(r.ranges.cpu().numpy().view(np.uint32), ranges)
    return db, rect, touched, K


def _check_sampled_lists(r, scene, cam, db, rect, touched, n_tiles_sample, seed):
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
    return K


def _check_pixels(out, scene, cam, npix, seed, orc, max_excluded, label, max_loose=0.0):
    rng = np.random.default_rng(seed)
    pix = np.stack([rng.integers(0, cam.width, npix), rng.integers(0, cam.height, npix)], 1).astype(np.int32)
    chk = orc.render_checked(pix)
    g = gpu_pixels(out, pix)
    return compare_pixels(g, chk, check_nc=True, max_excluded=max_excluded, max_loose=max_loose, label=label)


# ---------------------------------------------------------------------------
# finite differences, one primitive at a time
# ---------------------------------------------------------------------------
def _fd_pixels(orc, cam, i, rect, rng, per_prim, cand_max=2048):
    """Up to per_prim pixels where primitive i contributes and the oracle's
    result is unambiguous (one correct result, a conditioning tolerance
    under 1e-4), and an oracle finite-difference session on them."""
    tx0, tx1, ty0, ty1 = rect
    x0, x1 = tx0 * 16, min((tx1 + 1) * 16, cam.width)
    y0, y1 = ty0 * 16, min((ty1 + 1) * 16, cam.height)
    npx = (x1 - x0) * (y1 - y0)
    if npx <= cand_max:
        ys, xs = np.mgrid[y0:y1, x0:x1]
        cand = np.stack([xs.ravel(), ys.ravel()], 1)
    else:
        cand = np.unique(np.stack([rng.integers(x0, x1, cand_max), rng.integers(y0, y1, cand_max)], 1), axis=0)
    cand = np.ascontiguousarray(cand, np.int32)
    ag = orc.pair_alpha(i, cand)
    hit = cand[ag >= CFG.alpha_min * 1.01]
    if len(hit) == 0:
        return hit, None
    hit = np.ascontiguousarray(hit[rng.permutation(len(hit))[:3 * per_prim]])
    with orc.fd_session(i, hit) as fd:
        _, amb, tol = fd.render(with_tol=True)
    good = ~amb & (tol[:, :8].max(1) < 1e-4)
    pix = np.ascontiguousarray(hit[good][:per_prim])
    return pix, (orc.fd_session(i, pix) if len(pix) else None)


class _FD:
    """Central differences of the oracle against the GPU gradient, for one
    primitive and one sparse cotangent at a time."""

    def __init__(self, scene, cam, r, orc, rgb_only):
        self.scene, self.cam, self.r, self.orc = scene, cam, r, orc
        self.rgb_only = rgb_only
        H, W, d = cam.height, cam.width, r.device
        self.cot = {"rgb": torch.zeros((3, H, W), device=d), "depth": torch.zeros((H, W), device=d),
                    "normal": torch.zeros((3, H, W), device=d), "alpha": torch.zeros((H, W), device=d)}
        n, nb = scene.n, scene.sh.shape[1]
        self.grads = {"means": torch.empty((n, 3), device=d), "log_scales": torch.empty((n, 3), device=d),
                      "quats": torch.empty((n, 4), device=d), "opacity_logits": torch.empty(n, device=d),
                      "sh": torch.empty((n, nb, 3), device=d)}
        self.records = []   # (field, fd, gpu)
        self.skipped = 0

    def _loss(self, out, c):
        return float(np.sum(out[:, :8] * c))

    def prim(self, i, pix, fd, rng, n_params):
        sc = self.scene
        P = len(pix)
        c = rng.normal(size=(P, 8))
        if self.rgb_only:
            c[:, 3:] = 0.0
        x, y = torch.from_numpy(pix[:, 0]).long(), torch.from_numpy(pix[:, 1]).long()
        ct = torch.from_numpy(c.astype(np.float32)).to(self.r.device)
        for k in self.cot.values():
            k.zero_()
        for ch in range(3):
            self.cot["rgb"][ch, y, x] = ct[:, ch]
            self.cot["normal"][ch, y, x] = ct[:, 4 + ch]
        self.cot["depth"][y, x] = ct[:, 3]
        self.cot["alpha"][y, x] = ct[:, 7]
        c = ct.double().cpu().numpy()   # the float32 values the GPU sees
        if self.rgb_only:
            self.r.backward(self.cot["rgb"], None, None, None, grads=self.grads)
        else:
            self.r.backward(self.cot["rgb"], self.cot["depth"], self.cot["normal"], self.cot["alpha"],
                            grads=self.grads)
        G = {k: v[i].double().cpu().numpy() for k, v in self.grads.items()}
        base = {k: getattr(sc, k)[i].astype(np.float64) for k in ("means", "log_scales", "quats", "sh")}
        base["opacity_logits"] = float(sc.opacity_logits[i])
        params = [(f, ()) for f in ("opacity_logits",)]
        params += [(f, (k,)) for f, m in (("means", 3), ("log_scales", 3), ("quats", 4)) for k in range(m)]
        params += [("sh", (a, b)) for a in range(sc.sh.shape[1]) for b in range(3)]
        if n_params < len(params):
            params = [params[k] for k in rng.choice(len(params), n_params, replace=False)]
        h = 1e-5
        for fname, comp in params:
            Ls, ncs = [], []
            for sgn in (1.0, -1.0):
                p = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in base.items()}
                if fname == "opacity_logits":
                    p[fname] += sgn * h
                else:
                    p[fname][comp] += sgn * h
                self.orc.set_prim(i, p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["sh"],
                                  sc.types[i])
                out, amb = fd.render()
                Ls.append(self._loss(out, c))
                ncs.append((out[:, 9].copy(), amb.copy()))
            self.orc.set_prim(i, base["means"], base["log_scales"], base["quats"], base["opacity_logits"],
                              base["sh"], sc.types[i])
            if not (np.array_equal(ncs[0][0], ncs[1][0]) and not ncs[0][1].any() and not ncs[1][1].any()):
                self.skipped += 1   # a decision changed inside the step: the difference is not a derivative
                continue
            fd = (Ls[0] - Ls[1]) / (2 * h)
            g = float(G[fname] if fname == "opacity_logits" else G[fname][comp])
            self.records.append((fname, fd, g))

    def assert_ok(self, min_checks):
        checked = len(self.records)
        assert checked >= min_checks, (checked, min_checks)
        assert checked >= 0.9 * (checked + self.skipped), (checked, self.skipped)
        rep = {}
        for fname in FIELDS:
            rows = [(fd, g) for f, fd, g in self.records if f == fname]
            if not rows:
                continue
            fd = np.array([a for a, _ in rows])
            g = np.array([b for _, b in rows])
            rms = np.sqrt(np.mean(fd ** 2))
            rel = np.linalg.norm(g - fd) / max(np.linalg.norm(fd), 1e-300)
            bad = np.abs(g - fd) > 1e-3 * np.abs(fd) + 1e-3 * rms
            rep[fname] = (len(rows), float(rel), int(bad.sum()))
            assert rel <= 1e-3, (fname, rel)
            assert not bad.any(), (fname, [rows[k] for k in np.nonzero(bad)[0][:5]])
        print(f"[fd] checks {checked} skipped {self.skipped} " +
              " ".join(f"{k}: n={v[0]} rel={v[1]:.2e}" for k, v in rep.items()), flush=True)
        return rep


def _fd_run(scene, cam, r, orc, rect, prims, n_full, per_prim, seed, rgb_only_every=2, min_frac=0.5):
    """All parameters for the first n_full primitives, 5 random ones for the
    rest; every rgb_only_every-th primitive with an rgb-only cotangent (the
    image-loss backward), the others with all four maps."""
    rng = np.random.default_rng(seed)
    fds = [_FD(scene, cam, r, orc, rgb_only=False), _FD(scene, cam, r, orc, rgb_only=True)]
    used = np.zeros(len(prims), bool)
    for k, i in enumerate(prims):
        i = int(i)
        pix, fd = _fd_pixels(orc, cam, i, rect[i], rng, per_prim)
        if len(pix) == 0:
            continue
        used[k] = True
        with fd:
            fds[1 if k % rgb_only_every == 0 else 0].prim(i, pix, fd, rng, 59 if k < n_full else 5)
    torch.cuda.synchronize()
    r.check()
    assert used.mean() >= min_frac, (int(used.sum()), len(prims))
    for f in fds:
        f.assert_ok(min_checks=1)
    return used, sum(len(f.records) for f in fds)


def test_scene_scale_3m_fwd_bwd():
    scene, cam = S.scene_scale()
    r = Rasterizer("cuda", keep_keys=False)
    st = SceneTensors.from_numpy(scene)
    out = r.forward(st, cam, CFG)
    torch.cuda.synchronize()
    r.check()
    _check_contract(r, scene, cam)
    db, rect, touched, K = _check_full_lists(r, scene, cam)
    assert K > 20_000_000
    orc = O.Oracle(scene, cam, CFG)
    # measured on this scene: no pixel excluded, none with an unplaceable stop
    _check_pixels(out, scene, cam, npix=4000, seed=1, orc=orc, max_excluded=0.0, label="3M scene")
    # 2,000 primitives: all 59 parameters for 200 of them, 5 for the rest
    rng = np.random.default_rng(2)
    binned = np.nonzero(touched > 0)[0]
    prims = rng.choice(binned, 2000, replace=False)
    used, checks = _fd_run(scene, cam, r, orc, rect, prims, n_full=200, per_prim=12, seed=3, min_frac=0.8)
    assert checks >= 0.8 * (200 * 59 + 1800 * 5), checks


def test_stress_6m_4k_fwd_bwd():
    scene, cam = S.stress_scene()
    r = Rasterizer("cuda", keep_keys=False)
    st = SceneTensors.from_numpy(scene)
    out = r.forward(st, cam, CFG)
    torch.cuda.synchronize()
    r.check()
    db, rect, touched = _check_contract(r, scene, cam)
    K = _check_sampled_lists(r, scene, cam, db, rect, touched, n_tiles_sample=12, seed=3)
    assert K > 1_000_000_000
    orc = O.Oracle(scene, cam, CFG)
    # measured on this scene: no pixel excluded; 8.9% whose stop point the
    # conditioning errors of its ribbons leave unplaceable (compared with the
    # stop's effect in the tolerance, contributor count unchecked)
    _check_pixels(out, scene, cam, npix=2000, seed=4, orc=orc, max_excluded=0.0, max_loose=0.18, label="stress")
    # stratified: screen-sized splats (the mask path), medium and small ones
    rng = np.random.default_rng(5)
    strata = [(touched > 256, 64), ((touched > 16) & (touched <= 256), 64), ((touched > 0) & (touched <= 16), 96)]
    picks = [rng.choice(np.nonzero(m)[0], k, replace=False) for m, k in strata]
    # interleave the strata so the 20 full-parameter primitives span all three
    order = np.argsort(np.concatenate([np.arange(len(p)) / len(p) for p in picks]), kind="stable")
    prims = np.concatenate(picks)[order]
    stratum = np.concatenate([np.full(len(p), j) for j, p in enumerate(picks)])[order]
    used, checks = _fd_run(scene, cam, r, orc, rect, prims, n_full=20, per_prim=8, seed=6, min_frac=0.6)
    assert (used & (stratum == 0)).sum() >= 50 and (used & (stratum == 1)).sum() >= 50, \
        [(int((used & (stratum == j)).sum())) for j in range(3)]
    assert checks >= 0.6 * (20 * 59 + 204 * 5), checks
