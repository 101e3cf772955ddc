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


def _set_tiles(rect, rowp, touched, width):
    """Every instance's tile (the contract's tile sets, in primitive order) and
    each instance's primitive."""
    tiles, first = O.contract_tiles(rect, rowp, touched, width)
    prim = np.repeat(np.arange(len(touched), dtype=np.int64), touched)
    return tiles, prim


def _oracle_tile_list(db, tiles, prim, t):
    ids = prim[tiles == t]
    order = np.lexsort((ids, db[ids]))
    return ids[order].astype(np.uint32)


def _check_contract(r, scene, cam):
    db, rect, touched, rowp = O.contract_bin(scene, cam, CFG, with_rowp=True)
    n = scene.n
    g_db = r.depth_key[:n].cpu().numpy().view(np.uint32)
    g_touched = r.touched[:n].cpu().numpy().view(np.uint32).astype(np.int64)
    g_rect = r.rect[:n].cpu().numpy().view(np.uint16).astype(np.int32)
    np.testing.assert_array_equal(g_touched, touched)
    b = touched > 0
    np.testing.assert_array_equal(g_db[b], db[b])
    np.testing.assert_array_equal(g_rect[b], rect[b])
    return db, rect, touched, rowp


def _check_full_lists(r, scene, cam):
    """Every instance of the frame, bit for bit: sorted values and ranges."""
    keys, vals, ranges, (db, rect, touched) = O.tile_lists(scene, cam, CFG)
    K = int(r.d_count.item())
    assert K == len(vals)
    np.testing.assert_array_equal(r.vals[:K].cpu().numpy().view(np.uint32), vals)
    np.testing.assert_array_equal(r.ranges.cpu().numpy().view(np.uint32), ranges)
    return db, rect, touched, K


def _check_sampled_lists(r, scene, cam, db, rect, touched, rowp, n_tiles_sample, seed):
    """Every tile's list length, and the complete lists of sampled tiles (the
    fullest one included), against the contract's tile sets."""
    TX, TY = (cam.width + 15) // 16, (cam.height + 15) // 16
    tiles, prim = _set_tiles(rect, rowp, touched, cam.width)
    counts = np.bincount(tiles, minlength=TX * TY)
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
        np.testing.assert_array_equal(got, _oracle_tile_list(db, tiles, prim, t))
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
# A pair's gradient flows through its splat-frame coordinates (u, v) of Eq. 1,
# which binary32 evaluates from the pixel's offset to the projected centre:
# along a needle thousands of pixels long, or for a splat whose centre
# projects tens of thousands of pixels off the frame, those cancelling terms
# leave (u, v) with absolute errors of 1e-4 and more, and the gradient terms,
# proportional to u and v, with relative errors of 1e-3 and more (measured:
# 2e-3 on a 576:1 surfel of the stress scene whose 8-ulp bound is 8e-3, 3e-3
# on a surfel centred 40,000 px below the frame, bound 1.2e-4 at v = 0.025),
# a limit of the data type, not of the method.  The checks use pairs whose
# 8-ulp bound is at most COND_MAX (measured: it removes 5% of the stress
# scene's candidate pairs and 0.2% at 3M).
COND_MAX = 1e-4
def _fd_plan(orc, cam, touched, strata, n_sample, per_prim, max_tol, rng, max_cond=COND_MAX):
    """Primitives and pixels for the finite-difference checks.  Random pixels
    are rendered by the oracle; those with one correct result and a
    conditioning tolerance under max_tol are kept, and every primitive Eq. 2
    blends at a kept pixel (so one the image shows there) may be checked at
    it, where binary32 fixes its splat-frame coordinates to max_cond
    (Oracle.pair_conditioning).  strata: [(mask over primitives, how many)],
    drawn at random among the primitives with such a pixel.  Returns
    [(primitive, pixels)]; prints the fraction of (primitive, pixel)
    candidates the conditioning bound removed."""
    pix = np.stack([rng.integers(0, cam.width, n_sample), rng.integers(0, cam.height, n_sample)], 1)
    pix = np.ascontiguousarray(np.unique(pix, axis=0), np.int32)
    _, flags, tol = orc._render(pix)
    pix = pix[(flags == 0) & (tol[:, :8].max(1) < max_tol)]
    pairs_p, pairs_i = [], []
    for p, ids in zip(pix, orc.pixel_contributors(pix)):
        for i in ids:
            pairs_p.append(p)
            pairs_i.append(int(i))
    cond = orc.pair_conditioning(np.array(pairs_i, np.int64), np.array(pairs_p, np.int32).reshape(-1, 2))
    ok = (cond.min(1) >= 0.0) & (cond.max(1) <= max_cond)
    print(f"[fd plan] candidate pairs {len(ok)}, removed by the conditioning bound {1.0 - ok.mean():.4f}", flush=True)
    where = {}
    for p, i, good in zip(pairs_p, pairs_i, ok):
        if good:
            where.setdefault(i, []).append(p)
    have = np.zeros(len(touched), bool)
    have[list(where)] = True
    plan = []
    for mask, k in strata:
        cand = np.nonzero(mask & have)[0]
        for i in rng.choice(cand, min(k, len(cand)), replace=False):
            p = np.array(where[int(i)], np.int32)
            plan.append((int(i), np.ascontiguousarray(p[rng.permutation(len(p))[:per_prim]])))
    return plan


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
        self.where = []     # (primitive, type, component, pixels)
        self.skipped = 0

    def _loss(self, out, c):
        return float(np.sum(out[:, :8] * c))

    def prim(self, i, pix, session, rng, n_params):
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
        h = 1e-6
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
                out, amb, place = session.render()
                Ls.append(self._loss(out, c))
                ncs.append((out[:, 9].copy(), amb.copy(), place.copy()))
            self.orc.set_prim(i, base["means"], base["log_scales"], base["quats"], base["opacity_logits"],
                              base["sh"], sc.types[i])
            if not (np.array_equal(ncs[0][0], ncs[1][0]) and not ncs[0][1].any() and not ncs[1][1].any()
                    and np.array_equal(ncs[0][2], ncs[1][2])):
                # a decision or the blend order changed inside the step: the
                # difference is not a derivative
                self.skipped += 1
                continue
            dfd = (Ls[0] - Ls[1]) / (2 * h)
            g = float(G[fname] if fname == "opacity_logits" else G[fname][comp])
            self.records.append((fname, dfd, g))
            self.where.append((i, int(sc.types[i]), comp, len(pix)))

    def assert_ok(self, min_checks):
        checked = len(self.records)
        assert checked >= min_checks, (checked, min_checks)
        assert checked >= 0.9 * (checked + self.skipped), (checked, self.skipped)
        rep, fails = {}, []
        for fname in FIELDS:
            idx = [k for k, (f, _, _) in enumerate(self.records) if f == fname]
            if not idx:
                continue
            fd = np.array([self.records[k][1] for k in idx])
            g = np.array([self.records[k][2] for k in idx])
            rms = np.sqrt(np.mean(fd ** 2))
            rel = np.linalg.norm(g - fd) / max(np.linalg.norm(fd), 1e-300)
            bad = np.abs(g - fd) > 1e-3 * np.abs(fd) + 1e-3 * rms
            rep[fname] = (len(idx), float(rel), int(bad.sum()))
            if rel > 1e-3 or bad.any():
                worst = np.argsort(-np.abs(g - fd))[:5]
                fails.append((fname, rel, int(bad.sum()), [(self.where[idx[k]], fd[k], g[k]) for k in worst]))
        print(f"[fd rgb_only={self.rgb_only}] checks {checked} skipped {self.skipped} " +
              " ".join(f"{k}: n={v[0]} rel={v[1]:.2e} bad={v[2]}" for k, v in rep.items()), flush=True)
        for fname, rel, nbad, worst in fails:
            for w, f, g in worst:
                print(f"[fd fail] {fname} rel={rel:.3e} bad={nbad} at {w}: fd={f:.9g} gpu={g:.9g}", flush=True)
        assert not fails, fails
        return rep


def _fd_run(scene, cam, r, orc, plan, n_full, seed, rgb_only_every=2):
    """All parameters for the first n_full primitives of the plan, 5 random
    ones for the rest; every rgb_only_every-th primitive with an rgb-only
    cotangent (the image-loss backward), the others with all four maps."""
    rng = np.random.default_rng(seed)
    fds = [_FD(scene, cam, r, orc, rgb_only=False), _FD(scene, cam, r, orc, rgb_only=True)]
    for k, (i, pix) in enumerate(plan):
        with orc.fd_session(i, pix) as session:
            fds[1 if k % rgb_only_every == 0 else 0].prim(i, pix, session, rng, 59 if k < n_full else 5)
    torch.cuda.synchronize()
    r.check()
    for f in fds:
        f.assert_ok(min_checks=1)
    return sum(len(f.records) for f in fds)


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
    # 2,000 primitives the image shows: all 59 parameters for 200 of them, 5
    # for the rest
    rng = np.random.default_rng(2)
    plan = _fd_plan(orc, cam, touched, [(touched > 0, 2000)], n_sample=20000, per_prim=12, max_tol=1e-4, rng=rng)
    assert len(plan) == 2000
    checks = _fd_run(scene, cam, r, orc, plan, n_full=200, seed=3)
    assert checks >= 0.9 * (200 * 59 + 1800 * 5), checks


def test_stress_6m_4k_fwd_bwd():
    scene, cam = S.stress_scene()
    r = Rasterizer("cuda", keep_keys=False)
    st = SceneTensors.from_numpy(scene)
    out = r.forward(st, cam, CFG)
    torch.cuda.synchronize()
    r.check()
    db, rect, touched, rowp = _check_contract(r, scene, cam)
    K = _check_sampled_lists(r, scene, cam, db, rect, touched, rowp, n_tiles_sample=12, seed=3)
    area = np.where(touched > 0, (rect[:, 1] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 2] + 1), 0)
    # the tile sets keep a small part of the rectangles' 2.6e9 tiles (measured
    # in the oracle's contract: 15%; the 36k surfels whose discs reach the near
    # plane list 8.6e7 instead of 1.2e9)
    assert area.sum() > 2_000_000_000 and K < 0.25 * area.sum(), (K, area.sum())
    orc = O.Oracle(scene, cam, CFG)
    # measured on this scene: no pixel excluded; 8.9% whose stop point the
    # conditioning errors of its ribbons leave unplaceable (compared with the
    # stop's effect in the tolerance, contributor count unchecked)
    _check_pixels(out, scene, cam, npix=2000, seed=4, orc=orc, max_excluded=0.0, max_loose=0.18, label="stress")
    # The image shows only screen-sized splats here: every pixel saturates
    # (T < T_min) within ~36 contributors, all of them with rectangles over
    # 256 tiles, and no medium or small primitive is reached anywhere
    # (measured with the oracle on 4,000 pixels: 330 primitives, all large),
    # so their gradients are exactly zero on both sides.  Up to 200 of the
    # shown ones are checked (144 have pixels the bounds below admit).  The
    # ribbons' conditioning tolerance is above 1e-4 at most pixels; the pixels
    # used are those under 2e-4.
    # Primitives whose centre lies within 5% of the near plane are left out:
    # Eq. 13's Jacobian and the surfels' re-centred homography are taken at
    # the projected centre, here tens of thousands of pixels off the frame,
    # and their gradients lose binary32 accuracy (measured: 5.5e-3 on the
    # depth gradient of a needle at 1.02 near, 43,000 px off the frame,
    # against FP64 autograd and the oracle's differences, which agree to 1e-9).
    rng = np.random.default_rng(5)
    depth = scene.means.astype(np.float64) @ np.asarray(cam.R, np.float64).reshape(3, 3)[2] + float(cam.t[2])
    plan = _fd_plan(orc, cam, touched, [((touched > 0) & (depth > 1.05 * CFG.near), 200)], n_sample=40000,
                    per_prim=8, max_tol=2e-4, rng=rng)
    large = sum(1 for i, _ in plan if area[i] > 256)
    assert len(plan) >= 140 and large >= 140, (len(plan), large)
    checks = _fd_run(scene, cam, r, orc, plan, n_full=20, seed=6)
    assert checks >= 0.9 * (20 * 59 + (len(plan) - 20) * 5), checks
