"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
not by the oracle itself.  CPU only."""
import math

import numpy as np
import pytest

import synthetic as S
from oracle import autograd_ref as AR
from oracle import native as O

CFG = S.RenderConfig()


def one_prim_scene(mean, log_scales, quat, logit, rgb=(0.8, 0.4, 0.2), type_=1, deg=0):
    k = (deg + 1) ** 2
    sh = np.zeros((1, k, 3), np.float32)
    sh[0, 0, :] = (np.asarray(rgb) - 0.5) / (0.5 / math.sqrt(math.pi))
    return S.Scene(np.array([mean], np.float32), np.array([log_scales], np.float32),
                   np.array([quat], np.float32), np.array([logit], np.float32), sh,
                   np.array([type_], np.uint8), deg)


def cat_scenes(scenes):
    return S.Scene(*(np.concatenate([getattr(s, f) for s in scenes]) for f in
                     ("means", "log_scales", "quats", "opacity_logits", "sh", "types")),
                   scenes[0].sh_degree)


def pixel_centres(cam):
    yy, xx = np.mgrid[0:cam.height, 0:cam.width]
    return xx + 0.5, yy + 0.5


# ---------------------------------------------------------------------------
# contract exp / log against libm (error bound, not self-consistency)
# ---------------------------------------------------------------------------
def test_contract_exp_log_accuracy():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(-87, 88, 4000), rng.uniform(-1, 1, 2000),
                         [0.0, 1.0, -1.0, 0.5, -87.0, 88.0]]).astype(np.float32)
    for x in xs:
        got = O.contract_exp(x)
        ref = math.exp(float(x))
        assert abs(got - ref) <= 4 * np.spacing(np.float32(ref)), (x, got, ref)
    ys = np.concatenate([rng.uniform(1, 255, 4000), np.exp(rng.uniform(-30, 30, 2000)),
                         [1.0, 2.0, 255.0, math.sqrt(2)]]).astype(np.float32)
    for y in ys:
        got = O.contract_log(y)
        ref = math.log(float(y))
        # absolute bound near 1 (log -> 0), relative elsewhere
        assert abs(got - ref) <= 4 * np.spacing(np.float32(max(abs(ref), 1e-3))) + 2e-8, (y, got, ref)
    assert O.contract_exp(0.0) == 1.0 and O.contract_log(1.0) == 0.0


# ---------------------------------------------------------------------------
# SH basis: scipy's complex harmonics and orthonormality
# ---------------------------------------------------------------------------
def _scipy_real_sh(deg, dirs):
    from scipy.special import sph_harm_y
    theta = np.arccos(np.clip(dirs[:, 2], -1, 1))
    phi = np.mod(np.arctan2(dirs[:, 1], dirs[:, 0]), 2 * np.pi)
    cols = []
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                cols.append(math.sqrt(2) * Y.real)
            elif m < 0:
                cols.append(math.sqrt(2) * Y.imag)
            else:
                cols.append(Y.real)
    return np.stack(cols, 1)


def test_sh_basis_matches_scipy_and_is_orthonormal():
    rng = np.random.default_rng(1)
    d = rng.normal(size=(500, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ref = _scipy_real_sh(3, d)
    c_basis = O.sh_basis(3, d)
    import torch
    t_basis = AR.sh_basis(3, torch.tensor(d)).numpy()
    np.testing.assert_allclose(c_basis, ref, atol=1e-12)
    np.testing.assert_allclose(t_basis, ref, atol=1e-12)
    # orthonormality on the sphere: Gauss-Legendre in cos(theta) x uniform phi
    xg, wg = np.polynomial.legendre.leggauss(16)
    nphi = 32
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(xg, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None]).reshape(-1)
    B = O.sh_basis(3, dirs)
    G = (B * w[:, None]).T @ B
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
def test_isotropic_3d_gaussian_closed_form():
    """On the optical axis at depth z with isotropic scale s the EWA
    covariance is (f s / z)^2 I exactly (App. C, Eq. 13), so each pixel is
    alpha exp(-r^2 / (2 sigma^2)) up to the 1/255 cutoff (Sec. 3.1)."""
    cam = S.pinhole(96, 96, 60.0)
    z, s, logit = 3.0, 0.05, 1.2
    sc = one_prim_scene((0.0, 0.0, z), (math.log(s),) * 3, (1, 0, 0, 0), logit)
    m = O.Oracle(sc, cam, CFG).render_maps()
    X, Y = pixel_centres(cam)
    sig = cam.fx * np.float64(np.float32(s)) / z
    # exp(log s) in float32 -> double: use the same s the oracle sees
    s64 = math.exp(float(np.float32(math.log(s))))
    sig = cam.fx * s64 / z
    r2 = (X - cam.cx) ** 2 + (Y - cam.cy) ** 2
    alpha = 1 / (1 + math.exp(-float(np.float32(logit))))
    a = alpha * np.exp(-r2 / (2 * sig ** 2))
    a = np.where(a >= CFG.alpha_min, np.minimum(a, CFG.alpha_max), 0.0)
    assert not m["amb"].any()
    np.testing.assert_allclose(m["alpha"], a, atol=1e-12)
    np.testing.assert_allclose(m["depth"], a * z, atol=1e-12)
    col = 0.5 + (0.5 / math.sqrt(math.pi)) * float(np.float32((0.8 - 0.5) / (0.5 / math.sqrt(math.pi))))
    np.testing.assert_allclose(m["rgb"][0], a * col, atol=1e-12)
    # isotropic: the normal is the z axis (tie rule) facing the camera
    np.testing.assert_allclose(m["normal"][2], -a, atol=1e-12)


@pytest.mark.parametrize("twist", [0.0, 0.7])
def test_face_on_surfel_closed_form(twist):
    """A surfel facing the camera at depth z: the ray through pixel p meets the
    plane at ((p-c) z / f); (u, v) are that point in the splat's frame divided
    by (s_u, s_v) (App. C), so d = u^2 + v^2 in closed form per axis."""
    cam = S.pinhole(80, 64, 55.0)
    z, su, sv, logit = 2.5, 0.08, 0.03, 2.0
    cx0, cy0 = 0.1, -0.05
    q = (math.cos(twist / 2), 0.0, 0.0, math.sin(twist / 2))
    sc = one_prim_scene((cx0, cy0, z), (math.log(su), math.log(sv), S.SURFEL_LOG_SZ), q, logit, type_=0)
    m = O.Oracle(sc, cam, CFG).render_maps()
    X, Y = pixel_centres(cam)
    mu = sc.means[0].astype(np.float64)
    PX = (X - cam.cx) / cam.fx * mu[2] - mu[0]
    PY = (Y - cam.cy) / cam.fy * mu[2] - mu[1]
    q64 = sc.quats[0].astype(np.float64)
    q64 /= np.linalg.norm(q64)
    ang = 2 * math.atan2(q64[3], q64[0])
    u = (math.cos(ang) * PX + math.sin(ang) * PY) / math.exp(float(sc.log_scales[0, 0]))
    v = (-math.sin(ang) * PX + math.cos(ang) * PY) / math.exp(float(sc.log_scales[0, 1]))
    alpha = 1 / (1 + math.exp(-float(sc.opacity_logits[0])))
    a = alpha * np.exp(-0.5 * (u * u + v * v))
    a = np.where(a >= CFG.alpha_min, np.minimum(a, CFG.alpha_max), 0.0)
    ok = ~m["amb"]
    assert ok.mean() > 0.99
    np.testing.assert_allclose(m["alpha"][ok], a[ok], atol=1e-12)
    np.testing.assert_allclose(m["depth"][ok], (a * mu[2])[ok], atol=1e-11)
    np.testing.assert_allclose(m["normal"][2][ok], -a[ok], atol=1e-12)


def test_edge_on_surfel_vanishes():
    """A surfel whose plane contains the camera centre: every ray meets the
    plane at the camera centre (depth 0) or lies in it, so the contribution is
    exactly zero everywhere."""
    cam = S.pinhole(64, 64, 60.0)
    # plane x = 0 (normal along x): local z axis -> world x
    q = (math.cos(math.pi / 4), 0.0, math.sin(math.pi / 4), 0.0)
    sc = one_prim_scene((0.0, 0.05, 3.0), (math.log(0.5), math.log(0.5), S.SURFEL_LOG_SZ), q, 3.0, type_=0)
    m = O.Oracle(sc, cam, CFG).render_maps()
    assert np.all(m["alpha"] == 0.0) and np.all(m["rgb"] == 0.0)
    # same splat rotated a little: now visible
    q2 = (math.cos(math.pi / 4 - 0.05), 0.0, math.sin(math.pi / 4 - 0.05), 0.0)
    sc2 = one_prim_scene((0.0, 0.05, 3.0), (math.log(0.5), math.log(0.5), S.SURFEL_LOG_SZ), q2, 3.0, type_=0)
    assert O.Oracle(sc2, cam, CFG).render_maps()["alpha"].max() > 0.5


def test_3d_converges_to_surfel_when_fronto_parallel():
    """A fronto-parallel 3D Gaussian whose z scale tends to 0 renders as the
    surfel with the same parameters: on a plane of constant depth the affine
    projection is exact.  Off the optical axis the difference is O(s_z^2)."""
    cam = S.pinhole(96, 80, 60.0)
    mean, q = (0.35, -0.2, 3.0), (math.cos(0.3), 0.0, 0.0, math.sin(0.3))
    ls = [math.log(0.06), math.log(0.025), 0.0]
    diffs = []
    for sz in (1e-2, 1e-3, 1e-4):
        ls[2] = math.log(sz)
        g3 = O.Oracle(one_prim_scene(mean, ls, q, 1.5, type_=1), cam, CFG).render_maps()
        g2 = O.Oracle(one_prim_scene(mean, ls, q, 1.5, type_=0), cam, CFG).render_maps()
        ok = ~(g3["amb"] | g2["amb"])
        diffs.append(np.abs(g3["alpha"] - g2["alpha"])[ok].max())
    assert diffs[-1] < 1e-6
    assert diffs[0] > diffs[1] > diffs[2]


def test_oblique_flat_gaussian_differs_from_surfel_except_at_centre():
    """The affine projection distorts everywhere except at the centre
    (Sec. 3.1): an oblique flat 3D Gaussian and the surfel with the same
    parameters agree at the centre pixel and differ around it."""
    cam = S.pinhole(128, 128, 70.0)
    z = 2.0
    # centre projects exactly onto the centre of pixel (70, 58)
    px, py = 70.5, 58.5
    mean = ((px - cam.cx) / cam.fx * z, (py - cam.cy) / cam.fy * z, z)
    mean = tuple(float(np.float32(v)) for v in mean)
    ang = 1.1  # strong tilt about the x axis
    q = (math.cos(ang / 2), math.sin(ang / 2), 0.0, 0.0)
    ls = (math.log(0.25), math.log(0.25), math.log(1e-6))
    g3 = O.Oracle(one_prim_scene(mean, ls, q, 2.0, type_=1), cam, CFG).render_maps()
    g2 = O.Oracle(one_prim_scene(mean, ls, q, 2.0, type_=0), cam, CFG).render_maps()
    assert abs(g3["alpha"][58, 70] - g2["alpha"][58, 70]) < 1e-6
    assert np.abs(g3["alpha"] - g2["alpha"]).max() > 0.05


def test_bruteforce_blend_eq2():
    """Eq. 2 enumerated term by term, C = sum_i c_i a_i prod_{j<i}(1 - a_j),
    over up to 8 face-on surfels with closed-form contributions, sorted by
    depth; no transmittance termination is reached."""
    cam = S.pinhole(16, 16, 60.0)
    rng = np.random.default_rng(5)
    prims, closed = [], []
    X, Y = pixel_centres(cam)
    for i in range(8):
        z = 2.0 + 0.25 * i
        mu = (rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), z)
        s = (rng.uniform(0.1, 0.3), rng.uniform(0.1, 0.3))
        logit = rng.uniform(-1.5, 0.0)
        rgb = rng.uniform(0, 1, 3)
        sc = one_prim_scene(mu, (math.log(s[0]), math.log(s[1]), S.SURFEL_LOG_SZ), (1, 0, 0, 0), logit, rgb, type_=0)
        prims.append(sc)
        m = sc.means[0].astype(np.float64)
        u = ((X - cam.cx) / cam.fx * m[2] - m[0]) / math.exp(float(sc.log_scales[0, 0]))
        v = ((Y - cam.cy) / cam.fy * m[2] - m[1]) / math.exp(float(sc.log_scales[0, 1]))
        a = (1 / (1 + math.exp(-float(sc.opacity_logits[0])))) * np.exp(-0.5 * (u * u + v * v))
        a = np.where(a >= CFG.alpha_min, np.minimum(a, CFG.alpha_max), 0.0)
        col = 0.5 + (0.5 / math.sqrt(math.pi)) * sc.sh[0, 0].astype(np.float64)
        closed.append((z, a, col))
    order = rng.permutation(8)
    scene = cat_scenes([prims[i] for i in order])
    m = O.Oracle(scene, cam, CFG).render_maps()
    closed.sort(key=lambda t: t[0])
    C = np.zeros((3, 16, 16))
    for i, (z, a, col) in enumerate(closed):
        trans = np.ones((16, 16))
        for j in range(i):
            trans = trans * (1 - closed[j][1])
        C += col[:, None, None] * a * trans
    assert not m["amb"].any()
    np.testing.assert_allclose(m["rgb"], C, atol=1e-12)


def test_order_of_input_invariance():
    sc, cam = S.tiny_scene(0)
    m0 = O.Oracle(sc, cam, CFG).render_maps()
    perm = np.random.default_rng(9).permutation(sc.n)
    m1 = O.Oracle(sc.subset(perm), cam, CFG).render_maps()
    ok = ~(m0["amb"] | m1["amb"])
    for k in ("rgb", "depth", "normal", "alpha"):
        np.testing.assert_allclose(m0[k][..., ok], m1[k][..., ok], atol=1e-13)
    # the contract's lists are identical up to the relabelling
    k0, v0, r0, _ = O.tile_lists(sc, cam, CFG)
    k1, v1, r1, _ = O.tile_lists(sc.subset(perm), cam, CFG)
    np.testing.assert_array_equal(k0, k1)
    np.testing.assert_array_equal(r0, r1)
    np.testing.assert_array_equal(v0, perm[v1])


def test_torch_formulation_matches_c_oracle():
    """Two independent FP64 formulations of the same image function."""
    sc, cam = S.tiny_scene(0)
    m = O.Oracle(sc, cam, CFG).render_maps()
    r = AR.render(sc, cam, CFG)
    H, W = cam.height, cam.width
    np.testing.assert_allclose(r["rgb"].detach().numpy().T.reshape(3, H, W), m["rgb"], atol=1e-12)
    np.testing.assert_allclose(r["depth"].detach().numpy().reshape(H, W), m["depth"], atol=1e-12)
    np.testing.assert_allclose(r["normal"].detach().numpy().T.reshape(3, H, W), m["normal"], atol=1e-12)
    np.testing.assert_allclose(r["alpha"].detach().numpy().reshape(H, W), m["alpha"], atol=1e-12)


def _set_pairs(sc, cam):
    """(primitive, tile) pairs of the contract's tile sets, encoded
    primitive * tiles + tile, sorted."""
    db, rect, touched, rowp = O.contract_bin(sc, cam, CFG, with_rowp=True)
    tiles, _ = O.contract_tiles(rect, rowp, touched, cam.width)
    ntiles = ((cam.width + 15) // 16) * ((cam.height + 15) // 16)
    prim = np.repeat(np.arange(sc.n), touched)
    return np.sort(prim.astype(np.int64) * ntiles + tiles), ntiles, rect, touched


def _assert_sets_hold_contributions(sc, cam, min_pairs):
    """Every (pixel, primitive) pair whose FP64 contribution clears the 1/255
    threshold outside the ambiguity band lies in a tile of the primitive's
    FP32 tile set (and so of its rectangle)."""
    enc, ntiles, rect, touched = _set_pairs(sc, cam)
    yy, xx = np.mgrid[0:cam.height, 0:cam.width]
    pix = np.stack([xx.ravel(), yy.ravel()], 1)
    araw, ok = AR.pair_alpha(sc, cam, CFG, pix)
    sure = ok & (araw >= CFG.alpha_min * (1 + 2e-4))
    p_idx, g_idx = np.nonzero(sure)
    tx = pix[p_idx, 0] // CFG.tile
    ty = pix[p_idx, 1] // CFG.tile
    TX = (cam.width + 15) // 16
    r = rect[g_idx]
    inside = (r[:, 0] <= tx) & (tx <= r[:, 1]) & (r[:, 2] <= ty) & (ty <= r[:, 3])
    assert inside.all(), np.count_nonzero(~inside)
    want = g_idx.astype(np.int64) * ntiles + ty * TX + tx
    pos = np.searchsorted(enc, want)
    found = (pos < len(enc)) & (enc[np.minimum(pos, len(enc) - 1)] == want)
    assert found.all(), np.count_nonzero(~found)
    assert len(p_idx) > min_pairs
    return enc, touched


def test_contract_is_conservative():
    """Tile sets and rectangles hold every contributing pair (tiny scenes)."""
    for seed in (0, 1):
        sc, cam = S.tiny_scene(seed)
        _assert_sets_hold_contributions(sc, cam, 1000)


def test_tile_sets_are_conservative_for_needles():
    """Heavy-tailed scales (needles and ribbons at every angle, both types):
    the tile sets still hold every contributing pair, and drop most of the
    rectangles' tiles."""
    rng = np.random.default_rng(21)
    n = 400
    means = np.stack([rng.uniform(-0.8, 0.8, n), rng.uniform(-0.6, 0.6, n), rng.uniform(2.0, 4.0, n)], 1)
    ls = rng.normal(-3.0, 0.3, (n, 3)) + np.where(rng.random((n, 3)) < 0.3, rng.uniform(1.0, 2.5, (n, 3)), 0.0)
    types = (rng.random(n) < 0.5).astype(np.uint8)
    ls[types == 0, 2] = S.SURFEL_LOG_SZ
    q = rng.normal(size=(n, 4))
    sh = np.zeros((n, 1, 3))
    scene = S.Scene(means.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                    rng.normal(1.5, 1.0, n).astype(np.float32), sh.astype(np.float32), types, 0)
    cam = S.pinhole(160, 128, 60.0)
    enc, touched = _assert_sets_hold_contributions(scene, cam, 5000)
    db, rect, _ = O.contract_bin(scene, cam, CFG)
    b = touched > 0
    area = (rect[b, 1] - rect[b, 0] + 1) * (rect[b, 3] - rect[b, 2] + 1)
    assert np.all(touched[b] <= area)
    assert touched.sum() < 0.8 * area.sum(), (touched.sum(), area.sum())


def test_tile_set_of_a_disc_is_its_tile_rows_chords():
    """An isotropic 3D Gaussian facing the camera: its footprint is a disc of
    radius R = sqrt(dmax) sigma_px, and row ty of its tile set must cover the
    tiles the disc's chord over that tile row reaches (pixel centres), and
    no tile beyond the chord of radius R (1 + 2^-9) + 1/16."""
    cam = S.pinhole(320, 256, 60.0)
    for (x, y, logit, ls) in [(0.05, -0.03, 2.0, -2.2), (-0.31, 0.2, 0.3, -2.6), (0.0, 0.0, 4.0, -1.9)]:
        z = 3.0
        scene = S.Scene(np.array([[x, y, z]], np.float32), np.full((1, 3), ls, np.float32),
                        np.array([[1, 0, 0, 0]], np.float32), np.array([logit], np.float32),
                        np.zeros((1, 1, 3), np.float32), np.ones(1, np.uint8), 0)
        db, rect, touched, rowp = O.contract_bin(scene, cam, CFG, with_rowp=True)
        tiles, _ = O.contract_tiles(rect, rowp, touched, cam.width)
        TX = (cam.width + 15) // 16
        alpha = 1.0 / (1.0 + np.exp(-logit))
        R = np.sqrt(2.0 * np.log(alpha / CFG.alpha_min)) * np.exp(ls) * cam.fx / z
        cx, cy = cam.fx * x / z + cam.cx, cam.fy * y / z + cam.cy
        got = {}
        for t in tiles:
            got.setdefault(int(t) // TX, []).append(int(t) % TX)

        def chord_tiles(rad, ty):
            # pixel centres (i + 0.5, j + 0.5) of tile row ty within radius rad
            ys = np.arange(16 * ty, 16 * ty + 16) + 0.5
            xs = np.arange(cam.width) + 0.5
            inside = (xs[None] - cx) ** 2 + (ys[:, None] - cy) ** 2 <= rad * rad
            cols = np.nonzero(inside.any(0))[0]
            return set((cols // 16).tolist())

        rows = range(int(rect[0, 2]), int(rect[0, 3]) + 1)
        for ty in rows:
            lo = chord_tiles(R * (1 - 1e-6), ty)
            hi = chord_tiles(R * (1 + 2 ** -9) + 1 / 16, ty)
            have = set(got.get(ty, []))
            assert lo <= have <= hi, (ty, sorted(lo), sorted(have), sorted(hi))


def test_contract_is_conservative_for_surfels_reaching_the_near_plane():
    """Large surfels whose discs cross the near plane take the contract's
    extent bound (contributing hits need depth > near); it must still cover
    every contributing pair."""
    rng = np.random.default_rng(8)
    n = 300
    means = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.4, 0.4, n), rng.uniform(0.22, 1.2, n)], 1)
    ls = np.stack([rng.normal(-1.2, 0.4, n), rng.normal(-1.2, 0.4, n), np.full(n, S.SURFEL_LOG_SZ)], 1)
    q = rng.normal(size=(n, 4))
    sh = np.zeros((n, 1, 3))
    scene = S.Scene(means.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                    rng.normal(1.0, 1.0, n).astype(np.float32), sh.astype(np.float32),
                    np.zeros(n, np.uint8), 0)
    cam = S.pinhole(96, 80, 70.0)
    enc, touched = _assert_sets_hold_contributions(scene, cam, 1000)
    # the branch is exercised: many discs reach the near plane, and their
    # tile sets (disc mode) drop part of their rectangles
    m = means.astype(np.float64)
    assert (m[:, 2] - 3 * np.exp(ls[:, :2]).max(1) < CFG.near).sum() > 30
    db, rect, _, rowp = O.contract_bin(scene, cam, CFG, with_rowp=True)
    disc = (touched > 0) & (rowp[:, 11] == 2)
    area = (rect[:, 1] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 2] + 1)
    assert disc.sum() > 30 and touched[disc].sum() < 0.9 * area[disc].sum()


def test_disc_mode_tile_sets_of_large_near_surfels():
    """Large surfels crossing the near plane at every orientation, seen over
    a wider frame: every contributing pair lies in the disc-mode tile set,
    which keeps well under the rectangles' tiles."""
    rng = np.random.default_rng(12)
    n = 120
    means = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.5, 0.5, n), rng.uniform(0.25, 1.5, n)], 1)
    ls = np.stack([rng.normal(-0.3, 0.5, n), rng.normal(-1.5, 1.0, n), np.full(n, S.SURFEL_LOG_SZ)], 1)
    q = rng.normal(size=(n, 4))
    sh = np.zeros((n, 1, 3))
    scene = S.Scene(means.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                    rng.normal(1.0, 1.0, n).astype(np.float32), sh.astype(np.float32),
                    np.zeros(n, np.uint8), 0)
    cam = S.pinhole(320, 224, 70.0)
    enc, touched = _assert_sets_hold_contributions(scene, cam, 20000)
    db, rect, _, rowp = O.contract_bin(scene, cam, CFG, with_rowp=True)
    disc = (touched > 0) & (rowp[:, 11] == 2)
    area = (rect[:, 1] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 2] + 1)
    assert disc.sum() > 40 and touched[disc].sum() < 0.7 * area[disc].sum(), (disc.sum(), touched[disc].sum(),
                                                                              area[disc].sum())


def test_tile_list_structure():
    sc, cam = S.tiny_scene(2)
    keys, vals, ranges, (db, rect, touched) = O.tile_lists(sc, cam, CFG)
    assert len(keys) == touched.sum()
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)
    TX = (cam.width + 15) // 16
    for t in range(len(ranges)):
        s, e = ranges[t]
        assert np.all((keys[s:e] >> np.uint64(32)) == t)
        d = (keys[s:e] & np.uint64(0xffffffff)).view(np.uint64)
        assert np.all(d == db[vals[s:e]])
        tx, ty = t % TX, t // TX
        rr = rect[vals[s:e]]
        assert np.all((rr[:, 0] <= tx) & (tx <= rr[:, 1]) & (rr[:, 2] <= ty) & (ty <= rr[:, 3]))
    # every binned primitive is listed touched times, once per tile of its set
    assert np.array_equal(np.bincount(vals, minlength=sc.n), touched)


def test_contract_depth_order_matches_fp64_depth():
    sc, cam = S.tiny_scene(3)
    db, _, _ = O.contract_bin(sc, cam, CFG)
    z32 = db.view(np.float32).astype(np.float64)
    z64 = sc.means.astype(np.float64) @ np.asarray(cam.R, np.float64)[2] + float(cam.t[2])
    np.testing.assert_allclose(z32, z64, rtol=2e-7)


# ---------------------------------------------------------------------------
# scale modulation of 2D Gaussians (Sec. 3.2, Eqs. 6-7)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("sz,lam,theta,Tz", [
    (0.9, 1.0, 1.05, 1e-3),    # gate closed: alpha unchanged
    (1.2, 1.0, 1.05, 1e-3),    # gate open: alpha * exp(-s_z)
    (1.05, 1.7, 1.05, 0.1),    # gate at one half, lambda_z != 1
    (1.10, 2.3, 1.05, 0.05),   # gate sigmoid(1)
    (0.95, 0.6, 1.05, 0.08),   # gate sigmoid(-1.25)
])
def test_scale_modulation_closed_form(sz, lam, theta, Tz):
    """A face-on surfel whose buffered s_z sits anywhere around theta_z: every
    pixel is the face-on closed form with alpha replaced by
    alpha * exp(-lambda_z * sigmoid((s_z - theta_z) / T_z) * s_z)."""
    import dataclasses
    cfg = dataclasses.replace(CFG, lambda_z=lam, theta_z=theta, T_z=Tz)
    cam = S.pinhole(64, 48, 55.0)
    z, su, sv, logit = 2.0, 0.07, 0.05, 2.5
    sc = one_prim_scene((0.05, -0.02, z), (math.log(su), math.log(sv), math.log(sz)), (1, 0, 0, 0), logit,
                        type_=0)
    m = O.Oracle(sc, cam, cfg).render_maps()
    X, Y = pixel_centres(cam)
    mu = sc.means[0].astype(np.float64)
    u = ((X - cam.cx) / cam.fx * mu[2] - mu[0]) / math.exp(float(sc.log_scales[0, 0]))
    v = ((Y - cam.cy) / cam.fy * mu[2] - mu[1]) / math.exp(float(sc.log_scales[0, 1]))
    s_z = math.exp(float(sc.log_scales[0, 2]))
    gate = 1.0 / (1.0 + math.exp(-(s_z - theta) / Tz))
    alpha = 1 / (1 + math.exp(-float(sc.opacity_logits[0]))) * math.exp(-lam * gate * s_z)
    a = alpha * np.exp(-0.5 * (u * u + v * v))
    a = np.where(a >= cfg.alpha_min, np.minimum(a, cfg.alpha_max), 0.0)
    ok = ~m["amb"]
    assert ok.mean() > 0.99
    np.testing.assert_allclose(m["alpha"][ok], a[ok], atol=1e-12)
    # the torch formulation agrees with the C oracle on the same config
    r = AR.render(sc, cam, cfg)
    np.testing.assert_allclose(r["alpha"].detach().numpy().reshape(cam.height, cam.width)[ok], a[ok], atol=1e-12)


def test_scale_modulation_leaves_3d_gaussians_alone():
    """Eqs. 6-7 act on 2D Gaussians only: a 3D Gaussian with s_z above
    theta_z renders the same with and without the modulation."""
    import dataclasses
    cam = S.pinhole(48, 48, 60.0)
    sc = one_prim_scene((0.0, 0.0, 4.0), (math.log(0.08), math.log(0.05), math.log(1.3)), (0.9, 0.1, 0.2, 0.3),
                        1.0, type_=1)
    m0 = O.Oracle(sc, cam, dataclasses.replace(CFG, lambda_z=0.0)).render_maps()
    m1 = O.Oracle(sc, cam, dataclasses.replace(CFG, lambda_z=2.0, T_z=0.1)).render_maps()
    assert m0["alpha"].max() > 0.3
    np.testing.assert_array_equal(m0["alpha"], m1["alpha"])


@pytest.mark.parametrize("sz,lam,Tz", [(1.05, 1.7, 0.1), (1.12, 0.8, 0.05), (0.97, 2.0, 0.04)])
def test_scale_modulation_gradient_closed_form(sz, lam, Tz):
    """d alpha_pix / d log s_z of Eqs. 6-7 in closed form at pixels of a
    face-on surfel: with g = sigmoid((s - theta)/T) and s = exp(l),
    d alpha* / d l = -lambda alpha* s (g + s g (1 - g) / T), and alpha_pix =
    alpha* exp(-d/2) below the clamp.  The torch formulation's autograd must
    reproduce it."""
    import dataclasses
    cfg = dataclasses.replace(CFG, lambda_z=lam, theta_z=1.05, T_z=Tz)
    cam = S.pinhole(32, 32, 55.0)
    sc = one_prim_scene((0.0, 0.0, 2.0), (math.log(0.15), math.log(0.12), math.log(sz)), (1, 0, 0, 0), 0.3,
                        type_=0)
    cot = {"rgb": np.zeros((3, 32, 32)), "depth": np.zeros((32, 32)), "normal": np.zeros((3, 32, 32)),
           "alpha": np.zeros((32, 32))}
    pix = [(16, 16), (18, 15), (13, 19)]
    for (x, y) in pix:
        cot["alpha"][y, x] = 1.0
    out, grads = AR.vjp(sc, cam, cfg, cot)
    s = math.exp(float(sc.log_scales[0, 2]))
    g = 1.0 / (1.0 + math.exp(-(s - 1.05) / Tz))
    dlog = -lam * s * (g + s * g * (1.0 - g) / Tz)
    expect = sum(out["alpha"][y, x] for (x, y) in pix) * dlog
    assert all(0.0 < out["alpha"][y, x] < CFG.alpha_max for (x, y) in pix)
    assert abs(grads["log_scales"][0, 2] - expect) <= 1e-10 * abs(expect)
    # and the C oracle's central difference
    orc = O.Oracle(sc, cam, cfg)
    h = 1e-6
    vals = []
    for sgn in (1, -1):
        ls = sc.log_scales[0].astype(np.float64).copy()
        ls[2] += sgn * h
        orc.set_prim(0, sc.means[0].astype(np.float64), ls, sc.quats[0].astype(np.float64),
                     float(sc.opacity_logits[0]), sc.sh[0].astype(np.float64), 0)
        o, _ = orc.render(np.array(pix, np.int32))
        vals.append(o[:, 7].sum())
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - expect) <= 1e-6 * abs(expect)


# ---------------------------------------------------------------------------
# view-dependent colour (Sec. 3.1): degree-1 SH in closed form
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("az", [0.0, 35.0, 160.0])
def test_sh_degree1_view_direction_closed_form(az):
    """Colour at degree 1 is 0.5 + C0 f_0 + k1 (-f_{1,-1} d_y + f_{1,0} d_z -
    f_{1,1} d_x), k1 = sqrt(3 / 4 pi), with d the unit vector from the camera
    centre to the primitive's mean in world coordinates.  An isotropic 3D
    Gaussian at the world origin seen from an orbiting camera: the centre
    pixel's rgb divided by its alpha is that colour, and a flipped view
    direction would move every odd-degree term's sign."""
    cam = S.orbit_camera(az, 25.0, 3.0, 33, 33, 40.0)
    sc = one_prim_scene((0.0, 0.0, 0.0), (math.log(0.1),) * 3, (1, 0, 0, 0), 1.0, type_=1, deg=1)
    f = np.array([[0.2, -0.1, 0.3], [0.5, 0.25, -0.4], [-0.3, 0.6, 0.15], [0.35, -0.45, 0.2]], np.float32)
    sc.sh[0] = f
    m = O.Oracle(sc, cam, CFG).render_maps()
    R = np.asarray(cam.R, np.float64)
    t = np.asarray(cam.t, np.float64)
    centre = -R.T @ t
    d = (np.zeros(3) - centre)
    d /= np.linalg.norm(d)
    k0, k1 = 0.5 / math.sqrt(math.pi), math.sqrt(3.0 / (4.0 * math.pi))
    f64 = f.astype(np.float64)
    col = 0.5 + k0 * f64[0] + k1 * (-f64[1] * d[1] + f64[2] * d[2] - f64[3] * d[0])
    col = np.maximum(col, 0.0)
    cy, cx = 16, 16
    a = m["alpha"][cy, cx]
    assert a > 0.3
    np.testing.assert_allclose(m["rgb"][:, cy, cx] / a, col, rtol=1e-12)
    # the sign matters: the opposite direction gives a different colour
    wrong = np.maximum(0.5 + k0 * f64[0] - k1 * (-f64[1] * d[1] + f64[2] * d[2] - f64[3] * d[0]), 0.0)
    assert np.abs(wrong - col).max() > 0.05
    r = AR.render(sc, cam, CFG, pixels=np.array([[cx, cy]]))
    np.testing.assert_allclose(r["rgb"].detach().numpy()[0] / r["alpha"].detach().numpy()[0], col, rtol=1e-12)


# ---------------------------------------------------------------------------
# ambiguous threshold decisions: every correct result is listed
# ---------------------------------------------------------------------------
def test_alpha_threshold_decision_lists_both_results():
    """An isotropic 3D Gaussian whose contribution at one pixel lies 1e-5
    (relative) above alpha_min: a binary32 evaluation may land on either side
    of the threshold, so the pixel has two correct results, with and without
    the pair (Sec. 3.1 contribution rule), and the renderer lists both."""
    cam = S.pinhole(48, 48, 60.0)
    z, s = 3.0, 0.1
    s64 = math.exp(float(np.float32(math.log(s))))
    sig = cam.fx * s64 / z
    px, py = 26, 24  # pixel centre (26.5, 24.5); the Gaussian sits at (24, 24)
    r2 = (px + 0.5 - cam.cx) ** 2 + (py + 0.5 - cam.cy) ** 2
    target = CFG.alpha_min * (1 + 1e-5)
    alpha = target * math.exp(r2 / (2 * sig ** 2))
    logit = float(np.float32(math.log(alpha / (1 - alpha))))
    sc = one_prim_scene((0.0, 0.0, z), (math.log(s),) * 3, (1, 0, 0, 0), logit)
    chk = O.Oracle(sc, cam, CFG).render_checked(np.array([[px, py], [24, 24]], np.int32))
    assert chk["flags"][0] & 1 and not chk["flags"][0] & 2
    assert not chk["flags"][1]
    v = chk["variants"][0]
    a_exact = (1 / (1 + math.exp(-logit))) * math.exp(-r2 / (2 * sig ** 2))
    assert abs(a_exact - CFG.alpha_min) < 1e-4 * CFG.alpha_min
    got = sorted(v[:, 7])
    assert len(v) == 2
    assert got[0] == 0.0 and abs(got[1] - a_exact) < 1e-15


def test_termination_decision_lists_both_results():
    """Two opaque face-on surfels at the same pixel: each contributes the clamp
    0.99, so the transmittance after the second is (0.01)^2 = T_min exactly and
    whether the pixel stops before it is ambiguous (Eq. 2 with the T_min
    rule): alpha is 0.99 or 0.9999."""
    cam = S.pinhole(32, 32, 60.0)
    prims = [one_prim_scene((0.0, 0.0, z), (math.log(3.0), math.log(3.0), S.SURFEL_LOG_SZ), (1, 0, 0, 0), 9.0,
                            type_=0) for z in (2.0, 2.5)]
    sc = cat_scenes(prims)
    chk = O.Oracle(sc, cam, CFG).render_checked(np.array([[16, 16]], np.int32))
    assert chk["flags"][0] & 1
    v = chk["variants"][0]
    np.testing.assert_allclose(sorted(v[:, 7]), [0.99, 1 - 0.01 ** 2], atol=1e-12)
    np.testing.assert_array_equal(sorted(v[:, 9]), [1, 2])
