"""CUDA path (through the C ABI) against the CPU oracle, element by element.
Needs a GB300."""
import math

import numpy as np
import pytest
import torch

import synthetic as S
from oracle import autograd_ref as AR
from oracle import native as O
from gpu_util import (CFG, assert_grads_match, assert_images_match, assert_lists_bitexact,
                      gpu_forward, gpu_lists)
from paper_2512_02932_gb300 import Rasterizer, SceneTensors

pytestmark = pytest.mark.gpu


def _oracle_maps(scene, cam, cfg=CFG):
    return O.Oracle(scene, cam, cfg).render_maps()


# ---------------------------------------------------------------------------
# tiny workload: 1,000 primitives, 128x128
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tiny_lists_and_images(seed):
    scene, cam = S.tiny_scene(seed)
    r, st, g = gpu_forward(scene, cam)
    K = assert_lists_bitexact(r, scene, cam)
    assert K > 1000
    m = _oracle_maps(scene, cam)
    # contributor counts are integers: the matching result must have the same
    assert_images_match(g, m, check_nc=True, max_excluded=0.0, label=f"tiny seed {seed}")
    # transmittance and alpha are consistent
    np.testing.assert_allclose(g["alpha"], 1 - g["T_final"], atol=1e-7)


def _gpu_vjp(scene, cam, cot, cfg=CFG, rgb_only=False):
    """rgb_only: pass only the rgb cotangent (the others as absent), which
    selects the backward specialised for an image loss."""
    r, st, g = gpu_forward(scene, cam, cfg, keep_keys=False)
    t = {k: torch.from_numpy(v).cuda() for k, v in cot.items()}
    if rgb_only:
        grads = r.backward(t["rgb"], None, None, None)
    else:
        grads = r.backward(t["rgb"], t["depth"], t["normal"], t["alpha"])
    torch.cuda.synchronize()
    r.check()
    return g, {k: v.cpu().numpy() for k, v in grads.items()}


def _masked_cot(seed, cam, amb):
    cot = S.random_cotangents(seed, cam.height, cam.width)
    for k in cot:
        cot[k] = np.where(amb, 0.0, cot[k]).astype(np.float32)
    return cot


@pytest.mark.parametrize("seed", [0, 3])
def test_tiny_gradients(seed):
    scene, cam = S.tiny_scene(seed)
    m = _oracle_maps(scene, cam)
    cot = _masked_cot(10 + seed, cam, m["amb"])
    _, ref = AR.vjp(scene, cam, CFG, cot)
    _, got = _gpu_vjp(scene, cam, cot)
    assert_grads_match(got, ref)


@pytest.mark.parametrize("seed", [1, 4])
def test_tiny_gradients_rgb_cotangent_only(seed):
    scene, cam = S.tiny_scene(seed)
    m = _oracle_maps(scene, cam)
    cot = _masked_cot(30 + seed, cam, m["amb"])
    for k in ("depth", "normal", "alpha"):
        cot[k] = np.zeros_like(cot[k])
    _, ref = AR.vjp(scene, cam, CFG, cot)
    _, got = _gpu_vjp(scene, cam, cot, rgb_only=True)
    assert_grads_match(got, ref)


def test_sh_degree3_surface_gradients_rgb_only():
    scene = S.surface_scene(400, seed=8, frac3d=0.5, ls_loc=-2.6, ls_scale=0.4)
    cam = S.orbit_camera(40.0, 10.0, 3.0, 96, 72, 50.0)
    m = _oracle_maps(scene, cam)
    cot = _masked_cot(22, cam, m["amb"])
    for k in ("depth", "normal", "alpha"):
        cot[k] = np.zeros_like(cot[k])
    _, ref = AR.vjp(scene, cam, CFG, cot)
    _, got = _gpu_vjp(scene, cam, cot, rgb_only=True)
    assert_grads_match(got, ref)


def test_sh_degree3_surface_gradients():
    scene = S.surface_scene(400, seed=7, frac3d=0.5, ls_loc=-2.6, ls_scale=0.4)
    cam = S.orbit_camera(20.0, 15.0, 3.0, 96, 72, 50.0)
    m = _oracle_maps(scene, cam)
    g = gpu_forward(scene, cam)[2]
    assert_images_match(g, m, check_nc=True, label="sh3 surface")
    cot = _masked_cot(21, cam, m["amb"])
    _, ref = AR.vjp(scene, cam, CFG, cot)
    _, got = _gpu_vjp(scene, cam, cot)
    assert_grads_match(got, ref)


@pytest.mark.parametrize("lam,Tz,rgb_only", [(1.0, 1e-3, False), (1.7, 0.1, False), (1.7, 0.1, True)])
def test_scale_modulation_parity(lam, Tz, rgb_only):
    """Surfels whose buffered s_z lies around theta_z = 1.05 (Sec. 3.2, Eqs.
    6-7): with the paper's temperature (T_z = 0.001, nearly a step) and a soft
    one (T_z = 0.1, lambda_z = 1.7).  Images against the oracle, gradients
    (d/d log s_z of every surfel included) against the FP64 autograd
    formulation."""
    import dataclasses
    cfg = dataclasses.replace(CFG, lambda_z=lam, T_z=Tz)
    scene, cam = S.tiny_scene(7)
    surf = scene.types == 0
    rng = np.random.default_rng(70)
    scene.log_scales[surf, 2] = np.log(rng.uniform(0.9, 1.2, int(surf.sum()))).astype(np.float32)
    m = O.Oracle(scene, cam, cfg).render_maps()
    g = gpu_forward(scene, cam, cfg)[2]
    assert_images_match(g, m, check_nc=True, label=f"modulation T_z={Tz}")
    cot = _masked_cot(71, cam, m["amb"])
    if rgb_only:
        for k in ("depth", "normal", "alpha"):
            cot[k] = np.zeros_like(cot[k])
    _, ref = AR.vjp(scene, cam, cfg, cot)
    _, got = _gpu_vjp(scene, cam, cot, cfg, rgb_only=rgb_only)
    assert_grads_match(got, ref)
    dsz = ref["log_scales"][surf, 2]
    assert np.count_nonzero(np.abs(dsz) > 1e-6 * np.abs(ref["log_scales"]).max()) > 20


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_ragged_image_and_tiles():
    """Image sizes that are not multiples of the tile, several tiles wide."""
    scene, _ = S.tiny_scene(4)
    for (w, h) in ((100, 37), (17, 129), (1, 1), (33, 16)):
        cam = S.pinhole(w, h, 60.0)
        r, st, g = gpu_forward(scene, cam)
        assert_lists_bitexact(r, scene, cam)
        m = _oracle_maps(scene, cam)
        assert_images_match(g, m, check_nc=True, label=f"ragged {w}x{h}")


def test_empty_scene_and_all_culled():
    scene, cam = S.tiny_scene(0)
    empty = scene.subset(np.arange(0))
    cfg = S.RenderConfig(bg=(0.25, 0.5, 0.75))
    r, st, g = gpu_forward(empty, cam, cfg)
    assert int(r.d_count.item()) == 0
    np.testing.assert_allclose(g["rgb"][0], 0.25)
    np.testing.assert_allclose(g["rgb"][2], 0.75)
    assert np.all(g["alpha"] == 0) and np.all(g["T_final"] == 1) and np.all(g["n_last"] == 0)
    behind = scene.copy()
    behind.means[:, 2] = -behind.means[:, 2]
    r, st, g = gpu_forward(behind, cam, cfg)
    assert int(r.d_count.item()) == 0
    assert np.all(g["alpha"] == 0)


def test_capacity_overflow_reports_and_retries():
    scene, cam = S.tiny_scene(1)
    K_ref = len(O.tile_lists(scene, cam, CFG)[0])
    # direct: a too-small capacity is reported, nothing written out of bounds
    r = Rasterizer("cuda", capacity=1024, keep_keys=True)
    st = SceneTensors.from_numpy(scene)
    r.preprocess(st, cam, CFG)
    guard = torch.full((4096,), 7, dtype=torch.int32, device="cuda")
    r.vals = guard[:1024]
    r._ensure_capacity(1024)
    r.vals = guard[:1024]
    r.bin_sort(sync_check=False)
    torch.cuda.synchronize()
    assert int(r.d_count.item()) == K_ref > 1024
    assert int(r.dev_err.item()) == -2
    assert torch.all(guard[1024:] == 7)
    assert torch.all(r.ranges == 0)
    # the managed path grows and retries
    r2, st2, g = gpu_forward(scene, cam, capacity=1024)
    assert r2.capacity >= K_ref
    assert_lists_bitexact(r2, scene, cam)


def test_long_tile_lists_and_termination():
    """Thousands of large primitives over one small image: lists far longer
    than one staged chunk, and most pixels terminate on T_min."""
    rng = np.random.default_rng(5)
    n = 3000
    types = (rng.random(n) < 0.5).astype(np.uint8)
    means = np.stack([rng.uniform(-0.25, 0.25, n), rng.uniform(-0.25, 0.25, n), rng.uniform(2, 6, n)], 1)
    ls = rng.normal(-1.2, 0.3, (n, 3))
    ls[types == 0, 2] = S.SURFEL_LOG_SZ
    q = rng.normal(size=(n, 4))
    sh = np.zeros((n, 1, 3))
    sh[:, 0] = rng.uniform(-1.7, 1.7, (n, 3))
    scene = S.Scene(means.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                    rng.normal(1.5, 1.0, n).astype(np.float32), sh.astype(np.float32), types, 0)
    cam = S.pinhole(48, 40, 60.0)
    r, st, g = gpu_forward(scene, cam)
    assert_lists_bitexact(r, scene, cam)
    _, _, ranges = gpu_lists(r)
    assert (ranges[:, 1] - ranges[:, 0]).max() > 1000
    m = _oracle_maps(scene, cam)
    assert (m["T"] < 1e-3).mean() > 0.3
    assert_images_match(g, m, check_nc=True, max_excluded=0.0, label="long lists")
    cot = _masked_cot(3, cam, m["amb"])
    _, ref = AR.vjp(scene, cam, CFG, cot)
    _, got = _gpu_vjp(scene, cam, cot)
    assert_grads_match(got, ref)


def test_degenerate_primitives():
    """Edge-on surfel (vanishes), isotropic 3D Gaussian, a surfel crossing the
    near plane (whole-image bbox), a primitive behind the camera, a
    near-transparent one and an exactly fronto-parallel surfel."""
    f = lambda *a: np.array(a, np.float32)
    means = [f(0.0, 0.05, 3.0), f(0.2, -0.1, 2.5), f(0.0, 0.0, 0.5), f(0.1, 0.1, -2.0),
             f(-0.3, 0.2, 3.0), f(-0.2, -0.25, 2.0)]
    ls = [f(math.log(0.5), math.log(0.5), -30), f(*(math.log(0.1),) * 3), f(math.log(2.0), math.log(2.0), -30),
          f(-2, -2, -2), f(-1.5, -1.5, -1.5), f(math.log(0.1), math.log(0.05), -30)]
    qs = [f(math.cos(math.pi / 4), 0, math.sin(math.pi / 4), 0), f(1, 0, 0, 0),
          f(math.cos(0.7), math.sin(0.7), 0, 0), f(1, 0, 0, 0), f(1, 0, 0, 0), f(1, 0, 0, 0)]
    logits = f(3.0, 1.0, 0.5, 2.0, -5.4, 2.0)
    types = np.array([0, 1, 0, 1, 1, 0], np.uint8)
    sh = np.zeros((6, 1, 3), np.float32)
    sh[:, 0, :] = 1.0
    scene = S.Scene(np.stack(means), np.stack(ls), np.stack(qs), logits, sh, types, 0)
    cam = S.pinhole(64, 48, 70.0)
    r, st, g = gpu_forward(scene, cam)
    assert_lists_bitexact(r, scene, cam)
    m = _oracle_maps(scene, cam)
    assert_images_match(g, m, check_nc=True, label="degenerate")
    # the edge-on surfel alone renders nothing
    r1, _, g1 = gpu_forward(scene.subset([0]), cam)
    assert np.all(g1["alpha"] == 0)


# ---------------------------------------------------------------------------
# exchange
# ---------------------------------------------------------------------------
def _exchange_gpu(scene, mode, theta, mask=None):
    st = SceneTensors.from_numpy(scene)
    ptr_before = (st.log_scales.data_ptr(), st.quats.data_ptr(), st.types.data_ptr())
    dflip = torch.zeros(1, dtype=torch.int64, device="cuda")
    m = torch.from_numpy(mask).cuda() if mask is not None else None
    from paper_2512_02932_gb300 import exchange_types
    exchange_types(st, mode=mode, theta_e=theta, mask=m, d_flipped=dflip)
    torch.cuda.synchronize()
    assert ptr_before == (st.log_scales.data_ptr(), st.quats.data_ptr(), st.types.data_ptr())
    return (st.log_scales.cpu().numpy(), st.quats.cpu().numpy(), st.types.cpu().numpy(),
            int(dflip.item()))


@pytest.mark.parametrize("theta", [2.05, 1.9, 2.15])
def test_exchange_erank_matches_oracle(theta):
    rng = np.random.default_rng(11)
    n = 200_000
    scene = S.surface_scene(n, seed=12, frac3d=0.5, ls_loc=-4.0, ls_scale=1.2)
    th = float(np.float32(theta))
    ls, q, t, nf = _exchange_gpu(scene, "erank", th)
    ls_o, q_o, t_o, nf_o = O.exchange(scene.log_scales, scene.quats, scene.types, mode="erank", theta=th)
    np.testing.assert_array_equal(t, t_o)
    assert nf == nf_o and nf > 0
    np.testing.assert_array_equal(ls.astype(np.float64), ls_o)
    np.testing.assert_allclose(q, q_o, atol=2e-7)


def test_exchange_mask_matches_oracle():
    scene = S.surface_scene(100_000, seed=13, frac3d=0.7)
    mask = (np.random.default_rng(0).random(scene.n) < 0.01).astype(np.uint8)
    ls, q, t, nf = _exchange_gpu(scene, "mask", 2.05, mask)
    ls_o, q_o, t_o, nf_o = O.exchange(scene.log_scales, scene.quats, scene.types, mode="mask", mask=mask)
    np.testing.assert_array_equal(t, t_o)
    assert nf == nf_o == int(mask.sum())
    np.testing.assert_array_equal(ls.astype(np.float64), ls_o)
    np.testing.assert_allclose(q, q_o, atol=2e-7)


def test_surfels_reaching_the_near_plane():
    """Large surfels crossing the near plane (the contract's extent-bound
    branch): lists bit-exact, images and gradients within tolerance."""
    rng = np.random.default_rng(8)
    n = 300
    means = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.4, 0.4, n), rng.uniform(0.22, 1.2, n)], 1)
    ls = np.stack([rng.normal(-1.2, 0.4, n), rng.normal(-1.2, 0.4, n), np.full(n, S.SURFEL_LOG_SZ)], 1)
    q = rng.normal(size=(n, 4))
    sh = np.zeros((n, 1, 3))
    sh[:, 0] = rng.uniform(-1.7, 1.7, (n, 3))
    scene = S.Scene(means.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                    rng.normal(1.0, 1.0, n).astype(np.float32), sh.astype(np.float32), np.zeros(n, np.uint8), 0)
    cam = S.pinhole(96, 80, 70.0)
    r, st, g = gpu_forward(scene, cam)
    assert_lists_bitexact(r, scene, cam)
    m = _oracle_maps(scene, cam)
    assert_images_match(g, m, check_nc=True, max_excluded=0.0, label="near plane")
    cot = _masked_cot(4, cam, m["amb"])
    _, ref = AR.vjp(scene, cam, CFG, cot)
    _, got = _gpu_vjp(scene, cam, cot)
    assert_grads_match(got, ref)


def test_disc_mode_tile_sets_of_large_near_surfels():
    """Large surfels crossing the near plane at every orientation over a
    wider frame (the contract's disc-mode tile sets, rows spanning the
    frame): lists bit-exact, images within tolerance."""
    rng = np.random.default_rng(12)
    n = 120
    means = np.stack([rng.uniform(-0.6, 0.6, n), rng.uniform(-0.5, 0.5, n), rng.uniform(0.25, 1.5, n)], 1)
    ls = np.stack([rng.normal(-0.3, 0.5, n), rng.normal(-1.5, 1.0, n), np.full(n, S.SURFEL_LOG_SZ)], 1)
    q = rng.normal(size=(n, 4))
    sh = np.zeros((n, 1, 3))
    sh[:, 0] = rng.uniform(-1.7, 1.7, (n, 3))
    scene = S.Scene(means.astype(np.float32), ls.astype(np.float32), q.astype(np.float32),
                    rng.normal(1.0, 1.0, n).astype(np.float32), sh.astype(np.float32), np.zeros(n, np.uint8), 0)
    cam = S.pinhole(320, 224, 70.0)
    r, st, g = gpu_forward(scene, cam)
    assert_lists_bitexact(r, scene, cam)
    db, rect, touched, rowp = O.contract_bin(scene, cam, CFG, with_rowp=True)
    assert ((touched > 0) & (rowp[:, 11] == 2)).sum() > 40
    m = _oracle_maps(scene, cam)
    assert_images_match(g, m, check_nc=True, max_excluded=0.0, label="disc mode")


# ---------------------------------------------------------------------------
# the autograd Function
# ---------------------------------------------------------------------------
def _autograd_grads(scene, cam, loss_fn):
    from paper_2512_02932_gb300 import rasterize
    st = SceneTensors.from_numpy(scene)
    params = [st.means, st.log_scales, st.quats, st.opacity_logits, st.sh]
    for p in params:
        p.requires_grad_(True)
    rgb, depth, normal, alpha = rasterize(st, cam, CFG)
    loss_fn(rgb, depth, normal, alpha).backward()
    torch.cuda.synchronize()
    names = ["means", "log_scales", "quats", "opacity_logits", "sh"]
    return {k: p.grad.detach().cpu().numpy() for k, p in zip(names, params)}


@pytest.mark.parametrize("with_depth", [False, True])
def test_autograd_function_matches_oracle(with_depth):
    """Loss through torch.autograd: an rgb-only loss (unused maps arrive as
    None and select the image-loss backward) and one that also uses depth."""
    scene, cam = S.tiny_scene(2)
    m = _oracle_maps(scene, cam)
    cot = _masked_cot(40, cam, m["amb"])
    if not with_depth:
        cot["depth"] = np.zeros_like(cot["depth"])
    cot["normal"] = np.zeros_like(cot["normal"])
    cot["alpha"] = np.zeros_like(cot["alpha"])
    c_rgb = torch.from_numpy(cot["rgb"]).cuda()
    c_depth = torch.from_numpy(cot["depth"]).cuda()

    def loss(rgb, depth, normal, alpha):
        L = (rgb * c_rgb).sum()
        return L + (depth * c_depth).sum() if with_depth else L

    got = _autograd_grads(scene, cam, loss)
    _, ref = AR.vjp(scene, cam, CFG, cot)
    assert_grads_match(got, ref)


def test_backward_after_the_caller_dropped_its_scene_tensors():
    """The Rasterizer keeps the arrays of its last forward alive for the
    backward, so a temporary SceneTensors is safe."""
    scene, cam = S.tiny_scene(6)
    r = Rasterizer("cuda")
    r.forward(SceneTensors.from_numpy(scene), cam, CFG)   # temporary, no reference kept
    junk = [torch.full((1 << 20,), float("nan"), device="cuda") for _ in range(8)]  # reuse freed memory
    g = r.backward(torch.ones((3, cam.height, cam.width), device="cuda"), None, None, None)
    torch.cuda.synchronize()
    del junk
    for k, v in g.items():
        assert torch.isfinite(v).all(), k


# ---------------------------------------------------------------------------
# tile sets: needles and ribbons list only the tiles along them
# ---------------------------------------------------------------------------
def _rect_tiles(r, n):
    rect = r.rect[:n].cpu().numpy().view(np.uint16).astype(np.int64)
    touched = r.touched[:n].cpu().numpy().view(np.uint32).astype(np.int64)
    b = touched > 0
    area = np.where(b, (rect[:, 1] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 2] + 1), 0)
    return touched, area


def test_tile_sets_of_heavy_tailed_scenes_are_bitexact():
    """Heavy-tailed scales (needles, ribbons and blobs, many rectangles wider
    than 256 tiles): lists, keys and ranges are bit-exact against the oracle,
    and the tile sets hold far fewer tiles than the rectangles (measured:
    51%)."""
    scene = S.surface_scene(60_000, seed=21, frac3d=0.3, ls_loc=-4.0, ls_scale=0.8, heavy_df=3)
    cam = S.orbit_camera(15.0, 25.0, 2.6, 1024, 640, 55.0)
    r, st, g = gpu_forward(scene, cam, CFG)
    K = assert_lists_bitexact(r, scene, cam, CFG)
    touched, area = _rect_tiles(r, scene.n)
    assert (area > 256).sum() > 100 and K < 0.6 * area.sum(), (K, area.sum())
    # the deferred emit (sets over 256 tiles or 8 rows) is exercised
    assert (touched > 256).sum() > 50


@pytest.mark.parametrize("loc", [-2.8, -2.5])
def test_tile_sets_with_ragged_edges_match_the_oracle(loc):
    """Mostly small primitives, some large, a ragged image edge: lists
    bit-exact, images within the parity bound."""
    scene = S.surface_scene(20_000, seed=23, frac3d=0.6, ls_loc=loc, ls_scale=0.5)
    cam = S.orbit_camera(200.0, 10.0, 2.8, 650, 371, 50.0)
    r, st, g = gpu_forward(scene, cam, CFG)
    assert_lists_bitexact(r, scene, cam, CFG)
    m = _oracle_maps(scene, cam, CFG)
    assert_images_match(g, m, check_nc=True, max_excluded=0.0, label=f"tile sets {loc}")


def test_tile_sets_when_every_primitive_is_large():
    """Every binned primitive's rectangle spans more than 256 tiles (the
    deferred, block-per-primitive emit for most of them)."""
    rng = np.random.default_rng(31)
    scene, _ = S.tiny_scene(31, n=700)
    n = scene.n
    scene.means[:] = np.stack([rng.uniform(-0.2, 0.2, n), rng.uniform(-0.2, 0.2, n),
                               rng.uniform(3.0, 4.0, n)], axis=1).astype(np.float32)
    scene.types[:] = 1
    scene.log_scales[:] = rng.uniform(-0.7, -0.4, size=(n, 3)).astype(np.float32)
    scene.opacity_logits[:] = 3.0
    cam = S.pinhole(1024, 640, 60.0)
    r, st, g = gpu_forward(scene, cam, CFG)
    K = assert_lists_bitexact(r, scene, cam, CFG)
    touched, area = _rect_tiles(r, n)
    assert (touched > 0).sum() == n and (area > 256).all() and K > 0


def test_tile_set_lists_without_keys():
    """Without the optional 64-bit keys: values and ranges bit-exact."""
    scene = S.surface_scene(60_000, seed=21, frac3d=0.3, ls_loc=-4.0, ls_scale=0.8, heavy_df=3)
    cam = S.orbit_camera(15.0, 25.0, 2.6, 1024, 640, 55.0)
    r, st, g = gpu_forward(scene, cam, CFG, keep_keys=False)
    keys, vals, ranges, _ = O.tile_lists(scene, cam, CFG)
    K = int(r.d_count.item())
    assert K == len(vals)
    np.testing.assert_array_equal(r.vals[:K].cpu().numpy().view(np.uint32), vals)
    np.testing.assert_array_equal(r.ranges.cpu().numpy().view(np.uint32), ranges)


def test_capacity_overflow_on_a_heavy_tailed_scene():
    """Overflow: reported, nothing written past the buffer, ranges cleared;
    the managed retry gives the oracle's lists."""
    scene = S.surface_scene(60_000, seed=21, frac3d=0.3, ls_loc=-4.0, ls_scale=0.8, heavy_df=3)
    cam = S.orbit_camera(15.0, 25.0, 2.6, 1024, 640, 55.0)
    K_ref = len(O.tile_lists(scene, cam, CFG)[1])
    cap = K_ref // 2
    r = Rasterizer("cuda", capacity=cap, keep_keys=True)
    r.preprocess(SceneTensors.from_numpy(scene), cam, CFG)
    r._ensure_capacity(cap)
    guard = torch.full((cap + 8192,), 7, dtype=torch.int32, device="cuda")
    r.vals = guard[:cap]
    r.bin_sort(sync_check=False)
    torch.cuda.synchronize()
    assert int(r.d_count.item()) == K_ref > cap
    assert int(r.dev_err.item()) == -2
    assert torch.all(guard[cap:] == 7)
    assert torch.all(r.ranges == 0)
    r2, st2, g = gpu_forward(scene, cam, CFG, capacity=cap)
    assert r2.capacity >= K_ref
    assert_lists_bitexact(r2, scene, cam, CFG)
