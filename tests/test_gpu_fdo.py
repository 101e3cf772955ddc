"""Frequency-decoupled optimisation on the GPU (EGGS §3.3, Eq. 8, Algorithm
1; App. E) against the oracle: the image-loss kernel (values and gradient
images, even/odd/degenerate shapes and the full 1600x1064 frame), and the
fused Algorithm 1 backward (tiny scenes against the oracle's three FP64
vector-Jacobian products, and sampled primitives of the 3M scene against
the oracle's Algorithm 1 applied to the separately computed GPU gradients).
Needs a GB300."""
import numpy as np
import pytest
import torch

import synthetic as S
from gpu_util import CFG, assert_grads_match, gpu_forward
from oracle import autograd_ref as AR
from oracle import fdo as F
from oracle import native as O
from paper_2512_02932_gb300 import Rasterizer, SceneTensors
from paper_2512_02932_gb300 import fdo as G

pytestmark = pytest.mark.gpu

W3 = (0.8, 0.2, 0.4)


@pytest.mark.parametrize("shape", [(3, 64, 48), (3, 37, 51), (1, 6, 9), (3, 1, 5), (2, 2, 2),
                                   (3, 1064, 1600)])
def test_image_losses_match_oracle(shape):
    rng = np.random.default_rng(sum(shape))
    img = rng.uniform(0, 1, size=shape).astype(np.float32)
    tgt = rng.uniform(0, 1, size=shape).astype(np.float32)
    out = G.image_losses(torch.from_numpy(img).cuda(), torch.from_numpy(tgt).cuda(), *W3)
    torch.cuda.synchronize()
    got = out["loss"].cpu().numpy()
    ref = np.array(F.image_losses(img, tgt))
    np.testing.assert_allclose(got, ref, rtol=2e-5, atol=1e-12)
    refg = F.loss_grads(img, tgt, W3)
    for k, name in enumerate(("g_l1", "g_low", "g_high")):
        g = out[name].cpu().numpy().astype(np.float64)
        scale = max(np.abs(refg[k]).max(), 1e-30)
        assert np.abs(g - refg[k]).max() <= 1e-5 * scale, (name, np.abs(g - refg[k]).max(), scale)


def _oracle_fdo(scene, cam, cots):
    gc = AR.vjp(scene, cam, CFG, cots["color"])[1]
    gl = AR.vjp(scene, cam, CFG, cots["low"])[1]
    gh = AR.vjp(scene, cam, CFG, cots["high"])[1]
    return F.algorithm1(gc, gl, gh, scene.types)


def _rgb_cot(seed, cam, amb):
    c = S.random_cotangents(seed, cam.height, cam.width)
    rgb = np.where(amb[None], 0.0, c["rgb"]).astype(np.float32)
    z = np.zeros((cam.height, cam.width), np.float32)
    return {"rgb": rgb, "depth": z, "normal": np.zeros_like(rgb), "alpha": z}


def _check_fdo_small(scene, cam):
    m = O.Oracle(scene, cam, CFG).render_maps()
    cots = {k: _rgb_cot(50 + j, cam, m["amb"]) for j, k in enumerate(("color", "low", "high"))}
    ref, conflict, margin = _oracle_fdo(scene, cam, cots)
    r, st, _ = gpu_forward(scene, cam, keep_keys=False)
    t = [torch.from_numpy(cots[k]["rgb"]).cuda() for k in ("color", "low", "high")]
    ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
    got = G.fdo_backward(r, *t, d_conflicts=ctr)
    torch.cuda.synchronize()
    r.check()
    got = {k: v.cpu().numpy() for k, v in got.items()}
    # a conflict decided by a dot product within rounding of zero may go either way
    near = margin < 1e-4
    for d in (got, ref):
        for k in d:
            d[k][near] = 0.0
    assert_grads_match(got, ref)
    n_conf = int(ctr.item())
    assert abs(n_conf - int(conflict.sum())) <= int((near & (margin < np.inf)).sum())
    assert 0 < conflict.sum() < scene.n
    return n_conf


@pytest.mark.parametrize("seed", [0, 1])
def test_fdo_backward_tiny_matches_oracle(seed):
    scene, cam = S.tiny_scene(seed)
    _check_fdo_small(scene, cam)


def test_fdo_backward_sh3_surface_matches_oracle():
    scene = S.surface_scene(400, seed=9, frac3d=0.5, ls_loc=-2.6, ls_scale=0.4)
    cam = S.orbit_camera(10.0, 20.0, 3.0, 96, 72, 50.0)
    _check_fdo_small(scene, cam)


def test_fdo_step_is_losses_plus_backward():
    scene, cam = S.tiny_scene(3)
    st = SceneTensors.from_numpy(scene)
    tgt = torch.rand((3, cam.height, cam.width), device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    r = Rasterizer("cuda")
    maps, loss, grads = G.fdo_step(st, cam, CFG, tgt, r)
    ls = G.image_losses(maps["rgb"], tgt, 1.0, G.LAMBDA_LOW, G.LAMBDA_HIGH)
    g2 = G.fdo_backward(r, ls["g_l1"], ls["g_low"], ls["g_high"])
    torch.cuda.synchronize()
    # block sums and record gradients are accumulated by atomics, whose order varies
    np.testing.assert_allclose(loss.cpu().numpy(), ls["loss"].cpu().numpy(), rtol=1e-9)
    for k in grads:
        a, b = grads[k].cpu().numpy(), g2[k].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-5 * max(np.abs(b).max(), 1e-30), k
    ref = F.image_losses(maps["rgb"].cpu().numpy(), tgt.cpu().numpy())
    np.testing.assert_allclose(loss.cpu().numpy(), ref, rtol=2e-5)


def test_fdo_backward_3m_against_oracle_algorithm1():
    """At the 3M scene: the fused kernel's projected sum for sampled
    primitives equals the oracle's Algorithm 1 applied to the three
    gradients the plain backward computes from the same cotangents."""
    scene, cam = S.scene_scale()
    st = SceneTensors.from_numpy(scene)
    r = Rasterizer("cuda", keep_keys=False)
    maps = r.forward(st, cam, CFG)
    tgt = torch.rand((3, cam.height, cam.width), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    ls = G.image_losses(maps["rgb"], tgt, 1.0, G.LAMBDA_LOW, G.LAMBDA_HIGH)
    ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
    fused = {k: v.clone() for k, v in G.fdo_backward(r, ls["g_l1"], ls["g_low"], ls["g_high"], d_conflicts=ctr).items()}
    parts = [{k: v.cpu().numpy() for k, v in r.backward(ls[name], None, None, None).items()}
             for name in ("g_l1", "g_low", "g_high")]
    torch.cuda.synchronize()
    r.check()
    touched = r.touched[: scene.n].cpu().numpy() > 0
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(np.nonzero(touched)[0], 3000, replace=False))
    sub = [{k: v[idx] for k, v in p.items()} for p in parts]
    ref, conflict, margin = F.algorithm1(sub[0], sub[1], sub[2], scene.types[idx])
    got = {k: v.cpu().numpy()[idx] for k, v in fused.items()}
    ok = margin >= 1e-4
    for d in (got, ref):
        for k in d:
            d[k][~ok] = 0.0
    assert_grads_match(got, ref)
    n_conf = int(ctr.item())
    assert 0 < n_conf < touched.sum()
    # culled primitives get zero gradients
    m = fused["means"].cpu().numpy()
    assert (~touched).any() and np.all(m[~touched] == 0.0)
