"""The training loop's kernels against the oracle (Adam, the densification
statistic, densification, opacity reset), and a short synthetic training
run through Trainer (loss falls, densification and exchange run, no device
error).  Needs a GB300."""
import ctypes as C
import math

import numpy as np
import pytest
import torch

import synthetic as S
from gpu_util import CFG
from oracle import train as T
from paper_2512_02932_gb300 import Rasterizer, SceneTensors, abi
from paper_2512_02932_gb300.rasterizer import _ptr, _stream
from paper_2512_02932_gb300.train import KEYS, TrainConfig, Trainer

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("count,offset,period,head", [(1, 0, 0, 0), (7, 0, 0, 0), (1027, 0, 0, 0),
                                                      (1000, 1, 0, 0), (48 * 37, 0, 48, 3), (48 * 5 + 3, 1, 48, 3)])
def test_adam_matches_oracle(count, offset, period, head):
    rng = np.random.default_rng(count + offset)
    buf = {k: torch.zeros(count + 8, dtype=torch.float32, device="cuda") for k in ("p", "g", "m", "v")}
    view = {k: v[offset:offset + count] for k, v in buf.items()}
    p = rng.normal(size=count).astype(np.float32)
    view["p"].copy_(torch.from_numpy(p))
    m = np.zeros(count)
    v = np.zeros(count)
    lr, lr_tail = 1e-2, 1e-3
    pos = np.arange(count) % period if period else np.zeros(count, int)
    lrs = np.where((period > 0) & (pos >= head), lr_tail, lr)
    pf = p.astype(np.float64)
    for t in range(1, 5):
        g = rng.normal(size=count).astype(np.float32)
        view["g"].copy_(torch.from_numpy(g))
        grp = (abi.hgs_adam_group * 1)(abi.hgs_adam_group(_ptr(view["p"]), _ptr(view["g"]), _ptr(view["m"]),
                                                          _ptr(view["v"]), count, lr, period, head, lr_tail))
        abi.check(abi.hgs_adam_step(1, grp, t, 0.9, 0.999, 1e-15, _stream()), "adam")
        torch.cuda.synchronize()
        # compare one step from the device's own previous state
        p_ref, m_ref, v_ref = T.adam_step(pf, g, m, v, t, lrs)
        got_p = view["p"].cpu().numpy().astype(np.float64)
        # binary32 rounding of terms of magnitude |g| (m) and |p| (p) before they cancel
        gmax = float(np.abs(g).max())
        np.testing.assert_allclose(view["m"].cpu().numpy(), m_ref, rtol=1e-6, atol=2e-7 * gmax)
        np.testing.assert_allclose(view["v"].cpu().numpy(), v_ref, rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(got_p, p_ref, rtol=1e-6, atol=2e-7 * float(np.abs(pf).max()))
        pf = got_p
        m = view["m"].cpu().numpy().astype(np.float64)
        v = view["v"].cpu().numpy().astype(np.float64)
    # untouched guard elements
    assert float(buf["p"][:offset].abs().sum()) == 0.0 and float(buf["p"][offset + count:].abs().sum()) == 0.0


def _random_train_scene(n, seed):
    sc = S.surface_scene(n, seed=seed, frac3d=0.6)
    rng = np.random.default_rng(seed)
    sc.log_scales[:] = rng.normal(-4.0, 1.2, size=sc.log_scales.shape).astype(np.float32)
    sc.log_scales[sc.types == 0, 2] = S.SURFEL_LOG_SZ
    sc.opacity_logits[:] = rng.normal(0.0, 3.0, size=n).astype(np.float32)
    return sc


def test_densify_matches_oracle():
    n = 20_000
    sc = _random_train_scene(n, 3)
    rng = np.random.default_rng(4)
    acc = (rng.exponential(3e-4, size=n) * rng.integers(0, 4, n)).astype(np.float32)
    cnt = rng.integers(0, 4, n).astype(np.float32)
    st = SceneTensors.from_numpy(sc)
    mom = {f"{w}_{k}": torch.from_numpy(rng.normal(size=getattr(sc, k).shape).astype(np.float32)).cuda()
           for w in ("m", "v") for k in KEYS}
    tr = Trainer.__new__(Trainer)
    tr.device = torch.device("cuda")
    tr.tcfg = TrainConfig(extent=1.0, percent_dense=0.03)
    tr.gen = torch.Generator(device="cuda").manual_seed(9)
    tr.scene, tr.moments = st, mom
    tr.accum = torch.from_numpy(acc).cuda()
    tr.count = torch.from_numpy(cnt).cuda()
    gen_state = tr.gen.get_state()
    actions, offsets, m = tr.densify(1e-4)
    torch.cuda.synchronize()
    g2 = torch.Generator(device="cuda")
    g2.set_state(gen_state)
    z = torch.randn((n, 2, 3), generator=g2, device="cuda").cpu().numpy()
    params = {k: getattr(sc, k) for k in KEYS}
    moments = {k: v.cpu().numpy() for k, v in mom.items()}
    ref, tref, mref, aref = T.densify(params, sc.types, moments, acc, cnt, z, 1e-4, 0.03, 0.005)
    np.testing.assert_array_equal(actions.cpu().numpy(), aref)
    assert set(np.unique(aref)) == {0, 1, 2, 3}
    assert m == len(tref)
    np.testing.assert_array_equal(tr.scene.types.cpu().numpy(), tref)
    split = np.repeat(aref == 3, np.where(aref == 0, 0, np.where(aref == 1, 1, 2)))
    for k in KEYS:
        got = getattr(tr.scene, k).cpu().numpy()
        np.testing.assert_array_equal(got[~split], ref[k][~split].astype(np.float32), err_msg=k)
        np.testing.assert_allclose(got[split], ref[k][split], rtol=1e-5, atol=1e-6, err_msg=k)
    for k, v in tr.moments.items():
        np.testing.assert_array_equal(v.cpu().numpy(), mref[k].astype(np.float32), err_msg=k)


def test_grad_stats_and_reset_opacity():
    scene, cam = S.tiny_scene(5)
    r = Rasterizer("cuda")
    st = SceneTensors.from_numpy(scene)
    maps = r.forward(st, cam, CFG)
    g = torch.randn_like(maps["rgb"])
    r.backward(g, None, None, None)
    acc = torch.full((scene.n,), 0.5, device="cuda")
    cnt = torch.ones(scene.n, device="cuda")
    abi.check(abi.hgs_grad_stats(scene.n, _ptr(r.grad_ws), C.byref(r.proj_struct()), _ptr(acc), _ptr(cnt),
                                 _stream()), "stats")
    torch.cuda.synchronize()
    G = r.grad_ws[: scene.n].cpu().numpy().astype(np.float64)
    touched = r.touched[: scene.n].cpu().numpy() > 0
    ref = 0.5 + np.where(touched, np.hypot(G[:, 4], G[:, 5]), 0.0)
    np.testing.assert_allclose(acc.cpu().numpy(), ref, rtol=1e-6)
    np.testing.assert_array_equal(cnt.cpu().numpy(), 1.0 + touched)
    lg = st.opacity_logits.clone()
    mm, vv = torch.ones_like(lg), torch.ones_like(lg)
    abi.check(abi.hgs_reset_opacity(scene.n, _ptr(lg), 0.01, _ptr(mm), _ptr(vv), _stream()), "reset")
    torch.cuda.synchronize()
    np.testing.assert_allclose(lg.cpu().numpy(), T.reset_opacity(scene.opacity_logits, 0.01), rtol=1e-6)
    assert float(mm.abs().sum()) == 0 and float(vv.abs().sum()) == 0


@pytest.mark.parametrize("fdo", [False, True])
def test_training_run_reduces_loss(fdo):
    """A perturbed copy of a synthetic scene is trained towards four views of
    the original, with the schedule compressed (densify every 40 iterations
    from 40, exchange every 60)."""
    gt = S.surface_scene(30_000, seed=11, frac3d=0.7, ls_loc=-3.6, ls_scale=0.5)
    cams = [S.orbit_camera(a, 20.0, 3.0, 256, 192, 50.0) for a in (0.0, 90.0, 180.0, 270.0)]
    r = Rasterizer("cuda")
    gts = SceneTensors.from_numpy(gt)
    targets = [r.forward(gts, c, CFG)["rgb"].clone() for c in cams]
    init = S.surface_scene(30_000, seed=11, frac3d=0.7, ls_loc=-3.6, ls_scale=0.5)
    rng = np.random.default_rng(12)
    init.means += rng.normal(0, 0.01, init.means.shape).astype(np.float32)
    init.sh[:, 0, :] = 0.0
    tc = TrainConfig(extent=3.0, densify_from=40, densify_until=200, densify_every=40, opacity_reset_every=0,
                     exchange_from=60, exchange_every=60, fdo=fdo, lr_sh_dc=1e-2)
    tr = Trainer(SceneTensors.from_numpy(init), CFG, tc)
    n0 = tr.scene.n
    first = last = None
    for it in range(240):
        k = it % 4
        loss = tr.step(cams[k], targets[k])
        if it < 4:
            first = (first or 0.0) + float(loss[0])
        if it >= 236:
            last = (last or 0.0) + float(loss[0])
    torch.cuda.synchronize()
    tr.rast.check()
    assert last < 0.6 * first, (first, last)
    assert tr.scene.n != n0
    for k in KEYS:
        assert torch.isfinite(getattr(tr.scene, k)).all(), k
