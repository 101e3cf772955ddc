"""The FP64 autograd formulation's gradients against central finite
differences of the C oracle (an independent implementation of the same image
function).  CPU only."""
import dataclasses

import numpy as np
import pytest

import synthetic as S
from oracle import autograd_ref as AR
from oracle import native as O

CFG = S.RenderConfig()


def _loss(out, amb, cot, H, W):
    o = out.reshape(H, W, 10)
    return (np.sum(np.moveaxis(o[..., 0:3], -1, 0) * cot["rgb"]) + np.sum(o[..., 3] * cot["depth"])
            + np.sum(np.moveaxis(o[..., 4:7], -1, 0) * cot["normal"]) + np.sum(o[..., 7] * cot["alpha"]))


def _scenes():
    sc, _ = S.tiny_scene(0)
    sc = sc.subset(np.arange(300))
    cam = S.pinhole(64, 64, 60.0)
    yield "tiny-deg0", sc, cam, CFG
    sc3 = S.surface_scene(300, seed=7, frac3d=0.5, ls_loc=-2.6, ls_scale=0.4)
    cam3 = S.orbit_camera(20.0, 15.0, 3.0, 64, 48, 50.0)
    yield "surface-deg3", sc3, cam3, CFG
    # surfels whose buffered s_z lies in the gate of Eqs. 6-7
    scm = sc.copy()
    scm.log_scales[scm.types == 0, 2] = np.log(np.random.default_rng(4).uniform(0.9, 1.2, (scm.types == 0).sum()))
    yield "tiny-modulated", scm, cam, dataclasses.replace(CFG, lambda_z=1.7, T_z=0.1)


@pytest.mark.parametrize("case", list(_scenes()), ids=lambda c: c[0])
def test_autograd_matches_finite_differences(case):
    name, sc, cam, cfg = case
    H, W = cam.height, cam.width
    cot = S.random_cotangents(11, H, W)
    _, grads = AR.vjp(sc, cam, cfg, cot)
    orc = O.Oracle(sc, cam, cfg)
    base_out, _ = orc.render()
    rng = np.random.default_rng(3)
    # primitives that touch the image
    vis = np.nonzero(np.abs(grads["opacity_logits"]) > 1e-6)[0]
    assert len(vis) > 20
    fields = [("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1), ("sh", None)]
    checked = skipped = 0
    for i in rng.choice(vis, size=16, replace=False):
        for fname, ncomp in fields:
            arr = getattr(sc, fname)
            if fname == "sh":
                comps = [tuple(rng.integers([0, 0], [arr.shape[1], 3]))]
            elif ncomp == 1:
                comps = [()]
            else:
                comps = [(int(rng.integers(ncomp)),)]
            if fname == "log_scales" and sc.types[i] == 0:
                # s_z of a surfel enters only through the modulation (Eqs. 6-7)
                comps = [(int(rng.integers(2)),)] + ([(2,)] if name == "tiny-modulated" else [])
            for c in comps:
                base = {k: getattr(sc, k)[i].astype(np.float64).copy() for k in
                        ("means", "log_scales", "quats", "sh")}
                base["opacity_logits"] = float(sc.opacity_logits[i])
                h = 1e-6
                Ls, nc = [], []
                for sgn in (1, -1):
                    p = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in base.items()}
                    if fname == "opacity_logits":
                        p[fname] = p[fname] + sgn * h
                    else:
                        p[fname][c] += sgn * h
                    orc.set_prim(i, p["means"], p["log_scales"], p["quats"], p["opacity_logits"],
                                 p["sh"], sc.types[i])
                    out, amb = orc.render()
                    Ls.append(_loss(out, amb, cot, H, W))
                    nc.append(out[:, 9].copy())
                orc.set_prim(i, base["means"], base["log_scales"], base["quats"],
                             base["opacity_logits"], base["sh"], sc.types[i])
                if not np.array_equal(nc[0], nc[1]):
                    skipped += 1  # a contributor crossed a threshold: FD ill-posed
                    continue
                fd = (Ls[0] - Ls[1]) / (2 * h)
                g = grads[fname][i] if fname == "opacity_logits" else grads[fname][i][c]
                scale = np.abs(grads[fname]).max()
                assert abs(fd - g) <= 1e-5 * abs(g) + 1e-6 * scale, (name, fname, i, c, fd, g)
                checked += 1
    assert checked >= 60 and skipped <= 4
