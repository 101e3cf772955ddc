"""Independent FP64 formulation of the hybrid rasterizer in torch (CPU),
differentiated by autograd.  Test infrastructure only.

It renders the same image function as hgs_oracle.c by a different route:
vectorised over (pixel, primitive) pairs, with the 2D ray-splat intersection
solved by Cramer's rule (triple products) rather than elimination, and the
blend written as an exclusive cumulative product rather than a loop:

  d_i    Eq. 1: (x-mu')^T Sigma'^-1 (x-mu') for t=1 (App. C, Eq. 13),
         u^2 + v^2 for t=0 (App. C, Eqs. 14-15)
  a~_i   min(alpha_max, alpha_i exp(-d_i/2)); contributes iff >= alpha_min
         (Sec. 3.1, with the 3DGS thresholds as the reading)
  C(x)   Eq. 2, terminated before the first contributor that would take the
         transmittance below T_min

The discrete decisions (which pairs contribute, where a pixel stops) are taken
without gradient, exactly as in the GPU kernels; everything else is
differentiated.  Pinned against central finite differences of the C oracle
(tests/test_oracle_grad.py) and value-for-value against the C oracle.

Memory is O(pixels_per_chunk x N): intended for N <= ~2000, images <= 128^2.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import native

_PI = math.pi


def _rot(q):
    q = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    return torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1).reshape(-1, 3, 3)


def sh_basis(deg, d):
    """Real SH basis (index l*l+l+m), written from the Legendre forms:
    Y_l^0 = sqrt((2l+1)/4pi) P_l(z); m != 0 uses sqrt(2) times the complex
    harmonic's real/imaginary part, Condon-Shortley phase included."""
    x, y, z = d.unbind(1)
    out = [torch.full_like(x, math.sqrt(1 / (4 * _PI)))]
    if deg >= 1:
        c = math.sqrt(3 / (4 * _PI))
        out += [-c * y, c * z, -c * x]
    if deg >= 2:
        a = math.sqrt(15 / (4 * _PI))
        b = math.sqrt(5 / (16 * _PI))
        e = math.sqrt(15 / (16 * _PI))
        out += [a * x * y, -a * y * z, b * (3 * z * z - 1), -a * x * z, e * (x * x - y * y)]
    if deg >= 3:
        a = math.sqrt(35 / (32 * _PI))
        b = math.sqrt(105 / (4 * _PI))
        c = math.sqrt(21 / (32 * _PI))
        e = math.sqrt(7 / (16 * _PI))
        f = math.sqrt(105 / (16 * _PI))
        out += [-a * y * (3 * x * x - y * y), b * x * y * z, -c * y * (5 * z * z - 1),
                e * z * (5 * z * z - 3), -c * x * (5 * z * z - 1), f * z * (x * x - y * y),
                -a * x * (x * x - 3 * y * y)]
    return torch.stack(out, 1)


def _params(scene, requires_grad=True):
    P = {
        "means": torch.tensor(scene.means, dtype=torch.float64),
        "log_scales": torch.tensor(scene.log_scales, dtype=torch.float64),
        "quats": torch.tensor(scene.quats, dtype=torch.float64),
        "opacity_logits": torch.tensor(scene.opacity_logits, dtype=torch.float64),
        "sh": torch.tensor(scene.sh, dtype=torch.float64),
    }
    for v in P.values():
        v.requires_grad_(requires_grad)
    return P


def _per_prim(P, types, cam, cfg):
    Rc = torch.tensor(np.asarray(cam.R, np.float64))
    tc = torch.tensor(np.asarray(cam.t, np.float64))
    mu = P["means"]
    ls = P["log_scales"]
    s = torch.exp(ls)
    R = _rot(P["quats"])
    alpha = torch.sigmoid(P["opacity_logits"])
    t2d = torch.as_tensor(types == 0)
    # scale modulation of 2D Gaussians (Eqs. 6-7)
    sz = s[:, 2]
    szs = torch.sigmoid((sz - cfg.theta_z) / cfg.T_z) * sz
    alpha = torch.where(t2d, alpha * torch.exp(-cfg.lambda_z * szs), alpha)
    muc = mu @ Rc.T + tc
    A = Rc[None] @ R  # columns: camera-space axes a_k
    # colour from SH, view direction from the camera centre
    cc = -(Rc.T @ tc)
    dv = mu - cc
    dv = dv / dv.norm(dim=1, keepdim=True)
    Y = sh_basis(scene_deg(P), dv)
    col = torch.clamp((P["sh"] * Y[:, :, None]).sum(1) + 0.5, min=0.0)
    # normal: axis of the smallest scale (z for 2D), oriented to the camera
    lsn = ls.detach().numpy()
    k = np.where(types == 0, 2,
                 np.where((lsn[:, 2] <= lsn[:, 0]) & (lsn[:, 2] <= lsn[:, 1]), 2,
                          np.where(lsn[:, 0] <= lsn[:, 1], 0, 1)))
    kk = torch.as_tensor(k)
    nrm = A[torch.arange(len(k)), :, kk]
    sgn = torch.where((nrm * muc).sum(1) > 0, -1.0, 1.0).detach()
    nrm = nrm * sgn[:, None]
    return dict(muc=muc, A=A, s=s, alpha=alpha, col=col, nrm=nrm)


def scene_deg(P):
    nb = P["sh"].shape[1]
    return int(round(math.sqrt(nb))) - 1


def render(scene, cam, cfg, pixels=None, params=None, chunk=1024):
    """Render `pixels` ((P,2) int, default full frame row-major).  Returns a dict
    of torch float64 tensors: rgb (P,3), depth (P,), normal (P,3), alpha (P,),
    plus `params` (leaf tensors with requires_grad)."""
    if params is None:
        params = _params(scene)
    types = np.asarray(scene.types)
    W, H = cam.width, cam.height
    if pixels is None:
        yy, xx = np.mgrid[0:H, 0:W]
        pixels = np.stack([xx.ravel(), yy.ravel()], 1)
    pixels = np.asarray(pixels)
    pp = _per_prim(params, types, cam, cfg)
    muc, A, s, alpha, col, nrm = (pp[k] for k in ("muc", "A", "s", "alpha", "col", "nrm"))
    fx, fy, cx, cy = cam.fx, cam.fy, cam.cx, cam.cy
    i3 = np.nonzero(types == 1)[0]
    i2 = np.nonzero(types == 0)[0]
    # 3D: EWA projection (App. C, Eq. 13)
    X, Y, Z = muc[i3].unbind(1)
    V = A[i3] @ torch.diag_embed(s[i3] ** 2) @ A[i3].transpose(1, 2)
    zero = torch.zeros_like(X)
    J = torch.stack([torch.stack([fx / Z, zero, -fx * X / Z ** 2], 1),
                     torch.stack([zero, fy / Z, -fy * Y / Z ** 2], 1)], 1)
    S2 = J @ V @ J.transpose(1, 2) + cfg.dilation * torch.eye(2, dtype=torch.float64)
    det = S2[:, 0, 0] * S2[:, 1, 1] - S2[:, 0, 1] * S2[:, 1, 0]
    ok3 = (det > 0).detach() & (Z > cfg.near).detach()
    det = torch.where(ok3, det, torch.ones_like(det))
    ca, cb, cc_ = S2[:, 1, 1] / det, -S2[:, 0, 1] / det, S2[:, 0, 0] / det
    mx, my = fx * X / Z + cx, fy * Y / Z + cy
    # 2D: tangent axes scaled, plane through mu_c
    a2 = A[i2, :, 0] * s[i2, 0:1]
    b2 = A[i2, :, 1] * s[i2, 1:2]
    m2 = muc[i2]
    ok2 = (m2[:, 2] > cfg.near).detach()
    bxm = torch.cross(b2, -m2, dim=1)  # for tau
    # global order: (contract binary32 depth bits, id); visibility is the
    # contract's binary32 decision (a primitive it does not bin is not drawn)
    db, _, touched = native.contract_bin(scene, cam, cfg)
    binned = torch.as_tensor(touched > 0)
    ok3 = ok3 & binned[torch.as_tensor(i3)]
    ok2 = ok2 & binned[torch.as_tensor(i2)]
    order = np.lexsort((np.arange(scene.n), db))
    pos = np.empty(scene.n, np.int64)
    pos[order] = np.arange(scene.n)
    p3, p2 = torch.as_tensor(pos[i3]), torch.as_tensor(pos[i2])
    outs = {"rgb": [], "depth": [], "normal": [], "alpha": []}
    col_o, nrm_o, alpha_o = col[order], nrm[order], alpha[order]
    bg = torch.tensor(cfg.bg, dtype=torch.float64)
    for c0 in range(0, len(pixels), chunk):
        pix = pixels[c0:c0 + chunk]
        px = torch.tensor(pix[:, 0] + 0.5, dtype=torch.float64)[:, None]
        py = torch.tensor(pix[:, 1] + 0.5, dtype=torch.float64)[:, None]
        Pn = px.shape[0]
        d = torch.zeros(Pn, scene.n, dtype=torch.float64)
        z = torch.zeros(Pn, scene.n, dtype=torch.float64)
        ok = torch.zeros(Pn, scene.n, dtype=torch.bool)
        if len(i3):
            dx, dy = px - mx[None], py - my[None]
            d3 = ca * dx * dx + 2 * cb * dx * dy + cc_ * dy * dy
            d = d.index_put((torch.arange(Pn)[:, None], p3[None]), d3)
            z = z.index_put((torch.arange(Pn)[:, None], p3[None]), Z[None].expand(Pn, -1))
            ok[:, p3] = ok3[None].expand(Pn, -1)
        if len(i2):
            ray = torch.stack([(px - cx) / fx, (py - cy) / fy, torch.ones_like(px)], -1)  # (P,1,3)
            nr = -ray
            c1xc2 = torch.cross(b2[None].expand(Pn, -1, -1), nr.expand(-1, len(i2), -1), dim=2)
            dett = (a2[None] * c1xc2).sum(2)
            rhs = -m2
            u_num = (rhs[None] * c1xc2).sum(2)
            rxc2 = torch.cross(rhs[None].expand(Pn, -1, -1), nr.expand(-1, len(i2), -1), dim=2)
            v_num = (a2[None] * rxc2).sum(2)
            t_num = (a2 * bxm).sum(1)[None]
            scale = (a2.norm(dim=1) * b2.norm(dim=1))[None] * ray.norm(dim=2)
            okd = (dett.abs() > 1e-12 * scale).detach()
            dsafe = torch.where(okd, dett, torch.ones_like(dett))
            u, v, tau = u_num / dsafe, v_num / dsafe, t_num / dsafe
            d2 = u * u + v * v
            okk = okd & (tau > cfg.near).detach() & ok2[None]
            d2 = torch.where(okk, d2, torch.full_like(d2, 1e30))
            d = d.index_put((torch.arange(Pn)[:, None], p2[None]), d2)
            z = z.index_put((torch.arange(Pn)[:, None], p2[None]), torch.where(okk, tau, torch.zeros_like(tau)))
            ok[:, p2] = okk
        araw = alpha_o[None] * torch.exp(-0.5 * d)
        contrib = (ok & (araw >= cfg.alpha_min)).detach()
        at = torch.clamp(araw, max=cfg.alpha_max)
        with torch.no_grad():
            am = torch.where(contrib, at, torch.zeros_like(at))
            cp = torch.cumprod(1 - am, dim=1)
            Tex = torch.cat([torch.ones(Pn, 1, dtype=torch.float64), cp[:, :-1]], 1)
            stop = contrib & (Tex * (1 - am) < cfg.T_min)
            idx = torch.arange(scene.n)[None].expand(Pn, -1)
            first = torch.where(stop, idx, torch.full_like(idx, scene.n)).min(1, keepdim=True).values
            keep = contrib & (idx < first)
        ak = torch.where(keep, at, torch.zeros_like(at))
        cp = torch.cumprod(1 - ak, dim=1)
        Tex = torch.cat([torch.ones(Pn, 1, dtype=torch.float64), cp[:, :-1]], 1)
        w = ak * Tex
        Tf = cp[:, -1]
        outs["rgb"].append(w @ col_o + Tf[:, None] * bg[None])
        outs["depth"].append((w * z).sum(1))
        outs["normal"].append(w @ nrm_o)
        outs["alpha"].append(1 - Tf)
    res = {k: torch.cat(v, 0) for k, v in outs.items()}
    res["params"] = params
    return res


def vjp(scene, cam, cfg, cot, chunk=1024):
    """Gradients of sum(cot * outputs) over the full frame with respect to the
    raw parameters.  cot: dict of numpy maps rgb (3,H,W), depth (H,W),
    normal (3,H,W), alpha (H,W).  Returns (outputs as planar maps, grads dict
    of float64 numpy arrays)."""
    params = _params(scene)
    W, H = cam.width, cam.height
    yy, xx = np.mgrid[0:H, 0:W]
    pixels = np.stack([xx.ravel(), yy.ravel()], 1)
    maps = {"rgb": [], "depth": [], "normal": [], "alpha": []}
    crgb = torch.tensor(cot["rgb"].reshape(3, -1).T, dtype=torch.float64)
    cd = torch.tensor(cot["depth"].reshape(-1), dtype=torch.float64)
    cn = torch.tensor(cot["normal"].reshape(3, -1).T, dtype=torch.float64)
    ca = torch.tensor(cot["alpha"].reshape(-1), dtype=torch.float64)
    step = chunk * 4
    for c0 in range(0, len(pixels), step):
        sl = slice(c0, c0 + step)
        r = render(scene, cam, cfg, pixels[sl], params=params, chunk=chunk)
        L = ((r["rgb"] * crgb[sl]).sum() + (r["depth"] * cd[sl]).sum()
             + (r["normal"] * cn[sl]).sum() + (r["alpha"] * ca[sl]).sum())
        L.backward()
        for k in maps:
            maps[k].append(r[k].detach().numpy())
    out = {
        "rgb": np.concatenate(maps["rgb"]).T.reshape(3, H, W),
        "depth": np.concatenate(maps["depth"]).reshape(H, W),
        "normal": np.concatenate(maps["normal"]).T.reshape(3, H, W),
        "alpha": np.concatenate(maps["alpha"]).reshape(H, W),
    }
    grads = {k: v.grad.numpy().copy() if v.grad is not None else np.zeros(v.shape)
             for k, v in params.items()}
    return out, grads


def pair_alpha(scene, cam, cfg, pixels):
    """Unclamped alpha*exp(-d/2) for every (pixel, primitive) pair in input
    order, with the geometric validity mask (centre in front, finite
    intersection in front of the near plane).  (P, N) float64 numpy arrays."""
    with torch.no_grad():
        params = _params(scene, requires_grad=False)
        types = np.asarray(scene.types)
        pp = _per_prim(params, types, cam, cfg)
        muc, A, s, alpha = pp["muc"], pp["A"], pp["s"], pp["alpha"]
        fx, fy, cx, cy = cam.fx, cam.fy, cam.cx, cam.cy
        pixels = np.asarray(pixels)
        px = torch.tensor(pixels[:, 0] + 0.5, dtype=torch.float64)[:, None]
        py = torch.tensor(pixels[:, 1] + 0.5, dtype=torch.float64)[:, None]
        Pn, N = len(pixels), scene.n
        d = torch.full((Pn, N), 1e30, dtype=torch.float64)
        ok = torch.zeros((Pn, N), dtype=torch.bool)
        i3 = np.nonzero(types == 1)[0]
        i2 = np.nonzero(types == 0)[0]
        if len(i3):
            X, Y, Z = muc[i3].unbind(1)
            V = A[i3] @ torch.diag_embed(s[i3] ** 2) @ A[i3].transpose(1, 2)
            zero = torch.zeros_like(X)
            J = torch.stack([torch.stack([fx / Z, zero, -fx * X / Z ** 2], 1),
                             torch.stack([zero, fy / Z, -fy * Y / Z ** 2], 1)], 1)
            S2 = J @ V @ J.transpose(1, 2) + cfg.dilation * torch.eye(2, dtype=torch.float64)
            det = S2[:, 0, 0] * S2[:, 1, 1] - S2[:, 0, 1] ** 2
            ok3 = (det > 0) & (Z > cfg.near)
            det = torch.where(ok3, det, torch.ones_like(det))
            dx, dy = px - (fx * X / Z + cx)[None], py - (fy * Y / Z + cy)[None]
            d[:, i3] = (S2[:, 1, 1] * dx * dx - 2 * S2[:, 0, 1] * dx * dy + S2[:, 0, 0] * dy * dy) / det
            ok[:, i3] = ok3[None].expand(Pn, -1)
        if len(i2):
            a2 = A[i2, :, 0] * s[i2, 0:1]
            b2 = A[i2, :, 1] * s[i2, 1:2]
            m2 = muc[i2]
            ray = torch.stack([(px - cx) / fx, (py - cy) / fy, torch.ones_like(px)], -1)
            nr = -ray
            c1xc2 = torch.cross(b2[None].expand(Pn, -1, -1), nr.expand(-1, len(i2), -1), dim=2)
            dett = (a2[None] * c1xc2).sum(2)
            u = (-m2[None] * c1xc2).sum(2) / dett
            rxc2 = torch.cross((-m2)[None].expand(Pn, -1, -1), nr.expand(-1, len(i2), -1), dim=2)
            v = (a2[None] * rxc2).sum(2) / dett
            tau = (a2 * torch.cross(b2, -m2, dim=1)).sum(1)[None] / dett
            okk = torch.isfinite(u) & torch.isfinite(v) & (tau > cfg.near) & (m2[:, 2] > cfg.near)[None]
            d[:, i2] = torch.where(okk, u * u + v * v, torch.full_like(u, 1e30))
            ok[:, i2] = okk
        _, _, touched = native.contract_bin(scene, cam, cfg)
        ok = ok & torch.as_tensor(touched > 0)[None]
        araw = alpha[None] * torch.exp(-0.5 * d)
        return araw.numpy(), ok.numpy()
