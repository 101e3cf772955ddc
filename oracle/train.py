"""Oracle for the training loop around the rasterizer (EGGS App. A: the 3DGS
training setup, with Adaptive Type Exchange every 500 iterations and
densification every 100 iterations from 500 to 15K).  Test infrastructure:
only tests/ may use it.  Shares nothing with the CUDA path.

  adam_step        one Adam update (Kingma & Ba, Algorithm 1) in the
                   bias-corrected form the 3DGS optimizer uses
  densify          the 3DGS densification rules: clone, split, prune
  reset_opacity    the periodic opacity reset of the 3DGS schedule

Readings (the paper defers to 3DGS and 2DGS defaults without restating
them):
  * the gradient statistic is the mean, over the iterations a primitive was
    binned, of the norm of its loss gradient with respect to its projected
    centre in pixels; the densify threshold is given in the same unit;
  * "size" of a primitive is its largest active scale (a surfel's two
    in-plane scales; a 3D Gaussian's three);
  * a split replaces the primitive by two, each centred at mu + R (s * z) with
    z a standard normal draw (passed in), scales divided by 1.6, the other
    parameters copied; a clone adds one exact copy; new primitives start
    with zero optimizer moments;
  * all decisions are taken in binary32, as on the device.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32
KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-15):
    """Returns (p', m', v') for one Adam step number `step` (1-based):
    m' = b1 m + (1-b1) g, v' = b2 v + (1-b2) g^2,
    p' = p - (lr / (1 - b1^t)) m' / (sqrt(v') / sqrt(1 - b2^t) + eps)."""
    p, g, m, v = (np.asarray(x, np.float64) for x in (p, g, m, v))
    m2 = beta1 * m + (1.0 - beta1) * g
    v2 = beta2 * v + (1.0 - beta2) * g * g
    bc1 = 1.0 - beta1 ** step
    bc2 = 1.0 - beta2 ** step
    p2 = p - (lr / bc1) * m2 / (np.sqrt(v2) / np.sqrt(bc2) + eps)
    return p2, m2, v2


def quat_to_rot(q):
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def thresholds(size_thresh, min_opacity):
    """The size and opacity thresholds mapped onto the stored parameters:
    binary32 log(size_thresh) for the log-scales and logit(min_opacity) for
    the opacity logits (both maps are monotonic, so the decisions are the
    definitions' decisions, taken on the stored values)."""
    return F32(np.log(size_thresh)), F32(np.log(min_opacity / (1.0 - min_opacity)))


def densify_actions(grad_accum, vis_count, log_scales, opacity_logits, types, grad_thresh, size_thresh,
                    min_opacity):
    """Per primitive: 0 = remove, 1 = keep, 2 = keep + clone, 3 = split (two
    new primitives replace it).  Decided in binary32: the mean gradient as
    one rounded division, size and opacity compared on the stored log-scale
    and logit (`thresholds`)."""
    acc = np.asarray(grad_accum, F32)
    cnt = np.asarray(vis_count, F32)
    with np.errstate(divide="ignore", invalid="ignore"):
        mean_g = np.where(cnt > 0, acc / np.where(cnt > 0, cnt, F32(1)), F32(0)).astype(F32)
    ls = np.asarray(log_scales, F32)
    types = np.asarray(types)
    # largest active log-scale (a surfel's two in-plane axes)
    lmax = np.where(types == 1, ls.max(1), ls[:, :2].max(1)).astype(F32)
    logits = np.asarray(opacity_logits, F32)
    ls_t, lg_t = thresholds(size_thresh, min_opacity)
    hot = mean_g >= F32(grad_thresh)
    big = lmax > ls_t
    act_code = np.ones(len(ls), np.int64)
    act_code[hot & ~big] = 2
    act_code[hot & big] = 3
    act_code[(logits < lg_t) & (act_code == 1)] = 0
    return act_code


def densify(params: dict, types, moments: dict, grad_accum, vis_count, normals_z, grad_thresh,
            size_thresh, min_opacity):
    """Apply the actions in primitive order: a kept primitive is copied with
    its moments, a clone is followed by its copy (zero moments), a split
    emits its two samples (zero moments).  normals_z: [N,2,3] standard
    normal draws, one triple per split sample.  Returns (params', types',
    moments', actions)."""
    act = densify_actions(grad_accum, vis_count, params["log_scales"], params["opacity_logits"], types,
                          grad_thresh, size_thresh, min_opacity)
    out = {k: [] for k in KEYS}
    mom = {k: [] for k in moments}
    tout = []
    n = len(types)
    for i in range(n):
        a = act[i]
        if a == 0:
            continue
        if a in (1, 2):
            for k in KEYS:
                out[k].append(np.asarray(params[k][i], np.float64))
            for k in moments:
                mom[k].append(np.asarray(moments[k][i], np.float64))
            tout.append(types[i])
        if a == 2:
            for k in KEYS:
                out[k].append(np.asarray(params[k][i], np.float64))
            for k in moments:
                mom[k].append(np.zeros_like(np.asarray(moments[k][i], np.float64)))
            tout.append(types[i])
        if a == 3:
            mu = np.asarray(params["means"][i], np.float64)
            ls = np.asarray(params["log_scales"][i], np.float64)
            s = np.exp(ls)
            if types[i] == 0:
                s = s * np.array([1.0, 1.0, 0.0])     # a surfel samples in its plane
            R = quat_to_rot(params["quats"][i])
            for j in range(2):
                z = np.asarray(normals_z[i, j], np.float64)
                out["means"].append(mu + R @ (s * z))
                ls_new = ls.copy()
                ls_new[:2] -= np.log(1.6)
                if types[i] == 1:
                    ls_new[2] -= np.log(1.6)
                out["log_scales"].append(ls_new)
                for k in ("quats", "opacity_logits", "sh"):
                    out[k].append(np.asarray(params[k][i], np.float64))
                for k in moments:
                    mom[k].append(np.zeros_like(np.asarray(moments[k][i], np.float64)))
                tout.append(types[i])
    shapes = {k: np.asarray(params[k]).shape[1:] for k in KEYS}
    res = {k: (np.array(out[k]) if out[k] else np.zeros((0,) + shapes[k])) for k in KEYS}
    mres = {k: (np.array(mom[k]) if mom[k] else np.zeros((0,) + np.asarray(moments[k]).shape[1:])) for k in moments}
    return res, np.array(tout, np.uint8), mres, act


def reset_opacity(opacity_logits, ceiling=0.01):
    """alpha <- min(alpha, ceiling), expressed on the logit."""
    lg = np.asarray(opacity_logits, np.float64)
    cap = np.log(ceiling / (1.0 - ceiling))
    return np.minimum(lg, cap)
