"""Oracle for frequency-decoupled optimisation (EGGS §3.3, Eq. 8, Algorithm 1;
App. E), in float64.  Test infrastructure: only tests/, the smoke check and
the bench's CPU leg may use it.  Shares nothing with the CUDA path.

  haar_matrices   the level-1 Haar analysis matrices L and H of App. E
  dwt_bands       I_LL = L I L^T, I_LH = H I L^T, I_HL = L I H^T, I_HH = H I H^T
  image_losses    L1, L_low, L_high as plain definitions over those bands
  loss_grads      their gradient images, by float64 autograd of the same definitions
  algorithm1      Algorithm 1 over per-primitive gradient vectors, step by step

Readings (the paper is silent):
  * the Haar pair is l = (1, 1)/sqrt2, h = (1, -1)/sqrt2 (App. E prints
    "l and h are the same", read as the standard orthogonal pair);
  * L_i = ||I^_i - I_i||^2 is taken as the mean over the band's elements, with
    I_h the three detail bands together; an odd last row or column is outside
    the level-1 transform (it enters L1 only);
  * g_i in Algorithm 1 is the concatenation of all of the primitive's
    parameter gradients (means, log-scales, quaternion, opacity logit, SH).
"""
from __future__ import annotations

import numpy as np
import torch

PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def haar_matrices(n: int):
    """L and H of App. E for a length-n signal (n even): row k of L has
    (1/sqrt2, 1/sqrt2) at columns 2k, 2k+1; row k of H has (1/sqrt2, -1/sqrt2)."""
    assert n % 2 == 0
    r = 1.0 / np.sqrt(2.0)
    L = np.zeros((n // 2, n))
    Hm = np.zeros((n // 2, n))
    for k in range(n // 2):
        L[k, 2 * k] = L[k, 2 * k + 1] = r
        Hm[k, 2 * k] = r
        Hm[k, 2 * k + 1] = -r
    return L, Hm


def dwt_bands(img):
    """img [C,H,W] -> dict of the four bands, each [C,H//2,W//2] (the even
    part of the image)."""
    img = np.asarray(img, np.float64)
    Cn, Hh, Ww = img.shape
    H2, W2 = Hh // 2 * 2, Ww // 2 * 2
    Lr, Hr = haar_matrices(H2)
    Lc, Hc = haar_matrices(W2)
    x = img[:, :H2, :W2]
    return {"LL": Lr @ x @ Lc.T, "LH": Hr @ x @ Lc.T, "HL": Lr @ x @ Hc.T, "HH": Hr @ x @ Hc.T}


def _losses_torch(img, tgt):
    Cn, Hh, Ww = img.shape
    H2, W2 = Hh // 2 * 2, Ww // 2 * 2
    l1 = (img - tgt).abs().mean()
    if H2 == 0 or W2 == 0:
        z = img.sum() * 0.0
        return l1, z, z
    Lr, Hr = (torch.from_numpy(m) for m in haar_matrices(H2))
    Lc, Hc = (torch.from_numpy(m) for m in haar_matrices(W2))
    d = (img - tgt)[:, :H2, :W2]
    ll = Lr @ d @ Lc.T
    lh, hl, hh = Hr @ d @ Lc.T, Lr @ d @ Hc.T, Hr @ d @ Hc.T
    low = (ll ** 2).mean()
    high = torch.cat([lh.reshape(-1), hl.reshape(-1), hh.reshape(-1)]).pow(2).mean()
    return l1, low, high


def image_losses(img, tgt):
    """(L1, L_low, L_high) of image vs target, [C,H,W] arrays."""
    a = torch.as_tensor(np.asarray(img, np.float64))
    b = torch.as_tensor(np.asarray(tgt, np.float64))
    return tuple(float(v) for v in _losses_torch(a, b))


def loss_grads(img, tgt, weights=(1.0, 1.0, 1.0)):
    """Gradient images (w_l1 dL1/dimg, w_low dL_low/dimg, w_high dL_high/dimg),
    each [C,H,W] float64, by autograd of the definitions above (d|x|/dx at 0
    is 0, as torch takes it)."""
    out = []
    for k in range(3):
        a = torch.as_tensor(np.asarray(img, np.float64)).clone().requires_grad_(True)
        b = torch.as_tensor(np.asarray(tgt, np.float64))
        L = _losses_torch(a, b)[k] * weights[k]
        (g,) = torch.autograd.grad(L, a, allow_unused=True)
        out.append(np.zeros(a.shape) if g is None else g.numpy())
    return tuple(out)


def flatten(grads: dict, i: int):
    """The concatenated parameter gradient of primitive i."""
    return np.concatenate([np.asarray(grads[k][i], np.float64).reshape(-1) for k in PARAM_KEYS])


def algorithm1(g_color: dict, g_low: dict, g_high: dict, types):
    """Algorithm 1, per primitive: on a conflict (g_low . g_high < 0) project
    g_high onto the normal of g_low for a surfel (t = 0, Eq. 9), g_low onto
    the normal of g_high for a 3D Gaussian (Eq. 10); the update is
    g_color + g_low + g_high.  Returns (update dict shaped like the inputs,
    boolean conflict array, conflict margin |g_low . g_high| / (|g_low| |g_high|))."""
    types = np.asarray(types)
    n = len(types)
    shapes = {k: np.asarray(g_color[k]).shape for k in PARAM_KEYS}
    sizes = [int(np.prod(shapes[k][1:])) for k in PARAM_KEYS]
    out = {k: np.zeros(shapes[k]) for k in PARAM_KEYS}
    conflict = np.zeros(n, bool)
    margin = np.zeros(n)
    for i in range(n):
        gc, gl, gh = flatten(g_color, i), flatten(g_low, i), flatten(g_high, i)
        dot = float(gl @ gh)
        nl, nh = float(np.linalg.norm(gl)), float(np.linalg.norm(gh))
        margin[i] = abs(dot) / (nl * nh) if nl > 0 and nh > 0 else np.inf
        if dot < 0:
            conflict[i] = True
            if types[i] == 0:
                gh = gh - dot / (gl @ gl) * gl
            else:
                gl = gl - dot / (gh @ gh) * gh
        upd = gc + gl + gh
        off = 0
        for k, sz in zip(PARAM_KEYS, sizes):
            out[k][i] = upd[off:off + sz].reshape(shapes[k][1:])
            off += sz
    return out, conflict, margin
