"""Frequency-decoupled optimisation on the GB300 path (EGGS §3.3, Eq. 8,
Algorithm 1; App. E).

  image_losses   L1 and the level-1 Haar DWT band losses of a rendered image,
                 with their (weighted) gradient images, in one kernel
                 (hgs_image_losses)
  fdo_backward   Algorithm 1: three rgb cotangents replayed through the
                 rasterizer, the per-primitive conflict projection, and the
                 sum written once (hgs_render_bwd_fdo)
  fdo_step       forward + losses + Algorithm 1 backward for one view

The appearance loss here is the L1 term of L_color; the D-SSIM term is not
part of this path.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import abi
from .rasterizer import GRAD_FLOATS, Rasterizer, SceneTensors, _ptr, _stream

LAMBDA_LOW = 0.2
LAMBDA_HIGH = 0.4


def image_losses(image: torch.Tensor, target: torch.Tensor, w_l1=1.0, w_low=1.0, w_high=1.0,
                 want_grads=True, out=None):
    """Losses (device float64 [3]: L1, L_low, L_high) and, if want_grads, the
    gradient images w_l1 dL1/dimage, w_low dL_low/dimage, w_high dL_high/dimage
    ([C,H,W] float32 each).  image/target: [C,H,W] float32 on the device."""
    if image.dim() != 3 or image.shape != target.shape:
        raise ValueError("image and target must be [C,H,W] of the same shape")
    image = image.contiguous()
    target = target.contiguous()
    Cn, H, W = image.shape
    d = image.device
    if out is None:
        out = {"loss": torch.empty(3, dtype=torch.float64, device=d)}
        if want_grads:
            for k in ("g_l1", "g_low", "g_high"):
                out[k] = torch.empty((Cn, H, W), dtype=torch.float32, device=d)
    g = [_ptr(out[k]) if want_grads else None for k in ("g_l1", "g_low", "g_high")]
    abi.check(abi.hgs_image_losses(_ptr(image), _ptr(target), Cn, H, W, float(w_l1), float(w_low),
                                   float(w_high), _ptr(out["loss"]), *g, _stream()), "hgs_image_losses")
    return out


def fdo_backward(rast: Rasterizer, g_color, g_low, g_high, grads=None, d_conflicts=None):
    """Algorithm 1 for the most recent forward of `rast`: raw-parameter
    gradients g^color + g^low + g^high with the conflicting frequency
    component projected per primitive type.  d_conflicts: optional device
    uint64 [1] counter (incremented once per conflicting primitive)."""
    n = rast.n
    deg = rast._scene_s.sh_degree
    nb = (deg + 1) ** 2
    d = rast.device
    if grads is None:
        grads = {
            "means": torch.empty((n, 3), dtype=torch.float32, device=d),
            "log_scales": torch.empty((n, 3), dtype=torch.float32, device=d),
            "quats": torch.empty((n, 4), dtype=torch.float32, device=d),
            "opacity_logits": torch.empty(n, dtype=torch.float32, device=d),
            "sh": torch.empty((n, nb, 3), dtype=torch.float32, device=d),
        }
    ws = getattr(rast, "grad_ws3", None)
    if ws is None or ws.shape[0] != 3 * max(n, 1):
        ws = torch.empty((3 * max(n, 1), GRAD_FLOATS), dtype=torch.float32, device=d)
        rast.grad_ws3 = ws
    cots = [t.contiguous() for t in (g_color, g_low, g_high)]
    out = abi.hgs_scene_grad(grads["means"].data_ptr(), grads["log_scales"].data_ptr(),
                             grads["quats"].data_ptr(), grads["opacity_logits"].data_ptr(),
                             grads["sh"].data_ptr())
    bins = rast.bin_struct()
    rast._keep_fdo = (cots, out, bins)
    abi.check(abi.hgs_render_bwd_fdo(C.byref(rast._scene_s), C.byref(rast._proj_s), C.byref(bins),
                                     C.byref(rast._cam_s), C.byref(rast._cfg_s), C.byref(rast._img_s),
                                     *[_ptr(t) for t in cots], _ptr(ws), C.byref(out), _ptr(d_conflicts),
                                     _ptr(rast.dev_err), _stream()), "hgs_render_bwd_fdo")
    return grads


def fdo_step(scene: SceneTensors, cam, cfg, target: torch.Tensor, rast: Rasterizer,
             lambda_low=LAMBDA_LOW, lambda_high=LAMBDA_HIGH, d_conflicts=None):
    """One view of frequency-decoupled training: render, the losses of Eq. 8
    (appearance term: L1), and the Algorithm 1 backward.  Returns the forward
    maps, the loss tensor (L1, L_low, L_high; unweighted) and the gradients."""
    maps = rast.forward(scene, cam, cfg)
    ls = image_losses(maps["rgb"], target, 1.0, lambda_low, lambda_high)
    grads = fdo_backward(rast, ls["g_l1"], ls["g_low"], ls["g_high"], d_conflicts=d_conflicts)
    return maps, ls["loss"], grads
