"""The training loop around the rasterizer (EGGS App. A): the 3DGS setup --
Adam with per-parameter learning rates, densification every 100 iterations
from 500 to 15K, opacity reset every 3000 -- with Adaptive Type Exchange
every 500 iterations from 500 (erank threshold 2.05) and, optionally,
frequency-decoupled optimisation (L1 + 0.2 L_low + 0.4 L_high with the
Algorithm 1 backward).  Every step runs in this library's kernels:

  Trainer.step         forward, image losses, backward, gradient statistic,
                       fused Adam, then the schedule's densify / reset /
                       exchange
  Trainer.densify      plan (actions, exclusive scan, new count), one read of
                       the new count, apply into freshly allocated arrays

Learning rates and thresholds follow the 3DGS defaults (the paper defers to
them): means 1.6e-4 -> 1.6e-6 x extent (log-linear over 30K steps), SH DC
2.5e-3 and higher orders 2.5e-3 / 20, opacity 0.05, scales 5e-3, rotations
1e-3; densify gradient 2e-4 in NDC units (converted to pixels per view),
split above 1% of the scene extent, prune below opacity 0.005.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import torch

from . import abi
from . import fdo as FDO
from .rasterizer import Rasterizer, SceneTensors, _ptr, _stream, exchange_types

KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


@dataclass
class TrainConfig:
    extent: float = 1.0
    lr_means_init: float = 1.6e-4
    lr_means_final: float = 1.6e-6
    lr_steps: int = 30_000
    lr_sh_dc: float = 2.5e-3
    lr_sh_rest: float = 2.5e-3 / 20.0
    lr_opacity: float = 0.05
    lr_scales: float = 5e-3
    lr_quats: float = 1e-3
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    densify_from: int = 500
    densify_until: int = 15_000
    densify_every: int = 100
    densify_grad_ndc: float = 2e-4
    percent_dense: float = 0.01
    min_opacity: float = 0.005
    opacity_reset_every: int = 3000
    exchange_from: int = 500
    exchange_every: int = 500
    theta_e: float = 2.05
    fdo: bool = False
    lambda_low: float = FDO.LAMBDA_LOW
    lambda_high: float = FDO.LAMBDA_HIGH


class Trainer:
    """Owns the trainable arrays, their Adam moments and the densification
    statistics on the device; `scene` (SceneTensors) is replaced after each
    densification."""

    def __init__(self, scene: SceneTensors, render_cfg, tcfg: TrainConfig | None = None, device="cuda",
                 seed: int = 0):
        self.device = torch.device(device)
        self.cfg = render_cfg
        self.tcfg = tcfg or TrainConfig()
        self.rast = Rasterizer(self.device)
        self.gen = torch.Generator(device=self.device).manual_seed(seed)
        self.it = 0
        self.adam_t = 0
        self._adopt(scene, None)

    # -- state ------------------------------------------------------------
    def _adopt(self, scene: SceneTensors, moments):
        self.scene = scene
        p = self.params()
        self.moments = moments or {f"{w}_{k}": torch.zeros_like(p[k]) for w in ("m", "v") for k in KEYS}
        n = scene.n
        self.accum = torch.zeros(max(n, 1), dtype=torch.float32, device=self.device)
        self.count = torch.zeros(max(n, 1), dtype=torch.float32, device=self.device)

    def params(self):
        s = self.scene
        return {"means": s.means, "log_scales": s.log_scales, "quats": s.quats, "opacity_logits": s.opacity_logits,
                "sh": s.sh}

    def lr_means(self):
        t = self.tcfg
        f = min(1.0, self.it / max(1, t.lr_steps))
        return math.exp((1 - f) * math.log(t.lr_means_init) + f * math.log(t.lr_means_final)) * t.extent

    # -- one iteration ----------------------------------------------------
    def step(self, cam, target):
        """One training iteration on one view.  Returns the loss tensor
        (device float64: L1, L_low, L_high)."""
        t = self.tcfg
        self.it += 1
        maps = self.rast.forward(self.scene, cam, self.cfg)
        if t.fdo:
            ls = FDO.image_losses(maps["rgb"], target, 1.0, t.lambda_low, t.lambda_high)
            grads = FDO.fdo_backward(self.rast, ls["g_l1"], ls["g_low"], ls["g_high"])
            rec = self.rast.grad_ws3  # first set: the appearance loss's record gradients
        else:
            ls = FDO.image_losses(maps["rgb"], target, 1.0, 0.0, 0.0, want_grads=True)
            grads = self.rast.backward(ls["g_l1"], None, None, None)
            rec = self.rast.grad_ws
        if self.it < t.densify_until:
            abi.check(abi.hgs_grad_stats(self.scene.n, _ptr(rec), C.byref(self.rast.proj_struct()),
                                         _ptr(self.accum), _ptr(self.count), _stream()), "hgs_grad_stats")
        self.adam(grads)
        self.schedule(cam)
        return ls["loss"]

    def adam(self, grads):
        t = self.tcfg
        self.adam_t += 1
        p = self.params()
        nb3 = p["sh"].shape[1] * 3
        lrs = {"means": (self.lr_means(), 0, 0, 0.0), "log_scales": (t.lr_scales, 0, 0, 0.0),
               "quats": (t.lr_quats, 0, 0, 0.0), "opacity_logits": (t.lr_opacity, 0, 0, 0.0),
               "sh": (t.lr_sh_dc, nb3, 3, t.lr_sh_rest) if nb3 >= 4 else (t.lr_sh_dc, 0, 0, 0.0)}
        groups = (abi.hgs_adam_group * 5)()
        for j, k in enumerate(KEYS):
            lr, period, head, tail = lrs[k]
            groups[j] = abi.hgs_adam_group(_ptr(p[k]), _ptr(grads[k]), _ptr(self.moments[f"m_{k}"]),
                                           _ptr(self.moments[f"v_{k}"]), p[k].numel(), lr, period, head, tail)
        self._keep_groups = (groups, grads)
        abi.check(abi.hgs_adam_step(5, groups, self.adam_t, t.beta1, t.beta2, t.eps, _stream()), "hgs_adam_step")

    def schedule(self, cam):
        t, it = self.tcfg, self.it
        if t.densify_from <= it < t.densify_until and it % t.densify_every == 0:
            grad_px = t.densify_grad_ndc / (0.5 * max(cam.width, cam.height))
            self.densify(grad_px)
        if t.opacity_reset_every and it % t.opacity_reset_every == 0:
            self.reset_opacity()
        if it >= t.exchange_from and it % t.exchange_every == 0:
            exchange_types(self.scene, mode="erank", theta_e=t.theta_e)

    # -- densification -----------------------------------------------------
    def densify(self, grad_thresh_px):
        t = self.tcfg
        s = self.scene
        n = s.n
        d = self.device
        cfg = abi.hgs_densify_cfg(grad_thresh_px, math.log(t.percent_dense * t.extent),
                                  math.log(t.min_opacity / (1.0 - t.min_opacity)))
        nb = C.c_size_t()
        abi.check(abi.hgs_densify_workspace(n, C.byref(nb)), "hgs_densify_workspace")
        ws = torch.empty(int(nb.value), dtype=torch.uint8, device=d)
        actions = torch.empty(max(n, 1), dtype=torch.int32, device=d)
        offsets = torch.empty(n + 1, dtype=torch.int64, device=d)
        d_new = torch.zeros(1, dtype=torch.int64, device=d)
        ss = s.struct()
        abi.check(abi.hgs_densify_plan(C.byref(ss), _ptr(self.accum), _ptr(self.count), C.byref(cfg), _ptr(actions),
                                       _ptr(offsets), _ptr(ws), nb.value, _ptr(d_new), _stream()), "hgs_densify_plan")
        z = torch.randn((max(n, 1), 2, 3), generator=self.gen, device=d, dtype=torch.float32)
        m = int(d_new.item())  # the one host read of a densification
        new = SceneTensors(*(torch.empty((m,) + tuple(getattr(s, k).shape[1:]), dtype=torch.float32, device=d)
                             for k in KEYS), torch.empty(m, dtype=torch.uint8, device=d), s.sh_degree)
        mom = {k: torch.empty((m,) + tuple(v.shape[1:]), dtype=torch.float32, device=d) for k, v in self.moments.items()}
        ain = self._arrays(s, self.moments)
        aout = self._arrays(new, mom)
        abi.check(abi.hgs_densify_apply(n, s.sh_degree, C.byref(ain), C.byref(aout), _ptr(z), _ptr(actions),
                                        _ptr(offsets), _stream()), "hgs_densify_apply")
        self._adopt(new, mom)
        return actions, offsets, m

    @staticmethod
    def _arrays(s: SceneTensors, mom):
        order = [f"{w}_{k}" for w in ("m", "v") for k in KEYS]
        return abi.hgs_train_arrays(_ptr(s.means), _ptr(s.log_scales), _ptr(s.quats), _ptr(s.opacity_logits),
                                    _ptr(s.sh), _ptr(s.types), (C.c_void_p * 10)(*[_ptr(mom[k]) for k in order]))

    def reset_opacity(self, ceiling=0.01):
        s = self.scene
        abi.check(abi.hgs_reset_opacity(s.n, _ptr(s.opacity_logits), ceiling, _ptr(self.moments["m_opacity_logits"]),
                                        _ptr(self.moments["v_opacity_logits"]), _stream()), "hgs_reset_opacity")
