"""Device-buffer management around the C ABI, and the autograd Function.

PyTorch supplies device memory and the current CUDA stream; every step of the
hybrid rasterizer (preprocess, binning, blending, backward, exchange) runs in
libhgs's CUDA kernels.  There is no CPU or PyTorch fallback: on a machine
without CUDA, or without the library, these calls raise.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import abi

REC_FLOATS = 20
GRAD_FLOATS = 16
TILE = 16


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def camera_struct(cam) -> abi.hgs_camera:
    """Any object with R (3x3), t (3), fx, fy, cx, cy, width, height."""
    c = abi.hgs_camera()
    R = np.asarray(cam.R, np.float32).reshape(9)
    t = np.asarray(cam.t, np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def config_struct(cfg=None) -> abi.hgs_config:
    c = abi.hgs_config()
    abi.hgs_default_config(C.byref(c))
    if cfg is None:
        return c
    c.near_z = cfg.near
    c.alpha_min = cfg.alpha_min
    c.alpha_max = cfg.alpha_max
    c.T_min = cfg.T_min
    c.lambda_z = cfg.lambda_z
    c.theta_z = cfg.theta_z
    c.T_z = cfg.T_z
    c.dilation = cfg.dilation
    for i in range(3):
        c.bg[i] = float(cfg.bg[i])
    c.tile = int(cfg.tile)
    return c


@dataclass
class SceneTensors:
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    sh: torch.Tensor
    types: torch.Tensor
    sh_degree: int

    @property
    def n(self):
        return int(self.means.shape[0])

    @staticmethod
    def from_numpy(scene, device="cuda"):
        f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)
        return SceneTensors(f(scene.means), f(scene.log_scales), f(scene.quats),
                            f(scene.opacity_logits), f(scene.sh), f(scene.types), int(scene.sh_degree))

    def struct(self) -> abi.hgs_scene:
        for t in (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("scene tensors must be contiguous float32 CUDA tensors")
        if not (self.types.is_cuda and self.types.dtype == torch.uint8):
            raise ValueError("types must be a uint8 CUDA tensor")
        return abi.hgs_scene(self.means.data_ptr(), self.log_scales.data_ptr(), self.quats.data_ptr(),
                             self.opacity_logits.data_ptr(), self.sh.data_ptr(), self.types.data_ptr(),
                             self.n, self.sh_degree)

    def mut_struct(self) -> abi.hgs_scene_mut:
        return abi.hgs_scene_mut(self.log_scales.data_ptr(), self.quats.data_ptr(),
                                 self.types.data_ptr(), self.n)


class Rasterizer:
    """Holds the per-frame device buffers (projected records, binning
    workspace, instance lists, per-pixel auxiliaries) and runs the C ABI.

    One forward may be in flight per Rasterizer: backward() uses the buffers
    of the most recent forward()."""

    def __init__(self, device="cuda", capacity: int = 0, keep_keys: bool = False,
                 sync_check: bool = True):
        """sync_check=False skips the per-frame read of the instance count:
        the caller guarantees enough capacity and calls check() later (an
        overflow is still detected on the device and reported there)."""
        self.device = torch.device(device)
        self.capacity = int(capacity)
        self.keep_keys = keep_keys
        self.sync_check = sync_check
        self.n = -1
        # when a list, every backward appends the (start, end) CUDA events it
        # records around its record-gradient stage on the current stream
        self.bwd_events = None
        self.hw = None
        self.dev_err = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.d_count = torch.zeros(1, dtype=torch.int64, device=self.device)
        self.generation = 0
        self.last_K = 0
        self.ws = None
        self.vals = None
        self.keys = None

    # -- buffers ---------------------------------------------------------
    def _ensure_prims(self, n):
        if n == self.n:
            return
        d = self.device
        m = max(n, 1)
        self.rec = torch.empty((m, REC_FLOATS), dtype=torch.float32, device=d)
        self.depth_key = torch.empty(m, dtype=torch.int32, device=d)
        self.rect = torch.empty((m, 4), dtype=torch.int16, device=d)
        self.touched = torch.empty(m, dtype=torch.int32, device=d)
        self.tileset = torch.empty((m, 12), dtype=torch.float32, device=d)
        self.grad_ws = torch.empty((m, GRAD_FLOATS), dtype=torch.float32, device=d)
        self.n = n
        self.ws = None

    def _ensure_image(self, W, H):
        if self.hw == (W, H):
            return
        d = self.device
        self.T_final = torch.empty((H, W), dtype=torch.float32, device=d)
        self.n_last = torch.empty((H, W), dtype=torch.int32, device=d)
        self.n_contrib = torch.empty((H, W), dtype=torch.int32, device=d)
        TX, TY = (W + TILE - 1) // TILE, (H + TILE - 1) // TILE
        self.ranges = torch.empty((TX * TY, 2), dtype=torch.int32, device=d)
        self.tile_sched = torch.empty(2 * TX * TY + 1, dtype=torch.int32, device=d)
        self.hw = (W, H)
        self.ws = None

    def _ensure_capacity(self, cap):
        if self.vals is not None and self.vals.numel() >= cap and self.ws is not None:
            return
        cap = max(int(cap), 1024)
        self.capacity = cap
        self.vals = torch.empty(cap, dtype=torch.int32, device=self.device)
        self.keys = torch.empty(cap, dtype=torch.int64, device=self.device) if self.keep_keys else None
        W, H = self.hw
        tiles = ((W + TILE - 1) // TILE) * ((H + TILE - 1) // TILE)
        nb = C.c_size_t()
        abi.check(abi.hgs_bin_sort_workspace(self.n, cap, tiles, C.byref(nb)), "hgs_bin_sort_workspace")
        self.ws = torch.empty(int(nb.value), dtype=torch.uint8, device=self.device)

    def proj_struct(self):
        return abi.hgs_projected(self.rec.data_ptr(), self.depth_key.data_ptr(), self.rect.data_ptr(),
                                 self.touched.data_ptr(), self.tileset.data_ptr())

    def bin_struct(self):
        return abi.hgs_binning(self.vals.data_ptr(), self.keys.data_ptr() if self.keys is not None else None,
                               self.ranges.data_ptr(), self.d_count.data_ptr())

    # -- forward -------------------------------------------------------------
    def preprocess(self, scene: SceneTensors, cam, cfg=None):
        self._ensure_prims(scene.n)
        self._ensure_image(cam.width, cam.height)
        # the backward reads the same parameter arrays: keep them alive with
        # the raw pointers the ABI structs hold
        self._scene_ref = scene
        self._scene_s = scene.struct()
        self._cam_s = camera_struct(cam)
        self._cfg_s = config_struct(cfg)
        self._proj_s = self.proj_struct()
        abi.check(abi.hgs_preprocess(C.byref(self._scene_s), C.byref(self._cam_s), C.byref(self._cfg_s),
                                     C.byref(self._proj_s), _ptr(self.dev_err), _stream()), "hgs_preprocess")

    def bin_sort(self, sync_check=True):
        if self.ws is None or self.vals is None or self.vals.numel() < self.capacity:
            cap = self.capacity or max(1 << 16, 8 * max(self.n, 1))
            self._ensure_capacity(cap)
        while True:
            bins = self.bin_struct()
            abi.check(abi.hgs_bin_sort(self.n, C.byref(self._proj_s), C.byref(self._cam_s),
                                       C.byref(self._cfg_s), _ptr(self.ws), self.ws.numel(),
                                       self.capacity, C.byref(bins), _ptr(self.dev_err), _stream()),
                      "hgs_bin_sort")
            if not sync_check:
                return
            K = int(self.d_count.item())
            self.last_K = K
            if K <= self.capacity:
                return
            # grow and redo: the overflowed call wrote nothing out of bounds
            self.dev_err.zero_()
            self.vals = None
            self._ensure_capacity(int(K * 1.25) + 1024)

    def render(self):
        W, H = self.hw
        d = self.device
        out = {
            "rgb": torch.empty((3, H, W), dtype=torch.float32, device=d),
            "depth": torch.empty((H, W), dtype=torch.float32, device=d),
            "normal": torch.empty((3, H, W), dtype=torch.float32, device=d),
            "alpha": torch.empty((H, W), dtype=torch.float32, device=d),
        }
        img = abi.hgs_image(out["rgb"].data_ptr(), out["depth"].data_ptr(), out["normal"].data_ptr(),
                            out["alpha"].data_ptr(), self.T_final.data_ptr(), self.n_last.data_ptr(),
                            self.n_contrib.data_ptr(), self.tile_sched.data_ptr())
        self._img_s = img
        bins = self.bin_struct()
        abi.check(abi.hgs_render_fwd(self.n, C.byref(self._proj_s), C.byref(bins), C.byref(self._cam_s),
                                     C.byref(self._cfg_s), C.byref(img), _ptr(self.dev_err), _stream()),
                  "hgs_render_fwd")
        self.generation += 1
        return out

    def forward(self, scene: SceneTensors, cam, cfg=None, sync_check=None):
        self.preprocess(scene, cam, cfg)
        self.bin_sort(sync_check=self.sync_check if sync_check is None else sync_check)
        out = self.render()
        out["T_final"] = self.T_final
        out["n_last"] = self.n_last
        out["n_contrib"] = self.n_contrib
        return out

    # -- backward ------------------------------------------------------------
    def backward(self, g_rgb=None, g_depth=None, g_normal=None, g_alpha=None, grads=None, stages=False):
        """Gradients of the raw parameters.  stages=True issues the two ABI
        stages (record gradients, then preprocess backward) separately and
        returns (grads, fn_records, fn_preprocess) callables for timing."""
        return self._backward(g_rgb, g_depth, g_normal, g_alpha, grads, stages)

    def _backward(self, g_rgb, g_depth, g_normal, g_alpha, grads, stages):
        n = self.n
        deg = self._scene_s.sh_degree
        nb = (deg + 1) ** 2
        d = self.device
        if grads is None:
            grads = {
                "means": torch.empty((n, 3), dtype=torch.float32, device=d),
                "log_scales": torch.empty((n, 3), dtype=torch.float32, device=d),
                "quats": torch.empty((n, 4), dtype=torch.float32, device=d),
                "opacity_logits": torch.empty(n, dtype=torch.float32, device=d),
                "sh": torch.empty((n, nb, 3), dtype=torch.float32, device=d),
            }
        keep = [t.contiguous() if t is not None else None for t in (g_rgb, g_depth, g_normal, g_alpha)]
        dl = abi.hgs_image_grad(*[(t.data_ptr() if t is not None else None) for t in keep])
        out = abi.hgs_scene_grad(grads["means"].data_ptr(), grads["log_scales"].data_ptr(),
                                 grads["quats"].data_ptr(), grads["opacity_logits"].data_ptr(),
                                 grads["sh"].data_ptr())
        bins = self.bin_struct()
        self._keep_grads = (keep, dl, out, bins)
        if stages:
            def records():
                abi.check(abi.hgs_render_bwd_records(C.byref(self._scene_s), C.byref(self._proj_s), C.byref(bins),
                                                     C.byref(self._cam_s), C.byref(self._cfg_s),
                                                     C.byref(self._img_s), C.byref(dl), _ptr(self.grad_ws),
                                                     _ptr(self.dev_err), _stream()), "hgs_render_bwd_records")

            def prep():
                abi.check(abi.hgs_preprocess_bwd(C.byref(self._scene_s), C.byref(self._proj_s),
                                                 C.byref(self._cam_s), C.byref(self._cfg_s), _ptr(self.grad_ws),
                                                 C.byref(out), _ptr(self.dev_err), _stream()), "hgs_preprocess_bwd")
            return grads, records, prep
        if self.bwd_events is not None:
            st = torch.cuda.current_stream(self.device)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            abi.check(abi.hgs_render_bwd_records(C.byref(self._scene_s), C.byref(self._proj_s), C.byref(bins),
                                                 C.byref(self._cam_s), C.byref(self._cfg_s), C.byref(self._img_s),
                                                 C.byref(dl), _ptr(self.grad_ws), _ptr(self.dev_err), _stream()),
                      "hgs_render_bwd_records")
            e1.record(st)
            self.bwd_events.append((e0, e1))
            abi.check(abi.hgs_preprocess_bwd(C.byref(self._scene_s), C.byref(self._proj_s), C.byref(self._cam_s),
                                             C.byref(self._cfg_s), _ptr(self.grad_ws), C.byref(out),
                                             _ptr(self.dev_err), _stream()), "hgs_preprocess_bwd")
            return grads
        abi.check(abi.hgs_render_bwd(C.byref(self._scene_s), C.byref(self._proj_s), C.byref(bins),
                                     C.byref(self._cam_s), C.byref(self._cfg_s), C.byref(self._img_s),
                                     C.byref(dl), _ptr(self.grad_ws), C.byref(out), _ptr(self.dev_err),
                                     _stream()), "hgs_render_bwd")
        return grads

    def check(self):
        """Synchronise and raise if a kernel reported a data-dependent error."""
        e = C.c_int32(0)
        st = abi.hgs_check(_ptr(self.dev_err), C.byref(e), _stream())
        if st != abi.HGS_OK:
            self.dev_err.zero_()
            raise abi.HgsError(st, "device error")


def exchange_types(scene: SceneTensors, mode="erank", theta_e=2.05, mask=None, d_flipped=None):
    """Adaptive Type Exchange in place on the scene's own tensors."""
    x = abi.hgs_exchange_cfg(abi.HGS_EXCHANGE_ERANK if mode == "erank" else abi.HGS_EXCHANGE_MASK,
                             float(theta_e), mask.data_ptr() if mask is not None else None)
    s = scene.mut_struct()
    abi.check(abi.hgs_exchange_types(C.byref(s), C.byref(x), _ptr(d_flipped), None, _stream()),
              "hgs_exchange_types")


class RasterizeFunction(torch.autograd.Function):
    """(means, log_scales, quats, opacity_logits, sh) -> (rgb, depth, normal,
    alpha); `types` is a non-differentiable uint8 buffer."""

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, types, rast, cam, cfg, sh_degree):
        scene = SceneTensors(means.detach(), log_scales.detach(), quats.detach(),
                             opacity_logits.detach(), sh.detach(), types, sh_degree)
        out = rast.forward(scene, cam, cfg)
        # maps the loss does not use arrive as None (not zero images), so an
        # image-only loss runs the backward specialised for it
        ctx.set_materialize_grads(False)
        ctx.rast = rast
        ctx.gen = rast.generation
        ctx.scene = scene
        return out["rgb"], out["depth"], out["normal"], out["alpha"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_normal, g_alpha):
        rast = ctx.rast
        if rast.generation != ctx.gen:
            raise RuntimeError("Rasterizer buffers were reused by a later forward before backward")
        g = rast.backward(g_rgb, g_depth, g_normal, g_alpha)
        return g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"], None, None, None, None, None


def rasterize(scene: SceneTensors, cam, cfg=None, rast: Rasterizer | None = None):
    rast = rast or Rasterizer(scene.means.device)
    return RasterizeFunction.apply(scene.means, scene.log_scales, scene.quats, scene.opacity_logits,
                                   scene.sh, scene.types, rast, cam, cfg, scene.sh_degree)
