"""Continuous-batching render server over scenes resident on the device.

Requests (scene id, camera) arrive over time.  The loop admits waiting
requests into a batch in arrival order while the batch stays within its
budgets (requests per batch, primitives, stacked tile rows and an estimate of
tile instances), and renders the whole batch with hgs_render_batch: one
preprocess, one sort and one render launch for all its scenes and
resolutions.  Batches run on a small pool of CUDA streams, so a batch admitted
while another is still on the GPU overlaps with it.  Completion is observed
with CUDA events; latency is completion minus arrival.

`plain=True` gives the baseline the server is compared with: one request per
launch sequence (hgs_preprocess, hgs_bin_sort, hgs_render_fwd) on one stream.
"""
from __future__ import annotations

import ctypes as C
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import abi
from .rasterizer import Rasterizer, SceneTensors, camera_struct, config_struct

TILE = 16


@dataclass
class ServingConfig:
    max_batch: int = 8            # requests per launch (<= HGS_MAX_BATCH)
    streams: int = 2              # batches in flight
    prim_budget: int = 8_000_000  # primitives per batch (workspace rows)
    row_budget: int = 8 * 68      # stacked 16-px tile rows per batch
    capacity: int = 120_000_000   # tile instances per batch
    safety: float = 1.3           # instance estimate margin at admission


@dataclass
class Request:
    rid: int
    t_arrival: float
    scene_id: int
    cam: object
    t_launch: float = 0.0
    t_done: float = 0.0
    attempts: int = 0
    failed: bool = False
    out: dict = field(default_factory=dict)


def take_batch(pending, n_of, rows_of, k_of, scfg):
    """Admission: take waiting requests in arrival order while the batch stays
    within the request, primitive, tile-row and instance budgets (the first
    request is always taken, so nothing starves)."""
    batch, prims, rows, kest = [], 0, 0, 0.0
    while pending and len(batch) < min(scfg.max_batch, abi.HGS_MAX_BATCH):
        r = pending[0]
        n, rr, k = n_of(r), rows_of(r), k_of(r) * scfg.safety
        if batch and (prims + n > scfg.prim_budget or rows + rr > scfg.row_budget
                      or kest + k > scfg.capacity):
            break
        batch.append(pending.popleft())
        prims += n
        rows += rr
        kest += k
    return batch


def _out_planes(W, H, device):
    return {"rgb": torch.empty((3, H, W), dtype=torch.float32, device=device),
            "depth": torch.empty((H, W), dtype=torch.float32, device=device),
            "normal": torch.empty((3, H, W), dtype=torch.float32, device=device),
            "alpha": torch.empty((H, W), dtype=torch.float32, device=device),
            "T_final": torch.empty((H, W), dtype=torch.float32, device=device),
            "n_last": torch.empty((H, W), dtype=torch.int32, device=device)}


def _request_struct(scene: SceneTensors, cam, out):
    img = abi.hgs_image(out["rgb"].data_ptr(), out["depth"].data_ptr(), out["normal"].data_ptr(),
                        out["alpha"].data_ptr(), out["T_final"].data_ptr(), out["n_last"].data_ptr(), None)
    return abi.hgs_request(scene.struct(), camera_struct(cam), img)


class BatchRenderer:
    """One workspace per stream, sized for the batch budgets."""

    def __init__(self, device, cfg, scfg: ServingConfig):
        self.device = torch.device(device)
        self.cfg_s = config_struct(cfg)
        self.scfg = scfg
        # workspace for the budgets: a request list with the budgeted primitives
        # and tile rows (the layout depends only on those sums and the width)
        probe = abi.hgs_request()
        probe.scene.n = scfg.prim_budget
        probe.scene.sh_degree = 3
        probe.cam.width = 2048
        probe.cam.height = scfg.row_budget * TILE
        nb = C.c_size_t()
        abi.check(abi.hgs_render_batch_workspace(1, C.byref(probe), scfg.capacity, C.byref(nb)),
                  "hgs_render_batch_workspace")
        self.ws_bytes = int(nb.value)
        self.slots = []
        for _ in range(scfg.streams):
            self.slots.append({
                "stream": torch.cuda.Stream(device=self.device),
                "ws": torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device),
                "d_count": torch.zeros(1, dtype=torch.int64, device=self.device),
                "dev_err": torch.zeros(1, dtype=torch.int32, device=self.device),
                "h_count": torch.zeros(1, dtype=torch.int64).pin_memory(),
                "h_err": torch.zeros(1, dtype=torch.int32).pin_memory(),
                "busy": False,
            })

    def launch(self, slot, scenes, cams, outs, capacity=None):
        """Enqueue one batched render on the slot's stream; returns its event."""
        n = len(scenes)
        arr = (abi.hgs_request * n)(*[_request_struct(s, c, o) for s, c, o in zip(scenes, cams, outs)])
        s = slot["stream"]
        with torch.cuda.stream(s):
            slot["dev_err"].zero_()
            st = abi.hgs_render_batch(n, arr, C.byref(self.cfg_s), C.c_void_p(slot["ws"].data_ptr()),
                                      self.ws_bytes, int(capacity or self.scfg.capacity),
                                      C.c_void_p(slot["d_count"].data_ptr()),
                                      C.c_void_p(slot["dev_err"].data_ptr()), C.c_void_p(s.cuda_stream))
            abi.check(st, "hgs_render_batch")
            slot["h_count"].copy_(slot["d_count"], non_blocking=True)
            slot["h_err"].copy_(slot["dev_err"], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(s)
        slot["busy"] = True
        slot["_keep"] = arr
        return ev


class Server:
    def __init__(self, scenes, cfg, scfg: ServingConfig | None = None, device="cuda", plain=False):
        self.scenes = scenes
        self.cfg = cfg
        self.scfg = scfg or ServingConfig()
        self.device = torch.device(device)
        self.plain = plain
        if plain:
            # the same fixed instance capacity as a batch, no per-frame read
            # of the instance count: an overflow is seen on the device and
            # the request is rendered again with room for it
            self.rast = Rasterizer(self.device, capacity=self.scfg.capacity, sync_check=False)
            self.stream = torch.cuda.Stream(device=self.device)
            self.h_err = torch.zeros(1, dtype=torch.int32).pin_memory()
            self.h_count = torch.zeros(1, dtype=torch.int64).pin_memory()
        else:
            self.br = BatchRenderer(self.device, cfg, self.scfg)
        # running estimate of tile instances per (scene, pixel): admission
        self.k_per_px = {i: 16.0 * s.n / (1280 * 720) for i, s in enumerate(scenes)}

    def _k_est(self, r):
        return self.k_per_px[r.scene_id] * r.cam.width * r.cam.height

    def _rows(self, r):
        return (r.cam.height + TILE - 1) // TILE

    def _take_batch(self, pending):
        return take_batch(pending, lambda r: self.scenes[r.scene_id].n, self._rows, self._k_est, self.scfg)

    # -- plain baseline: one request per launch sequence -----------------
    def _run_plain(self, reqs, realtime, keep):
        t0 = time.perf_counter()
        for r in reqs:
            if realtime:
                while time.perf_counter() - t0 < r.t_arrival:
                    time.sleep(2e-5)
            now = time.perf_counter() - t0
            r.t_launch = max(now, r.t_arrival)
            while True:
                with torch.cuda.stream(self.stream):
                    self.rast.dev_err.zero_()
                    out = self.rast.forward(self.scenes[r.scene_id], r.cam, self.cfg)
                    self.h_err.copy_(self.rast.dev_err, non_blocking=True)
                    self.h_count.copy_(self.rast.d_count, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(self.stream)
                while not ev.query():
                    time.sleep(2e-5)
                if int(self.h_err.item()) != abi.HGS_ERR_CAPACITY:
                    break
                self.rast._ensure_capacity(int(int(self.h_count.item()) * 1.25) + 1024)
            r.t_done = time.perf_counter() - t0
            if keep:
                r.out = {k: v.clone() for k, v in out.items()}
        return reqs

    # -- continuous batching ---------------------------------------------
    def _run_batched(self, reqs, realtime, keep):
        br = self.br
        t0 = time.perf_counter()
        pending = deque()
        inflight = []  # (slot, event, batch, outs)
        i = 0
        retry = deque()
        while i < len(reqs) or pending or inflight or retry:
            now = time.perf_counter() - t0
            while i < len(reqs) and (not realtime or reqs[i].t_arrival <= now):
                pending.append(reqs[i])
                i += 1
            # retire finished batches
            for item in list(inflight):
                slot, ev, batch, outs = item
                if ev.query():
                    t = time.perf_counter() - t0
                    inflight.remove(item)
                    slot["busy"] = False
                    K = int(slot["h_count"].item())
                    if int(slot["h_err"].item()) == abi.HGS_ERR_CAPACITY:
                        # estimate was short: learn and render these again alone;
                        # a request that overflows alone cannot be served
                        for r in batch:
                            self.k_per_px[r.scene_id] *= 2.0
                            if len(batch) == 1 and r.attempts > 1:
                                r.failed, r.t_done = True, t
                            else:
                                retry.append(r)
                        continue
                    px = sum(r.cam.width * r.cam.height for r in batch)
                    for r in batch:  # per-scene instance density, slow decay
                        est = K / max(px, 1)
                        self.k_per_px[r.scene_id] = max(0.9 * self.k_per_px[r.scene_id], est)
                    for r, o in zip(batch, outs):
                        r.t_done = t
                        if keep:
                            r.out = o
            # launch on a free slot
            free = [s for s in br.slots if not s["busy"]]
            if free and (retry or pending):
                batch = [retry.popleft()] if retry else self._take_batch(pending)
                now = time.perf_counter() - t0
                for r in batch:
                    r.t_launch = now
                    r.attempts += 1
                outs = [_out_planes(r.cam.width, r.cam.height, self.device) for r in batch]
                scenes = [self.scenes[r.scene_id] for r in batch]
                ev = br.launch(free[0], scenes, [r.cam for r in batch], outs)
                inflight.append((free[0], ev, batch, outs))
                continue
            time.sleep(2e-5)
        return reqs

    def run(self, requests, realtime=True, keep=False):
        """requests: iterable of (t_arrival, scene_id, cam).  Returns the
        Request list (t_arrival, t_launch, t_done filled) and a stats dict."""
        reqs = [Request(k, float(t), int(sid), cam) for k, (t, sid, cam) in enumerate(requests)]
        reqs.sort(key=lambda r: r.t_arrival)
        torch.cuda.synchronize(self.device)
        if self.plain:
            self._run_plain(reqs, realtime, keep)
        else:
            self._run_batched(reqs, realtime, keep)
        torch.cuda.synchronize(self.device)
        return reqs, stats(reqs)


def stats(reqs):
    failed = sum(r.failed for r in reqs)
    reqs = [r for r in reqs if not r.failed]
    lat = np.array([r.t_done - r.t_arrival for r in reqs]) * 1e3
    span = max(r.t_done for r in reqs) - min(r.t_arrival for r in reqs)
    return {"requests": len(reqs), "frames_per_s": len(reqs) / span if span > 0 else float("nan"),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "span_s": span, "failed": failed}


def render_batch_once(scenes, cams, cfg, device="cuda", capacity=60_000_000):
    """Render the (scene, camera) pairs as one batch; returns their outputs."""
    scfg = ServingConfig(max_batch=len(scenes), streams=1,
                         prim_budget=max(1, sum(s.n for s in scenes)),
                         row_budget=sum((c.height + TILE - 1) // TILE for c in cams),
                         capacity=capacity)
    br = BatchRenderer(device, cfg, scfg)
    outs = [_out_planes(c.width, c.height, torch.device(device)) for c in cams]
    ev = br.launch(br.slots[0], scenes, cams, outs)
    ev.synchronize()
    err = int(br.slots[0]["h_err"].item())
    if err != 0:
        raise abi.HgsError(err, "hgs_render_batch")
    return outs, int(br.slots[0]["h_count"].item())
