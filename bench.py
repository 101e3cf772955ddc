"""Benchmark of the hybrid 2D/3D Gaussian rasterizer on GB300.

Default workload: the scene-scale training step -- 3,000,000 primitives (70%
3D Gaussians, 30% 2D surfels, SH degree 3) on a unit-sphere shell plus ground
plane, one 1600x1064 pinhole view (fov 50 deg), forward + backward through the
autograd Function on an L1 loss against a random target image, with a
mask-mode type exchange of 1% of the flags every 100 steps.  One step is one
pass of the whole hot path: preprocess, binning (scan, emit, radix sort, tile
ranges), blend forward, blend backward, preprocess backward (+ exchange).

Prints one JSON line (see the keys below).  `--impl reference` times the CPU
oracle instead (the reference arm of this build).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/iter @3M prims 1600x1064; served frames/s + p50/p99 latency"


def workload(args):
    return (f"scene-scale training step: {args.n} prims (70% 3D / 30% 2D, SH deg 3), "
            f"{args.width}x{args.height}, fwd+bwd, L1 loss")


def base_config(args, world):
    """The config both arms print (the GPU arm and the reference arm)."""
    return {"workload": workload(args), "n_prims": args.n, "width": args.width, "height": args.height,
            "sh_degree": 3, "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2 (scene 708 MB, records 240 MB, lists > 100 MB)"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--prims", dest="n", type=int, default=3_000_000)
    p.add_argument("--width", type=int, default=1600)
    p.add_argument("--height", type=int, default=1064)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-sample-pixels", type=int, default=20000)
    p.add_argument("--profile-phases", action="store_true", default=True)
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-fdo", action="store_true")
    p.add_argument("--no-train", action="store_true")
    p.add_argument("--no-stress", action="store_true")
    p.add_argument("--binning-probe", action="store_true",
                   help="time only the binning of the stress scene recipe at --prims primitives and "
                        "--width x --height, over --steps calls (one JSON line)")
    p.add_argument("--serving-seconds", type=float, default=20.0)
    p.add_argument("--serving-rate", type=float, default=200.0)
    return p.parse_args()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed
    region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.samples = []
        self.proc = None
        self.gpu_index = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # the timed region starts only once samples are flowing
        t0 = time.time()
        while not self.samples and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for k, nm in enumerate(names):
                if s[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


# ---------------------------------------------------------------------------
def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        # the reference arm runs on rank 0 alone and needs no process group
        import torch.distributed as dist
        dist.init_process_group(backend="nccl")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device=None):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
def cpu_baseline(scene, cam, cfg, sample_pixels, seed=0):
    """The oracle as it stands, on a bounded sample: FP64 per-primitive
    preparation of all N primitives plus the per-pixel render of a random pixel
    sample, extrapolated to one full-frame forward."""
    from oracle import native as O
    rng = np.random.default_rng(seed)
    W, H = cam.width, cam.height
    pix = np.stack([rng.integers(0, W, sample_pixels), rng.integers(0, H, sample_pixels)], 1)
    t0 = time.perf_counter()
    orc = O.Oracle(scene, cam, cfg)
    t1 = time.perf_counter()
    orc.render(pix)
    t2 = time.perf_counter()
    orc.close()
    per_frame = (t1 - t0) + (t2 - t1) * (W * H) / sample_pixels
    return {
        "value": round(per_frame * 1e3, 3), "unit": "ms", "cores": O.num_threads(),
        "kind": "oracle",
        "sample": (f"forward only, extrapolated from {sample_pixels} sampled pixels: FP64 C oracle, "
                   f"prepare all {scene.n} prims ({t1 - t0:.2f} s) + render the sampled pixels "
                   f"({t2 - t1:.2f} s), scaled to one {W}x{H} frame; the backward is not included (the "
                   f"oracle's gradients are finite differences and FP64 autograd on small scenes)"),
        "forward_only": True, "extrapolated": True, "measured_s": round(t2 - t0, 3),
        "host_cpus": os.cpu_count(),
    }


def reference_arm(args, world, rank):
    import synthetic as S
    if rank != 0:
        return
    scene, cam = S.scene_scale(args.n, seed=1)
    cam = S.orbit_camera(30.0, 20.0, 3.0, args.width, args.height, 50.0)
    cfg = S.RenderConfig()
    per_step, measured = [], []
    sample = max(2000, args.cpu_sample_pixels // max(1, args.steps))
    res = None
    for k in range(args.warmup + args.steps):
        res = cpu_baseline(scene, cam, cfg, sample, seed=k)
        if k >= args.warmup:
            per_step.append(res["value"])
            measured.append(res["measured_s"])
    v = float(np.median(per_step))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": base_config(args, world),
            "cpu_baseline": {"value": v, "unit": "ms", "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"], "forward_only": True, "extrapolated": True,
                             "measured_s_per_step": round(float(np.median(measured)), 3)},
            "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def run_serving(args, dev, cfg):
    """Serving workload: 4 resident scenes (200k, 500k, 1M, 3M primitives,
    3D shares 50-80%, SH degree 3), Poisson arrivals with random orbit poses
    and resolutions from {512^2, 800x600, 1280x720, 1920x1080}; the batched
    server against the one-request-per-launch renderer, in real time, then
    both saturated (all requests waiting at t = 0)."""
    import synthetic as S
    from paper_2512_02932_gb300 import SceneTensors
    from paper_2512_02932_gb300.serving import Server, ServingConfig
    scenes = [SceneTensors.from_numpy(sc, dev) for sc in S.serving_scenes()]
    reqs = S.serving_requests(seed=3, rate_hz=args.serving_rate, duration_s=args.serving_seconds)
    out = {"workload": f"4 resident scenes (200k/500k/1M/3M prims), Poisson {args.serving_rate:g} req/s "
                       f"for {args.serving_seconds:g} s, mixed resolutions", "requests": len(reqs)}
    warm = reqs[:16]
    for name, plain in (("batched", False), ("plain", True)):
        srv = Server(scenes, cfg, ServingConfig(), device=dev, plain=plain)
        srv.run(warm, realtime=False)
        _, st = srv.run(reqs, realtime=True)
        _, sat = srv.run([(0.0, sid, cam) for (_, sid, cam) in reqs[:400]], realtime=False)
        out[name] = {"frames_per_s": round(st["frames_per_s"], 2), "p50_ms": round(st["p50_ms"], 3),
                     "p99_ms": round(st["p99_ms"], 3), "mean_ms": round(st["mean_ms"], 3),
                     "saturated_frames_per_s": round(sat["frames_per_s"], 2),
                     "saturated_p50_ms": round(sat["p50_ms"], 3), "failed": st["failed"]}
        del srv
        torch_sync(dev)
    return out


def torch_sync(dev):
    import torch
    torch.cuda.synchronize(dev)


def launches_per_step(rast, exchange_steps, steps):
    tiles = rast.ranges.shape[0]
    tile_bits = max(1, math.ceil(math.log2(tiles))) if tiles > 1 else 1
    passes = (tile_bits + 7) // 8
    # 4 depth passes and the tile passes (chunk histogram, chunk scan,
    # scatter each), offsets scan (3), emit (2), range fix-up, optional
    # 64-bit keys.  Render forward and backward: tile work, tile order and
    # the kernel each; preprocess forward and backward one each.
    bin_sort = 3 * (4 + passes) + 3 + 2 + 1 + (1 if rast.keys is not None else 0)
    per = 1 + bin_sort + 3 + 3 + 1
    return per * steps + exchange_steps


def busy_launch(dev, iters):
    """Queue a short FMA-only kernel (no memory traffic) so that the work
    queued after it starts without waiting for the host."""
    import ctypes as C

    import torch

    from paper_2512_02932_gb300 import abi
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = torch.empty(sms * 8, dtype=torch.float32, device=dev)
    fl = C.c_double()
    s = torch.cuda.current_stream(dev)
    abi.check(abi.hgs_fp32_probe(sms * 8, iters, C.c_void_p(out.data_ptr()), C.byref(fl),
                                 C.c_void_p(s.cuda_stream)), "hgs_fp32_probe")
    return out


def alu_peak(dev, kind=0):
    """Peak rate of one unit, measured in this run by hgs_alu_probe (8
    independent chains per thread, 8 CTAs of 256 threads per SM) sized to run
    ~10 ms, best of three CUDA-event timings.  kind: HGS_PROBE_FFMA (FP32
    flops), _FFMA2, _EX2 or _RCP (special-function ops).  Returns (T ops/s,
    description)."""
    import ctypes as C

    import torch

    from paper_2512_02932_gb300 import abi
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks, dtype=torch.float32, device=dev)
    ops = C.c_double()
    s = torch.cuda.current_stream(dev)

    def run(iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        abi.check(abi.hgs_alu_probe(kind, blocks, iters, C.c_void_p(out.data_ptr()), C.byref(ops),
                                    C.c_void_p(s.cuda_stream)), "hgs_alu_probe")
        e1.record(s)
        torch.cuda.synchronize(dev)
        return ops.value / (e0.elapsed_time(e1) * 1e-3) / 1e12, e0.elapsed_time(e1)

    _, ms = run(2000)
    iters = max(1000, int(2000 * 10.0 / max(ms, 1e-3)))
    best = max(run(iters)[0] for _ in range(3))
    name = {0: "FFMA", 1: "FFMA2", 2: "EX2", 3: "RCP"}[kind]
    return best, f"measured: hgs_alu_probe {name}, {blocks} CTAs x 256 threads x 8 chains x {iters} steps"


def hbm_phases(phases, n, n_binned, K, tile_passes, peak, peak_src):
    """Achieved HBM bandwidth of the memory-bound phases from their
    algorithmic bytes (each array read or written once) and their CUDA-event
    times.  preprocess: 45 B read + 16 B written per primitive, + 192 B of SH
    read + 80 B of record and 32 B of tile-set parameters written per binned
    one.  preprocess_bwd: 385 B read per binned primitive (parameters, SH,
    record, record gradient) + 4 B per culled one, 236 B written per
    primitive.  bin_sort: four depth passes over the binned primitives (4 B
    histogram read + 8 B read + 8 B written) and two scans (8 B) and the
    emit's reads (id, offset, rectangle, count, tile set: 48 B), per instance
    the emit (8 B written) and each tile pass (4 B histogram read + 8 B read
    + 8 B written, the last 4 B written)."""
    nb, nc = n_binned, n - n_binned
    byts = {
        "preprocess": 61 * n + 304 * nb,
        "preprocess_bwd": 385 * nb + 4 * nc + 236 * n,
        "bin_sort": (4 * 20 + 16 + 48) * nb + 8 * K + tile_passes * 20 * K - 4 * K,
    }
    out = {}
    for k, b in byts.items():
        if k in phases and phases[k] > 0:
            gbs = b / (phases[k] * 1e-3) / 1e9
            out[k] = {"bytes": int(b), "achieved_gbs": round(gbs, 1), "peak_gbs": peak,
                      "frac": round(gbs / peak, 4)}
    if "bin_sort" in out:
        # the same phase against an unfactored sort's bytes: emit 12 B and
        # ranges 8 B per instance, six 24-B passes of 8 digit bits over the
        # 64-bit keys, a 4-B scan per primitive
        sv = 164 * K + 4 * n
        gbs = sv / (phases["bin_sort"] * 1e-3) / 1e9
        out["bin_sort"]["unfactored_sort_bytes"] = int(sv)
        out["bin_sort"]["unfactored_frac"] = round(gbs / peak, 4)
    out["peak_source"] = peak_src
    return out


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def run_fdo(args, dev, st, cam, cfg, target):
    """Frequency-decoupled training step on the same workload: forward, the
    Eq. 8 image losses (L1 + Haar L_low/L_high, one kernel) and the Algorithm 1
    backward (three rgb replays + fused projection)."""
    import torch
    from paper_2512_02932_gb300 import Rasterizer, fdo
    rast = Rasterizer(dev, sync_check=True)
    ctr = torch.zeros(1, dtype=torch.int64, device=dev)
    for _ in range(3):
        fdo.fdo_step(st, cam, cfg, target, rast)
    torch.cuda.synchronize()
    reps = max(3, min(20, args.steps))
    names = ["forward", "losses", "bwd_fdo"]
    acc = {n: 0.0 for n in names}
    s = torch.cuda.current_stream()
    e_all0, e_all1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_all0.record(s)
    for k in range(reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(s)
        maps = rast.forward(st, cam, cfg)
        ev[1].record(s)
        ls = fdo.image_losses(maps["rgb"], target, 1.0, fdo.LAMBDA_LOW, fdo.LAMBDA_HIGH)
        ev[2].record(s)
        if k == reps - 1:
            ctr.zero_()
        fdo.fdo_backward(rast, ls["g_l1"], ls["g_low"], ls["g_high"], d_conflicts=ctr if k == reps - 1 else None)
        ev[3].record(s)
        torch.cuda.synchronize()
        for i, n in enumerate(names):
            acc[n] += ev[i].elapsed_time(ev[i + 1])
    e_all1.record(s)
    torch.cuda.synchronize()
    rast.check()
    ph = {n: round(v / reps, 4) for n, v in acc.items()}
    C_, H_, W_ = target.shape
    loss_bytes = 4 * C_ * H_ * W_ * (2 + 3)  # image + target read, three gradient images written
    gbs = loss_bytes / (ph["losses"] * 1e-3) / 1e9
    peak, src = hbm_peak()
    touched = int((rast.touched[: st.n] > 0).sum().item())
    return {"workload": "same scene and view; loss = L1 + 0.2 L_low + 0.4 L_high (Haar level 1), Algorithm 1 backward",
            "ms_per_step": round(sum(ph.values()), 4), "phases_ms": ph,
            "image_losses": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(gbs / peak, 4), "bytes": loss_bytes, "peak_source": src},
            "conflicting_fraction": round(int(ctr.item()) / max(touched, 1), 4),
            "losses": [round(float(v), 6) for v in ls["loss"].cpu().tolist()]}


def run_train(args, dev, scene_np, cam, cfg, target):
    """Full training iteration on the same workload through Trainer: forward,
    L1 loss, backward, densification statistic and the fused Adam update of
    all 59 floats per primitive (densify / reset / exchange disabled so the
    primitive count stays fixed)."""
    import torch
    from paper_2512_02932_gb300 import SceneTensors
    from paper_2512_02932_gb300.train import TrainConfig, Trainer
    tc = TrainConfig(densify_from=10 ** 9, opacity_reset_every=0, exchange_from=10 ** 9)
    tr = Trainer(SceneTensors.from_numpy(scene_np, dev), cfg, tc, device=dev)
    for _ in range(3):
        tr.step(cam, target)
    torch.cuda.synchronize()
    reps = max(3, min(20, args.steps))
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        tr.step(cam, target)
    e1.record(s)
    torch.cuda.synchronize()
    it_ms = e0.elapsed_time(e1) / reps
    # the optimizer alone, on the last gradients
    grads = tr._keep_groups[1]
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(s)
    for _ in range(reps):
        tr.adam(grads)
    a1.record(s)
    torch.cuda.synchronize()
    tr.rast.check()
    adam_ms = a0.elapsed_time(a1) / reps
    floats = sum(p.numel() for p in tr.params().values())
    adam_bytes = 28 * floats  # read p, g, m, v; write p, m, v
    gbs = adam_bytes / (adam_ms * 1e-3) / 1e9
    peak, src = hbm_peak()
    return {"workload": "same scene and view; Trainer.step: forward, L1, backward, statistic, Adam (59 floats/prim)",
            "ms_per_iteration": round(it_ms, 4), "adam_ms": round(adam_ms, 4),
            "adam": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(gbs / peak, 4), "bytes": adam_bytes, "peak_source": src}}


def run_stress(args, dev, cfg):
    """The stress workload: 6M primitives (90% surfels, heavy-tailed scales),
    3840x2160, forward + backward through the ABI stages, with per-phase CUDA
    events and the instance count."""
    import torch
    import synthetic as S
    from paper_2512_02932_gb300 import Rasterizer, SceneTensors
    scene, cam = S.stress_scene()
    st = SceneTensors.from_numpy(scene, dev)
    probe = Rasterizer(dev, sync_check=True)
    probe.forward(st, cam, cfg)
    K = probe.last_K
    del probe
    rast = Rasterizer(dev, capacity=int(K * 1.05) + (1 << 20), sync_check=False)
    g = torch.sign(torch.randn((3, cam.height, cam.width), device=dev)) / (3 * cam.height * cam.width)
    names = ["preprocess", "bin_sort", "render_fwd", "render_bwd", "preprocess_bwd"]
    acc = {n: 0.0 for n in names}
    s = torch.cuda.current_stream()
    reps = 3
    for k in range(reps + 1):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record(s)
        rast.preprocess(st, cam, cfg)
        ev[1].record(s)
        rast.bin_sort(sync_check=False)
        ev[2].record(s)
        rast.render()
        ev[3].record(s)
        _, f_rec, f_prep = rast.backward(g, None, None, None, stages=True)
        f_rec()
        ev[4].record(s)
        f_prep()
        ev[5].record(s)
        torch.cuda.synchronize()
        if k > 0:
            for i, n in enumerate(names):
                acc[n] += ev[i].elapsed_time(ev[i + 1])
    rast.check()
    ph = {n: round(v / reps, 3) for n, v in acc.items()}
    rg = rast.ranges.to(torch.int64) & 0xFFFFFFFF  # uint32 offsets (K may pass 2^31)
    lens = (rg[:, 1] - rg[:, 0]).to(torch.float64)
    ws_bytes = sum(t.numel() * t.element_size() for t in (rast.ws, rast.vals, rast.keys, rast.ranges, rast.rec,
                                                         rast.grad_ws) if t is not None)
    out = {"workload": "stress: 6M prims (90% 2D, log-scales -4.5 + 0.8 t_3), 3840x2160, fwd+bwd (rgb cotangent)",
           "ms_per_step": round(sum(ph.values()), 3), "phases_ms": ph, "instances_K": K,
           "tile_list_len": {"max": int(lens.max().item()), "p99": int(torch.quantile(lens, 0.99).item()),
                             "mean": round(float(lens.mean().item()), 1)},
           "device_buffers_gb": round(ws_bytes / 1e9, 2),
           "peak_allocated_gb": round(torch.cuda.max_memory_allocated(dev) / 1e9, 2)}
    del rast, st
    torch.cuda.empty_cache()
    return out


def binning_probe(args):
    """The binning alone on the stress scene's recipe (90% surfels, log-scales
    -4.5 + 0.8 t_3) at a chosen size: one checked frame, then --steps timed
    hgs_bin_sort calls (CUDA events).  A small case with the stress scene's
    per-tile statistics, for kernel captures."""
    import dataclasses

    import numpy as np
    import torch

    import synthetic as S
    from paper_2512_02932_gb300 import Rasterizer, SceneTensors
    dev = torch.device("cuda", 0)
    scene = S.surface_scene(args.n, seed=4, frac3d=0.1, ls_loc=-4.5, ls_scale=0.8, heavy_df=3)
    cam = S.orbit_camera(30.0, 20.0, 3.0, args.width, args.height, 50.0)
    cfg = S.RenderConfig()
    r = Rasterizer(dev)
    st = SceneTensors.from_numpy(scene, dev)
    r.forward(st, cam, cfg)
    torch.cuda.synchronize()
    ts = []
    for _ in range(max(1, args.steps)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r.preprocess(st, cam, cfg)
        e0.record()
        r.bin_sort(sync_check=False)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    r.check()
    t = r.touched[: scene.n].cpu().numpy().astype(np.int64)
    big = t > 256
    print(json.dumps({"binning_probe": {"prims": args.n, "width": args.width, "height": args.height,
                                        "instances_K": r.last_K, "prims_over_256_tiles": int(big.sum()),
                                        "their_instances": int(t[big].sum()),
                                        "bin_sort_ms": round(statistics.median(ts), 4)}}), flush=True)


def main():
    args = parse()
    world, rank, local = dist_init(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    if args.binning_probe:
        binning_probe(args)
        return
    import torch

    import synthetic as S
    from paper_2512_02932_gb300 import Rasterizer, SceneTensors, exchange_types, rasterize
    from paper_2512_02932_gb300.rasterizer import RasterizeFunction

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scene, _ = S.scene_scale(args.n, seed=1 + rank)
    cam = S.orbit_camera(30.0 + 10 * rank, 20.0, 3.0, args.width, args.height, 50.0)
    cfg = S.RenderConfig()
    st = SceneTensors.from_numpy(scene, dev)
    for t in (st.means, st.log_scales, st.quats, st.opacity_logits, st.sh):
        t.requires_grad_(True)
    target = torch.rand((3, args.height, args.width), device=dev, generator=torch.Generator(device=dev).manual_seed(7))
    mask_rng = torch.Generator(device=dev).manual_seed(11)

    # capacity from one checked frame, then no per-step host sync
    probe = Rasterizer(dev, sync_check=True)
    probe.forward(SceneTensors(st.means.detach(), st.log_scales.detach(), st.quats.detach(),
                               st.opacity_logits.detach(), st.sh.detach(), st.types, 3), cam, cfg)
    K0 = probe.last_K
    del probe
    rast = Rasterizer(dev, capacity=int(K0 * 1.5) + (1 << 20), sync_check=False)

    n_exchange = [0]

    def step(k):
        rgb, depth, normal, alpha = rasterize(st, cam, cfg, rast)
        loss = (rgb - target).abs().mean()
        loss.backward()
        if k % 100 == 0:
            with torch.no_grad():
                mask = (torch.rand(st.n, device=dev, generator=mask_rng) < 0.01).to(torch.uint8)
                exchange_types(SceneTensors(st.means.detach(), st.log_scales.detach(), st.quats.detach(),
                                            st.opacity_logits.detach(), st.sh.detach(), st.types, 3),
                               mode="mask", mask=mask)
                n_exchange[0] += 1
        for t in (st.means, st.log_scales, st.quats, st.opacity_logits, st.sh):
            t.grad = None
        return loss

    # warm-up covers one exchange too (its first call pays one-time module loads)
    for k in range(args.warmup):
        step(0 if k == 0 else k + 100)
    torch.cuda.synchronize()
    rast.check()

    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    n_exchange[0] = 0
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    rast.bwd_events = []  # the render backward's own duration inside the timed steps
    ev0.record()
    step_ev[0].record()
    for k in range(args.steps):
        step(k)
        step_ev[k + 1].record()
    ev1.record()
    torch.cuda.synchronize()
    barrier(world)
    ms_total = ev0.elapsed_time(ev1)
    bwd_timed = [a.elapsed_time(b) for a, b in rast.bwd_events]
    rast.bwd_events = None
    clk = clocks.stop()
    rast.check()
    ms_total = max_over_ranks(ms_total, world, dev)
    ms_per_step = ms_total / args.steps
    step_ms = [step_ev[k].elapsed_time(step_ev[k + 1]) for k in range(args.steps)]
    K = int(rast.d_count.item())
    n_last_sum = int(rast.n_last.to(torch.int64).sum().item())
    n_binned = int((rast.touched[: scene.n] != 0).sum().item())
    tile_passes = (max(1, math.ceil(math.log2(rast.ranges.shape[0]))) + 7) // 8

    # per-phase timing on the launching stream (same workload, separate loop):
    # CUDA events around each ABI call; the backward's two stages separately.
    # (The roofline's render_bwd time is taken inside the timed steps.)
    phases = {}
    if args.profile_phases:
        s = torch.cuda.current_stream()
        dsc = SceneTensors(st.means.detach(), st.log_scales.detach(), st.quats.detach(),
                           st.opacity_logits.detach(), st.sh.detach(), st.types, 3)
        g = torch.sign(torch.randn((3, args.height, args.width), device=dev)) / target.numel()
        names = ["preprocess", "bin_sort", "render_fwd", "render_bwd", "preprocess_bwd"]
        acc = {n: 0.0 for n in names}
        reps = max(3, min(10, args.steps))
        for _ in range(reps):
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
            # ~0.3 ms of FMA work first, so the first phase is queued before
            # its start event runs and its time holds no host-side gap
            keep_busy = busy_launch(dev, 4000)
            evs[0].record(s)
            rast.preprocess(dsc, cam, cfg)
            evs[1].record(s)
            rast.bin_sort(sync_check=False)
            evs[2].record(s)
            rast.render()
            evs[3].record(s)
            _, f_rec, f_prep = rast.backward(g, None, None, None, stages=True)
            f_rec()
            evs[4].record(s)
            f_prep()
            evs[5].record(s)
            torch.cuda.synchronize()
            for i, n in enumerate(names):
                acc[n] += evs[i].elapsed_time(evs[i + 1])
        phases = {n: round(v / reps, 4) for n, v in acc.items()}
        n_contrib_sum = int(rast.n_contrib.to(torch.int64).sum().item())
        n_last_sum = int(rast.n_last.to(torch.int64).sum().item())

    # end to end through the public API with host buffers: every step copies
    # its inputs (scene parameters + target) from pinned host memory and reads
    # its loss back.  The copy of step k+1's inputs runs on a copy stream into
    # the second of two device input sets while step k computes (a training
    # loop's input pipeline); step k waits only for its own inputs.
    e2e = None
    if not args.no_e2e:
        keys = ("means", "log_scales", "quats", "opacity_logits", "sh", "types")
        host = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k))).pin_memory() for k in keys}
        host_target = target.cpu().pin_memory()
        h2d = sum(v.numel() * v.element_size() for v in host.values()) + host_target.numel() * 4
        dev_in = [{k: torch.empty_like(v, device=dev) for k, v in host.items()} for _ in range(2)]
        dev_target = [torch.empty_like(host_target, device=dev) for _ in range(2)]
        loss_host = torch.empty(1, dtype=torch.float32).pin_memory()
        comp = torch.cuda.current_stream()
        copy_s = torch.cuda.Stream(device=dev)
        copied = [torch.cuda.Event() for _ in range(2)]
        used = [torch.cuda.Event() for _ in range(2)]

        def issue_copy(b):
            with torch.cuda.stream(copy_s):
                copy_s.wait_event(used[b])
                for k, v in host.items():
                    dev_in[b][k].copy_(v, non_blocking=True)
                dev_target[b].copy_(host_target, non_blocking=True)
                copied[b].record(copy_s)

        def e2e_compute(b):
            comp.wait_event(copied[b])
            sc = SceneTensors(*(dev_in[b][k] for k in keys), 3)
            params = [sc.means, sc.log_scales, sc.quats, sc.opacity_logits, sc.sh]
            for p in params:
                p.requires_grad_(True)
            rgb, depth, normal, alpha = RasterizeFunction.apply(*params, sc.types, rast, cam, cfg, 3)
            loss = (rgb - dev_target[b]).abs().mean()
            loss.backward()
            loss_host.copy_(loss.detach().reshape(1), non_blocking=True)
            used[b].record(comp)
            for p in params:
                p.requires_grad_(False)
                p.grad = None

        def run(k_steps):
            issue_copy(0)
            for k in range(k_steps):
                if k + 1 < k_steps:
                    issue_copy((k + 1) % 2)
                e2e_compute(k % 2)

        for e in used:
            e.record(comp)
        run(2)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ksteps = max(3, args.steps // 2)
        barrier(world)
        e0.record(comp)
        copy_s.wait_event(e0)
        run(ksteps)
        e1.record(comp)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1) / ksteps, world, dev)
        e2e = {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": 4, "steps": ksteps,
               "pipeline": "inputs of step k+1 copied on a second stream while step k computes"}

    roofline = None
    if phases:
        # dominant kernel: the blend backward the L1 step runs (rgb-only
        # cotangent; one warp per tile, tiles longest first), bound by FP32
        # issue.  Algorithmic FP32 work (FMA = 2 flops): 16 flops per (pixel,
        # list entry) the pixel consumed (70/30 mix of the 12-flop 3D and
        # 24-flop surfel evaluation) + 56 per contributing pair (46 of
        # gradient, ~10 of the per-record sum over pixels).  Peaks measured in
        # this run by hgs_alu_probe (FFMA for FP32; EX2 and RCP for the
        # special-function unit), with 152 SMs x 128 lanes x 2 x the max SM
        # clock beside them for context.
        sm_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
        derived = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        peak, peak_source = alu_peak(dev, 0)
        ex2_peak, _ = alu_peak(dev, 2)
        rcp_peak, _ = alu_peak(dev, 3)
        flops = 16.0 * n_last_sum + 56.0 * n_contrib_sum
        # the kernel's mean duration inside the timed steps (CUDA events on its
        # stream around the record-gradient stage), else the per-phase loop's
        kernel_ms = statistics.mean(bwd_timed) if bwd_timed else phases["render_bwd"]
        sec = kernel_ms * 1e-3
        achieved = flops / sec / 1e12
        # a coarser count, the same for every evaluated pair: ~61 operations
        # (2.5 x the forward's 20 (3D) / 35 (surfel) at the 70/30 mix)
        coarse = 61.0 * n_last_sum / sec / 1e12
        # special-function work: one EX2 per (pixel, entry), one RCP per
        # surfel entry (30% of the entries at this mix, an estimate) and one
        # RCP per contributing pair (the transmittance recovered by division)
        ex2_ops, rcp_ops = float(n_last_sum), 0.3 * n_last_sum + float(n_contrib_sum)
        mufu_busy = (ex2_ops / (ex2_peak * 1e12) + rcp_ops / (rcp_peak * 1e12)) / sec
        roofline = {"kernel": "render_bwd_rgb4_kernel", "bound": "alu", "achieved": round(achieved, 3),
                    "kernel_ms": round(kernel_ms, 4),
                    "kernel_ms_source": "timed steps" if bwd_timed else "per-phase loop",
                    "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                    "traffic": None,
                    "peak_source": peak_source,
                    "peak_derived": round(derived, 2),
                    "flop_convention": "16 flops per (pixel, list entry) consumed + 56 per contributing pair",
                    "units": {"pixel_list_entries": n_last_sum, "contributing_pairs": n_contrib_sum,
                              "flops_per_entry": 16, "flops_per_contributing_pair": 56},
                    "pairs_per_s": round(n_last_sum / sec, 1),
                    "per_entry_convention": {"ops_per_entry": 61, "achieved": round(coarse, 3),
                                             "frac": round(coarse / peak, 4)},
                    "special_function": {"ex2_ops": ex2_ops, "rcp_ops": rcp_ops,
                                         "peak_ex2_tops": round(ex2_peak, 3), "peak_rcp_tops": round(rcp_peak, 3),
                                         "busy_frac": round(mufu_busy, 4)}}
    serving = None
    if not args.no_serving and world == 1:
        serving = run_serving(args, dev, cfg)
    fdo_line = None
    if not args.no_fdo and world == 1:
        dsc = SceneTensors(st.means.detach(), st.log_scales.detach(), st.quats.detach(),
                           st.opacity_logits.detach(), st.sh.detach(), st.types, 3)
        fdo_line = run_fdo(args, dev, dsc, cam, cfg, target)
    train_line = None
    if not args.no_train and world == 1:
        train_line = run_train(args, dev, scene, cam, cfg, target)
    stress_line = None
    if not args.no_stress and world == 1:
        stress_line = run_stress(args, dev, cfg)
    line = {
        "metric": METRIC, "value": round(ms_per_step, 4), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": base_config(args, world),
        "workload_stats": {"instances_K": K, "pixel_list_entries": n_last_sum, "binned_prims": n_binned},
        "phases_ms": phases,
        "hbm_phases": hbm_phases(phases, scene.n, n_binned, K, tile_passes, *hbm_peak()) if phases else None,
        "step_ms": {"min": round(min(step_ms), 4), "median": round(statistics.median(step_ms), 4),
                    "max": round(max(step_ms), 4), "first": round(step_ms[0], 4)},
        "roofline": roofline,
        "serving": serving,
        "fdo": fdo_line,
        "train": train_line,
        "stress": stress_line,
        "gpu_launches": launches_per_step(rast, n_exchange[0], args.steps),
        "clocks": clk,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline(scene, cam, cfg, args.cpu_sample_pixels)
        except Exception as exc:  # the checker is optional for the GPU number
            line["cpu_baseline"] = {"error": repr(exc)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
