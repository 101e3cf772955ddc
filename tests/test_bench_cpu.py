"""bench.py's multi-process plumbing on CPU: max over ranks and the barrier
with two gloo ranks, and the reference arm under torchrun with two ranks
(rank 0 alone prints its line, the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        out[rank] = bench.max_over_ranks(1.5 + rank, world)
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        assert dict(out) == {0: 2.5, 1: 2.5}


def test_max_over_ranks_single_process_is_identity():
    assert bench.max_over_ranks(3.25, 1) == 3.25


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--prims", "3000", "--width", "64", "--height", "48", "--cpu-sample-pixels", "2000"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["config"]["n_prims"] == 3000 and d["config"]["width"] == 64
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_hbm_phases_counts_the_documented_bytes():
    """The memory-bound phases' algorithmic bytes: preprocess 61 B per
    primitive + 304 B per binned one; its backward 385 B per binned + 4 B per
    culled + 236 B per primitive; the sort 144 B per binned primitive + 8 B
    per instance for the emit + 20 B per instance and tile pass, less 4 B
    (the last pass writes no keys)."""
    ph = {"preprocess": 1.0, "preprocess_bwd": 2.0, "bin_sort": 4.0}
    n, nb, K = 1000, 600, 10_000
    out = bench.hbm_phases(ph, n, nb, K, 2, 1000.0, "test")
    assert out["preprocess"]["bytes"] == 61 * n + 304 * nb
    assert out["preprocess_bwd"]["bytes"] == 385 * nb + 4 * (n - nb) + 236 * n
    assert out["bin_sort"]["bytes"] == 144 * nb + 8 * K + 2 * 20 * K - 4 * K
    b = out["preprocess"]["bytes"]
    assert abs(out["preprocess"]["achieved_gbs"] - b / 1e-3 / 1e9) < 0.1
    assert abs(out["preprocess"]["frac"] - out["preprocess"]["achieved_gbs"] / 1000.0) < 1e-3
    assert bench.hbm_phases({}, n, nb, K, 2, 1000.0, "test") == {"peak_source": "test"}
