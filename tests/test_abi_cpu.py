"""The C-ABI library loads and exports every entry point include/hgs.h
declares; host-side validation answers without touching a GPU.  CPU only."""
import ctypes as C
import os
import re

import pytest

from paper_2512_02932_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "hgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hgs_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = abi.load()
    names = declared_symbols()
    assert len(names) >= 9
    for name in names:
        assert hasattr(L, name), name
        assert name in abi.SYMBOLS, f"{name} not bound in abi.py"


def test_library_is_built_for_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(abi.load()._name)


def test_defaults_and_status_strings():
    c = abi.hgs_config()
    abi.hgs_default_config(C.byref(c))
    assert c.tile == 16 and abs(c.alpha_min - 1 / 255) < 1e-9 and abs(c.theta_z - 1.05) < 1e-6
    assert abi.hgs_status_string(abi.HGS_ERR_CAPACITY) == b"HGS_ERR_CAPACITY"
    assert abi.hgs_status_string(12345) == b"HGS_ERR_UNKNOWN"


def test_workspace_query_is_host_only():
    nb = C.c_size_t()
    assert abi.hgs_bin_sort_workspace(1000, 5000, 64, C.byref(nb)) == 0
    small = nb.value
    assert abi.hgs_bin_sort_workspace(3_000_000, 20_000_000, 6700, C.byref(nb)) == 0
    assert nb.value > small > 0
    assert abi.hgs_bin_sort_workspace(-1, 10, 1, C.byref(nb)) == abi.HGS_ERR_INVALID_ARG


def test_capacity_beyond_32_bit_offsets_is_rejected():
    """List offsets are 32-bit: a capacity above 2^32 - 1 is rejected by every
    entry point that sizes buffers from it, before any size can wrap and
    before anything is launched (no GPU is touched here)."""
    nb = C.c_size_t(7)
    for cap in (abi.HGS_MAX_CAPACITY + 1, 1 << 62, (1 << 63) - 1):
        assert abi.hgs_bin_sort_workspace(1000, cap, 64, C.byref(nb)) == abi.HGS_ERR_INVALID_ARG
    assert nb.value == 7
    assert abi.hgs_bin_sort_workspace(1000, abi.HGS_MAX_CAPACITY, 64, C.byref(nb)) == 0
    cam = abi.hgs_camera()
    cam.R[0] = cam.R[4] = cam.R[8] = 1.0
    cam.fx = cam.fy = 100.0
    cam.width = cam.height = 64
    cfg = abi.hgs_config()
    abi.hgs_default_config(C.byref(cfg))
    proj = abi.hgs_projected(16, 16, 16, 16, 16)
    out = abi.hgs_binning(16, None, 16, 16)
    cap = 1 << 62
    assert abi.hgs_bin_sort(10, C.byref(proj), C.byref(cam), C.byref(cfg), C.c_void_p(16), 1 << 30, cap,
                            C.byref(out), None, None) == abi.HGS_ERR_INVALID_ARG
    assert abi.hgs_bin_sort_static(10, C.byref(proj), C.byref(cam), C.byref(cfg), cap, C.byref(out),
                                   None, None) == abi.HGS_ERR_INVALID_ARG
    req = (abi.hgs_request * 1)()
    req[0].scene.n = 10
    req[0].cam.width = req[0].cam.height = 64
    assert abi.hgs_render_batch_workspace(1, req, 1000, C.byref(nb)) == 0
    assert abi.hgs_render_batch_workspace(1, req, cap, C.byref(nb)) == abi.HGS_ERR_INVALID_ARG


def test_invalid_arguments_rejected_before_launch():
    cam = abi.hgs_camera()
    cfg = abi.hgs_config()
    abi.hgs_default_config(C.byref(cfg))
    proj = abi.hgs_projected()
    scene = abi.hgs_scene()
    scene.n = 10
    scene.sh_degree = 0
    # NULL arrays
    assert abi.hgs_preprocess(C.byref(scene), C.byref(cam), C.byref(cfg), C.byref(proj), None, None) \
        == abi.HGS_ERR_INVALID_ARG
    # bad SH degree
    scene.sh_degree = 4
    assert abi.hgs_preprocess(C.byref(scene), C.byref(cam), C.byref(cfg), C.byref(proj), None, None) \
        == abi.HGS_ERR_INVALID_ARG
    # tile other than 16
    scene.n = 0
    scene.sh_degree = 0
    cam.width = cam.height = 16
    cam.fx = cam.fy = 10.0
    cfg.tile = 8
    assert abi.hgs_preprocess(C.byref(scene), C.byref(cam), C.byref(cfg), C.byref(proj), None, None) \
        == abi.HGS_ERR_UNSUPPORTED
    # camera with zero size
    cfg.tile = 16
    cam.width = 0
    assert abi.hgs_preprocess(C.byref(scene), C.byref(cam), C.byref(cfg), C.byref(proj), None, None) \
        == abi.HGS_ERR_INVALID_ARG
    # exchange without a mask in mask mode
    sm = abi.hgs_scene_mut(1, 16, 1, 5)
    x = abi.hgs_exchange_cfg(abi.HGS_EXCHANGE_MASK, 2.05, None)
    assert abi.hgs_exchange_types(C.byref(sm), C.byref(x), None, None, None) == abi.HGS_ERR_INVALID_ARG
    # the FP32 probe needs a launch size and an output
    fl = C.c_double()
    assert abi.hgs_fp32_probe(0, 10, None, C.byref(fl), None) == abi.HGS_ERR_INVALID_ARG
    assert abi.hgs_fp32_probe(4, 0, None, C.byref(fl), None) == abi.HGS_ERR_INVALID_ARG
    # the unit probes also need a known kind
    for kind in (-1, 4):
        assert abi.hgs_alu_probe(kind, 4, 10, C.c_void_p(16), C.byref(fl), None) == abi.HGS_ERR_INVALID_ARG
    assert abi.hgs_alu_probe(abi.HGS_PROBE_EX2, 0, 10, C.c_void_p(16), C.byref(fl), None) \
        == abi.HGS_ERR_INVALID_ARG
    # the binning needs the tile-set array, 16-byte aligned (checked before
    # anything launches)
    cam.width = 16
    out = abi.hgs_binning(16, None, 16, 16)
    for ts in (None, 24):
        proj16 = abi.hgs_projected(16, 16, 16, 16, ts)
        assert abi.hgs_bin_sort(10, C.byref(proj16), C.byref(cam), C.byref(cfg), C.c_void_p(16), 1 << 30, 1000,
                                C.byref(out), None, None) == abi.HGS_ERR_INVALID_ARG
        assert abi.hgs_bin_sort_static(10, C.byref(proj16), C.byref(cam), C.byref(cfg), 1000, C.byref(out),
                                       None, None) == abi.HGS_ERR_INVALID_ARG
    # an empty scene is valid and launches nothing
    scene.n = 0
    assert abi.hgs_preprocess(C.byref(scene), C.byref(cam), C.byref(cfg), C.byref(proj), None, None) == 0
