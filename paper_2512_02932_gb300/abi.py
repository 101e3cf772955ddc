"""ctypes binding of libhgs (include/hgs.h): the same entry points, same
names, argument marshalling only.  Every step of the rasterizer runs in the
library's CUDA kernels; this module has no compute path of its own and raises
if the library cannot be loaded.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

HGS_OK = 0
HGS_ERR_INVALID_ARG = -1
HGS_ERR_CAPACITY = -2
HGS_ERR_CUDA = -3
HGS_ERR_TIMEOUT = -4
HGS_ERR_UNSUPPORTED = -5
HGS_EXCHANGE_ERANK = 0
HGS_EXCHANGE_MASK = 1
HGS_BIN_SORT_STATIC_BYTES = 64 << 20
HGS_MAX_CAPACITY = 0xffffffff
HGS_MAX_BATCH = 16
HGS_PROBE_FFMA, HGS_PROBE_FFMA2, HGS_PROBE_EX2, HGS_PROBE_RCP = 0, 1, 2, 3

P = C.c_void_p


class hgs_scene(C.Structure):
    _fields_ = [("means", P), ("log_scales", P), ("quats", P), ("opacity_logits", P), ("sh", P),
                ("types", P), ("n", C.c_int64), ("sh_degree", C.c_int32)]


class hgs_scene_mut(C.Structure):
    _fields_ = [("log_scales", P), ("quats", P), ("types", P), ("n", C.c_int64)]


class hgs_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class hgs_config(C.Structure):
    _fields_ = [("near_z", C.c_float), ("alpha_min", C.c_float), ("alpha_max", C.c_float),
                ("T_min", C.c_float), ("lambda_z", C.c_float), ("theta_z", C.c_float),
                ("T_z", C.c_float), ("dilation", C.c_float), ("bg", C.c_float * 3),
                ("tile", C.c_int32)]


class hgs_projected(C.Structure):
    _fields_ = [("rec", P), ("depth_key", P), ("rect", P), ("touched", P), ("tileset", P)]


class hgs_binning(C.Structure):
    _fields_ = [("vals", P), ("keys", P), ("ranges", P), ("d_count", P)]


class hgs_image(C.Structure):
    _fields_ = [("rgb", P), ("depth", P), ("normal", P), ("alpha", P), ("T_final", P), ("n_last", P),
                ("n_contrib", P), ("tile_sched", P)]


class hgs_image_grad(C.Structure):
    _fields_ = [("rgb", P), ("depth", P), ("normal", P), ("alpha", P)]


class hgs_scene_grad(C.Structure):
    _fields_ = [("means", P), ("log_scales", P), ("quats", P), ("opacity_logits", P), ("sh", P)]


class hgs_request(C.Structure):
    _fields_ = [("scene", hgs_scene), ("cam", hgs_camera), ("out", hgs_image)]


class hgs_exchange_cfg(C.Structure):
    _fields_ = [("mode", C.c_int32), ("theta_e", C.c_float), ("mask", P)]


class hgs_adam_group(C.Structure):
    _fields_ = [("param", P), ("grad", P), ("m", P), ("v", P), ("count", C.c_int64), ("lr", C.c_float),
                ("period", C.c_int32), ("head", C.c_int32), ("lr_tail", C.c_float)]


class hgs_densify_cfg(C.Structure):
    _fields_ = [("grad_thresh", C.c_float), ("log_size_thresh", C.c_float), ("logit_min_opacity", C.c_float)]


class hgs_train_arrays(C.Structure):
    _fields_ = [("means", P), ("log_scales", P), ("quats", P), ("opacity_logits", P), ("sh", P),
                ("types", P), ("moments", P * 10)]


SYMBOLS = {
    "hgs_default_config": (None, [C.POINTER(hgs_config)]),
    "hgs_status_string": (C.c_char_p, [C.c_int]),
    "hgs_check": (C.c_int, [P, C.POINTER(C.c_int32), P]),
    "hgs_preprocess": (C.c_int, [C.POINTER(hgs_scene), C.POINTER(hgs_camera), C.POINTER(hgs_config),
                                 C.POINTER(hgs_projected), P, P]),
    "hgs_bin_sort_workspace": (C.c_int, [C.c_int64, C.c_int64, C.c_int32, C.POINTER(C.c_size_t)]),
    "hgs_bin_sort": (C.c_int, [C.c_int64, C.POINTER(hgs_projected), C.POINTER(hgs_camera),
                               C.POINTER(hgs_config), P, C.c_size_t, C.c_int64, C.POINTER(hgs_binning),
                               P, P]),
    "hgs_bin_sort_static": (C.c_int, [C.c_int64, C.POINTER(hgs_projected), C.POINTER(hgs_camera),
                                      C.POINTER(hgs_config), C.c_int64, C.POINTER(hgs_binning), P, P]),
    "hgs_render_fwd": (C.c_int, [C.c_int64, C.POINTER(hgs_projected), C.POINTER(hgs_binning),
                                 C.POINTER(hgs_camera), C.POINTER(hgs_config), C.POINTER(hgs_image), P, P]),
    "hgs_render_bwd": (C.c_int, [C.POINTER(hgs_scene), C.POINTER(hgs_projected), C.POINTER(hgs_binning),
                                 C.POINTER(hgs_camera), C.POINTER(hgs_config), C.POINTER(hgs_image),
                                 C.POINTER(hgs_image_grad), P, C.POINTER(hgs_scene_grad), P, P]),
    "hgs_render_batch_workspace": (C.c_int, [C.c_int, C.POINTER(hgs_request), C.c_int64, C.POINTER(C.c_size_t)]),
    "hgs_render_batch": (C.c_int, [C.c_int, C.POINTER(hgs_request), C.POINTER(hgs_config), P, C.c_size_t,
                                   C.c_int64, P, P, P]),
    "hgs_render_bwd_records": (C.c_int, [C.POINTER(hgs_scene), C.POINTER(hgs_projected), C.POINTER(hgs_binning),
                                         C.POINTER(hgs_camera), C.POINTER(hgs_config), C.POINTER(hgs_image),
                                         C.POINTER(hgs_image_grad), P, P, P]),
    "hgs_preprocess_bwd": (C.c_int, [C.POINTER(hgs_scene), C.POINTER(hgs_projected), C.POINTER(hgs_camera),
                                     C.POINTER(hgs_config), P, C.POINTER(hgs_scene_grad), P, P]),
    "hgs_exchange_types": (C.c_int, [C.POINTER(hgs_scene_mut), C.POINTER(hgs_exchange_cfg), P, P, P]),
    "hgs_image_losses": (C.c_int, [P, P, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                                   P, P, P, P, P]),
    "hgs_fp32_probe": (C.c_int, [C.c_int32, C.c_int32, P, C.POINTER(C.c_double), P]),
    "hgs_alu_probe": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, P, C.POINTER(C.c_double), P]),
    "hgs_render_bwd_fdo": (C.c_int, [C.POINTER(hgs_scene), C.POINTER(hgs_projected), C.POINTER(hgs_binning),
                                     C.POINTER(hgs_camera), C.POINTER(hgs_config), C.POINTER(hgs_image),
                                     P, P, P, P, C.POINTER(hgs_scene_grad), P, P, P]),
    "hgs_adam_step": (C.c_int, [C.c_int32, C.POINTER(hgs_adam_group), C.c_int32, C.c_double, C.c_double,
                                C.c_double, P]),
    "hgs_grad_stats": (C.c_int, [C.c_int64, P, C.POINTER(hgs_projected), P, P, P]),
    "hgs_densify_workspace": (C.c_int, [C.c_int64, C.POINTER(C.c_size_t)]),
    "hgs_densify_plan": (C.c_int, [C.POINTER(hgs_scene), P, P, C.POINTER(hgs_densify_cfg), P, P, P, C.c_size_t,
                                   P, P]),
    "hgs_densify_apply": (C.c_int, [C.c_int64, C.c_int32, C.POINTER(hgs_train_arrays),
                                    C.POINTER(hgs_train_arrays), P, P, P, P]),
    "hgs_reset_opacity": (C.c_int, [C.c_int64, P, C.c_float, P, P, P]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True):
    """Load libhgs.so (building it with nvcc first if it is missing or stale).
    Raises RuntimeError if the CUDA library cannot be built or loaded."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_needed and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libhgs.so is missing ({_build.LIB}); build it with "
                           "paper_2512_02932_gb300.build.build()")
    L = C.CDLL(_build.LIB)
    for name, (res, args) in SYMBOLS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class HgsError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        name = load().hgs_status_string(status).decode()
        super().__init__(f"{where}: {name} ({status})")


def check(status, where=""):
    if status != HGS_OK:
        raise HgsError(status, where)
    return status


def _fwd(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    f.__doc__ = f"Direct call of {name} (see include/hgs.h)."
    return f


hgs_default_config = _fwd("hgs_default_config")
hgs_status_string = _fwd("hgs_status_string")
hgs_check = _fwd("hgs_check")
hgs_preprocess = _fwd("hgs_preprocess")
hgs_bin_sort_workspace = _fwd("hgs_bin_sort_workspace")
hgs_bin_sort = _fwd("hgs_bin_sort")
hgs_bin_sort_static = _fwd("hgs_bin_sort_static")
hgs_render_fwd = _fwd("hgs_render_fwd")
hgs_render_bwd = _fwd("hgs_render_bwd")
hgs_render_bwd_records = _fwd("hgs_render_bwd_records")
hgs_preprocess_bwd = _fwd("hgs_preprocess_bwd")
hgs_exchange_types = _fwd("hgs_exchange_types")
hgs_render_batch_workspace = _fwd("hgs_render_batch_workspace")
hgs_render_batch = _fwd("hgs_render_batch")
hgs_image_losses = _fwd("hgs_image_losses")
hgs_render_bwd_fdo = _fwd("hgs_render_bwd_fdo")
hgs_adam_step = _fwd("hgs_adam_step")
hgs_grad_stats = _fwd("hgs_grad_stats")
hgs_densify_workspace = _fwd("hgs_densify_workspace")
hgs_densify_plan = _fwd("hgs_densify_plan")
hgs_densify_apply = _fwd("hgs_densify_apply")
hgs_reset_opacity = _fwd("hgs_reset_opacity")
hgs_fp32_probe = _fwd("hgs_fp32_probe")
hgs_alu_probe = _fwd("hgs_alu_probe")
