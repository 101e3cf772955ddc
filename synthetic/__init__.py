"""Seeded synthetic inputs for the hybrid 2D/3D Gaussian rasterizer.

This module only draws random numbers and lays them out: scenes (SoA float32
parameter arrays plus a uint8 type flag), pinhole cameras and the render
configuration.  It contains none of the rasterizer's arithmetic, so both the
CUDA path and the CPU oracle may consume what it produces.

Parameter layout (one row per primitive, C-contiguous float32):
  means           (N, 3)   world-space centre mu
  log_scales      (N, 3)   log s; a 2D surfel stores the sentinel -30 on z
                           (s_z ~ 1e-13, the "s_z = 0" initialisation of
                           Sec. 3.1 kept finite)
  quats           (N, 4)   rotation quaternion (w, x, y, z), not normalised
  opacity_logits  (N,)     opacity = sigmoid(logit)
  sh              (N, (l+1)^2, 3)  SH coefficients, coefficient-major
  types           (N,)     uint8: 0 = 2D surfel, 1 = 3D Gaussian (Sec. 3.1)

Camera convention: OpenCV (x right, y down, z forward); world-to-camera
x_c = R x_w + t; pixel (i, j) has its centre at (i + 0.5, j + 0.5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

SURFEL_LOG_SZ = -30.0
SQRT_PI = math.sqrt(math.pi)  # DC coefficient range that spans RGB [0, 1]


@dataclass
class Camera:
    R: np.ndarray  # (3, 3) float32 world-to-camera rotation
    t: np.ndarray  # (3,) float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def as_array16(self) -> np.ndarray:
        """R (row-major 9), t (3), fx, fy, cx, cy as float32[16]."""
        return np.concatenate([
            np.asarray(self.R, np.float32).reshape(9),
            np.asarray(self.t, np.float32).reshape(3),
            np.array([self.fx, self.fy, self.cx, self.cy], np.float32),
        ]).astype(np.float32)


@dataclass
class RenderConfig:
    """Render settings; the paper leaves all of these unstated except the
    scale-modulation pair theta_z = 1.05, T_z = 0.001 (App. A)."""
    near: float = 0.2
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    T_min: float = 1e-4
    lambda_z: float = 1.0
    theta_z: float = 1.05
    T_z: float = 1e-3
    dilation: float = 0.0
    bg: tuple = (0.0, 0.0, 0.0)
    tile: int = 16

    def as_oracle_array(self) -> np.ndarray:
        return np.array([self.near, self.alpha_min, self.alpha_max, self.T_min,
                         self.lambda_z, self.theta_z, self.T_z, self.dilation,
                         *self.bg], np.float64)


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    types: np.ndarray
    sh_degree: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity_logits[idx].copy(),
                     self.sh[idx].copy(), self.types[idx].copy(), self.sh_degree,
                     dict(self.meta))

    def copy(self) -> "Scene":
        return self.subset(np.arange(self.n))

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.means, self.log_scales, self.quats,
                                      self.opacity_logits, self.sh, self.types))


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------
def pinhole(width: int, height: int, fov_x_deg: float, R=None, t=None) -> Camera:
    """Pinhole camera with horizontal field of view fov_x and square pixels."""
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) / 2.0)
    R = np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32)
    t = np.zeros(3, np.float32) if t is None else np.asarray(t, np.float32)
    return Camera(R, t, float(np.float32(fx)), float(np.float32(fx)),
                  width / 2.0, height / 2.0, width, height)


def look_at(position, target=(0.0, 0.0, 0.0), down=(0.0, 1.0, 0.0)):
    """World-to-camera (R, t) for a camera at `position` looking at `target`;
    world +y is "down" (OpenCV)."""
    p = np.asarray(position, np.float64)
    f = np.asarray(target, np.float64) - p
    f /= np.linalg.norm(f)
    right = np.cross(np.asarray(down, np.float64), f)
    right /= np.linalg.norm(right)
    dn = np.cross(f, right)
    R = np.stack([right, dn, f]).astype(np.float64)
    t = -R @ p
    return R.astype(np.float32), t.astype(np.float32)


def orbit_camera(azimuth_deg, elevation_deg, radius, width, height, fov_x_deg=50.0):
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    pos = (radius * math.cos(el) * math.sin(az), -radius * math.sin(el),
           radius * math.cos(el) * math.cos(az))
    R, t = look_at(pos)
    return pinhole(width, height, fov_x_deg, R, t)


# --------------------------------------------------------------------------
# orientation helpers (input construction only)
# --------------------------------------------------------------------------
def _quat_mul(a, b):
    w1, x1, y1, z1 = a[:, 0], a[:, 1], a[:, 2], a[:, 3]
    w2, x2, y2, z2 = b[:, 0], b[:, 1], b[:, 2], b[:, 3]
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], axis=1)


def _quats_z_to(normals, twist):
    """Quaternions whose local z axis is `normals`, with a twist about it."""
    n = normals / np.linalg.norm(normals, axis=1, keepdims=True)
    qa = np.stack([1.0 + n[:, 2], -n[:, 1], n[:, 0], np.zeros(len(n))], axis=1)
    bad = (1.0 + n[:, 2]) < 1e-6
    qa[bad] = np.array([0.0, 1.0, 0.0, 0.0])
    qa /= np.linalg.norm(qa, axis=1, keepdims=True)
    qt = np.stack([np.cos(twist / 2), np.zeros_like(twist), np.zeros_like(twist),
                   np.sin(twist / 2)], axis=1)
    return _quat_mul(qa, qt)


def _types(rng, n, frac3d):
    n3 = int(round(n * frac3d))
    t = np.zeros(n, np.uint8)
    t[:n3] = 1
    return t[rng.permutation(n)]


def _log_scales(rng, types, loc, scale, heavy_df=None):
    n = len(types)
    if heavy_df is None:
        ls = rng.normal(loc, scale, size=(n, 3))
    else:
        ls = loc + scale * rng.standard_t(heavy_df, size=(n, 3))
    ls[types == 0, 2] = SURFEL_LOG_SZ
    return ls.astype(np.float32)


def _sh(rng, n, degree, hi_sigma=0.05):
    k = (degree + 1) ** 2
    sh = np.zeros((n, k, 3), np.float32)
    sh[:, 0, :] = rng.uniform(-SQRT_PI, SQRT_PI, size=(n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, hi_sigma, size=(n, k - 1, 3))
    return sh


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------
def tiny_scene(seed: int = 0, n: int = 1000):
    """1,000 primitives (half 3D, half 2D, shuffled), means x,y ~ U[-1,1] and
    z ~ U[2,4] in camera space, log-scales N(-3, 0.5), random unit
    quaternions, logit ~ N(0,1), SH degree 0 with RGB uniform in [0,1];
    identity camera, fov 60 deg, 128x128."""
    rng = np.random.default_rng(seed)
    types = np.zeros(n, np.uint8)
    types[: n // 2] = 1
    types = types[rng.permutation(n)]
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n),
                      rng.uniform(2, 4, n)], axis=1).astype(np.float32)
    ls = _log_scales(rng, types, -3.0, 0.5)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logits = rng.normal(0.0, 1.0, n).astype(np.float32)
    sh = _sh(rng, n, 0)
    scene = Scene(means, ls, q.astype(np.float32), logits, sh, types, 0,
                  {"workload": "tiny", "seed": seed})
    cam = pinhole(128, 128, 60.0)
    return scene, cam


def surface_scene(n: int, seed: int, frac3d: float = 0.7, sh_degree: int = 3,
                  ls_loc: float = -4.5, ls_scale: float = 0.7, heavy_df=None,
                  logit_loc: float = 1.0, logit_scale: float = 1.5):
    """Primitives on a unit sphere shell (radial noise 0.01) and a ground plane
    y = +1 over [-3,3]^2 (half each), oriented along the surface normal with
    normal noise 0.01 and a random twist."""
    rng = np.random.default_rng(seed)
    types = _types(rng, n, frac3d)
    n_s = n // 2
    n_p = n - n_s
    d = rng.normal(size=(n_s, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = 1.0 + rng.normal(0.0, 0.01, size=(n_s, 1))
    sphere = d * r
    plane = np.stack([rng.uniform(-3, 3, n_p), np.ones(n_p), rng.uniform(-3, 3, n_p)], axis=1)
    means = np.concatenate([sphere, plane]).astype(np.float32)
    normals = np.concatenate([d, np.tile(np.array([[0.0, -1.0, 0.0]]), (n_p, 1))])
    normals = normals + rng.normal(0.0, 0.01, size=normals.shape)
    q = _quats_z_to(normals, rng.uniform(0, 2 * np.pi, n)).astype(np.float32)
    ls = _log_scales(rng, types, ls_loc, ls_scale, heavy_df)
    logits = rng.normal(logit_loc, logit_scale, n).astype(np.float32)
    sh = _sh(rng, n, sh_degree)
    return Scene(means, ls, q, logits, sh, types, sh_degree,
                 {"workload": "surface", "seed": seed, "frac3d": frac3d})


def scene_scale(n: int = 3_000_000, seed: int = 1):
    """3M primitives (70% 3D / 30% 2D), log-scales N(-4.5, 0.7), SH degree 3,
    logit N(1, 1.5); orbit camera radius 3, elevation 20 deg, 1600x1064, fov 50."""
    scene = surface_scene(n, seed)
    scene.meta["workload"] = f"scene {n} prims 1600x1064"
    cam = orbit_camera(30.0, 20.0, 3.0, 1600, 1064, 50.0)
    return scene, cam


def stress_scene(n: int = 6_000_000, seed: int = 4, width: int = 3840, height: int = 2160):
    """6M primitives, 90% 2D, heavy-tailed log-scales -4.5 + 0.8 t_3 (not
    clipped), 3840x2160."""
    scene = surface_scene(n, seed, frac3d=0.1, ls_loc=-4.5, ls_scale=0.8, heavy_df=3)
    scene.meta["workload"] = f"stress {n} prims {width}x{height}"
    cam = orbit_camera(30.0, 20.0, 3.0, width, height, 50.0)
    return scene, cam


SERVING_SIZES = (200_000, 500_000, 1_000_000, 3_000_000)
SERVING_MIX = (0.5, 0.6, 0.7, 0.8)
SERVING_RES = ((512, 512), (800, 600), (1280, 720), (1920, 1080))


def serving_scenes(seed: int = 3, sizes=SERVING_SIZES, mixes=SERVING_MIX):
    return [surface_scene(n, seed * 100 + k, frac3d=f) for k, (n, f) in enumerate(zip(sizes, mixes))]


def serving_requests(seed: int = 3, rate_hz: float = 200.0, duration_s: float = 20.0,
                     n_scenes: int = 4, resolutions=SERVING_RES):
    """Poisson arrivals; each request: (t_arrival, scene id, camera)."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        sid = int(rng.integers(n_scenes))
        w, h = resolutions[int(rng.integers(len(resolutions)))]
        cam = orbit_camera(float(rng.uniform(0, 360)), float(rng.uniform(-30, 30)),
                           float(rng.uniform(2.5, 4.0)), w, h, 50.0)
        out.append((t, sid, cam))
    return out


def random_cotangents(seed: int, height: int, width: int):
    """Upstream gradients for (rgb[3], depth, normal[3], alpha) maps."""
    rng = np.random.default_rng(seed)
    return {
        "rgb": rng.normal(size=(3, height, width)).astype(np.float32),
        "depth": (0.1 * rng.normal(size=(height, width))).astype(np.float32),
        "normal": rng.normal(size=(3, height, width)).astype(np.float32),
        "alpha": rng.normal(size=(height, width)).astype(np.float32),
    }


__all__ = ["Camera", "RenderConfig", "Scene", "pinhole", "look_at", "orbit_camera",
           "tiny_scene", "surface_scene", "scene_scale", "stress_scene",
           "serving_scenes", "serving_requests", "random_cotangents", "SURFEL_LOG_SZ",
           "replace"]
