"""ctypes front end of the C oracle (hgs_oracle.c).  Test infrastructure only.

Functions and what pins them (tests/test_oracle_*.py):
  Oracle.render      FP64 per-pixel renderer, Eq. 1, Sec. 3.1 contribution,
                     Eq. 2 blending, App. C projections; render_checked adds
                     every correct result where a threshold decision is
                     ambiguous, and the conditioning tolerance.  Pinned by closed forms
                     (isotropic 3D Gaussian, face-on surfel), the edge-on surfel
                     vanishing, 3D->2D convergence as s_z -> 0, brute-force
                     compositing, order-of-input invariance, and the
                     independent torch formulation (autograd_ref).
  contract_bin       FP32 binning contract.  Pinned by conservativeness against
                     the FP64 renderer and by exp/log accuracy against libm.
  tile_lists         Sort of the contract's (tile | depth bits, id) pairs:
                     numpy lexsort, a library primitive.
  sh_basis           Real SH basis (Sec. 3.1 "decoded from f"), pinned against
                     scipy's complex spherical harmonics and orthonormality.
  exchange / erank   Eqs. 3-5, App. D.  Pinned by the erank values the paper
                     states (3 isotropic, 2 flat, ~2.6 crossing) and by
                     Sigma* = Sigma, det R* > 0.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.orc_prepare.restype = P
        L.orc_prepare.argtypes = [C.c_int64, P, P, P, P, P, P, C.c_int, P, C.c_int, C.c_int, P]
        L.orc_render.restype = None
        L.orc_render.argtypes = [P, C.c_int64, P, P, P, P]
        L.orc_render_variants.restype = None
        L.orc_render_variants.argtypes = [P, C.c_int64, P, P, P]
        L.orc_max_variants.restype = C.c_int
        L.orc_max_variants.argtypes = []
        L.orc_pair_alpha.restype = None
        L.orc_pair_alpha.argtypes = [P, C.c_int64, C.c_int64, P, P]
        L.orc_pixel_contributors.restype = None
        L.orc_pair_conditioning.restype = None
        L.orc_pair_conditioning.argtypes = [P, C.c_int64, P, P, P]
        L.orc_pixel_contributors.argtypes = [P, C.c_int64, P, C.c_int, P, P]
        L.orc_fd_begin.restype = P
        L.orc_fd_begin.argtypes = [P, C.c_int64, C.c_int64, P]
        L.orc_fd_render.restype = None
        L.orc_fd_render.argtypes = [P, P, P, P, P, P]
        L.orc_fd_end.restype = None
        L.orc_fd_end.argtypes = [P]
        L.orc_set_prim.restype = None
        L.orc_set_prim.argtypes = [P, C.c_int64, P, P, P, C.c_double, P, C.c_int]
        L.orc_free.restype = None
        L.orc_free.argtypes = [P]
        L.orc_contract_bin.restype = None
        L.orc_contract_bin.argtypes = [C.c_int64, P, P, P, P, P, P, C.c_int, C.c_int, C.c_int, P, P, P, P, P]
        L.orc_contract_tiles.restype = None
        L.orc_contract_tiles.argtypes = [C.c_int64, P, P, P, P, C.c_int, C.c_int, P]
        L.orc_contract_exp.restype = C.c_float
        L.orc_contract_exp.argtypes = [C.c_float]
        L.orc_contract_log.restype = C.c_float
        L.orc_contract_log.argtypes = [C.c_float]
        L.orc_sh_basis.restype = None
        L.orc_sh_basis.argtypes = [C.c_int, C.c_int64, P, P]
        L.orc_erank.restype = C.c_double
        L.orc_erank.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_exchange.restype = C.c_int64
        L.orc_exchange.argtypes = [C.c_int64, P, P, P, C.c_int, C.c_double, P, P, P, P]
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return int(lib().orc_num_threads())


OUT_FIELDS = ("r", "g", "b", "depth", "nx", "ny", "nz", "alpha", "T", "n_contrib")


class Oracle:
    """FP64 renderer context for one (scene, camera, config)."""

    def __init__(self, scene, cam, cfg):
        L = lib()
        self.n = scene.n
        self.W, self.H = cam.width, cam.height
        self.deg = scene.sh_degree
        self._keep = [np.ascontiguousarray(scene.means, np.float64),
                      np.ascontiguousarray(scene.log_scales, np.float64),
                      np.ascontiguousarray(scene.quats, np.float64),
                      np.ascontiguousarray(scene.opacity_logits, np.float64),
                      np.ascontiguousarray(scene.sh, np.float64),
                      np.ascontiguousarray(scene.types, np.uint8),
                      cam.as_array16(), cfg.as_oracle_array()]
        m, ls, q, lg, sh, ty, cam16, cf = self._keep
        self.ctx = L.orc_prepare(self.n, _p(m), _p(ls), _p(q), _p(lg), _p(sh), _p(ty),
                                 self.deg, _p(cam16), self.W, self.H, _p(cf))

    def close(self):
        if self.ctx:
            lib().orc_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _render(self, pixels):
        if pixels is None:
            npix = self.W * self.H
            pp = None
        else:
            pixels = np.ascontiguousarray(pixels, np.int32)
            npix = len(pixels)
            pp = _p(pixels)
        out = np.zeros((npix, 10), np.float64)
        flags = np.zeros(npix, np.uint8)
        tol = np.zeros((npix, 10), np.float64)
        lib().orc_render(self.ctx, npix, pp, _p(out), _p(flags), _p(tol))
        return out, flags, tol

    def render(self, pixels=None):
        """pixels: (P, 2) int pixel indices (x, y) or None for the full frame
        (row-major).  Returns (out (P, 10) float64, amb (P,) bool): the result
        with every threshold decision taken the FP64 way, and whether the
        pixel met an ambiguous decision (other results are correct too)."""
        out, flags, _ = self._render(pixels)
        return out, flags != 0

    def render_checked(self, pixels=None):
        """Everything an image comparison needs for `pixels` (None = full
        frame, row-major): out (P, 10) and tol (P, 10), the FP64-decision
        result and its conditioning tolerance; flags (P,) (bit 0: ambiguous
        decisions met, bit 1: more than the renderer enumerates); variants:
        {pixel row: (nv, 20) every correct result and its tolerance} for the
        pixels with bit 0 set."""
        out, flags, tol = self._render(pixels)
        if pixels is None:
            yy, xx = np.mgrid[0:self.H, 0:self.W]
            pixels = np.stack([xx.ravel(), yy.ravel()], 1)
        pixels = np.ascontiguousarray(pixels, np.int32)
        rows = np.nonzero(flags & 1)[0]
        variants = {}
        if len(rows):
            mv = int(lib().orc_max_variants())
            sub = np.ascontiguousarray(pixels[rows], np.int32)
            nv = np.zeros(len(rows), np.int32)
            leaves = np.zeros((len(rows), mv, 20), np.float64)
            lib().orc_render_variants(self.ctx, len(rows), _p(sub), _p(nv), _p(leaves))
            for k, r in enumerate(rows):
                variants[int(r)] = leaves[k, :nv[k]].copy()
        return {"pixels": pixels, "out": out, "tol": tol, "flags": flags, "variants": variants}

    def render_maps(self):
        """Full frame as planar maps: dict rgb (3,H,W), depth, normal (3,H,W),
        alpha, T, n_contrib, amb (H,W) (ambiguous decisions met, or a
        conditioning tolerance above 1e-4: pixels whose gradient the
        comparison leaves out), and `checked`, the render_checked() record of
        the frame."""
        chk = self.render_checked(None)
        out, flags = chk["out"], chk["flags"]
        H, W = self.H, self.W
        o = out.reshape(H, W, 10)
        amb = (flags != 0) | (chk["tol"][:, :8].max(1) > 1e-4)
        return {"rgb": np.moveaxis(o[..., 0:3], -1, 0), "depth": o[..., 3],
                "normal": np.moveaxis(o[..., 4:7], -1, 0), "alpha": o[..., 7],
                "T": o[..., 8], "n_contrib": o[..., 9], "amb": amb.reshape(H, W),
                "checked": chk}

    def pair_alpha(self, i, pixels):
        """alpha exp(-d/2) of primitive i alone at `pixels` (P, 2), 0 where
        it does not contribute."""
        pixels = np.ascontiguousarray(pixels, np.int32)
        out = np.zeros(len(pixels), np.float64)
        lib().orc_pair_alpha(self.ctx, int(i), len(pixels), _p(pixels), _p(out))
        return out

    def pixel_contributors(self, pixels, maxc=256):
        """For each pixel, the ids of the primitives Eq. 2 blends there (every
        decision the FP64 way), front to back: list of int arrays."""
        pixels = np.ascontiguousarray(pixels, np.int32)
        ids = np.zeros((len(pixels), maxc), np.int32)
        cnt = np.zeros(len(pixels), np.int32)
        lib().orc_pixel_contributors(self.ctx, len(pixels), _p(pixels), int(maxc), _p(ids), _p(cnt))
        return [ids[k, :cnt[k]].copy() for k in range(len(pixels))]

    def pair_conditioning(self, ids, pixels):
        """For (primitive, pixel) pairs: the binary32 conditioning bounds
        (du, dv) of the primitive's splat-frame coordinates at the pixel
        centre, (P, 2) float64 (-1 where a surfel's plane is missed)."""
        ids = np.ascontiguousarray(ids, np.int64)
        pixels = np.ascontiguousarray(pixels, np.int32)
        out = np.zeros((len(ids), 2), np.float64)
        lib().orc_pair_conditioning(self.ctx, len(ids), _p(ids), _p(pixels), _p(out))
        return out

    def fd_session(self, i, pixels):
        """A finite-difference session for primitive i at `pixels`: the other
        primitives' pairs there are evaluated and sorted once; render() then
        re-evaluates primitive i with its current parameters (set_prim) and
        blends, returning (out (P, 10), amb (P,) bool) as Oracle.render."""
        return _FDSession(self, i, pixels)

    def set_prim(self, i, mean, log_scale, quat, logit, sh, type_):
        a = [np.ascontiguousarray(x, np.float64) for x in (mean, log_scale, quat, sh)]
        lib().orc_set_prim(self.ctx, int(i), _p(a[0]), _p(a[1]), _p(a[2]), float(logit),
                           _p(a[3]), int(type_))


class _FDSession:
    def __init__(self, orc, i, pixels):
        self.orc = orc
        self.pixels = np.ascontiguousarray(pixels, np.int32)
        self.h = lib().orc_fd_begin(orc.ctx, int(i), len(self.pixels), _p(self.pixels))

    def render(self, with_tol=False):
        """(out (P, 10), amb (P,) bool, place (P,) int32: the primitive's place
        in each pixel's sorted pairs, -1 if absent[, tol (P, 10)])."""
        P = len(self.pixels)
        out = np.zeros((P, 10), np.float64)
        flags = np.zeros(P, np.uint8)
        tol = np.zeros((P, 10), np.float64)
        place = np.zeros(P, np.int32)
        lib().orc_fd_render(self.orc.ctx, self.h, _p(out), _p(flags), _p(tol), _p(place))
        return (out, flags != 0, place, tol) if with_tol else (out, flags != 0, place)

    def close(self):
        if self.h:
            lib().orc_fd_end(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def contract_bin(scene, cam, cfg, with_rowp=False):
    """FP32 binning contract for every primitive: (depth_bits u32 (N,),
    rect int32 (N,4) = tx0,tx1,ty0,ty1 (-1 if not binned), touched int64:
    the tiles of the primitive's tile set[, rowp float32 (N,12): the tile-set
    parameters])."""
    n = scene.n
    arrs = [np.ascontiguousarray(scene.means, np.float32),
            np.ascontiguousarray(scene.log_scales, np.float32),
            np.ascontiguousarray(scene.quats, np.float32),
            np.ascontiguousarray(scene.opacity_logits, np.float32),
            np.ascontiguousarray(scene.types, np.uint8)]
    cam16 = cam.as_array16()
    cfg32 = np.array([cfg.near, cfg.alpha_min, cfg.dilation], np.float32)
    db = np.zeros(n, np.uint32)
    rect = np.zeros((n, 4), np.int32)
    touched = np.zeros(n, np.int64)
    rowp = np.zeros((n, 12), np.float32)
    lib().orc_contract_bin(n, *[_p(a) for a in arrs], _p(cam16), cam.width, cam.height,
                           cfg.tile, _p(cfg32), _p(db), _p(rect), _p(touched), _p(rowp))
    return (db, rect, touched, rowp) if with_rowp else (db, rect, touched)


def contract_tiles(rect, rowp, touched, width, tile=16):
    """The tile ids of every binned primitive's tile set (row by row, left to
    right), concatenated in primitive order: (tiles (K,) uint32, first (N,)
    int64 offsets)."""
    touched = np.ascontiguousarray(touched, np.int64)
    first = np.ascontiguousarray(np.cumsum(touched) - touched, np.int64)
    K = int(touched.sum())
    tiles = np.zeros(max(K, 1), np.uint32)
    lib().orc_contract_tiles(len(touched), _p(np.ascontiguousarray(rect, np.int32)),
                             _p(np.ascontiguousarray(rowp, np.float32)), _p(touched), _p(first), int(width),
                             int(tile), _p(tiles))
    return tiles[:K], first


def tile_lists(scene, cam, cfg):
    """The binned instance list the contract defines: keys (K,) uint64 =
    tile_id << 32 | depth bits, vals (K,) uint32 primitive ids, sorted by
    (key, id); ranges (tiles, 2) uint32 [start, end)."""
    db, rect, touched, rowp = contract_bin(scene, cam, cfg, with_rowp=True)
    T = cfg.tile
    TX = (cam.width + T - 1) // T
    TY = (cam.height + T - 1) // T
    ids = np.nonzero(touched > 0)[0]
    cnt = touched[ids]
    rep = np.repeat(ids, cnt)
    tile, _ = contract_tiles(rect, rowp, touched, cam.width, T)
    keys = (tile.astype(np.uint64) << np.uint64(32)) | db[rep].astype(np.uint64)
    order = np.lexsort((rep, keys))
    keys = keys[order]
    vals = rep[order].astype(np.uint32)
    tiles_of = (keys >> np.uint64(32)).astype(np.int64)
    edges = np.searchsorted(tiles_of, np.arange(TX * TY + 1))
    ranges = np.stack([edges[:-1], edges[1:]], axis=1).astype(np.uint32)
    ranges[ranges[:, 0] == ranges[:, 1]] = 0  # an empty tile is [0, 0)
    return keys, vals, ranges, (db, rect, touched)


def contract_exp(x: float) -> float:
    return float(lib().orc_contract_exp(float(x)))


def contract_log(x: float) -> float:
    return float(lib().orc_contract_log(float(x)))


def sh_basis(deg: int, dirs: np.ndarray) -> np.ndarray:
    dirs = np.ascontiguousarray(dirs, np.float64)
    nb = (deg + 1) ** 2
    out = np.zeros((len(dirs), nb), np.float64)
    lib().orc_sh_basis(deg, len(dirs), _p(dirs), _p(out))
    return out


def erank(lsx, lsy, lsz) -> float:
    return float(lib().orc_erank(float(lsx), float(lsy), float(lsz)))


def exchange(log_scales, quats, types, mode="erank", theta=2.05, mask=None):
    """Adaptive Type Exchange in FP64.  Returns (log_scales f64, quats f64,
    types u8, n_flipped)."""
    ls = np.ascontiguousarray(log_scales, np.float32)
    q = np.ascontiguousarray(quats, np.float32)
    t = np.ascontiguousarray(types, np.uint8)
    n = len(t)
    m = np.ascontiguousarray(mask if mask is not None else np.zeros(n), np.uint8)
    ls_o = np.zeros((n, 3), np.float64)
    q_o = np.zeros((n, 4), np.float64)
    t_o = np.zeros(n, np.uint8)
    nf = lib().orc_exchange(n, _p(ls), _p(q), _p(t), 0 if mode == "erank" else 1, float(theta),
                            _p(m), _p(ls_o), _p(q_o), _p(t_o))
    return ls_o, q_o, t_o, int(nf)
