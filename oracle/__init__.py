"""FP64 CPU oracle for the Seele hot path (arxiv 2503.05168).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product package
never imports this module, and this module imports nothing from the product
package.  All arithmetic lives in ``seele_oracle.c`` (plain C, double
precision, one Gaussian / one pixel at a time); this file only marshals numpy
arrays through ctypes.

What each entry point follows in the paper:

* ``preprocess``       Sec. 3.1 "Preprocessing" (frustum cull, EWA projection
                       of Eqn. 2's Sigma', SH colour) and Sec. 3.3 (view-cluster
                       filter; online filtering of Eqns. 3-5).
* ``instances``        Sec. 3.1 "Sorting": per-tile lists in (fp32 depth, index)
                       order.
* ``render_tiled``     Sec. 3.1 "Rasterization", Eqns. 1-2 and the alpha_theta
                       / Gamma_theta rules; with ``cr`` Algorithm 1 (Sec. 3.4).
* ``pixel_outcomes``   the outcomes of a pixel of ``render_tiled`` when any
                       decision near its threshold goes the other way (the
                       decision-aware comparison with an FP32 render).
* ``render_bruteforce`` the same rules without tiles: every pixel walks every
                       visible Gaussian in global depth order.
* ``backward_*``       the chain rule through the above (Sec. 3.5 fine-tuning;
                       HP and CR decisions held fixed).
* ``select_clusters``  Sec. 3.3 "Algorithm": nearest cluster plus M neighbours.

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, library routines, brute force,
finite differences).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "seele_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

CAMERA_DTYPE = np.dtype(
    [("R", "f8", (9,)), ("t", "f8", (3,)), ("fx", "f8"), ("fy", "f8"), ("cx", "f8"), ("cy", "f8"),
     ("width", "i4"), ("height", "i4"), ("near_z", "f8")],
    align=True,
)
OPTIONS_DTYPE = np.dtype(
    [("tile_w", "i4"), ("tile_h", "i4"), ("opacity_filter", "i4"), ("cr", "i4"), ("group_w", "i4"),
     ("group_h", "i4"), ("use_mask", "i4"), ("sel_bits", "u4"), ("tile_test", "i4"), ("alpha_min", "f8"),
     ("alpha_max", "f8"), ("t_stop", "f8"), ("dilation", "f8"), ("frustum_slack", "f8")],
    align=True,
)
PROJ_DTYPE = np.dtype(
    [("visible", "i4"), ("radius", "i4"), ("rect", "i4", (4,)), ("ntiles", "i4"), ("depth32", "f4"),
     ("mean_cam", "f8", (3,)), ("uv", "f8", (2,)), ("cov2", "f8", (3,)), ("conic", "f8", (3,)),
     ("opacity", "f8"), ("rgb_raw", "f8", (3,)), ("rgb", "f8", (3,)), ("tg", "f8"), ("margin_px", "f8"),
     ("margin_rel", "f8")],
    align=True,
)
NCOUNT = 8
COUNTER_NAMES = ("visible", "instances", "alpha_evals", "blended", "leader_tests", "leader_skips",
                 "terminated", "clamped")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + OpenMP). Returns the .so path."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I32 = ctypes.c_int
        lib.oc_preprocess.argtypes = [I64, I32, P, P, P, P, P, P, P, P, P, I32]
        lib.oc_preprocess.restype = None
        lib.oc_count_instances.argtypes = [I64, P]
        lib.oc_count_instances.restype = I64
        lib.oc_build_instances.argtypes = [I64, P, P, I32, I32, P, P, P]
        lib.oc_build_instances.restype = None
        lib.oc_render_tiled.argtypes = [P, P, P, I32, I32, P, P, P, P, P, P, I32]
        lib.oc_render_tiled.restype = None
        lib.oc_pixel_outcomes.argtypes = [P, P, P, I32, I32, P, P, I64, ctypes.c_double, I32, P, P, I32]
        lib.oc_pixel_outcomes.restype = None
        lib.oc_render_bruteforce.argtypes = [I64, P, I32, I32, P, P, P, P, I32]
        lib.oc_render_bruteforce.restype = None
        lib.oc_backward_raster.argtypes = [I64, P, P, P, I32, I32, P, P, P]
        lib.oc_backward_raster.restype = None
        lib.oc_backward_preprocess.argtypes = [I64, I32, P, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.oc_backward_preprocess.restype = None
        lib.oc_select_clusters.argtypes = [I32, P, ctypes.c_double, P, I32]
        lib.oc_select_clusters.restype = ctypes.c_uint32
        lib.oc_sh_eval.argtypes = [I32, I64, P, P, P]
        lib.oc_pose_feature.argtypes = [P, ctypes.c_double, P]
        lib.oc_pose_feature.restype = None
        lib.oc_kmeans.argtypes = [I32, I32, P, I32, P, I32, P, P]
        lib.oc_kmeans.restype = I32
        lib.oc_topk_contributors.argtypes = [P, P, P, I32, I32, P, I32, P, P, P, P, I32]
        lib.oc_topk_contributors.restype = None
        lib.oc_contribution_skew.argtypes = [P, P, P, I32, I32, P, ctypes.c_double, P, P, P, P, P, I32]
        lib.oc_contribution_skew.restype = None
        lib.oc_sh_eval.restype = None
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


@dataclass
class Options:
    """Render options; defaults are the paper's constants (Sec. 3.1, Sec. 4.1)."""
    tile_w: int = 16
    tile_h: int = 16
    opacity_filter: bool = False
    cr: bool = False
    group_w: int = 2
    group_h: int = 2
    use_mask: bool = False
    sel_bits: int = 0xFFFFFFFF
    tile_test: str = "ellipse"          # or "rect": every tile of the bounding rect
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_stop: float = 1e-4
    dilation: float = 0.3
    frustum_slack: float = 1.3

    def to_struct(self):
        if self.cr and (self.tile_w % self.group_w or self.tile_h % self.group_h):
            raise ValueError("tile size must be a multiple of the pixel-group size")
        o = np.zeros((), OPTIONS_DTYPE)
        for k in ("tile_w", "tile_h", "group_w", "group_h"):
            o[k] = getattr(self, k)
        o["opacity_filter"] = int(self.opacity_filter)
        o["cr"] = int(self.cr)
        o["use_mask"] = int(self.use_mask)
        if self.tile_test not in ("ellipse", "rect"):
            raise ValueError("tile_test must be 'ellipse' or 'rect'")
        o["tile_test"] = int(self.tile_test == "ellipse")
        o["sel_bits"] = self.sel_bits & 0xFFFFFFFF
        for k in ("alpha_min", "alpha_max", "t_stop", "dilation", "frustum_slack"):
            o[k] = getattr(self, k)
        return o


def camera_struct(cam) -> np.ndarray:
    """``cam``: mapping with world_to_cam (3x4), fx, fy, cx, cy, width, height, near."""
    c = np.zeros((), CAMERA_DTYPE)
    w2c = np.asarray(cam["world_to_cam"], dtype=np.float64).reshape(3, 4)
    c["R"] = w2c[:, :3].reshape(9)
    c["t"] = w2c[:, 3]
    for k in ("fx", "fy", "cx", "cy"):
        c[k] = float(cam[k])
    c["width"] = int(cam["width"])
    c["height"] = int(cam["height"])
    c["near_z"] = float(cam.get("near", 0.2))
    return c


@dataclass
class Scene64:
    """Scene attributes promoted to float64 (the oracle's working precision)."""
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int
    mask: np.ndarray | None = None
    centroids: np.ndarray | None = None
    pos_scale: float = 1.0

    @property
    def n(self):
        return self.means.shape[0]

    @staticmethod
    def from_scene(s) -> "Scene64":
        n = s["means"].shape[0]
        deg = int(s["sh_degree"])
        nc = (deg + 1) ** 2
        mask = s.get("cluster_mask")
        return Scene64(
            means=_f64(s["means"], (n, 3)), log_scales=_f64(s["log_scales"], (n, 3)),
            quats=_f64(s["quats"], (n, 4)), opacity_logits=_f64(s["opacity_logits"], (n,)),
            sh=_f64(s["sh"], (n, nc, 3)), sh_degree=deg,
            mask=None if mask is None else np.ascontiguousarray(mask, dtype=np.uint32),
            centroids=None if s.get("centroids") is None else _f64(s["centroids"], (-1, 6)),
            pos_scale=float(s.get("pos_scale", 1.0)),
        )


def preprocess(scene: Scene64, cam, opts: Options, nthreads: int = 1) -> np.ndarray:
    out = np.zeros(scene.n, PROJ_DTYPE)
    cams = camera_struct(cam)
    o = opts.to_struct()
    _L().oc_preprocess(scene.n, scene.sh_degree, _p(scene.means), _p(scene.log_scales), _p(scene.quats),
                       _p(scene.opacity_logits), _p(scene.sh), _p(scene.mask), _p(cams), _p(o), _p(out),
                       nthreads)
    return out


def tile_grid(cam, opts: Options):
    W, H = int(cam["width"]), int(cam["height"])
    return (W + opts.tile_w - 1) // opts.tile_w, (H + opts.tile_h - 1) // opts.tile_h


def instances(proj: np.ndarray, cam, opts: Options):
    """Sorted (tile, Gaussian) list and per-tile [start, end) ranges."""
    tx, ty = tile_grid(cam, opts)
    lib = _L()
    K = lib.oc_count_instances(proj.shape[0], _p(proj))
    tile = np.zeros(max(K, 1), np.int32)
    gid = np.zeros(max(K, 1), np.int32)
    ranges = np.zeros((tx * ty, 2), np.int64)
    o = opts.to_struct()
    lib.oc_build_instances(proj.shape[0], _p(proj), _p(o), tx, ty, _p(tile), _p(gid), _p(ranges))
    return tile[:K], gid[:K], ranges


@dataclass
class Render:
    rgb: np.ndarray          # [3, H, W]
    T: np.ndarray            # [H, W]
    ncontrib: np.ndarray     # [H, W]
    margin: np.ndarray       # [H, W] min relative decision margin
    counters: dict = field(default_factory=dict)


def render_tiled(proj, gid, ranges, cam, opts: Options, nthreads: int = 1) -> Render:
    W, H = int(cam["width"]), int(cam["height"])
    rgb = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), np.int64)
    margin = np.zeros((H, W))
    cnt = np.zeros(NCOUNT, np.int64)
    o = opts.to_struct()
    gid = np.ascontiguousarray(gid, np.int32)
    ranges = np.ascontiguousarray(ranges, np.int64)
    _L().oc_render_tiled(_p(proj), _p(gid) if gid.size else None, _p(ranges), W, H, _p(o), _p(rgb), _p(T),
                         _p(nc), _p(margin), _p(cnt), nthreads)
    counters = dict(zip(COUNTER_NAMES, cnt.tolist()))
    counters["visible"] = int(proj["visible"].sum())
    counters["instances"] = int(gid.size)
    return Render(rgb, T, nc, margin, counters)


def pixel_outcomes(proj, gid, ranges, cam, opts: Options, pixels, tol: float = 1e-3, max_out: int = 256,
                   nthreads: int = 1):
    """Every outcome (r, g, b, T) a pixel of the tiled render can reach when
    any decision taken within ``tol`` (relative) of its threshold goes the
    other way (see oc_pixel_outcomes).  ``pixels``: flat indices y * W + x.
    Returns (outcomes [npix, max_out, 4], counts [npix]); outcome 0 is the
    ordinary render's pixel, a count of -1 means more than ``max_out``."""
    W, H = int(cam["width"]), int(cam["height"])
    pix = np.ascontiguousarray(pixels, np.int64).reshape(-1)
    out = np.zeros((pix.size, max_out, 4))
    n = np.zeros(pix.size, np.int32)
    if pix.size == 0:
        return out, n
    o = opts.to_struct()
    gid = np.ascontiguousarray(gid, np.int32)
    ranges = np.ascontiguousarray(ranges, np.int64)
    _L().oc_pixel_outcomes(_p(proj), _p(gid) if gid.size else None, _p(ranges), W, H, _p(o), _p(pix), pix.size,
                           float(tol), int(max_out), _p(out), _p(n), nthreads)
    return out, n


def render(scene: Scene64, cam, opts: Options, nthreads: int = 1):
    """preprocess -> instances -> tiled render. Returns (Render, proj, tile, gid, ranges)."""
    proj = preprocess(scene, cam, opts, nthreads)
    tile, gid, ranges = instances(proj, cam, opts)
    return render_tiled(proj, gid, ranges, cam, opts, nthreads), proj, tile, gid, ranges


def render_bruteforce(proj, cam, opts: Options, nthreads: int = 1):
    W, H = int(cam["width"]), int(cam["height"])
    rgb = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), np.int64)
    o = opts.to_struct()
    _L().oc_render_bruteforce(proj.shape[0], _p(proj), W, H, _p(o), _p(rgb), _p(T), _p(nc), nthreads)
    return rgb, T


def backward(scene: Scene64, cam, opts: Options, dL_drgb: np.ndarray, proj=None, gid=None, ranges=None):
    """Analytic FP64 gradients of sum(dL_drgb * rgb) w.r.t. the scene attributes.

    Returns dict with means, log_scales, quats, opacity_logits, sh and the
    screen-space gradients g2d[n, 9] = d(u, v, A, B, C, o, r, g, b)."""
    if proj is None:
        proj = preprocess(scene, cam, opts)
        _, gid, ranges = instances(proj, cam, opts)
    W, H = int(cam["width"]), int(cam["height"])
    dC = _f64(dL_drgb, (3, H, W))
    n = scene.n
    g2d = np.zeros((n, 9))
    o = opts.to_struct()
    camst = camera_struct(cam)
    gid = np.ascontiguousarray(gid, np.int32)
    lib = _L()
    lib.oc_backward_raster(n, _p(proj), _p(gid) if gid.size else None, _p(np.ascontiguousarray(ranges, np.int64)),
                           W, H, _p(o), _p(dC), _p(g2d))
    nc = (scene.sh_degree + 1) ** 2
    out = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacity_logits=np.zeros(n), sh=np.zeros((n, nc, 3)))
    lib.oc_backward_preprocess(n, scene.sh_degree, _p(scene.means), _p(scene.log_scales), _p(scene.quats),
                               _p(scene.opacity_logits), _p(scene.sh), _p(camst), _p(o), _p(proj), _p(g2d),
                               _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]),
                               _p(out["opacity_logits"]), _p(out["sh"]))
    out["g2d"] = g2d
    return out


def select_clusters(centroids: np.ndarray, pos_scale: float, cam, M: int) -> int:
    c = _f64(centroids, (-1, 6))
    camst = camera_struct(cam)
    return int(_L().oc_select_clusters(c.shape[0], _p(c), float(pos_scale), _p(camst), int(M)))


def sh_eval(lmax: int, dirs: np.ndarray, grad: bool = False):
    d = _f64(dirs, (-1, 3))
    nc = (lmax + 1) ** 2
    y = np.zeros((d.shape[0], nc))
    g = np.zeros((d.shape[0], nc, 3)) if grad else None
    _L().oc_sh_eval(lmax, d.shape[0], _p(d), _p(y), _p(g))
    return (y, g) if grad else y


# ------------------------------------------------------------------------------
# Offline view-dependent representation (Sec. 3.3 "Offline Clustering")
# ------------------------------------------------------------------------------

def pose_features(poses, pos_scale: float) -> np.ndarray:
    """(x / s, v) per pose: camera centre over the position scale and the unit
    viewing direction (beta = 1)."""
    out = np.zeros((len(poses), 6))
    for i, cam in enumerate(poses):
        f = np.zeros(6)
        _L().oc_pose_feature(_p(camera_struct(cam)), float(pos_scale), _p(f))
        out[i] = f
    return out


def position_scale(poses) -> float:
    """s = the largest camera distance from the origin over the samples."""
    f = pose_features(poses, 1.0)
    return float(np.max(np.linalg.norm(f[:, :3], axis=1)))


def kmeans(x: np.ndarray, k: int, u: np.ndarray, max_iter: int = 100):
    """k-means++ seeded by the uniforms u[0..k), then Lloyd iterations (see
    oc_kmeans).  Returns (centroids [k, dim], assignment [n], updates)."""
    x = _f64(x, (x.shape[0], -1))
    u = _f64(u, (-1,))
    assert u.shape[0] >= k and x.shape[0] >= 1
    cent = np.zeros((k, x.shape[1]))
    assign = np.zeros(x.shape[0], np.int32)
    it = _L().oc_kmeans(x.shape[0], x.shape[1], _p(x), k, _p(u), int(max_iter), _p(cent), _p(assign))
    return cent, assign, int(it)


def topk_contributors(proj, gid, ranges, cam, opts: Options, k: int, nthreads: int = 1):
    """Per-pixel top-k contributors (Gamma alpha) of a plain render: ids and
    contributions [H, W, k] (-1 / 0 when unused), counts [H, W] and the
    per-pixel decision margin including the k-th / (k+1)-th gap."""
    W, H = int(cam["width"]), int(cam["height"])
    ids = np.zeros((H, W, k), np.int32)
    w = np.zeros((H, W, k))
    cnt = np.zeros((H, W), np.int32)
    margin = np.zeros((H, W))
    o = opts.to_struct()
    gid = np.ascontiguousarray(gid, np.int32)
    ranges = np.ascontiguousarray(ranges, np.int64)
    _L().oc_topk_contributors(_p(proj), _p(gid) if gid.size else None, _p(ranges), W, H, _p(o), int(k), _p(ids),
                              _p(w), _p(cnt), _p(margin), nthreads)
    return ids, w, cnt, margin


def contribution_skew(proj, gid, ranges, cam, opts: Options, frac: float = 0.99, nthreads: int = 1):
    """Per pixel of a plain render (Sec. 1, Sec. 3.4 "Motivation"): the
    smallest number m of its largest contributions Gamma alpha that sum to
    frac of their total, the number of contributions, the list entries it
    walked, the total, and the decision margin (see oc_contribution_skew)."""
    W, H = int(cam["width"]), int(cam["height"])
    m = np.zeros((H, W), np.int32)
    blended = np.zeros((H, W), np.int32)
    walked = np.zeros((H, W), np.int32)
    total = np.zeros((H, W))
    margin = np.zeros((H, W))
    o = opts.to_struct()
    gid = np.ascontiguousarray(gid, np.int32)
    ranges = np.ascontiguousarray(ranges, np.int64)
    _L().oc_contribution_skew(_p(proj), _p(gid) if gid.size else None, _p(ranges), W, H, _p(o), float(frac), _p(m),
                              _p(blended), _p(walked), _p(total), _p(margin), nthreads)
    return dict(m=m, blended=blended, walked=walked, total=total, margin=margin)


def view_masks(scene: Scene64, poses, assign: np.ndarray, k: int, opts: Options | None = None,
               nthreads: int = 1):
    """Cluster bit mask per Gaussian: bit c is set when the Gaussian is among
    the top-k contributors of some pixel of some pose assigned to cluster c
    (Gaussians of every cluster are the shared ones; a zero mask drops the
    Gaussian).  Also returns, per Gaussian, the smallest margin of a pixel
    that made it a member (for decision-aware comparisons)."""
    opts = opts or Options()
    mask = np.zeros(scene.n, np.uint32)
    gmargin = np.full(scene.n, np.inf)
    for cam, c in zip(poses, assign):
        proj = preprocess(scene, cam, opts, nthreads)
        _, gid, ranges = instances(proj, cam, opts)
        ids, _, _, margin = topk_contributors(proj, gid, ranges, cam, opts, k, nthreads)
        sel = ids >= 0
        g = ids[sel]
        mask[g] |= np.uint32(1) << np.uint32(c)
        m = np.broadcast_to(margin[..., None], ids.shape)[sel]
        np.minimum.at(gmargin, g, m)
    return mask, gmargin
