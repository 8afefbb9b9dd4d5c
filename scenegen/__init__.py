"""Seeded synthetic scenes and cameras for the Seele hot path.

This module only draws inputs: Gaussian attributes, cluster memberships and
camera poses.  It holds none of the rendering arithmetic, and both the CUDA
path and the FP64 oracle consume what it returns.  The scenes stand in for
the trained 3DGS captures (Mip-NeRF360, Tanks&Temples, DeepBlending) the paper
evaluates on, which are not available here; their shapes follow the workload
list below.

Attribute distributions (shared by every workload unless stated):
  log-scales ~ N(ln 0.02, 0.5) per axis; quaternions = normalised N(0, 1)^4;
  opacity logits ~ N(0, 1.5); SH degree 3 with the DC coefficient ~ N(0.5, 0.2)
  per channel and higher-order coefficients ~ N(0, 0.05).

Workloads:
  uniform_10k      10k means uniform in [-1, 1]^3, one 256x256 camera at
                   (0, 0, -3) looking at the origin, 60 deg FOV.
  clusters_500k    500k means from 64 isotropic clusters (sigma 0.1, centres
                   uniform in [-2, 2]^3), eight 1280x720 cameras on a radius-4
                   orbit, 16 view clusters (see ``view_clusters``).
  unbounded_3m     3M: 80% in 64 dense clusters (sigma 0.15, centres in
                   [-3, 3]^3) and 20% on a background shell of radius 30-50 with
                   log-scales ~ N(ln 0.5, 0.5); 1920x1080 cameras on a radius-5
                   orbit.
  clusters_1m      1M shaped as clusters_500k, 1280x720, plus an L1 target
                   rendered from attributes perturbed by N(0, 0.01).
  multiview_2m     2M shaped as unbounded_3m; 64 cameras with resolutions drawn
                   from {640x360, 1280x720, 1920x1080}, random poses at radius
                   3-6 looking at the origin.
"""
from __future__ import annotations

import math

import numpy as np

SH_DEGREE = 3
N_SH = (SH_DEGREE + 1) ** 2


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def attributes(n: int, r: np.random.Generator, log_scale_mean=math.log(0.02), log_scale_std=0.5,
               sh_degree: int = SH_DEGREE) -> dict:
    nc = (sh_degree + 1) ** 2
    log_scales = (log_scale_mean + log_scale_std * r.standard_normal((n, 3))).astype(np.float32)
    q = r.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logits = (1.5 * r.standard_normal(n)).astype(np.float32)
    sh = np.empty((n, nc, 3), np.float32)
    sh[:, 0, :] = 0.5 + 0.2 * r.standard_normal((n, 3))
    if nc > 1:
        sh[:, 1:, :] = 0.05 * r.standard_normal((n, nc - 1, 3))
    return dict(log_scales=log_scales, quats=q.astype(np.float32), opacity_logits=logits, sh=sh,
                sh_degree=sh_degree)


def cluster_means(n: int, n_clusters: int, sigma: float, half_extent: float, r: np.random.Generator):
    centres = r.uniform(-half_extent, half_extent, (n_clusters, 3))
    which = r.integers(0, n_clusters, n)
    return (centres[which] + sigma * r.standard_normal((n, 3))).astype(np.float32)


def shell_means(n: int, r_min: float, r_max: float, r: np.random.Generator):
    d = r.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    rad = r.uniform(r_min, r_max, (n, 1))
    return (d * rad).astype(np.float32)


# ---------------------------------------------------------------- cameras --

def look_at(eye, target, width: int, height: int, fov_y_deg: float = 60.0, near: float = 0.2) -> dict:
    """Pinhole camera with x right, y down (world +y is down), z forward."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, z)
    if np.linalg.norm(x) < 1e-6:
        x = np.cross(np.array([0.0, 0.0, 1.0]), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ eye
    fy = 0.5 * height / math.tan(math.radians(fov_y_deg) / 2)
    w2c = np.concatenate([R, t[:, None]], axis=1)
    return dict(world_to_cam=w2c, fx=fy, fy=fy, cx=width / 2.0, cy=height / 2.0, width=int(width),
                height=int(height), near=near)


def orbit(n: int, radius: float, width: int, height: int, elevation_deg: float = 0.0, phase: float = 0.0):
    cams = []
    el = math.radians(elevation_deg)
    for k in range(n):
        th = 2 * math.pi * k / n + phase
        eye = (radius * math.cos(th) * math.cos(el), -radius * math.sin(el), radius * math.sin(th) * math.cos(el))
        cams.append(look_at(eye, (0, 0, 0), width, height))
    return cams


def random_poses(n: int, r_min: float, r_max: float, resolutions, r: np.random.Generator):
    cams = []
    for _ in range(n):
        az = r.uniform(0, 2 * math.pi)
        el = math.radians(r.uniform(-30, 30))
        rad = r.uniform(r_min, r_max)
        W, H = resolutions[r.integers(0, len(resolutions))]
        eye = (rad * math.cos(az) * math.cos(el), -rad * math.sin(el), rad * math.sin(az) * math.cos(el))
        cams.append(look_at(eye, (0, 0, 0), W, H))
    return cams


# ---------------------------------------------------------- view clusters --

def view_clusters(means: np.ndarray, n_clusters: int, radius: float, r: np.random.Generator,
                  shared_frac: float = 0.3, spread: int = 1):
    """Synthetic stand-in for the offline view-dependent representation.

    Cluster c is a camera pose on the orbit at azimuth 2 pi c / C (jittered so
    that no two centroid distances tie), described by the feature
    (position / radius, viewing direction).  A random ``shared_frac`` of the
    Gaussians is shared (every cluster bit set); every other Gaussian is
    exclusive to the cluster nearest its own azimuth and to ``spread``
    neighbours on each side.  Returns (mask uint32 [n], centroids [C, 6],
    pos_scale)."""
    assert n_clusters <= 32
    az_c = 2 * math.pi * np.arange(n_clusters) / n_clusters + r.uniform(-0.05, 0.05, n_clusters)
    pos = np.stack([np.cos(az_c), np.zeros(n_clusters), np.sin(az_c)], 1)
    view = -pos
    centroids = np.concatenate([pos, view], 1) + r.uniform(-1e-3, 1e-3, (n_clusters, 6))
    az_g = np.arctan2(means[:, 2].astype(np.float64), means[:, 0].astype(np.float64)) % (2 * math.pi)
    home = np.rint(az_g / (2 * math.pi) * n_clusters).astype(np.int64) % n_clusters
    mask = np.zeros(means.shape[0], np.uint32)
    for off in range(-spread, spread + 1):
        mask |= (np.uint32(1) << ((home + off) % n_clusters).astype(np.uint32)).astype(np.uint32)
    shared = r.random(means.shape[0]) < shared_frac
    mask[shared] = np.uint32(0xFFFFFFFF)
    return mask, centroids, float(radius)


def sample_poses(n: int, radius: float, width: int, height: int, r: np.random.Generator,
                 elevation_deg: float = 30.0, fov_y_deg: float = 60.0) -> list:
    """n random camera poses on a sphere of the given radius looking at the
    origin: azimuth U[0, 2 pi), elevation U[-elevation, elevation]."""
    az = r.uniform(0.0, 2 * math.pi, n)
    el = np.radians(r.uniform(-elevation_deg, elevation_deg, n))
    cams = []
    for a, e in zip(az, el):
        eye = (radius * math.cos(a) * math.cos(e), -radius * math.sin(e), radius * math.sin(a) * math.cos(e))
        cams.append(look_at(eye, (0.0, 0.0, 0.0), width, height, fov_y_deg))
    return cams


def kmeans_uniforms(k: int, r: np.random.Generator) -> np.ndarray:
    """The k uniforms in [0, 1) that drive k-means++ seeding."""
    return r.random(k)


# -------------------------------------------------------------- workloads --

def uniform_10k(seed: int = 0, n: int = 10_000, width: int = 256, height: int = 256) -> tuple[dict, list]:
    r = rng(seed)
    means = r.uniform(-1, 1, (n, 3)).astype(np.float32)
    scene = dict(means=means, **attributes(n, r))
    cams = [look_at((0, 0, -3), (0, 0, 0), width, height)]
    return scene, cams


def clusters_500k(seed: int = 0, n: int = 500_000, width: int = 1280, height: int = 720, n_cams: int = 8,
                  n_view_clusters: int = 16) -> tuple[dict, list]:
    r = rng(seed)
    means = cluster_means(n, 64, 0.1, 2.0, r)
    scene = dict(means=means, **attributes(n, r))
    mask, centroids, pos_scale = view_clusters(means, n_view_clusters, 4.0, r)
    scene.update(cluster_mask=mask, centroids=centroids, pos_scale=pos_scale)
    cams = orbit(n_cams, 4.0, width, height)
    return scene, cams


def unbounded_3m(seed: int = 0, n: int = 3_000_000, width: int = 1920, height: int = 1080,
                 n_cams: int = 8) -> tuple[dict, list]:
    r = rng(seed)
    n_dense = int(round(0.8 * n))
    n_shell = n - n_dense
    dense = cluster_means(n_dense, 64, 0.15, 3.0, r)
    shell = shell_means(n_shell, 30.0, 50.0, r)
    means = np.concatenate([dense, shell])
    attr = attributes(n, r)
    attr["log_scales"][n_dense:] = (math.log(0.5) + 0.5 * r.standard_normal((n_shell, 3))).astype(np.float32)
    scene = dict(means=means, **attr)
    cams = orbit(n_cams, 5.0, width, height, phase=0.3)
    return scene, cams


def clusters_1m(seed: int = 0, n: int = 1_000_000, width: int = 1280, height: int = 720):
    scene, cams = clusters_500k(seed, n=n, width=width, height=height, n_cams=1)
    r = rng(seed + 1)
    target = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    for k in ("means", "log_scales", "opacity_logits", "sh", "quats"):
        target[k] = (scene[k] + 0.01 * r.standard_normal(scene[k].shape)).astype(np.float32)
    target["quats"] /= np.linalg.norm(target["quats"], axis=1, keepdims=True)
    return scene, cams, target


def multiview_2m(seed: int = 0, n: int = 2_000_000, n_cams: int = 64):
    scene, _ = unbounded_3m(seed, n=n, n_cams=1)
    r = rng(seed + 7)
    cams = random_poses(n_cams, 3.0, 6.0, [(640, 360), (1280, 720), (1920, 1080)], r)
    return scene, cams


def subset(scene: dict, idx) -> dict:
    """Scene restricted to the Gaussians ``idx`` (arrays indexed, scalars kept)."""
    n = scene["means"].shape[0]
    out = {}
    for k, v in scene.items():
        out[k] = v[idx] if isinstance(v, np.ndarray) and v.shape[:1] == (n,) else v
    return out
