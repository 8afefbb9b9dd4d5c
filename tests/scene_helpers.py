"""Hand-built tiny scenes for the pin tests (inputs only, no rendering math)."""
import math

import numpy as np


def camera(f=100.0, width=64, height=64, cx=None, cy=None, R=None, t=None, near=0.2):
    R = np.eye(3) if R is None else np.asarray(R, np.float64)
    t = np.zeros(3) if t is None else np.asarray(t, np.float64)
    return dict(world_to_cam=np.concatenate([R, t[:, None]], 1), fx=f, fy=f,
                cx=width / 2.0 if cx is None else cx, cy=height / 2.0 if cy is None else cy,
                width=width, height=height, near=near)


def scene(means, log_scales=None, quats=None, opacity=None, dc=None, sh=None, sh_degree=0, mask=None):
    means = np.asarray(means, np.float64).reshape(-1, 3)
    n = means.shape[0]
    nc = (sh_degree + 1) ** 2
    if log_scales is None:
        log_scales = np.full((n, 3), math.log(0.05))
    log_scales = np.broadcast_to(np.asarray(log_scales, np.float64), (n, 3)).copy()
    if quats is None:
        quats = np.tile([1.0, 0, 0, 0], (n, 1))
    quats = np.asarray(quats, np.float64).reshape(n, 4)
    if opacity is None:
        opacity = np.full(n, 0.8)
    opacity = np.broadcast_to(np.asarray(opacity, np.float64), (n,))
    logits = np.log(opacity / (1 - opacity))
    if sh is None:
        sh = np.zeros((n, nc, 3))
        if dc is not None:
            sh[:, 0, :] = np.broadcast_to(np.asarray(dc, np.float64), (n, 3))
    s = dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=logits,
             sh=np.asarray(sh, np.float64).reshape(n, nc, 3), sh_degree=sh_degree)
    if mask is not None:
        s["cluster_mask"] = np.asarray(mask, np.uint32)
    return s
