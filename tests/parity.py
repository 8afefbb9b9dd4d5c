"""Helpers shared by the GPU parity tests: run the CUDA path and the FP64
oracle on the same seeded inputs and compare (decision-aware)."""
from __future__ import annotations

import math

import numpy as np

import oracle

LOG2E = 1.0 / math.log(2.0)

# Tolerances (written out here so every test uses the same bar):
# RGB max-abs on pixels whose every decision is at least MARGIN away from its
# threshold (relative), and mean-abs over every pixel.
RGB_MAX_ABS = 2e-3
RGB_MEAN_ABS = 1e-5
MARGIN = 1e-3


def gpu_render(r, mode="plain", **kw):
    """Render with an existing Renderer; returns per-camera numpy images,
    final T and the debug view (numpy)."""
    import torch
    T = torch.empty(r.n_pixels, dtype=torch.float32, device=r.device)
    flat = r.render(mode=mode, out_T=T, **kw)
    torch.cuda.synchronize()
    imgs = [x.cpu().numpy() for x in r.images(flat)]
    Ts, off = [], 0
    Tn = T.cpu().numpy()
    for c in r.cameras:
        k = c["width"] * c["height"]
        Ts.append(Tn[off:off + k].reshape(c["height"], c["width"]))
        off += k
    return imgs, Ts


def debug_numpy(r):
    d = r.debug_view()
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in d.items()}


def oracle_options(mode="plain", group=(2, 2), opacity_filter=False, cluster_filter=False, sel_bits=0xFFFFFFFF):
    return oracle.Options(cr=(mode == "cr"), group_w=group[0], group_h=group[1], opacity_filter=opacity_filter,
                          use_mask=cluster_filter, sel_bits=sel_bits)


def compare_images(gpu, ref, margin, max_abs=RGB_MAX_ABS, mean_abs=RGB_MEAN_ABS):
    """Returns (ok, report). ``margin`` is the oracle's per-pixel decision margin."""
    err = np.abs(gpu.astype(np.float64) - ref)
    clear = margin >= MARGIN
    mx = float(err[:, clear].max()) if clear.any() else 0.0
    mean = float(err.mean())
    rep = dict(max_abs_clear=mx, mean_abs=mean, ambiguous_frac=float(1 - clear.mean()),
               max_abs_all=float(err.max()))
    return (mx <= max_abs and mean <= mean_abs), rep


def records_to_proj(rec):
    """GPU raster records -> u, v, conic (A, B, C), opacity, rgb."""
    u, v = rec[:, 0], rec[:, 1]
    A = rec[:, 2] / (-0.5 * LOG2E)
    B = rec[:, 3] / (-LOG2E)
    C = rec[:, 4] / (-0.5 * LOG2E)
    o = np.exp2(rec[:, 5].astype(np.float64))
    return u, v, np.stack([A, B, C], 1), o, rec[:, 8:11]


def oracle_render_tiles(proj, cam, opts: oracle.Options, tiles, nthreads: int = 8):
    """The oracle's render of the given tiles only, for workloads too large to
    bin whole on the CPU: the Gaussians whose rect covers a sampled tile go
    through the oracle's own instance builder (tile test, (depth, index) sort),
    every other tile's list is emptied, and the oracle rasterizes the rest.
    Returns (Render, global Gaussian ids of each sampled tile's list)."""
    tx_n, _ = oracle.tile_grid(cam, opts)
    tiles = np.unique(np.asarray(tiles, np.int64))
    rect = proj["rect"]
    vis = proj["visible"] == 1
    sel = np.zeros(proj.shape[0], bool)
    for t in tiles:
        tx, ty = t % tx_n, t // tx_n
        sel |= vis & (rect[:, 0] <= tx) & (tx <= rect[:, 2]) & (rect[:, 1] <= ty) & (ty <= rect[:, 3])
    idx = np.nonzero(sel)[0]
    sub = np.ascontiguousarray(proj[idx])
    _, gid, ranges = oracle.instances(sub, cam, opts)
    keep = np.zeros(ranges.shape[0], bool)
    keep[tiles] = True
    ranges = ranges.copy()
    ranges[~keep] = 0
    ref = oracle.render_tiled(sub, gid, ranges, cam, opts, nthreads)
    lists = {int(t): idx[gid[ranges[t, 0]:ranges[t, 1]]] for t in tiles}
    return ref, lists
