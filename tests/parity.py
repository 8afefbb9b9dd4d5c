"""Helpers shared by the GPU parity tests: run the CUDA path and the FP64
oracle on the same seeded inputs and compare (decision-aware)."""
from __future__ import annotations

import math

import numpy as np

import oracle

LOG2E = 1.0 / math.log(2.0)

# Tolerances (written out here so every test uses the same bar):
# RGB (and T) max-abs on pixels whose every decision is at least MARGIN away
# from its threshold (relative), and mean-abs over every pixel.
RGB_MAX_ABS = 2e-3
RGB_MEAN_ABS = 1e-5
MARGIN = 1e-3
# A pixel with a decision closer than MARGIN to its threshold is compared with
# every outcome the oracle reaches by flipping such decisions (reading A13);
# it may stay unchecked only if no outcome matches, its closest decision is
# within UNCHECKED_MARGIN of a flip, and at most UNCHECKED_SHARE of the
# compared pixels are in that state.
UNCHECKED_MARGIN = 1e-5
UNCHECKED_SHARE = 1e-4


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


def check_render(gpu_rgb, gpu_T, ref, proj, gid, ranges, cam, opts, pixels=None, max_abs=RGB_MAX_ABS,
                 mean_abs=RGB_MEAN_ABS):
    """Decision-aware comparison of a GPU frame ([3, H, W] colour and [H, W]
    transmittance, or None) with the oracle's tiled render of the same lists.

    Every pixel is checked:
      * pixels whose decisions are all at least MARGIN from their thresholds
        against the oracle's pixel, max-abs ``max_abs`` on colour and T;
      * the others against every outcome of ``oracle.pixel_outcomes`` (each
        near decision taken either way): the GPU pixel must be within
        ``max_abs`` of one of them;
      * a pixel no outcome matches fails, unless its closest decision lies
        within UNCHECKED_MARGIN of a flip, or it has more outcomes than the
        oracle enumerates (then only the first ones, the ordinary render's
        among them, are compared), and such pixels stay below
        UNCHECKED_SHARE of the compared ones;
    and the mean-abs colour error over the compared pixels stays below
    ``mean_abs``.  ``pixels``: flat indices to compare (default all).
    Returns a report with ``ok``."""
    W, H = int(cam["width"]), int(cam["height"])
    pix = np.arange(W * H) if pixels is None else np.asarray(pixels, np.int64).reshape(-1)
    g = gpu_rgb.reshape(3, -1)[:, pix].T.astype(np.float64)
    o = ref.rgb.reshape(3, -1)[:, pix].T
    if gpu_T is not None:
        g = np.concatenate([g, np.asarray(gpu_T, np.float64).reshape(-1)[pix, None]], 1)
        o = np.concatenate([o, ref.T.reshape(-1)[pix, None]], 1)
    nch = g.shape[1]
    err0 = np.abs(g - o).max(1)
    margin = ref.margin.reshape(-1)[pix]
    clear = margin >= MARGIN
    amb = np.nonzero(~clear)[0]
    outs, n = oracle.pixel_outcomes(proj, gid, ranges, cam, opts, pix[amb], tol=MARGIN, nthreads=8)
    e = np.abs(outs[:, :, :nch] - g[amb, None, :]).max(2)
    capped = np.zeros(pix.size, bool)
    capped[amb] = n < 0
    listed = np.where(n < 0, outs.shape[1], n)   # a capped pixel: the outcomes enumerated before the cap
    e[np.arange(outs.shape[1])[None, :] >= listed[:, None]] = np.inf
    matched = np.zeros(pix.size, bool)
    matched[clear] = err0[clear] <= max_abs
    matched[amb] = e.min(1) <= max_abs
    flip_only = np.zeros(pix.size, bool)
    flip_only[amb] = matched[amb] & (e[:, 0] > max_abs)
    bad_clear = clear & ~matched
    unchecked = ~clear & ~matched
    failing_near = unchecked & (margin >= UNCHECKED_MARGIN) & ~capped
    share = float(unchecked.mean()) if pix.size else 0.0
    mean = float(np.abs(g[:, :3] - o[:, :3]).mean()) if pix.size else 0.0
    ok = not bad_clear.any() and not failing_near.any() and share <= UNCHECKED_SHARE and mean <= mean_abs
    rep = dict(ok=bool(ok), pixels=int(pix.size), clear=int(clear.sum()), near=int(amb.size),
               flip_only=int(flip_only.sum()), unchecked=int(unchecked.sum()), unchecked_share=share,
               capped=int(capped.sum()), max_abs_clear=float(err0[clear].max()) if clear.any() else 0.0,
               mean_abs=mean, failing_clear=int(bad_clear.sum()), failing_near=int(failing_near.sum()))
    if not ok:
        bad = np.nonzero(bad_clear | failing_near)[0][:5]
        rep["examples"] = [dict(pixel=int(pix[i]), err=float(err0[i]), margin=float(margin[i])) for i in bad]
    return rep


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
    Returns (Render, global Gaussian ids of each sampled tile's list, and the
    (projections, list ids, ranges) the oracle rendered from, for
    ``check_render``)."""
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
    return ref, lists, (sub, gid, ranges)
