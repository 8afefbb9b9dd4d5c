"""Benchmark of the Seele hot path on GB300: 1080p frames/s at 3M Gaussians.

A step is one frame of the whole path -- preprocessing, compaction, depth
sort, instance emission, tile sort, ranges and rasterization -- for one
1920x1080 camera of the 3M-Gaussian unbounded-style synthetic scene (2.4M
Gaussians in 64 dense clusters plus 0.6M on a radius 30-50 shell, SH degree 3,
16x16 tiles).  Steps cycle over 8 orbit cameras.  The headline path is the
contribution-aware rasterizer (Alg. 1, 2x2 groups) with the opacity-aware
online filter (Eqn. 5); the plain path (Sec. 3.1) is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (launched by torchrun) each rank renders its own cameras (views
are independent: no collective on the data path); value = frames of all
ranks / max-over-ranks time.  ``--impl reference`` times the FP64 CPU oracle
as it stands on this host's cores, on the same workload and metric.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "1080p frames/s at 3M Gaussians vs plain path; fwd+bwd ms; % of roofline"
UNIT = "frames/s"
WORKLOAD = ("unbounded_3m: 3M Gaussians (2.4M in 64 clusters sigma 0.15 in [-3,3]^3 + 0.6M on a r 30-50 shell), "
            "SH degree 3, 1920x1080, 16x16 tiles, 8 orbit cameras at r 5, seed 0")
def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "50", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for r in csv.reader(io.StringIO(open(self.path).read())):
                if len(r) >= 9:
                    rows.append([x.strip() for x in r])
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 0, 1, None
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return rank, local, ws, dist


def _barrier(dist):
    if dist is not None:
        dist.barrier()


def _reduce_device(dist):
    return "cpu" if dist.get_backend() == "gloo" else "cuda"


def _max_over_ranks(dist, v: float) -> float:
    """The slowest rank's time (whole-job throughput divides by it)."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(dist, v: float) -> float:
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=_reduce_device(dist))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def view_of(step: int, rank: int, world: int, n_views: int) -> int:
    """Camera rendered by `rank` at `step`: views are dealt round-robin, so the
    ranks of one step render distinct views and no data crosses ranks."""
    return (rank + step * world) % n_views


# ----------------------------------------------------------------- oracle --

def _oracle_band(s64, cam, opts, y0, h, nthreads):
    """Oracle frame restricted to rows [y0, y0 + h): the same camera with the
    principal point shifted, so it renders exactly those rows of the frame."""
    import oracle
    band = dict(cam)
    band["cy"] = float(cam["cy"]) - y0
    band["height"] = h
    t = time.perf_counter()
    oracle.render(s64, band, opts, nthreads)
    return time.perf_counter() - t


def cpu_baseline(scene, cams, bands=4, nthreads=None):
    """The FP64 oracle, as it stands, on all host cores: one full frame of
    camera 0 rendered as ``bands`` horizontal bands (same arithmetic as one
    frame; each band re-runs preprocessing, so this slightly favours the GPU)."""
    import oracle
    nthreads = nthreads or os.cpu_count()
    s64 = oracle.Scene64.from_scene(scene)
    opts = oracle.Options(cr=True, opacity_filter=True)
    H = int(cams[0]["height"])
    hb = H // bands
    total = 0.0
    for b in range(bands):
        y0 = b * hb
        total += _oracle_band(s64, cams[0], opts, y0, H - y0 if b == bands - 1 else hb, nthreads)
    return {"value": 1.0 / total, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"one full 1920x1080 frame (camera 0, contribution-aware + opacity filter) rendered as "
                      f"{bands} horizontal bands by the FP64 C oracle with OpenMP; {total:.1f} s"}


def cpu_baseline_views(n_gauss: int, poses: int = 2):
    """The FP64 oracle building the view representation's masks for a bounded
    sample of the poses the GPU builder processes (same scene, same 320x180
    poses), in seconds per pose on all host cores."""
    import oracle
    import scenegen
    scene, _ = scenegen.clusters_500k(n=n_gauss)
    s64 = oracle.Scene64.from_scene(scene)
    sample = scenegen.sample_poses(512, 4.0, 320, 180, scenegen.rng(7))[:poses]
    t0 = time.perf_counter()
    oracle.view_masks(s64, sample, np.zeros(poses, np.int32), 32, nthreads=os.cpu_count())
    return {"s_per_pose": (time.perf_counter() - t0) / poses, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{poses} of the 512 poses (320x180, top-32 contributors), {n_gauss} Gaussians"}


def _workload(n_gauss: int) -> str:
    if n_gauss == 3_000_000:
        return WORKLOAD
    return (f"unbounded, {n_gauss} Gaussians (80% in 64 clusters, 20% on a r 30-50 shell), SH degree 3, "
            f"1920x1080, 16x16 tiles, 8 orbit cameras at r 5, seed 0")


def run_reference(args):
    rank, _, ws, dist = _dist()
    if rank != 0:
        return
    import scenegen
    import oracle
    scene, cams = scenegen.unbounded_3m(n=args.n_gauss)
    s64 = oracle.Scene64.from_scene(scene)
    opts = oracle.Options(cr=True, opacity_filter=True)
    nthreads = os.cpu_count()
    bands = 4
    H = int(cams[0]["height"])
    hb = H // bands

    def step(i):
        cam = cams[(i // bands) % len(cams)]
        b = i % bands
        return _oracle_band(s64, cam, opts, b * hb, hb, nthreads)

    for i in range(args.warmup):
        step(i)
    total = sum(step(args.warmup + i) for i in range(args.steps))
    frames = args.steps / bands
    value = frames / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": _workload(args.n_gauss), "path": "CR 2x2 + opacity-aware filter",
                                            "step": "one horizontal quarter band of a frame"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": f"each step renders one 1920x270 band of a frame; {args.steps} bands"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------------- GPU --

def _timed_frames(r, cams, opts, steps, stream, rank, world, out):
    import torch
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(steps):
        r.set_cameras([cams[view_of(i, rank, world, len(cams))]])
        r.render(out=out, options=opts)
    end.record(stream)
    return start, end


def _source_hash(*names):
    h = hashlib.sha256()
    for n in names:
        h.update(open(os.path.join(ROOT, "paper_2503_05168_gb300", "csrc", n), "rb").read())
    return h.hexdigest()[:16]


def _traffic(kernel: str, src_hash: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of that kernel."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        e = t.get(kernel)
        if e and e.get("source_hash") == src_hash:
            return e["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


def _fwd_bwd(args, device):
    """ms of one forward + backward for an L1 loss, per raster mode."""
    import torch

    import scenegen
    from paper_2503_05168_gb300 import Renderer

    scene, cams, target = scenegen.clusters_1m(n=args.fwd_bwd_n)
    r = Renderer(device)
    r.load_scene(target)
    r.set_cameras(cams)
    tgt = r.render(mode="plain").clone()
    params = {k: torch.from_numpy(np.ascontiguousarray(scene[k])).cuda(device)
              for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    out = {}
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)

    def timed(step, k):
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        s.record()
        for _ in range(k):
            step()
        e.record()
        torch.cuda.synchronize()
        return s.elapsed_time(e) / k

    for mode in ("cr", "plain"):
        def make_step(tile):
            # training bins by tiles: the backward walks per-tile lists
            opts = r.make_options(mode=mode, opacity_filter=(mode == "cr"), binning="tiles", tile=tile)

            def step():
                r.load_scene(dict(params, sh_degree=3), borrow=True)
                img = r.render(options=opts)
                g = torch.sign(img - tgt) / img.numel()      # d(mean |img - target|)
                return r.render_backward(g)
            return opts, step

        # the tile shape is tuned for the whole step (a few timed steps each)
        tune = {tile: timed(make_step(tile)[1], 5) for tile in ((16, 16), (8, 8), (32, 8))}
        tile = min(tune, key=tune.get)
        opts, step = make_step(tile)
        k = max(3, min(args.steps, 20))
        out[f"{mode}_ms"] = timed(step, k)
        out[f"{mode}_tile"] = list(tile)
        out[f"{mode}_tuning_ms"] = {f"{a}x{b}": round(v, 4) for (a, b), v in tune.items()}
        # the backward alone on the last frame, and the frame's counted work
        img = r.render(options=opts)
        g = torch.sign(img - tgt) / img.numel()
        r.render_backward(g)
        torch.cuda.synchronize()
        s.record()
        for _ in range(k):
            r.render_backward(g)
        e.record()
        torch.cuda.synchronize()
        out[f"{mode}_bwd_ms"] = s.elapsed_time(e) / k
        r.render(mode=mode, opacity_filter=(mode == "cr"), binning="tiles", tile=tile, count=True)
        out[f"{mode}_work"] = {kk: r.last_stats[kk] for kk in ("n_visible", "n_instances", "leader_tests",
                                                                "pairs_evaluated", "pairs_blended")}
    out["workload"] = (f"clusters_1m: {args.fwd_bwd_n} Gaussians in 64 clusters, 1280x720, L1 loss vs a target "
                       f"rendered from attributes + N(0, 0.01); gradients for all attributes; CR path with the "
                       f"opacity filter, plain path without; tile binning, tile shape tuned per mode over "
                       f"16x16, 8x8 and 32x8 by timing the step")
    r.close()
    return out


def _ablation(args, device):
    """The paper's ablation (Tbl. 4) and pixel-group sweep (Fig. 7) on the
    clustered 500k scene with 16 view clusters, 8 orbit cameras at 1280x720:
    frames/s and PSNR against the plain render of each variant."""
    import torch

    import scenegen
    from paper_2503_05168_gb300 import Renderer

    scene, cams = scenegen.clusters_500k(n=args.ablation_n)
    for key in ("cluster_mask", "centroids", "pos_scale"):
        scene.pop(key)
    r = Renderer(device)
    r.load_scene(scene)
    # the offline view-dependent representation, built on the GPU (Sec. 3.3):
    # 512 poses on the r = 4 sphere (elevation within 30 deg) at 320x180,
    # 16 clusters, top-32 contributors per pixel
    poses = scenegen.sample_poses(512, 4.0, 320, 180, scenegen.rng(7))
    u = scenegen.kmeans_uniforms(16, scenegen.rng(8))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = r.build_view_clusters(poses, n_clusters=16, top_k=32, uniforms=u)
    build_s = time.perf_counter() - t0
    n = scene["means"].shape[0]
    full_bits = np.uint32((1 << 16) - 1)
    representation = {
        "build_s": build_s, "poses": 512, "pose_size": [320, 180], "clusters": 16, "top_k": 32,
        "kept_fraction": float(np.count_nonzero(rep["mask"]) / n),
        "shared_fraction": float(np.count_nonzero((rep["mask"] & full_bits) == full_bits) / n),
        "what": "seele_build_view_clusters: pose k-means + per-pixel top-k contributor pass over all poses"}
    scene.update(cluster_mask=rep["mask"], centroids=rep["centroids"], pos_scale=rep["pos_scale"])
    r.load_scene(scene)
    variants = {
        "plain": dict(mode="plain"),
        "hp_online": dict(mode="plain", opacity_filter=True),
        "hp_online_cluster": dict(mode="plain", opacity_filter=True, cluster_filter=True),
        "cr": dict(mode="cr"),
        "full": dict(mode="cr", opacity_filter=True, cluster_filter=True),
        "cr_group_1x1": dict(mode="cr", group=(1, 1)),
        "cr_group_2x4": dict(mode="cr", group=(2, 4)),
        "cr_group_4x4": dict(mode="cr", group=(4, 4)),
        "cr_group_4x8": dict(mode="cr", group=(4, 8)),
    }
    refs = []
    for c in cams:
        r.set_cameras([c])
        refs.append(r.render(mode="plain").clone())
    out = {}
    for name, kw in variants.items():
        imgs = []
        for c in cams:
            r.set_cameras([c])
            imgs.append(r.render(**kw).clone())
        mse = float(np.mean([torch.mean((a - b) ** 2).item() for a, b in zip(imgs, refs)]))
        opts = r.make_options(sync=False, **kw)
        k = max(2, min(args.steps, 10))
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        for i in range(k * len(cams)):
            r.set_cameras([cams[i % len(cams)]])
            r.render(options=opts)
        e.record()
        r.synchronize()
        ms = s.elapsed_time(e) / (k * len(cams))
        out[name] = {"fps": 1000.0 / ms, "psnr_vs_plain_db": (10 * math.log10(1.0 / mse) if mse > 0 else None)}
    base = out["plain"]["fps"]
    for v in out.values():
        v["speedup"] = v["fps"] / base
    out["workload"] = (f"clusters_500k: {args.ablation_n} Gaussians in 64 clusters, 16 view clusters built on the "
                       f"GPU from 512 sampled poses (nearest + 3 neighbours at render time), 8 orbit cameras at r 4, "
                       f"1280x720, mean over the cameras")
    out["representation"] = representation
    out["streaming"] = _streaming(scene, r, device)
    r.close()
    return out


def _streaming(scene, r_full, device):
    """Scene prefetching (Sec. 3.3): the same representation streamed -- the
    shared Gaussians and 6 cluster slots resident, each camera's pose
    extrapolated one frame ahead -- against the whole scene resident, along a
    smooth 120-frame orbit (frames/s of synchronous renders, full path)."""
    import torch

    import scenegen
    from paper_2503_05168_gb300 import Renderer
    path = scenegen.orbit(120, 4.0, 1280, 720, elevation_deg=10.0, phase=0.2)
    kw = dict(mode="cr", opacity_filter=True, cluster_filter=True)
    # slots of a quarter of the largest cluster, as many as the six largest
    # clusters fill (four selected at a time, two being prefetched)
    C = int(scene["centroids"].shape[0])
    m = np.asarray(scene["cluster_mask"], np.uint32) & np.uint32((1 << C) - 1)
    own = m[(m != 0) & (m != np.uint32((1 << C) - 1))]
    sizes = np.array([int(np.count_nonzero(own & np.uint32(1 << k))) for k in range(C)])
    chunk = max(1, int(math.ceil(sizes.max() / 4)))
    slots = int(min(64, np.sort(-(-sizes // chunk))[::-1][:6].sum()))
    rs = Renderer(device)
    rs.load_scene(scene, streamed_slots=slots, slot_gaussians=chunk, ahead=1)
    out_img = torch.empty(3 * 1280 * 720, device=r_full.device)

    def run(r):
        opts = r.make_options(**kw)
        for cam in path[:3]:  # warm-up (not timed)
            r.set_cameras([cam])
            r.render(out=out_img, options=opts)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for cam in path:
            r.set_cameras([cam])
            r.render(out=out_img, options=opts)
        torch.cuda.synchronize()
        return len(path) / (time.perf_counter() - t0)

    fps_full = run(r_full)
    fps_stream = run(rs)
    st = rs.stream_stats()
    rs.close()
    return {"fps_resident": fps_full, "fps_streamed": fps_stream, "overhead": 1.0 - fps_stream / fps_full,
            "resident_fraction": st["resident_bytes"] / st["full_bytes"], "stats": st,
            "clusters_per_kept_gaussian": float(sizes.sum() / max(1, own.size)),
            "kept_fraction": float(own.size / m.size), "shared_fraction": float(np.count_nonzero(
                m == np.uint32((1 << C) - 1)) / m.size),
            "what": "seele_load_scene_streamed (slots of a quarter of the largest cluster, as many as the six "
                    "largest clusters fill, 1 frame ahead) vs seele_load_scene, 120-frame orbit at r 4, 1280x720, "
                    "CR + opacity and cluster filters, synchronous renders; the paper reports 39.1% less model "
                    "memory at < 6% overhead"}


def _sensitivity(args, device):
    """Sensitivity sweeps of Sec. 4.4 on the clustered scene: number of view
    clusters x cluster neighbours M, and the number of primary contributors k
    of the offline representation (each point rebuilt on the GPU); frames/s
    of the full path (CR + both filters) and PSNR against the plain render of
    all Gaussians, mean over the 8 orbit cameras."""
    import torch

    import scenegen
    from paper_2503_05168_gb300 import Renderer

    scene, cams = scenegen.clusters_500k(n=args.ablation_n)
    for key in ("cluster_mask", "centroids", "pos_scale"):
        scene.pop(key)
    r = Renderer(device)
    r.load_scene(scene)
    refs = []
    for c in cams:
        r.set_cameras([c])
        refs.append(r.render(mode="plain").clone())
    poses = scenegen.sample_poses(512, 4.0, 320, 180, scenegen.rng(7))

    def point(n_clusters, k, M):
        rep = r.build_view_clusters(poses, n_clusters=n_clusters, top_k=k,
                                    uniforms=scenegen.kmeans_uniforms(n_clusters, scenegen.rng(8)))
        r.load_scene(dict(scene, cluster_mask=rep["mask"], centroids=rep["centroids"], pos_scale=rep["pos_scale"]))
        kw = dict(mode="cr", opacity_filter=True, cluster_filter=True, n_neighbors=M)
        imgs = []
        for c in cams:
            r.set_cameras([c])
            imgs.append(r.render(**kw).clone())
        mse = float(np.mean([torch.mean((a - b) ** 2).item() for a, b in zip(imgs, refs)]))
        opts = r.make_options(sync=False, **kw)
        reps = 4
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for i in range(reps * len(cams)):
            r.set_cameras([cams[i % len(cams)]])
            r.render(options=opts)
        e.record()
        r.synchronize()
        return {"fps": 1000.0 * reps * len(cams) / s.elapsed_time(e),
                "psnr_vs_plain_db": 10 * math.log10(1.0 / mse) if mse > 0 else None,
                "kept_fraction": float(np.count_nonzero(rep["mask"]) / scene["means"].shape[0])}

    out = {"clusters_x_neighbours": {}, "top_k": {}}
    for n_clusters in (8, 16, 24):
        for M in (1, 3):
            out["clusters_x_neighbours"][f"{n_clusters}x{M}"] = point(n_clusters, 32, M)
    for k in (8, 16, 32, 64):
        out["top_k"][str(k)] = point(16, k, 3)
    out["workload"] = (f"clusters_500k: {args.ablation_n} Gaussians, 512 sampled poses at 320x180 per build, "
                       f"8 orbit cameras at 1280x720; full path (CR + opacity and cluster filters)")
    r.close()
    return out


def _multiview(args, device, pipe_peaks):
    """64 cameras of mixed resolution rendered in one CUDA-graph launch per
    batch.  The batched autotuner (seele_autotune_ex) picks the tile shape,
    then the rasterizer schedule and batch depth, once for throughput and once
    for the median per-view latency; both choices are timed."""
    import torch

    import scenegen
    from paper_2503_05168_gb300 import Renderer

    scene, cams = scenegen.multiview_2m(n=args.multiview_n)
    r = Renderer(device)
    r.load_scene(scene, spatial=True)
    r.set_cameras(cams)
    n_views = len(cams)
    out = torch.empty(3 * r.n_pixels, device=r.device)
    t0 = time.perf_counter()
    o_thr, tune_thr = r.autotune_ex(objective="batch", cache=args.tune_cache, mode="cr", opacity_filter=True)
    o_lat, tune_lat = r.autotune_ex(objective="p50", cache=args.tune_cache, mode="cr", opacity_filter=True)
    tune_s = time.perf_counter() - t0

    def timed(o):
        kw = dict(mode="cr", opacity_filter=True, tile=(o.tile_w, o.tile_h),
                  schedule="queue" if o.schedule else "grid", batch_depth=o.batch_depth)
        r.render(**kw)                                # sizes the instance buffers
        gopts = r.make_options(graph=True, sync=False, **kw)
        for _ in range(3):
            r.render(out=out, options=gopts)
        r.synchronize()
        k = max(3, min(args.steps, 10))
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(k):
            r.render(out=out, options=gopts)
        e.record()
        r.synchronize()
        ms = s.elapsed_time(e) / k
        per_view = []
        for _ in range(3):
            r.render(out=out, options=r.make_options(graph=True, **kw))
            per_view += r.view_times()
        return kw, {"views_per_s": n_views * 1000.0 / ms, "ms_per_batch": ms,
                    "view_ms_p50": float(np.percentile(per_view, 50)),
                    "view_ms_p99": float(np.percentile(per_view, 99)),
                    "tile": [o.tile_w, o.tile_h], "schedule": "queue" if o.schedule else "grid",
                    "batch_depth": int(o.batch_depth)}

    kw_thr, thr = timed(o_thr)
    _, lat = timed(o_lat)
    # roofline of the batch's rasterizer: counted FP32 work over its event time
    stage = {}
    for _ in range(3):
        r.render(profile=True, **kw_thr)
        for kk, v in r.last_stats["stage_ms"].items():
            stage[kk] = stage.get(kk, 0.0) + v / 3
    r.render(count=True, **kw_thr)
    work = {kk: r.last_stats[kk] for kk in ("leader_tests", "pairs_evaluated", "pairs_blended")}
    ops = 8 * (work["pairs_evaluated"] + work["leader_tests"]) + 7 * work["pairs_blended"]
    achieved = ops / (stage["raster"] / 1000.0) / 1e12
    res = dict(thr)
    res.update({
        "latency_tuned": lat, "autotune": {"throughput": tune_thr, "latency": tune_lat, "seconds": tune_s},
        "views": n_views, "instances": r.last_stats["n_instances"] if r.last_stats else None,
        "stage_ms": {kk: round(v, 4) for kk, v in stage.items()},
        "roofline": {"bound": "alu", "kernel": "raster_fwd (CR 2x2, all views of the batch)", "unit": "TFLOP/s",
                     "achieved": achieved, "peak": pipe_peaks["fp32_tops"],
                     "frac": achieved / pipe_peaks["fp32_tops"], "raster_ms": stage["raster"],
                     "ops": ops, "work": work},
        "workload": (f"multiview_2m: {args.multiview_n} Gaussians (unbounded-style), {n_views} cameras with "
                     f"resolutions from {{640x360, 1280x720, 1920x1080}} at radius 3-6, one CUDA-graph launch "
                     f"per batch, CR + opacity filter, scene in spatial order; per-view ms = start of "
                     f"preprocessing to the view's last tile; configuration from seele_autotune_ex")})
    r.close()
    return res


def run_gpu(args):
    import torch

    import __graft_entry__
    import scenegen
    from paper_2503_05168_gb300 import Renderer

    rank, local, ws, dist = _dist()
    if rank == 0:
        __graft_entry__.build()
    _barrier(dist)
    torch.cuda.set_device(local)
    if args.fwd_bwd_only:
        if rank == 0:
            print(json.dumps({"fwd_bwd": _fwd_bwd(args, local)}), flush=True)
        return
    import paper_2503_05168_gb300 as seele
    # issue rates of the FMA, MUFU and ALU pipes on this device (the
    # denominators of the blending's roofline), and its SM count
    pipe_peaks = seele.measure_peaks(local)
    scene, cams = scenegen.unbounded_3m(n=args.n_gauss)
    r = Renderer(local)
    # stored in Morton order of the means (SEELE_SCENE_SPATIAL, computed at load)
    r.load_scene(scene, spatial=True)
    stream = torch.cuda.current_stream()
    # the timed frames are CUDA-graph replays of the whole frame (captured on
    # first use, replayed with each step's camera pose); asynchronous
    # launches without the graph are timed too
    cr_opts = r.make_options(mode="cr", opacity_filter=True, sync=False, graph=True)
    plain_opts = r.make_options(mode="plain", sync=False, graph=True)
    cr_async = r.make_options(mode="cr", opacity_filter=True, sync=False)
    out = torch.empty(3 * cams[0]["width"] * cams[0]["height"], device=r.device)

    # warm-up: synchronous renders grow the instance capacity, then the
    # timed kind of launch (the graph is captured here)
    for opts in (cr_opts, plain_opts, cr_async):
        for i in range(max(args.warmup, 3)):
            r.set_cameras([cams[view_of(i, rank, ws, len(cams))]])
            r.render(mode="cr" if opts.mode else "plain", opacity_filter=bool(opts.opacity_filter))
            r.render(out=out, options=opts)
        r.synchronize()
        # a new capture each time the options change: re-warm the graph last
        # used before timing it
    def timed(opts):
        for i in range(3):
            r.set_cameras([cams[view_of(i, rank, ws, len(cams))]])
            r.render(out=out, options=opts)
        r.synchronize()
        _barrier(dist)
        torch.cuda.synchronize()
        s, e = _timed_frames(r, cams, opts, args.steps, stream, rank, ws, out)
        torch.cuda.synchronize()
        r.synchronize()
        _barrier(dist)
        return s.elapsed_time(e) / 1000.0

    clocks = ClockSampler(local)
    clocks.start()
    t_cr = timed(cr_opts)
    clock_info = clocks.stop()
    t_plain = timed(plain_opts)
    t_async = timed(cr_async)
    # per-stage device times (CUDA events inside the library, same stream),
    # taken before the batched call below grows the instance capacity, so
    # that the sorts run on the grids of the timed single-view frames
    stage = {}
    n_prof = max(3, min(args.steps, 10))
    for i in range(n_prof):
        r.set_cameras([cams[view_of(i, rank, ws, len(cams))]])
        r.render(mode="cr", opacity_filter=True, profile=True)
        for k, v in r.last_stats["stage_ms"].items():
            stage[k] = stage.get(k, 0.0) + v / n_prof
    kernels_per_frame = r.last_stats["n_kernels"]
    n_vis, K = r.last_stats["n_visible"], r.last_stats["n_instances"]
    stage_plain = {}
    for i in range(n_prof):
        r.set_cameras([cams[view_of(i, rank, ws, len(cams))]])
        r.render(mode="plain", profile=True)
        for k, v in r.last_stats["stage_ms"].items():
            stage_plain[k] = stage_plain.get(k, 0.0) + v / n_prof
    # the 8 orbit views of the workload as one batched call per step (one
    # frame pass over all cameras; frames/s counts every view)
    batch_cams = [cams[(rank * 8 + j) % len(cams)] for j in range(8)]
    r.set_cameras(batch_cams)
    bopts = r.make_options(mode="cr", opacity_filter=True, sync=False, graph=True)
    bout = torch.empty(8 * 3 * cams[0]["width"] * cams[0]["height"], device=r.device)
    for _ in range(3):
        r.render(mode="cr", opacity_filter=True)
        r.render(out=bout, options=bopts)
    r.synchronize()
    _barrier(dist)
    torch.cuda.synchronize()
    bsteps = max(3, args.steps // 8)
    bs, be = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    bs.record(stream)
    for _ in range(bsteps):
        r.set_cameras(batch_cams)
        r.render(out=bout, options=bopts)
    be.record(stream)
    torch.cuda.synchronize()
    r.synchronize()
    fps_batch8 = 8 * bsteps * ws / _max_over_ranks(dist, bs.elapsed_time(be) / 1000.0)
    # two frames in flight: a second context shares the resident scene
    # (seele_share_scene) on its own stream and takes every other step, so
    # one frame's rasterization overlaps the next one's preprocessing and
    # sorting; same frames, same graph replays
    s2 = torch.cuda.Stream(local)
    r2 = Renderer(local, stream=s2)
    r2.share_scene(r)
    p_opts = r2.make_options(mode="cr", opacity_filter=True, sync=False, graph=True)
    out2 = torch.empty_like(out)
    for i in range(3):
        r2.set_cameras([cams[view_of(i, rank, ws, len(cams))]])
        r2.render(mode="cr", opacity_filter=True)
        r2.render(out=out2, options=p_opts)
    r.set_cameras([cams[view_of(0, rank, ws, len(cams))]])
    r.render(out=out, options=cr_opts)
    r.synchronize()
    r2.synchronize()
    _barrier(dist)
    torch.cuda.synchronize()
    ps, pe, p2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    ps.record(stream)
    s2.wait_event(ps)
    for i in range(args.steps):
        rr, o, oo = (r, cr_opts, out) if i % 2 == 0 else (r2, p_opts, out2)
        rr.set_cameras([cams[view_of(i, rank, ws, len(cams))]])
        rr.render(out=oo, options=o)
    p2.record(s2)
    stream.wait_event(p2)
    pe.record(stream)
    torch.cuda.synchronize()
    r.synchronize()
    r2.synchronize()
    fps_two_streams = args.steps * ws / _max_over_ranks(dist, ps.elapsed_time(pe) / 1000.0)
    r2.close()
    t_cr_max = _max_over_ranks(dist, t_cr)
    t_plain_max = _max_over_ranks(dist, t_plain)
    frames = args.steps * ws
    fps = frames / t_cr_max
    fps_plain = frames / t_plain_max
    fps_async = frames / _max_over_ranks(dist, t_async)

    # algorithmic work of the rasterizer (counting variant, untimed)
    r.set_cameras([cams[rank % len(cams)]])
    r.render(mode="cr", opacity_filter=True, count=True)
    work = {k: r.last_stats[k] for k in ("leader_tests", "pairs_evaluated", "pairs_blended")}
    work_K = r.last_stats["n_instances"]
    work_vis = r.last_stats["n_visible"]
    # (tile, Gaussian) instances of the same frame binned by tiles (untimed)
    r.render(mode="cr", opacity_filter=True, binning="tiles")
    K_tiles = r.last_stats["n_instances"]

    raster_event_ms = stage["raster"]
    raster_traffic = _traffic("raster_fwd", _source_hash("raster.cu", "raster_impl.cuh", "raster_queue.cu"))

    # quality: CR vs plain on the same frame
    img_cr = r.render(mode="cr", opacity_filter=True).cpu().numpy().astype(np.float64)
    img_pl = r.render(mode="plain").cpu().numpy().astype(np.float64)
    mse = float(np.mean((img_cr - img_pl) ** 2))
    psnr = 10 * math.log10(1.0 / mse) if mse > 0 else float("inf")

    # roofline of the dominant stage
    peaks = _peaks()
    dom = max(stage, key=stage.get)
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    n_gauss = int(scene["means"].shape[0])
    # algorithmic bytes per stage (block binning, one 1920x1080 camera:
    # 15 x 17 = 255 tile blocks, so the block sort is one 8-bit pass)
    n_blocks = 15 * 17
    block_passes = max(1, math.ceil(max(1, (n_blocks - 1).bit_length()) / 8))
    stage_bytes = {
        # position/logit in and tile + block counts out for every Gaussian; quat, scale,
        # 48 SH floats in and the 64 B record + 4 B depth out per visible one
        "preprocess": 16 * n_gauss + 8 * n_gauss + (32 + 192 + 68) * work_vis,
        "compact": 4 * n_gauss + 12 * work_vis,
        "depth_sort": 4 * 20 * work_vis,
        "tile_scan": 12 * work_vis,
        # order + offset + the record's ellipse and tile box in, 10 B per entry out
        "emit": 48 * work_vis + 10 * work_K,
        "tile_sort": block_passes * 22 * work_K,
        "ranges": 4 * work_K,
    }
    stage_roof = {k: {"GB_s": round(v / (stage[k] / 1000.0) / 1e9, 1),
                      "frac": round(v / (stage[k] / 1000.0) / 1e9 / hbm, 3)}
                  for k, v in stage_bytes.items() if stage.get(k, 0) > 0}
    pipes = pipe_peaks
    raster_s = raster_event_ms / 1000.0
    # counted work of the blending: 8 FP32 ops per exponent evaluation
    # (leader tests and pixel pairs) + 7 per blended pair; one ex2 per pixel
    # pair; one threshold compare per exponent and one stop compare per pair
    fp32_ops = 8 * (work["pairs_evaluated"] + work["leader_tests"]) + 7 * work["pairs_blended"]
    sfu_ops = work["pairs_evaluated"]
    alu_ops = work["pairs_evaluated"] + work["leader_tests"] + work["pairs_evaluated"]
    raster_bytes = raster_traffic if raster_traffic else 0
    floors = {"fp32": fp32_ops / (pipes["fp32_tops"] * 1e12), "sfu": sfu_ops / (pipes["sfu_tops"] * 1e12),
              "alu": alu_ops / (max(pipes["alu_fmnmx_tops"], pipes["alu_lop3_tops"]) * 1e12),
              "hbm": raster_bytes / (hbm * 1e9)}
    binding = max(floors, key=floors.get)
    sustained = float(peaks.get("clocks_under_load", {}).get("sm_mhz_median", 0.0) or 0.0)
    clk_max = float(pipes.get("sm_clock_max_mhz") or peaks.get("sm_max_mhz", 2070.0))
    achieved = fp32_ops / raster_s / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": pipes["fp32_tops"], "unit": "TFLOP/s",
            "frac": achieved / pipes["fp32_tops"],
            "traffic": raster_traffic, "kernel": "raster_fwd_kernel (CR 2x2)",
            "binding_pipe": binding,
            "frac_of_floor": {k: round(v / raster_s, 4) for k, v in floors.items()},
            "frac_sustained_clock": (achieved / (pipes["fp32_tops"] * sustained / clk_max)
                                     if sustained > 0 else None),
            "launch_ms": raster_event_ms,
            "note": f"achieved = counted FP32 ops of the blending ({fp32_ops / 1e9:.3f} G: 8 per exponent "
                    f"evaluation, leader tests and pixel pairs, + 7 per blended pair) / the kernel's mean CUDA-event "
                    f"time; peak = the FMA rate measured by seele_measure_peaks on this device "
                    f"({pipes['sm_count']} SMs; of measured); frac_of_floor: each pipe's counted work over its "
                    f"measured rate (sfu: {sfu_ops / 1e9:.3f} G ex2; alu: {alu_ops / 1e9:.3f} G compares), and the "
                    f"kernel's DRAM bytes over {hbm:.0f} GB/s; frac_sustained_clock: the FMA peak scaled to the "
                    f"{sustained:.0f} MHz median SM clock under sustained load"}
    if dom != "raster":
        roof["note"] += f"; the stage with most time is {dom}"

    # end to end through the public API with host buffers: scene upload from
    # pinned host memory (read in place by the load's repack kernel), render,
    # image read back into pinned host memory.  Timed two ways: one context,
    # each call synchronous; and two contexts on their own streams taking
    # alternate steps with asynchronous renders, so that one step's upload
    # overlaps the previous step's frame and read-back.
    pinned = {k: (torch.from_numpy(np.ascontiguousarray(v)).pin_memory() if isinstance(v, np.ndarray) else v)
              for k, v in scene.items()}
    host_imgs = [torch.empty(3 * 1920 * 1080, dtype=torch.float32).pin_memory() for _ in range(2)]
    h2d = sum(v.numel() * v.element_size() for v in pinned.values() if isinstance(v, torch.Tensor))
    d2h = host_imgs[0].numel() * 4
    e2e_steps = max(4, min(args.steps, 8))
    rs = [r, Renderer(local, stream=torch.cuda.Stream(local))]

    def upload_step(i, rr, opts):
        rr.load_scene(pinned)
        rr.set_cameras([cams[view_of(i, rank, ws, len(cams))]])
        if opts is None:
            rr.render(out=host_imgs[0], mode="cr", opacity_filter=True)
        else:
            rr.render(out=host_imgs[i % 2], options=opts)

    a_opts = [x.make_options(mode="cr", opacity_filter=True, sync=False) for x in rs]
    for i in range(2):   # warm-up: capacities grown by synchronous renders
        upload_step(i, rs[i], None)
        upload_step(i, rs[i], a_opts[i])
        rs[i].synchronize()
    _barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        upload_step(i, r, None)
    torch.cuda.synchronize()
    t_seq = _max_over_ranks(dist, time.perf_counter() - t0)
    _barrier(dist)
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        upload_step(i, rs[i % 2], a_opts[i % 2])
    for x in rs:
        x.synchronize()
    t_e2e = _max_over_ranks(dist, time.perf_counter() - t0)
    e2e = {"value": e2e_steps * ws / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "steps": e2e_steps,
           "what": "per step: seele_load_scene (COPY, the pinned host arrays read in place) + seele_set_cameras + "
                   "seele_render(ASYNC, out = pinned host image); two contexts on their own streams take "
                   "alternate steps; the clock stops when every image is on the host",
           "one_context_sync": {"value": e2e_steps * ws / t_seq, "unit": UNIT,
                                "what": "the same steps on one context, each call synchronous"}}
    # the serving loop: the scene stays resident (loaded once, like model
    # weights, in spatial order); per step the camera goes up and the image
    # comes back.  One context synchronous, and two contexts sharing the
    # scene with asynchronous graph replays
    r.load_scene(scene, spatial=True)
    rs[1].share_scene(r)
    g_opts = [x.make_options(mode="cr", opacity_filter=True, sync=False, graph=True) for x in rs]

    def serve_step(i, rr, opts):
        rr.set_cameras([cams[view_of(i, rank, ws, len(cams))]])
        if opts is None:
            rr.render(out=host_imgs[0], mode="cr", opacity_filter=True)
        else:
            rr.render(out=host_imgs[i % 2], options=opts)

    for i in range(4):
        serve_step(i, rs[i % 2], None)
        serve_step(i, rs[i % 2], g_opts[i % 2])
    for x in rs:
        x.synchronize()
    serve_steps = max(8, min(args.steps, 100))
    _barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(serve_steps):
        serve_step(i, r, None)
    torch.cuda.synchronize()
    t_seq = _max_over_ranks(dist, time.perf_counter() - t0)
    _barrier(dist)
    t0 = time.perf_counter()
    for i in range(serve_steps):
        serve_step(i, rs[i % 2], g_opts[i % 2])
    for x in rs:
        x.synchronize()
    t_serve = _max_over_ranks(dist, time.perf_counter() - t0)
    e2e["resident_scene"] = {"value": serve_steps * ws / t_serve, "unit": UNIT, "h2d_bytes_per_step": 80,
                             "d2h_bytes_per_step": int(d2h), "steps": serve_steps,
                             "what": "per step: seele_set_cameras + seele_render(ASYNC | GRAPH, out = pinned host "
                                     "image), scene resident (loaded once with SEELE_SCENE_SPATIAL and shared "
                                     "by two contexts on their own streams taking alternate steps); the clock "
                                     "stops when every image is on the host",
                             "one_context_sync": {"value": serve_steps * ws / t_seq, "unit": UNIT,
                                                  "what": "the same steps on one context, each render "
                                                          "synchronous"}}
    rs[1].close()

    # contribution skew (Sec. 1, Sec. 3.4): per pixel of a plain render of the
    # headline view, how many of its largest contributions make up 99% of it
    skew = None
    if rank == 0:
        r.set_cameras([cams[0]])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sk = r.contribution_skew(0.99)[0]
        t_skew = time.perf_counter() - t0
        b = sk["blended"].astype(np.float64)
        m = sk["m"].astype(np.float64)
        wk = sk["walked"].astype(np.float64)
        ls = sk["listed"].astype(np.float64)
        on = b > 0
        skew = {"frac": 0.99, "pixels": int(on.sum()),
                "m_mean": float(m[on].mean()), "blended_mean": float(b[on].mean()),
                "walked_mean": float(wk[on].mean()),
                "share_of_blended_mean": float((m[on] / b[on]).mean()),
                "share_of_walked_mean": float((m[on] / wk[on]).mean()),
                "share_of_walked_median": float(np.median(m[on] / wk[on])),
                "listed_mean": float(ls[on].mean()),
                "share_of_listed_mean": float((m[on] / ls[on]).mean()),
                "share_of_listed_median": float(np.median(m[on] / ls[on])),
                "ms": 1000.0 * t_skew,
                "what": "seele_contribution_skew on camera 0 of the workload, plain rules (t_g = 9), tile lists; "
                        "share = m / contributions, m / tile-list entries walked, or m / the pixel's tile-list "
                        "length, mean (and median) over covered pixels; "
                        "the paper reports 1.5% on MipNeRF360 captures"}

    # forward + backward for an L1 loss (the fine-tuning step of Sec. 3.5):
    # 1M Gaussians shaped as the clustered scene, 1280x720, target rendered
    # from attributes perturbed by N(0, 0.01)
    fwd_bwd = _fwd_bwd(args, local)
    multiview = _multiview(args, local, pipe_peaks) if args.multiview_n > 0 else None
    ablation = _ablation(args, local) if args.ablation_n > 0 else None
    sensitivity = _sensitivity(args, local) if args.ablation_n > 0 else None

    config = {"workload": _workload(args.n_gauss),
              "path": "contribution-aware (Alg. 1, 2x2 groups) + opacity-aware filter; ellipse tile test; block "
                      "binning (8x4-tile blocks with tile masks)",
              "launch": "one CUDA-graph replay of the whole frame per step (pose updated per step)",
              "l2": "inputs larger than L2 (720 MB of Gaussian attributes per frame)",
              "scene_order": "Morton order of the means, computed by the library at load (SEELE_SCENE_SPATIAL)",
              "parallelism": f"replicas x{ws} (cameras sharded, no collective)"}
    fb = fwd_bwd
    line = {
        "metric": METRIC, "value": fps, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_cr_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config,
        "plain_fps": fps_plain, "speedup_vs_plain": fps / fps_plain, "psnr_cr_vs_plain_db": psnr,
        "fwd_bwd": {"cr_ms": fb["cr_ms"], "plain_ms": fb["plain_ms"], "cr_bwd_ms": fb["cr_bwd_ms"],
                    "plain_bwd_ms": fb["plain_bwd_ms"], "speedup_vs_plain": fb["plain_ms"] / fb["cr_ms"],
                    "workload": f"clusters_1m, {args.fwd_bwd_n} Gaussians, 1280x720, L1 loss, all gradients"},
        "stage_ms": {k: round(v, 4) for k, v in stage.items()},
        "roofline": roof,
        "e2e": {k: e2e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step")},
        "e2e_resident_scene_fps": e2e["resident_scene"]["value"],
        "async_fps": fps_async, "batch8_fps": fps_batch8, "two_stream_fps": fps_two_streams,
        "multiview": ({**{k: multiview[k] for k in ("views_per_s", "view_ms_p50", "view_ms_p99", "tile",
                                                     "schedule", "batch_depth")},
                       "latency_tuned": {k: multiview["latency_tuned"][k] for k in
                                         ("views_per_s", "view_ms_p50", "view_ms_p99", "schedule", "batch_depth")},
                       "raster_frac": round(multiview["roofline"]["frac"], 4)} if multiview else None),
        "peaks": {k: (round(v, 3) if isinstance(v, float) else v) for k, v in pipe_peaks.items()},
        "gpu_launches": int(kernels_per_frame * args.steps),
        "clocks": clock_info,
    }
    details = {
        "stage_ms_plain": {k: round(v, 4) for k, v in stage_plain.items()},
        "n_visible": n_vis, "n_block_instances": K, "n_tile_instances": K_tiles, "raster_work": work,
        "stage_roofline_hbm": stage_roof, "e2e": e2e, "fwd_bwd": fwd_bwd, "multiview": multiview,
        "ablation": ablation, "sensitivity": sensitivity, "contribution_skew": skew,
        "launch_kinds": {"async_fps": "the same frames as plain stream launches",
                         "two_stream_fps": "the same frames alternating between two contexts sharing the scene, "
                                           "each on its own stream (two frames in flight)",
                         "batch8_fps": "the 8 orbit views as one batched call per step"},
    }
    # the CPU oracle as it stands, rank 0 at N = 1 only
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(scene, cams)
        if args.ablation_n > 0:
            details["cpu_baseline_view_representation"] = cpu_baseline_views(args.ablation_n)
    if rank == 0:
        # the long-form results go to stderr (and to --details): the JSON line
        # on stdout stays short enough to be read whole
        blob = json.dumps({"details": details})
        print(blob, file=sys.stderr, flush=True)
        if args.details:
            with open(args.details, "w") as fh:
                fh.write(blob + "\n")
        print(json.dumps(line), flush=True)
    r.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="seele", choices=["seele", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fwd-bwd-n", type=int, default=1_000_000)
    ap.add_argument("--fwd-bwd-only", action="store_true",
                    help="time only the forward + backward step (for profiling captures of the backward kernels)")
    ap.add_argument("--multiview-n", type=int, default=2_000_000, help="0 skips the multi-view measurement")
    ap.add_argument("--ablation-n", type=int, default=500_000, help="0 skips the ablation")
    ap.add_argument("--details", default=None, help="also write the long-form results (JSON) to this file")
    ap.add_argument("--tune-cache", default=None, help="JSON cache file of the batched autotuner")
    ap.add_argument("--n-gauss", type=int, default=3_000_000,
                    help="scene size (3M is the benchmark; smaller sizes are for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
