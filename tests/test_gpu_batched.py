"""Batched multi-view rendering: CUDA-graph capture and replay, tile shapes,
the autotuner and per-view completion times (through the C ABI)."""
import numpy as np
import pytest

import oracle
import scenegen
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Renderer():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_05168_gb300 import Renderer as R
    return R


def _cams(seed, sizes):
    rs = np.random.default_rng(seed)
    out = []
    for w, h in sizes:
        az, el, rad = rs.uniform(0, 2 * np.pi), rs.uniform(-0.4, 0.4), rs.uniform(2.8, 3.6)
        eye = (rad * np.cos(az) * np.cos(el), -rad * np.sin(el), rad * np.sin(az) * np.cos(el))
        out.append(scenegen.look_at(eye, (0, 0, 0), w, h))
    return out


SIZES = [(64, 48), (100, 70), (96, 96), (33, 17), (160, 90)]


def test_graph_replay_equals_plain_launches_and_follows_new_poses(Renderer):
    import torch
    sc, _ = scenegen.uniform_10k()
    r = Renderer()
    r.load_scene(sc)
    out = torch.empty(sum(3 * w * h for w, h in SIZES), device="cuda")
    for seed in (1, 2, 3):
        cams = _cams(seed, SIZES)  # same resolutions, new poses: the graph is replayed
        r.set_cameras(cams)
        ref = r.render(mode="cr", opacity_filter=True).clone()
        r.render(out=out, mode="cr", opacity_filter=True, graph=True)
        torch.cuda.synchronize()
        torch.testing.assert_close(out, ref, rtol=0, atol=0)
    # a new resolution forces a new capture
    cams = _cams(4, SIZES[:-1] + [(128, 72)])
    r.set_cameras(cams)
    ref = r.render(mode="plain").clone()
    out2 = torch.empty_like(ref)
    r.render(out=out2, mode="plain", graph=True)
    torch.cuda.synchronize()
    torch.testing.assert_close(out2, ref, rtol=0, atol=0)
    r.close()


def test_graph_replays_asynchronously(Renderer):
    import torch
    sc, _ = scenegen.uniform_10k(n=5000)
    r = Renderer()
    r.load_scene(sc)
    frames = [_cams(10 + i, SIZES) for i in range(4)]
    refs = []
    for cams in frames:
        r.set_cameras(cams)
        refs.append(r.render(mode="cr").clone())
    outs = [torch.empty_like(refs[0]) for _ in frames]
    # one output buffer per frame means one capture per buffer; replay twice
    for _ in range(2):
        for cams, o in zip(frames, outs):
            r.set_cameras(cams)
            r.render(out=o, mode="cr", graph=True, sync=False)
    r.synchronize()
    for o, ref in zip(outs, refs):
        torch.testing.assert_close(o, ref, rtol=0, atol=0)
    r.close()


@pytest.mark.parametrize("tile", [(32, 8), (32, 16)])
def test_tile_shapes_render_the_same_image(Renderer, tile):
    sc, cams = scenegen.uniform_10k()
    cams = cams + _cams(5, [(100, 70)])
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    for mode in ("plain", "cr"):
        a, _ = parity.gpu_render(r, mode=mode)
        b, _ = parity.gpu_render(r, mode=mode, tile=tile)
        for x, y in zip(a, b):
            d = np.abs(x - y)
            assert d.max() <= parity.RGB_MAX_ABS and (d == 0).mean() > 0.999
    # and against the oracle with that tile shape
    oo = oracle.Options(cr=True, tile_w=tile[0], tile_h=tile[1])
    ref, proj, _, gid, ranges = oracle.render(oracle.Scene64.from_scene(sc), cams[0], oo, nthreads=8)
    imgs, Ts = parity.gpu_render(r, mode="cr", tile=tile)
    rep = parity.check_render(imgs[0], Ts[0], ref, proj, gid, ranges, cams[0], oo)
    assert rep["ok"], str(rep)
    r.close()


def test_view_times_and_autotune(Renderer):
    sc, _ = scenegen.uniform_10k()
    cams = _cams(6, SIZES * 4)
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    opts, ms = r.autotune(mode="cr", opacity_filter=True)
    assert (opts.tile_w, opts.tile_h) in {(16, 16), (32, 8), (32, 16), (8, 8)} and ms > 0
    r.render(options=opts)
    t = r.view_times()
    assert len(t) == len(cams) and all(v > 0 for v in t) and max(t) < 1000
    r.close()


@pytest.mark.parametrize("binning", ["blocks", "tiles"])
def test_wide_batches_take_32_bit_unit_keys(Renderer, binning):
    """520 cameras of 16384x16 make 532,480 tiles and 66,560 tile blocks in one
    frame: unit ids no longer fit 16-bit keys and the unit sort takes 3 passes.
    Sampled cameras of the batch equal their single-camera renders (16-bit
    keys, one or two passes) bit for bit."""
    import torch
    sc, _ = scenegen.uniform_10k(n=4000)
    rs = np.random.default_rng(9)
    cams = []
    for i in range(520):
        eye = (rs.uniform(-0.5, 0.5), rs.uniform(-0.3, 0.3), -3.0)
        c = scenegen.look_at(eye, (0, 0, 0), 16384, 16)
        c["fx"] = c["fy"] = 4000.0
        cams.append(c)
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    flat = r.render(mode="cr", binning=binning)
    torch.cuda.synchronize()
    assert r.last_stats["n_instances"] > 0
    per = 3 * 16384 * 16
    for i in (0, 259, 519):
        batch = flat[i * per:(i + 1) * per].cpu().numpy()
        r.set_cameras([cams[i]])
        single = r.render(mode="cr", binning=binning).cpu().numpy()
        np.testing.assert_array_equal(batch, single)
        assert np.count_nonzero(single) > 0
    r.close()


# ------------------------------------------------- persistent queue schedule --

MIXED = [(640, 360), (320, 180), (160, 90), (640, 360), (96, 96), (320, 180), (200, 120), (160, 90), (48, 32),
         (320, 180)]


def _mixed_scene():
    # the unbounded-style scene of the batched workload, small: dense clusters
    # and a far shell, cameras at radius 3-6 looking at the origin
    sc, _ = scenegen.unbounded_3m(n=60_000)
    rs = np.random.default_rng(17)
    cams = []
    for w, h in MIXED:
        az, el, rad = rs.uniform(0, 2 * np.pi), rs.uniform(-0.5, 0.5), rs.uniform(3.0, 6.0)
        eye = (rad * np.cos(az) * np.cos(el), -rad * np.sin(el), rad * np.sin(az) * np.cos(el))
        cams.append(scenegen.look_at(eye, (0, 0, 0), w, h))
    return sc, cams


@pytest.mark.parametrize("mode", ["cr", "plain"])
def test_mixed_resolution_batch_matches_oracle_per_camera(Renderer, mode):
    """Ten cameras of five resolutions in one frame (grid and persistent queue
    schedules, CUDA-graph replay): every camera against the oracle on sampled
    tiles (the corner tiles, the ragged last row and column, the longest list
    and random ones), decision-aware on every sampled pixel."""
    import torch
    sc, cams = _mixed_scene()
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    kw = dict(mode=mode, opacity_filter=(mode == "cr"))
    r.render(**kw)
    out = torch.empty(3 * r.n_pixels, device="cuda")
    r.render(out=out, schedule="queue", batch_depth=3, graph=True, sync=False, **kw)
    r.render(out=out, schedule="queue", batch_depth=3, graph=True, sync=False, **kw)   # a replay
    r.synchronize()
    imgs = r.images(out)
    grid_imgs = r.images(r.render(**kw))
    s64 = oracle.Scene64.from_scene(sc)
    oo = parity.oracle_options(mode, opacity_filter=(mode == "cr"))
    rs = np.random.default_rng(5)
    for ci, cam in enumerate(cams):
        img = imgs[ci].cpu().numpy()
        np.testing.assert_array_equal(img, grid_imgs[ci].cpu().numpy())
        proj = oracle.preprocess(s64, cam, oo, nthreads=8)
        tx_n, ty_n = oracle.tile_grid(cam, oo)
        tiles = np.unique(np.concatenate([rs.choice(tx_n * ty_n, min(6, tx_n * ty_n), replace=False),
                                          [0, tx_n - 1, (ty_n - 1) * tx_n, tx_n * ty_n - 1]]))
        ref, _, (sub, gid, ranges) = parity.oracle_render_tiles(proj, cam, oo, tiles)
        W, H = cam["width"], cam["height"]
        pix = []
        for t in tiles:
            tx, ty = t % tx_n, t // tx_n
            yy, xx = np.mgrid[16 * ty:min(16 * ty + 16, H), 16 * tx:min(16 * tx + 16, W)]
            pix.append((yy * W + xx).reshape(-1))
        rep = parity.check_render(img, None, ref, sub, gid, ranges, cam, oo, pixels=np.concatenate(pix))
        assert rep["ok"], str((ci, rep))
    r.close()


@pytest.mark.parametrize("binning", ["blocks", "tiles"])
@pytest.mark.parametrize("depth", [0, 1, 4])
def test_queue_schedule_equals_grid_bit_for_bit(Renderer, binning, depth):
    sc, _ = scenegen.uniform_10k()
    cams = _cams(21, SIZES * 3)
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    for mode in ("plain", "cr"):
        a, ta = parity.gpu_render(r, mode=mode, binning=binning)
        b, tb = parity.gpu_render(r, mode=mode, binning=binning, schedule="queue", batch_depth=depth)
        for x, y in zip(a + ta, b + tb):
            np.testing.assert_array_equal(x, y)
    r.close()


def test_queue_groups_finish_in_order(Renderer):
    """batch_depth 1: cameras one at a time, least work first.  Six views that
    see no Gaussian (empty tile lists) and six that see the scene, all
    256x256: every empty view is finished before any loaded one; as one group
    (batch_depth 0) the longest lists go first instead."""
    sc, _ = scenegen.uniform_10k()
    loaded = _cams(31, [(256, 256)] * 6)
    empty = [scenegen.look_at((0.0, 0.0, -3.0 - 0.1 * i), (0.0, 0.0, -9.0), 256, 256) for i in range(6)]
    cams = [c for pair in zip(loaded, empty) for c in pair]   # interleaved: loaded views at even indices
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    r.render(mode="cr")
    for _ in range(3):
        r.render(mode="cr", schedule="queue", batch_depth=1)
        t = np.asarray(r.view_times())
        assert t[1::2].max() < t[0::2].min(), t
    r.close()


def test_autotune_ex_times_then_reads_its_cache(Renderer, tmp_path):
    import json
    sc, _ = scenegen.uniform_10k(n=5000)
    cams = _cams(41, SIZES * 2)
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    cache = tmp_path / "tune.json"
    o1, res1 = r.autotune_ex(objective="p50", cache=cache, mode="cr", opacity_filter=True)
    assert res1["from_cache"] == 0 and res1["candidates"] >= 5 and res1["batch_ms"] > 0
    assert 0 < res1["view_p50_ms"] <= res1["view_p99_ms"]
    assert (o1.tile_w, o1.tile_h) in {(16, 16), (32, 8), (32, 16), (8, 8)} and o1.schedule in (0, 1)
    entries = json.loads(cache.read_text())
    assert len(entries) == 1
    o2, res2 = r.autotune_ex(objective="p50", cache=cache, mode="cr", opacity_filter=True)
    assert res2["from_cache"] == 1
    assert (o2.tile_w, o2.tile_h, o2.schedule, o2.batch_depth) == (o1.tile_w, o1.tile_h, o1.schedule, o1.batch_depth)
    # another objective is another key
    r.autotune_ex(objective="batch", cache=cache, mode="cr", opacity_filter=True)
    assert len(json.loads(cache.read_text())) == 2
    # the chosen options render
    r.render(options=o2)
    r.close()
