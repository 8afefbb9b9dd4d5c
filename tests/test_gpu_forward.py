"""GPU parity of the forward hot path against the FP64 oracle (through the C ABI).

Bars: tile lists, sort order and ranges bit-exact where no rounding decision
is within reach of FP32 (reject-sampled tiny scenes); at larger sizes the same
lists up to the counted ambiguous cases; RGB within max-abs 2e-3 on pixels
whose decisions are >= 1e-3 (relative) from their thresholds and mean-abs
1e-5 over all pixels.
"""
import math

import numpy as np
import pytest

import oracle
import scenegen
from tests import parity
from tests.scene_helpers import camera, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Renderer():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_05168_gb300 import Renderer as R
    return R


def _ragged_scene(n=3000, seed=5, W=100, H=70):
    sc, _ = scenegen.uniform_10k(seed=seed, n=n)
    cam = scenegen.look_at((0.4, -0.3, -3.2), (0, 0, 0), W, H)
    cam["fx"] = cam["fy"] = 85.0
    return sc, cam


# ------------------------------------------------------------ preprocessing --

def test_preprocess_records_match_oracle(Renderer):
    sc, cams = scenegen.uniform_10k()
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    parity.gpu_render(r)
    d = parity.debug_numpy(r)
    proj = oracle.preprocess(oracle.Scene64.from_scene(sc), cams[0], oracle.Options())
    vis_g = d["tiles_touched"] > 0
    vis_o = proj["visible"] == 1
    clear = (proj["margin_px"] >= 1e-3) & (proj["margin_rel"] >= 1e-5)
    assert np.array_equal(vis_g[clear], vis_o[clear])
    both = vis_g & vis_o & clear
    assert both.sum() > 9000
    u, v, con, o, rgb = parity.records_to_proj(d["records"][both])
    np.testing.assert_allclose(u, proj["uv"][both, 0], atol=2e-3)
    np.testing.assert_allclose(v, proj["uv"][both, 1], atol=2e-3)
    cn = np.linalg.norm(proj["conic"][both], axis=1, keepdims=True)
    assert np.max(np.abs(con - proj["conic"][both]) / cn) < 1e-3
    np.testing.assert_allclose(o, proj["opacity"][both], rtol=1e-5)
    np.testing.assert_allclose(rgb, proj["rgb"][both], atol=1e-5)
    np.testing.assert_allclose(d["depth"][both], proj["mean_cam"][both, 2], rtol=1e-6)
    rect_o = proj["rect"][both]
    rg = d["rect"][both].view(np.uint32)
    rect_g = np.stack([rg[:, 0] & 0xFFFF, rg[:, 0] >> 16, rg[:, 1] & 0xFFFF, rg[:, 1] >> 16], 1)
    np.testing.assert_array_equal(rect_g, rect_o)
    np.testing.assert_array_equal(d["tiles_touched"][both], proj["ntiles"][both])
    r.close()


# ---------------------------------------------------------------- tile lists --

def _f32(s):
    return {k: (v.astype(np.float32) if isinstance(v, np.ndarray) and v.dtype == np.float64 else v)
            for k, v in s.items()}


def _is_clear(s, cam, n, opts=None):
    proj = oracle.preprocess(oracle.Scene64.from_scene(s), cam, opts or oracle.Options())
    vis = proj["visible"] == 1
    if vis.sum() < n // 2:
        return False
    if np.min(proj["margin_px"][np.isfinite(proj["margin_px"])]) < 1e-3:
        return False
    if np.min(proj["margin_rel"][np.isfinite(proj["margin_rel"])]) < 1e-4:
        return False
    d = np.sort(proj["depth32"][vis].view(np.uint32).astype(np.int64))
    return np.min(np.diff(d)) > 4


def _clear_tiny_scene(seed, n=48, W=64, H=48, f=50.0, n_big=0, opts=None):
    """Random tiny scene and two cameras with every rect, cull and depth-order
    decision far from a rounding flip (re-drawn until so) for the tiles of
    opts.  The first n_big Gaussians are wide ones near the middle of the
    view."""
    rs = np.random.default_rng(seed)
    cam = camera(f=f, width=W, height=H)
    cam2 = dict(cam, world_to_cam=np.concatenate([np.eye(3), [[0.3], [0.1], [0.5]]], 1))
    for _ in range(500):
        means = rs.uniform(-1, 1, (n, 3)) * [1.0, 0.7, 1.0] + [0, 0, 4]
        log_scales = rs.normal(math.log(0.08), 0.4, (n, 3))
        means[:n_big, :2] *= 0.2
        log_scales[:n_big] = rs.normal(math.log(0.5), 0.1, (n_big, 3))
        s = _f32(scene(means, log_scales=log_scales, quats=rs.standard_normal((n, 4)),
                       opacity=rs.uniform(0.05, 0.95, n), dc=rs.uniform(-1, 1, (n, 3))))
        if _is_clear(s, cam, n, opts) and _is_clear(s, cam2, n, opts):
            return s, [cam, cam2]
    raise RuntimeError("no clear scene found")


@pytest.mark.parametrize("tile_test", ["ellipse", "rect"])
@pytest.mark.parametrize("seed,size,n_big", [(0, (64, 48, 50.0), 0), (1, (64, 48, 50.0), 0),
                                             (2, (200, 120, 160.0), 0), (3, (200, 120, 160.0), 0),
                                             (4, (480, 320, 400.0), 3)])
def test_tile_lists_bit_exact(Renderer, seed, size, n_big, tile_test):
    """Tile lists, their order and ranges equal the oracle's, bit for bit.  The
    480x320 frames hold Gaussians spanning more than 255 tiles, whose counts
    do not fit the count byte the depth sort carries with each record id."""
    _check_tile_lists(Renderer, seed, size, n_big, tile_test)


@pytest.mark.parametrize("seed,size,n_blocks", [(5, (640, 720, 600.0), 460), (6, (1280, 720, 900.0), 920)])
def test_tile_lists_bit_exact_one_wide_block_pass(Renderer, seed, size, n_blocks):
    """8x8 tiles on frames of 257 to 1024 tile blocks: the block sort takes one
    pass with 9-bit (460 blocks) or 10-bit (920 blocks) digits; the tile lists
    expanded from it still equal the oracle's."""
    W, H, _ = size
    tx, ty = -(-W // 8), -(-H // 8)
    assert 2 * (-(-tx // 8)) * (-(-ty // 4)) == n_blocks
    _check_tile_lists(Renderer, seed, size, 3, "ellipse", tile=(8, 8))


def _check_tile_lists(Renderer, seed, size, n_big, tile_test, tile=(16, 16)):
    W, H, f = size
    oo = oracle.Options(tile_test=tile_test, tile_w=tile[0], tile_h=tile[1])
    s, cams = _clear_tiny_scene(seed, W=W, H=H, f=f, n_big=n_big, opts=oo)
    r = Renderer()
    r.load_scene(s)
    r.set_cameras(cams)
    parity.gpu_render(r, tile_test=tile_test, binning="tiles", tile=tile)
    d = parity.debug_numpy(r)
    n = s["means"].shape[0]
    exp_tile, exp_rec, exp_rng = [], [], []
    tile_off, k_off = 0, 0
    for ci, c in enumerate(cams):
        proj = oracle.preprocess(oracle.Scene64.from_scene(s), c, oo)
        tile_ids, gid, ranges = oracle.instances(proj, c, oo)
        exp_tile.append(tile_ids + tile_off)
        exp_rec.append(gid + ci * n)
        rr = ranges.copy()
        nonempty = rr[:, 1] > rr[:, 0]
        rr[nonempty] += k_off
        exp_rng.append(rr)
        tile_off += ranges.shape[0]
        k_off += tile_ids.size
    if n_big:
        assert d["tiles_touched"].max() > 255
    np.testing.assert_array_equal(d["inst_tile"], np.concatenate(exp_tile))
    np.testing.assert_array_equal(d["inst_record"], np.concatenate(exp_rec))
    # an empty tile's range may start anywhere; non-empty ones are exact
    exp = np.concatenate(exp_rng)
    got = d["tile_ranges"].astype(np.int64)
    np.testing.assert_array_equal(got[:, 1] - got[:, 0], exp[:, 1] - exp[:, 0])
    ne = exp[:, 1] > exp[:, 0]
    np.testing.assert_array_equal(got[ne], exp[ne])
    r.close()


@pytest.mark.parametrize("seed,size,n_big,tile", [(2, (200, 120, 160.0), 0, (16, 16)),
                                                  (3, (200, 120, 160.0), 0, (16, 16)),
                                                  (4, (480, 320, 400.0), 3, (16, 16)),
                                                  (6, (1280, 720, 900.0), 3, (8, 8))])
def test_block_lists_filtered_per_tile_are_the_tile_lists(Renderer, seed, size, n_big, tile):
    """Block binning: walking a tile's block list and keeping the entries whose
    mask has the tile's bit gives exactly the oracle's tile list, in order
    (the 200x120 frames span several 8x4-tile blocks each way; the 480x320
    ones hold records up to 20 tile rows tall across many blocks; the 1280x720
    pair at 8x8 tiles has 920 blocks, sorted in one pass of 10-bit digits)."""
    W, H, f = size
    oo = oracle.Options(tile_w=tile[0], tile_h=tile[1])
    s, cams = _clear_tiny_scene(seed, W=W, H=H, f=f, n_big=n_big, opts=oo)
    r = Renderer()
    r.load_scene(s)
    r.set_cameras(cams)
    parity.gpu_render(r, binning="blocks", tile=tile)
    d = parity.debug_numpy(r)
    n = s["means"].shape[0]
    rng = d["tile_ranges"].astype(np.int64)
    mask = d["inst_mask"].view(np.uint32)
    blk_off = 0
    for ci, c in enumerate(cams):
        tx_n, ty_n = oracle.tile_grid(c, oo)
        bx_n, by_n = -(-tx_n // 8), -(-ty_n // 4)
        proj = oracle.preprocess(oracle.Scene64.from_scene(s), c, oo)
        _, gid, ranges = oracle.instances(proj, c, oo)
        for t in range(tx_n * ty_n):
            tx, ty = t % tx_n, t // tx_n
            b = blk_off + (ty // 4) * bx_n + tx // 8
            bit = (ty % 4) * 8 + tx % 8
            sel = slice(rng[b, 0], rng[b, 1])
            keep = (mask[sel] >> bit) & 1 == 1
            got = d["inst_record"][sel][keep].astype(np.int64)
            np.testing.assert_array_equal(got, gid[ranges[t, 0]:ranges[t, 1]] + ci * n, err_msg=f"{ci} {t}")
        blk_off += bx_n * by_n
    assert blk_off == d["n_tiles"]
    # the rasterizer's group skip: summary g is the OR of the masks of entries 32 g .. 32 g + 31
    K = d["n_instances"]
    padded = np.zeros(-(-K // 32) * 32, np.uint32)
    padded[:K] = mask[:K]
    np.testing.assert_array_equal(d["mask_summary"].view(np.uint32),
                                  np.bitwise_or.reduce(padded.reshape(-1, 32), axis=1))
    r.close()


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (32, 16), (8, 8)])
def test_block_binning_renders_bit_identical_to_tile_binning(Renderer, tile):
    sc, _ = scenegen.uniform_10k()
    cams = [scenegen.look_at((0.5 * i, -0.2, -2.6), (0, 0, 0), w, h) for i, (w, h) in
            enumerate([(256, 256), (100, 70), (33, 17), (517, 301)])]
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    for kw in (dict(mode="plain"), dict(mode="cr"), dict(mode="cr", opacity_filter=True),
               dict(mode="cr", group=(2, 4)), dict(mode="cr", group=(1, 1)), dict(mode="cr", group=(4, 4)),
               dict(mode="cr", group=(4, 8)), dict(mode="plain", tile_test="rect")):
        a, ta = parity.gpu_render(r, tile=tile, binning="tiles", **kw)
        nca = parity.debug_numpy(r)["n_contrib"]
        b, tb = parity.gpu_render(r, tile=tile, binning="blocks", **kw)
        ncb = parity.debug_numpy(r)["n_contrib"]
        for x, y in zip(a + ta, b + tb):
            np.testing.assert_array_equal(x, y, err_msg=str(kw))
        np.testing.assert_array_equal(nca, ncb, err_msg=str(kw))
    r.close()


def test_tile_lists_at_scale_up_to_ambiguous_cases(Renderer):
    sc, cams = scenegen.uniform_10k()
    cam = cams[0]
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    parity.gpu_render(r, binning="tiles")
    d = parity.debug_numpy(r)
    proj = oracle.preprocess(oracle.Scene64.from_scene(sc), cam, oracle.Options())
    tile, gid, ranges = oracle.instances(proj, cam, oracle.Options())
    amb = (proj["margin_px"] < 1e-3) | (proj["margin_rel"] < 1e-5)
    dbits = proj["depth32"].view(np.uint32).astype(np.int64)
    n_amb_tiles, n_swaps = 0, 0
    for t in range(ranges.shape[0]):
        g_gpu = d["inst_record"][d["tile_ranges"][t, 0]:d["tile_ranges"][t, 1]]
        g_or = gid[ranges[t, 0]:ranges[t, 1]]
        a = g_gpu[~amb[g_gpu]]
        b = g_or[~amb[g_or]]
        if set(g_gpu.tolist()) != set(g_or.tolist()):
            n_amb_tiles += 1
        assert set(a.tolist()) == set(b.tolist()), t
        # order: equal, except swaps of neighbours within 2 ulp of oracle depth
        if not np.array_equal(a, b):
            pos = {g: i for i, g in enumerate(b)}
            seq = np.array([pos[g] for g in a])
            bad = np.nonzero(np.diff(seq) < 0)[0]
            for i in bad:
                assert abs(dbits[a[i]] - dbits[a[i + 1]]) <= 2, (t, a[i], a[i + 1])
            n_swaps += len(bad)
    assert n_amb_tiles <= 0.01 * ranges.shape[0] + 2
    r.close()


# -------------------------------------------------------------------- images --

CASES = [
    dict(mode="plain"),
    dict(mode="cr"),
    dict(mode="plain", opacity_filter=True),
    dict(mode="cr", opacity_filter=True),
    dict(mode="cr", group=(1, 1)),
    dict(mode="cr", group=(2, 4)),
    dict(mode="cr", group=(4, 4)),
    dict(mode="cr", group=(4, 8)),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "-".join(f"{k}={v}" for k, v in c.items()))
@pytest.mark.parametrize("where", ["uniform_10k", "ragged_100x70"])
def test_render_matches_oracle(Renderer, case, where):
    if where == "uniform_10k":
        sc, cams = scenegen.uniform_10k()
    else:
        sc, cam = _ragged_scene()
        cams = [cam]
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    imgs, Ts = parity.gpu_render(r, **case)
    oo = parity.oracle_options(case["mode"], case.get("group", (2, 2)), case.get("opacity_filter", False))
    ref, proj, _, gid, ranges = oracle.render(oracle.Scene64.from_scene(sc), cams[0], oo, nthreads=8)
    rep = parity.check_render(imgs[0], Ts[0], ref, proj, gid, ranges, cams[0], oo)
    assert rep["ok"], str(rep)
    r.close()


@pytest.mark.parametrize("case", [dict(mode="plain"), dict(mode="cr"), dict(mode="cr", group=(4, 4))],
                         ids=lambda c: "-".join(f"{k}={v}" for k, v in c.items()))
def test_eight_by_eight_tiles_match_oracle(Renderer, case):
    """8x8 tiles (one pixel per thread, groups spanning threads) against the
    oracle run on 8x8 tiles."""
    sc, cams = scenegen.uniform_10k()
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    imgs, Ts = parity.gpu_render(r, tile=(8, 8), **case)
    g = case.get("group", (2, 2))
    oo = oracle.Options(cr=case["mode"] == "cr", group_w=g[0], group_h=g[1], tile_w=8, tile_h=8)
    ref, proj, _, gid, ranges = oracle.render(oracle.Scene64.from_scene(sc), cams[0], oo, nthreads=8)
    rep = parity.check_render(imgs[0], Ts[0], ref, proj, gid, ranges, cams[0], oo)
    assert rep["ok"], str(rep)
    r.close()


def test_cr_one_pixel_groups_equal_plain_bit_exact(Renderer):
    sc, cams = scenegen.uniform_10k()
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    a, _ = parity.gpu_render(r, mode="plain")
    b, _ = parity.gpu_render(r, mode="cr", group=(1, 1))
    np.testing.assert_array_equal(a[0], b[0])
    r.close()


def test_opacity_filter_keeps_image_and_cuts_instances(Renderer):
    sc, cams = scenegen.uniform_10k()
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    a, _ = parity.gpu_render(r, mode="plain", binning="tiles")
    k0 = r.last_stats["n_instances"]
    b, _ = parity.gpu_render(r, mode="plain", opacity_filter=True, binning="tiles")
    k1 = r.last_stats["n_instances"]
    assert k1 < k0
    diff = np.abs(a[0] - b[0])
    assert diff.max() <= parity.RGB_MAX_ABS and (diff == 0).mean() > 0.999
    r.close()


@pytest.mark.parametrize("tile", [(16, 16), (32, 8)])
def test_ellipse_tile_test_keeps_image_and_cuts_instances(Renderer, tile):
    """Dropping the tiles the support ellipse does not reach removes only
    entries the rasterizer would skip, so the images are bit-identical."""
    sc, cams = scenegen.uniform_10k()
    cams = cams + [scenegen.look_at((0.9, -0.4, -2.5), (0, 0, 0), 200, 120)]
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    for kw in (dict(mode="plain"), dict(mode="cr", opacity_filter=True)):
        a, ta = parity.gpu_render(r, tile=tile, tile_test="rect", binning="tiles", **kw)
        k_rect = r.last_stats["n_instances"]
        b, tb = parity.gpu_render(r, tile=tile, tile_test="ellipse", binning="tiles", **kw)
        k_ell = r.last_stats["n_instances"]
        assert k_ell < 0.85 * k_rect, (k_ell, k_rect)
        for x, y in zip(a + ta, b + tb):
            np.testing.assert_array_equal(x, y)
    r.close()


def test_cluster_filter_matches_oracle(Renderer):
    sc, cams = scenegen.clusters_500k(n=60_000, width=320, height=180, n_cams=3)
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    imgs, Ts = parity.gpu_render(r, mode="cr", cluster_filter=True, opacity_filter=True)
    s64 = oracle.Scene64.from_scene(sc)
    for ci, cam in enumerate(cams):
        sel = oracle.select_clusters(s64.centroids, s64.pos_scale, cam, 3)
        oo = parity.oracle_options("cr", opacity_filter=True, cluster_filter=True, sel_bits=sel)
        ref, proj, _, gid, ranges = oracle.render(s64, cam, oo, nthreads=8)
        rep = parity.check_render(imgs[ci], Ts[ci], ref, proj, gid, ranges, cam, oo)
        assert rep["ok"], str((ci, rep))
    r.close()


def test_batched_cameras_equal_single_renders(Renderer):
    sc, _ = scenegen.uniform_10k()
    cams = [scenegen.look_at((0.5 * i, -0.2, -3), (0, 0, 0), w, h) for i, (w, h) in
            enumerate([(64, 48), (100, 70), (33, 17), (256, 128)])]
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    batch, _ = parity.gpu_render(r, mode="cr")
    for ci, c in enumerate(cams):
        r.set_cameras([c])
        single, _ = parity.gpu_render(r, mode="cr")
        np.testing.assert_array_equal(batch[ci], single[0])
    r.close()


# ---------------------------------------------------------- edge cases / API --

def test_degenerate_scenes(Renderer):
    r = Renderer()
    # every Gaussian behind the camera: black image, T = 1, no instances
    sc, cams = scenegen.uniform_10k(n=500)
    back = scenegen.look_at((0, 0, -3), (0, 0, -6), 64, 64)
    r.load_scene(sc)
    r.set_cameras([back])
    imgs, Ts = parity.gpu_render(r)
    assert np.all(imgs[0] == 0) and np.all(Ts[0] == 1) and r.last_stats["n_instances"] == 0
    # a single Gaussian, 1x1 image and a 17x1 image
    s1 = _f32(scene([[0, 0, 4]], dc=0.3))
    for W, H in ((1, 1), (17, 1)):
        cam = camera(f=10.0, width=W, height=H)
        r.load_scene(s1)
        r.set_cameras([cam])
        imgs, _ = parity.gpu_render(r)
        ref = oracle.render(oracle.Scene64.from_scene(s1), cam, oracle.Options())[0]
        np.testing.assert_allclose(imgs[0], ref.rgb, atol=2e-3)
    r.close()


@pytest.mark.parametrize("case", [dict(mode="plain"), dict(mode="cr"), dict(mode="cr", opacity_filter=True)],
                         ids=lambda c: "-".join(f"{k}={v}" for k, v in c.items()))
def test_extreme_attributes_match_oracle(Renderer, case):
    """Opacities above the 0.99 alpha clamp, sub-pixel scales (the 0.3 px^2
    dilation dominates the footprint), Gaussians larger than the image and
    elongated ones, mixed in one frame."""
    rs = np.random.default_rng(21)
    n = 400
    means = rs.uniform(-1, 1, (n, 3)) * [1.2, 0.9, 1.0] + [0, 0, 5]
    ls = rs.normal(math.log(0.05), 0.4, (n, 3))
    ls[:80] = math.log(1e-4)                        # far below a pixel
    ls[80:90] = math.log(2.5)                       # larger than the view
    ls[90:150, 0] = math.log(0.6)                   # needles: one long axis
    ls[90:150, 1:] = math.log(0.004)
    op = rs.uniform(0.05, 0.9, n)
    op[150:260] = 1.0 - rs.uniform(1e-6, 5e-3, 110)  # alpha clamps at the centre
    s = _f32(scene(means, log_scales=ls, quats=rs.standard_normal((n, 4)), opacity=op,
                   dc=rs.uniform(-1, 1, (n, 3))))
    cam = camera(f=120.0, width=160, height=128)
    r = Renderer()
    r.load_scene(s)
    r.set_cameras([cam])
    imgs, Ts = parity.gpu_render(r, **case)
    oo = parity.oracle_options(case["mode"], (2, 2), case.get("opacity_filter", False))
    ref, proj, _, gid, ranges = oracle.render(oracle.Scene64.from_scene(s), cam, oo, nthreads=8)
    rep = parity.check_render(imgs[0], Ts[0], ref, proj, gid, ranges, cam, oo)
    assert rep["ok"], str(rep)
    r.close()


def test_capacity_growth_is_transparent(Renderer):
    # a few huge Gaussians touch every tile: K = n * tiles >> 4 n, so the first
    # attempt overflows the initial capacity and the call grows and re-renders
    n = 16384
    rs = np.random.default_rng(0)
    s = _f32(scene(rs.uniform(-0.2, 0.2, (n, 3)) + [0, 0, 8], log_scales=[math.log(3.0)] * 3, opacity=0.5,
                   dc=rs.uniform(-1, 1, (n, 3))))
    cam = camera(f=75.0, width=256, height=256)
    r = Renderer()
    r.load_scene(s)
    r.set_cameras([cam])
    imgs, Ts = parity.gpu_render(r, binning="tiles")
    assert r.last_stats["retries"] == 1 and r.last_stats["n_instances"] > (1 << 20)
    oo = oracle.Options()
    ref, proj, _, gid, ranges = oracle.render(oracle.Scene64.from_scene(s), cam, oo, nthreads=8)
    rep = parity.check_render(imgs[0], Ts[0], ref, proj, gid, ranges, cam, oo)
    assert rep["ok"], str(rep)
    # a small frame on the grown context: the sorts' grids and count matrices
    # stay sized for the large capacity while only a few tiles hold elements
    s2 = _f32(scene(rs.uniform(-1, 1, (3000, 3)) + [0, 0, 4], log_scales=[math.log(0.05)] * 3, opacity=0.6,
                    dc=rs.uniform(-1, 1, (3000, 3))))
    r.load_scene(s2)
    for binning in ("tiles", "blocks"):
        imgs, Ts = parity.gpu_render(r, binning=binning)
        st = r.last_stats
        assert st["retries"] == 0 and 0 < st["n_instances"] < (1 << 16) and st["capacity"] > (1 << 20), st
        ref, proj, _, gid, ranges = oracle.render(oracle.Scene64.from_scene(s2), cam, oo, nthreads=8)
        rep = parity.check_render(imgs[0], Ts[0], ref, proj, gid, ranges, cam, oo)
        assert rep["ok"], (binning, str(rep))
    r.close()


def test_async_render_and_host_outputs(Renderer):
    import torch
    sc, cams = scenegen.uniform_10k()
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    ref = r.render(mode="cr").cpu().numpy()
    out = torch.empty(3 * r.n_pixels, device=r.device)
    r.render(out=out, mode="cr", sync=False)
    r.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)
    host = np.zeros(3 * r.n_pixels, np.float32)
    r.render(out=host, mode="cr")
    np.testing.assert_array_equal(host, ref)
    pinned = torch.zeros(3 * r.n_pixels, pin_memory=True)
    r.render(out=pinned, mode="cr")
    np.testing.assert_array_equal(pinned.numpy(), ref)
    r.close()


def test_scene_from_device_tensors_and_borrow(Renderer):
    import torch
    sc, cams = scenegen.uniform_10k(n=4000)
    r = Renderer()
    r.load_scene(sc)
    r.set_cameras(cams)
    ref = r.render(mode="plain").cpu().numpy()
    dev = {k: (torch.from_numpy(v).cuda() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    for borrow in (False, True):
        r.load_scene(dev, borrow=borrow)
        r.set_cameras(cams)
        np.testing.assert_array_equal(r.render(mode="plain").cpu().numpy(), ref)
    r.close()


def test_argument_and_state_errors(Renderer):
    from paper_2503_05168_gb300 import SeeleError
    r = Renderer()
    with pytest.raises(SeeleError, match="ERR_STATE"):
        r.render()
    sc, cams = scenegen.uniform_10k(n=100)
    r.load_scene(sc)
    with pytest.raises(SeeleError, match="ERR_STATE"):
        r.render()
    r.set_cameras(cams)
    with pytest.raises(SeeleError, match="ERR_ARG"):
        r.render(mode="cr", group=(3, 3))
    with pytest.raises(SeeleError, match="ERR_ARG"):
        r.render(tile=(16, 8))
    with pytest.raises(SeeleError, match="ERR_STATE"):
        r.render(cluster_filter=True)
    with pytest.raises(SeeleError, match="ERR_ARG"):
        r.set_cameras([dict(cams[0], width=0)])
    bad = dict(sc)
    bad["sh_degree"] = 5
    with pytest.raises(SeeleError, match="ERR_ARG"):
        r.load_scene(bad)
    r.close()
