"""Pins of the oracle's offline view-dependent representation (Sec. 3.3
"Offline Clustering") against facts fixed outside of it (CPU only):
k-means against scikit-learn's Lloyd iterations from the same seeds and
against the D^2 sampling law of its seeding; per-pixel top-k contributors
against a brute-force walk, the conservation of transmittance and the order
rule; the cluster masks against their definition and against the image they
must leave unchanged."""
import math

import numpy as np
import pytest

import oracle
import scenegen
from tests.scene_helpers import camera, scene


def _blobs(seed, k=5, per=40, dim=6, spread=0.05):
    rs = np.random.default_rng(seed)
    centres = rs.uniform(-1, 1, (k, dim))
    x = np.concatenate([c + spread * rs.standard_normal((per, dim)) for c in centres])
    return x, centres, np.repeat(np.arange(k), per)


def test_kmeans_lloyd_matches_scikit_learn_from_the_same_seeds():
    KMeans = pytest.importorskip("sklearn.cluster").KMeans
    x, _, _ = _blobs(0, k=6, per=30, spread=0.3)
    u = np.random.default_rng(1).random(6)
    seeds, assign0, it0 = oracle.kmeans(x, 6, u, max_iter=0)
    assert it0 == 0 and np.all(assign0 == -1)
    cent, assign, it = oracle.kmeans(x, 6, u, max_iter=100)
    km = KMeans(n_clusters=6, init=seeds, n_init=1, max_iter=100, tol=0.0, algorithm="lloyd").fit(x)
    np.testing.assert_array_equal(assign, km.labels_)
    np.testing.assert_allclose(cent, km.cluster_centers_, rtol=0, atol=1e-12)
    assert 0 < it < 100


def test_kmeans_fixed_point_and_separated_clusters():
    x, centres, label = _blobs(2, k=5, per=40, spread=0.02)
    cent, assign, _ = oracle.kmeans(x, 5, np.random.default_rng(3).random(5))
    # a fixed point: every point is nearest to its own centre, every centre
    # is the mean of its points
    d = ((x[:, None, :] - cent[None, :, :]) ** 2).sum(-1)
    np.testing.assert_array_equal(assign, np.argmin(d, 1))
    for j in range(5):
        np.testing.assert_allclose(cent[j], x[assign == j].mean(0), rtol=0, atol=1e-12)
    # well separated blobs are recovered up to a relabelling
    perm = {}
    for a, b in zip(assign, label):
        assert perm.setdefault(a, b) == b
    assert len(set(perm.values())) == 5


def test_kmeans_seeding_follows_the_squared_distance_law():
    """Given the first centre, the second is drawn with probability
    proportional to the squared distance to it (k-means++)."""
    rs = np.random.default_rng(4)
    x = rs.uniform(-1, 1, (7, 2))
    n_draw = 20000
    first = 3
    u0 = (first + 0.5) / 7
    hits = np.zeros(7)
    for u1 in (np.arange(n_draw) + 0.5) / n_draw:
        seeds, _, _ = oracle.kmeans(x, 2, np.array([u0, u1]), max_iter=0)
        hits[np.argmin(((x - seeds[1]) ** 2).sum(1))] += 1
    d2 = ((x - x[first]) ** 2).sum(1)
    np.testing.assert_allclose(hits / n_draw, d2 / d2.sum(), atol=2e-4)
    assert hits[first] == 0


def test_pose_feature_is_position_over_scale_and_view_direction():
    cam = scenegen.look_at((0.0, -1.0, 3.0), (0, 0, 0), 32, 32)
    f = oracle.pose_features([cam], 2.0)[0]
    np.testing.assert_allclose(f[:3], np.array([0.0, -1.0, 3.0]) / 2.0, atol=1e-12)
    v = -np.array([0.0, -1.0, 3.0]) / math.sqrt(10.0)
    np.testing.assert_allclose(f[3:], v, atol=1e-7)  # camera axes are stored in float32
    poses = scenegen.sample_poses(16, 4.0, 8, 8, np.random.default_rng(0))
    assert abs(oracle.position_scale(poses) - 4.0) < 1e-5


def _tiny(seed=0, n=40, W=32, H=24):
    rs = np.random.default_rng(seed)
    cam = camera(f=30.0, width=W, height=H)
    s = scene(rs.uniform(-0.6, 0.6, (n, 3)) + [0, 0, 4], log_scales=rs.normal(math.log(0.12), 0.3, (n, 3)),
              quats=rs.standard_normal((n, 4)), opacity=rs.uniform(0.1, 0.95, n), dc=rs.uniform(-1, 1, (n, 3)))
    return s, cam


def test_topk_contributors_brute_force_and_conservation():
    s, cam = _tiny()
    opts = oracle.Options()
    s64 = oracle.Scene64.from_scene(s)
    r, proj, tile, gid, ranges = oracle.render(s64, cam, opts)
    K = 64  # more than any pixel blends
    ids, w, cnt, _ = oracle.topk_contributors(proj, gid, ranges, cam, opts, K)
    assert cnt.max() < K
    # every blended Gaussian is listed: the contributions and the final
    # transmittance account for the whole pixel
    np.testing.assert_allclose(w.sum(-1) + r.T, 1.0, rtol=0, atol=1e-12)
    # brute force: all visible Gaussians in global (fp32 depth, index) order
    vis = np.nonzero(proj["visible"])[0]
    order = vis[np.lexsort((vis, proj["depth32"][vis].view(np.uint32)))]
    for y in range(0, cam["height"], 5):
        for x in range(0, cam["width"], 3):
            T, contrib = 1.0, []
            for g in order:
                P = proj[g]
                d = np.array([x + 0.5, y + 0.5]) - P["uv"]
                A, B, C = P["conic"]
                q = A * d[0] ** 2 + 2 * B * d[0] * d[1] + C * d[1] ** 2
                if q > P["tg"]:
                    continue
                al = min(opts.alpha_max, P["opacity"] * math.exp(-0.5 * q))
                if al < opts.alpha_min:
                    continue
                if T * (1 - al) < opts.t_stop:
                    break
                contrib.append((T * al, g))
                T *= 1 - al
            contrib.sort(key=lambda c: (-c[0], c[1]))
            c = cnt[y, x]
            assert c == len(contrib)
            np.testing.assert_array_equal(ids[y, x, :c], [g for _, g in contrib])
            np.testing.assert_allclose(w[y, x, :c], [v for v, _ in contrib], rtol=1e-12, atol=0)


def test_topk_keeps_the_largest_in_order():
    s, cam = _tiny(seed=1, n=80)
    opts = oracle.Options()
    r, proj, tile, gid, ranges = oracle.render(oracle.Scene64.from_scene(s), cam, opts)
    full_ids, full_w, full_cnt, _ = oracle.topk_contributors(proj, gid, ranges, cam, opts, 128)
    ids, w, cnt, margin = oracle.topk_contributors(proj, gid, ranges, cam, opts, 4)
    np.testing.assert_array_equal(cnt, np.minimum(full_cnt, 4))
    np.testing.assert_array_equal(ids, full_ids[..., :4])
    np.testing.assert_array_equal(w, full_w[..., :4])
    assert np.all(np.diff(w, axis=-1)[cnt[..., None] > np.arange(1, 4)] <= 0)
    more = full_cnt > 4
    gap = (full_w[..., 3] - full_w[..., 4]) / np.where(full_w[..., 3] > 0, full_w[..., 3], 1)
    assert np.all(margin[more] <= gap[more] + 1e-15)


def test_view_masks_union_and_image_preserved():
    """A Gaussian carries bit c exactly when it is a top-k contributor of a
    pose of cluster c; with k above every pixel's contributor count, each pose
    rendered from its own cluster's Gaussians equals the full render."""
    rs = np.random.default_rng(5)
    n = 90
    s = scene(rs.uniform(-1, 1, (n, 3)) * [2.0, 0.5, 0.5] + [0, 0, 4],
              log_scales=rs.normal(math.log(0.12), 0.3, (n, 3)), quats=rs.standard_normal((n, 4)),
              opacity=rs.uniform(0.1, 0.95, n), dc=rs.uniform(-1, 1, (n, 3)))
    s64 = oracle.Scene64.from_scene(s)
    poses = [scenegen.look_at(rs.normal(0, 0.05, 3), (tx, 0, 4), 24, 20, fov_y_deg=25.0)
             for tx in (-1.5, -1.2, 0.0, 0.3, 1.2, 1.5)]
    assign = np.array([0, 0, 1, 1, 2, 2], np.int32)
    opts = oracle.Options()
    mask, _ = oracle.view_masks(s64, poses, assign, 256)
    expect = np.zeros(s64.n, np.uint32)
    for cam, c in zip(poses, assign):
        r, proj, tile, gid, ranges = oracle.render(s64, cam, opts)
        ids, _, _, _ = oracle.topk_contributors(proj, gid, ranges, cam, opts, 256)
        expect[np.unique(ids[ids >= 0])] |= np.uint32(1 << c)
    np.testing.assert_array_equal(mask, expect)
    masked = oracle.Scene64.from_scene(dict(s, cluster_mask=mask))
    for cam, c in zip(poses, assign):
        full, pf = oracle.render(s64, cam, opts)[:2]
        sub, ps = oracle.render(masked, cam, oracle.Options(use_mask=True, sel_bits=1 << int(c)))[:2]
        np.testing.assert_array_equal(full.rgb, sub.rgb)
        np.testing.assert_array_equal(full.T, sub.T)
    # other clusters' Gaussians are outside the narrow views
    assert all(np.count_nonzero(mask & np.uint32(1 << c)) < np.count_nonzero(mask) for c in range(3))
    mask4, _ = oracle.view_masks(s64, poses, assign, 4)
    assert np.all(mask4 & ~mask == 0) and np.count_nonzero(mask4) < np.count_nonzero(mask)
