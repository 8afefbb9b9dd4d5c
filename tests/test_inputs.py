"""The seeded synthetic workloads follow their stated recipes: attribute
distributions, scene shapes and camera rigs (CPU)."""
import math

import numpy as np

import scenegen


def _centre(cam):
    w = np.asarray(cam["world_to_cam"], np.float64)
    R, t = w[:, :3], w[:, 3]
    return -R.T @ t, R[2]


def test_attribute_distributions():
    a = scenegen.attributes(200_000, scenegen.rng(0))
    n = 200_000
    assert a["log_scales"].shape == (n, 3) and a["quats"].shape == (n, 4) and a["sh"].shape == (n, 16, 3)
    assert all(a[k].dtype == np.float32 for k in ("log_scales", "quats", "opacity_logits", "sh"))
    assert a["sh_degree"] == 3
    assert abs(a["log_scales"].mean() - math.log(0.02)) < 0.01 and abs(a["log_scales"].std() - 0.5) < 0.01
    np.testing.assert_allclose(np.linalg.norm(a["quats"], axis=1), 1.0, atol=1e-6)
    assert abs(a["opacity_logits"].mean()) < 0.02 and abs(a["opacity_logits"].std() - 1.5) < 0.02
    assert abs(a["sh"][:, 0].mean() - 0.5) < 0.005 and abs(a["sh"][:, 0].std() - 0.2) < 0.005
    assert abs(a["sh"][:, 1:].mean()) < 0.001 and abs(a["sh"][:, 1:].std() - 0.05) < 0.001


def test_uniform_10k_recipe():
    sc, cams = scenegen.uniform_10k()
    assert sc["means"].shape == (10_000, 3) and np.abs(sc["means"]).max() <= 1.0
    (cam,) = cams
    c, fwd = _centre(cam)
    np.testing.assert_allclose(c, [0, 0, -3], atol=1e-9)
    np.testing.assert_allclose(fwd, [0, 0, 1], atol=1e-12)
    assert (cam["width"], cam["height"]) == (256, 256) and cam["near"] == 0.2
    assert math.isclose(cam["fy"], 128 / math.tan(math.radians(30)), rel_tol=1e-12) and cam["fx"] == cam["fy"]


def test_unbounded_recipe():
    n = 200_000
    sc, cams = scenegen.unbounded_3m(n=n)
    nd = int(round(0.8 * n))
    dense, shell = sc["means"][:nd].astype(np.float64), sc["means"][nd:].astype(np.float64)
    r = np.linalg.norm(shell, axis=1)
    assert r.min() >= 30 - 1e-3 and r.max() <= 50 + 1e-3
    assert np.abs(dense).max() < 3 + 6 * 0.15
    assert abs(sc["log_scales"][nd:].mean() - math.log(0.5)) < 0.01
    assert abs(sc["log_scales"][:nd].mean() - math.log(0.02)) < 0.01
    assert len(cams) == 8
    for cam in cams:
        c, fwd = _centre(cam)
        assert math.isclose(np.linalg.norm(c), 5.0, rel_tol=1e-9) and abs(c[1]) < 1e-9
        np.testing.assert_allclose(fwd, -c / 5.0, atol=1e-12)   # looks at the origin
        assert (cam["width"], cam["height"]) == (1920, 1080)


def test_clusters_and_training_target():
    sc, cams, tgt = scenegen.clusters_1m(n=50_000)
    assert sc["cluster_mask"].shape == (50_000,) and sc["centroids"].shape == (16, 6)
    d = (tgt["means"] - sc["means"]).astype(np.float64)
    assert abs(d.std() - 0.01) < 5e-4
    np.testing.assert_allclose(np.linalg.norm(tgt["quats"], axis=1), 1.0, atol=1e-6)
    (cam,) = cams
    c, _ = _centre(cam)
    assert math.isclose(np.linalg.norm(c), 4.0, rel_tol=1e-9) and (cam["width"], cam["height"]) == (1280, 720)
    # 64 clusters of sigma 0.1 with centres in [-2, 2]^3
    assert np.abs(sc["means"]).max() < 2 + 6 * 0.1


def test_multiview_recipe():
    _, cams = scenegen.multiview_2m(n=10_000)
    assert len(cams) == 64
    res = {(c["width"], c["height"]) for c in cams}
    assert res <= {(640, 360), (1280, 720), (1920, 1080)} and len(res) == 3
    for cam in cams:
        c, fwd = _centre(cam)
        rad = np.linalg.norm(c)
        assert 3.0 <= rad <= 6.0
        assert abs(math.degrees(math.asin(-c[1] / rad))) <= 30 + 1e-9
        np.testing.assert_allclose(fwd, -c / rad, atol=1e-12)


def test_sampled_poses_cover_the_band():
    cams = scenegen.sample_poses(512, 4.0, 320, 180, scenegen.rng(0))
    el = np.array([math.degrees(math.asin(-_centre(c)[0][1] / 4.0)) for c in cams])
    az = np.array([math.atan2(_centre(c)[0][2], _centre(c)[0][0]) for c in cams]) % (2 * math.pi)
    assert np.abs(el).max() <= 30 + 1e-9 and el.min() < -25 and el.max() > 25
    assert np.histogram(az, bins=8, range=(0, 2 * math.pi))[0].min() > 40
